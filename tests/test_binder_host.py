"""Host arithmetic of the Binder-cumulant study (no GPU): the cumulant of
known distributions and the crossing finder."""
import numpy as np

from paper_1906_06297_gb300 import binder


def test_binder_of_known_distributions():
    rng = np.random.default_rng(0)
    g = rng.normal(size=2_000_000)  # Gaussian: <m^4> = 3 <m^2>^2, U = 0
    u = binder.binder_from_moments(np.mean(g ** 2), np.mean(g ** 4))
    assert abs(u) < 0.01
    # two-peaked m = +-a: <m^4> = <m^2>^2, U = 2/3 (ordered phase limit)
    a = np.where(rng.random(1000) < 0.5, -0.7, 0.7)
    assert abs(binder.binder_from_moments(np.mean(a ** 2), np.mean(a ** 4)) - 2.0 / 3.0) < 1e-12


def test_crossings_by_linear_interpolation():
    beta = np.linspace(0.40, 0.48, 9)
    ua = 0.3 + 4.0 * (beta - 0.40)
    ub = 0.2 + 6.0 * (beta - 0.40)  # equal at beta = 0.45
    (x,) = binder.crossings(beta, ua, ub)
    assert abs(x - 0.45) < 1e-12
    assert binder.crossings(beta, ua, ua + 1.0) == []
    assert abs(binder.BETA_C - 0.44068679350977151) < 1e-15
