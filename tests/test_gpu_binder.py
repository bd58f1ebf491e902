"""The Binder cumulant crossing (Sec. 5.3, Fig. 6) from the batched sampler
with replica exchange: U_32(beta) and U_64(beta) cross at the critical
inverse temperature ln(1 + sqrt 2)/2 and take the known critical value
U* ~ 0.611 of the periodic square lattice there.  The paper runs 512^2 to
4096^2 for 16M to 1B sweeps; these sizes reach the same crossing in seconds."""
import numpy as np
import pytest

from paper_1906_06297_gb300 import binder

pytestmark = pytest.mark.gpu


def test_binder_curves_cross_at_beta_c():
    import paper_1906_06297_gb300 as ising

    ising.build()
    res = binder.binder_study(sizes=(32, 64), ladders=8, ladder_size=16, beta_lo=0.41, beta_hi=0.47,
                              sweeps=20000, thermalize=2000, record_every=2, chunks=10, seed=5)
    u32, u64 = np.array(res["U"]["32"]), np.array(res["U"]["64"])
    # disordered side: larger lattices lower; ordered side: higher; both rise with beta
    assert u64[0] < u32[0] and u64[-1] > u32[-1]
    assert u32[-1] > u32[0] + 0.2 and u64[-1] > u64[0] + 0.3
    (cross,) = res["crossings"]["32/64"]
    assert abs(cross - binder.BETA_C) < 0.01, res["crossings"]
    for side in ("32", "64"):
        assert 0.57 < res["U_at_beta_nearest_c"][side] < 0.65, res["U_at_beta_nearest_c"]
    assert max(res["U_err"]["64"]) < 0.02
