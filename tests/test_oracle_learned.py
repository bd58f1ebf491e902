"""Pins for the learned block-proposal oracle (oracle/learned.py).

- The hand-written backward pass against central finite differences (of the
  network without activation rounding, which is smooth; the rounded network
  uses the same formulas straight through the rounding).
- The bfloat16 activations: exactly representable, within half a bfloat16
  step of the unrounded values, and the logits close to the unrounded ones;
  the gradient of the rounded network (bfloat16 gradients into the 32-channel
  data gradients) close to the exact one, its layer-4 part equal to it.
- The block energy change against the full Hamiltonian (Eq. 1) before and
  after the flip.
- The Metropolis-Hastings block move, interleaved with checkerboard sweeps,
  samples the Boltzmann law exactly: 4x4 torus with 2x2 blocks against exact
  enumeration, for an arbitrary state-dependent proposal and for the network.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import exact, stats
from oracle import learned as ln


def energy(s):
    s = s.astype(np.int64)
    return -int((s * np.roll(s, -1, 0)).sum() + (s * np.roll(s, -1, 1)).sum())


def random_theta(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, ln.N_PARAMS)


def test_param_count():
    assert ln.N_PARAMS == 32 * 9 + 32 + 2 * (32 * 32 * 9 + 32) + 32 * 9 + 1


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = random_theta(1)
    spins = rng.choice([-1.0, 1.0], size=(2, 8, 8))
    dl = rng.normal(size=(2, 4))  # 8x8 lattice, 4x4 blocks
    _, cache = ln.forward(theta, spins, B=4, keep=True, round_act=False)
    g = ln.backward(theta, cache, dl)
    idx = np.concatenate([rng.choice(ln.N_PARAMS, 60, replace=False), [0, 300, 9600, ln.N_PARAMS - 1]])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (np.sum(dl * ln.forward(tp, spins, B=4, round_act=False)) -
              np.sum(dl * ln.forward(tm, spins, B=4, round_act=False))) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    theta = random_theta(3, 0.1)
    spins = rng.choice([-1.0, 1.0], size=(2, 8, 8))
    loss, g = ln.loss_and_grad(theta, spins, 0.44, B=4, round_act=False)
    for i in rng.choice(ln.N_PARAMS, 20, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += 1e-6
        tm[i] -= 1e-6
        fd = (ln.loss_and_grad(tp, spins, 0.44, B=4, round_act=False)[0] -
              ln.loss_and_grad(tm, spins, 0.44, B=4, round_act=False)[0]) / 2e-6
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(fd))


@pytest.mark.parametrize("L,B", [(8, 4), (16, 8), (16, 4)])
def test_block_energy_change_against_hamiltonian(L, B):
    rng = np.random.default_rng(L + B)
    for _ in range(5):
        s = rng.choice(np.array([-1, 1], np.int8), size=(L, L))
        for b in range((L // B) ** 2):
            sp = ln.flip_blocks(s[None].astype(float), [b], B)[0].astype(np.int8)
            assert ln.block_delta_E(s, b, B) == energy(sp) - energy(s)


def test_gelu_matches_its_definition():
    z = np.linspace(-4, 4, 17)
    phi = np.array([0.5 * (1 + math.erf(v / math.sqrt(2))) for v in z])
    np.testing.assert_allclose(ln.gelu(z), z * phi, rtol=0, atol=1e-15)
    h = 1e-6
    np.testing.assert_allclose(ln.gelu_grad(z), (ln.gelu(z + h) - ln.gelu(z - h)) / (2 * h), atol=1e-8)


def test_bf16_rounding():
    x = np.array([1.0, 1.00390625, 1.005859375, -2.5, 3.14159265], dtype=np.float32)
    r = ln.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125  # ties to even, then round up
    assert r[3] == -2.5 and abs(r[4] - 3.140625) < 1e-12


def test_activations_are_bf16_and_close_to_unrounded():
    rng = np.random.default_rng(5)
    theta = ln.bf16_round(random_theta(6, 0.2).astype(np.float32))
    spins = rng.choice([-1.0, 1.0], size=(2, 16, 16))
    lr, cr = ln.forward(theta, spins, B=8, keep=True)
    lu, cu = ln.forward(theta, spins, B=8, keep=True, round_act=False)
    for name in ("a1", "a2", "a3"):
        a = cr[name]
        bits = a.astype(np.float32).view(np.uint32)
        assert np.all(bits & 0xFFFF == 0), name  # exactly bfloat16
        assert np.array_equal(a.astype(np.float32).astype(np.float64), a)
    # a1 sees the same z1 in both networks: within half a bfloat16 step (8
    # significant bits: at most 2^-8 relative, plus the float32 step on the way)
    assert np.all(np.abs(cr["a1"] - cu["a1"]) <= 2.0 ** -8 * (1 + 1e-6) * np.abs(cu["a1"]) + 1e-300)
    assert np.abs(cr["a1"] - cu["a1"]).max() > 0  # rounding did happen
    # the logits move by a small fraction of their spread, not by a different network
    d = np.abs(lr - lu).max()
    assert 0 < d < 0.05 * (np.abs(lu).max() + 1e-12), (d, np.abs(lu).max())


def test_rounded_backward_is_close_to_the_exact_gradient():
    rng = np.random.default_rng(8)
    theta = ln.bf16_round(random_theta(9, 0.2).astype(np.float32))
    spins = rng.choice([-1.0, 1.0], size=(2, 16, 16))
    dl = rng.normal(size=(2, 4))
    _, cr = ln.forward(theta, spins, B=8, keep=True)
    gr = ln.backward(theta, cr, dl)
    cu = dict(cr, round=False)  # same rounded activations, unrounded gradients
    gu = ln.backward(theta, cu, dl)
    parts = ln.unflatten(np.arange(ln.N_PARAMS))
    w4 = np.concatenate([parts["W4"].ravel(), parts["b4"].ravel(), parts["W3"].ravel(), parts["b3"].ravel()])
    # W4, b4 and W3 see dz3 unrounded: identical
    np.testing.assert_array_equal(gr[w4.astype(int)], gu[w4.astype(int)])
    # W2 and W1 see gradients that went through bfloat16 (2^-8 relative per value)
    d = np.abs(gr - gu).max() / np.abs(gu).max()
    assert 0 < d < 1e-2, d


def _chain_bond_sums(logits_fn, beta, n_cycles, seed, L=4, B=2):
    s = oracle.init(L, oracle.MODE_RANDOM, seed)
    out = np.zeros(n_cycles, dtype=np.int64)
    acc = 0
    for t in range(n_cycles):
        oracle.run(s, beta, 1, seed, off=t, trace=False, nthreads=1)
        u1 = oracle.draw_stream(seed, 0, 0, t, 0, 3)
        u2 = oracle.draw_stream(seed, 0, 1, t, 0, 3)
        _, _, a = ln.block_move(s, logits_fn, beta, B, u1, u2)
        acc += int(a)
        out[t] = -energy(s)
    return out, acc / n_cycles


@pytest.mark.parametrize("kind", ["uniform", "state_dependent"])
def test_block_moves_keep_the_boltzmann_law(kind):
    beta, L, B = 0.45, 4, 2
    ex = exact.enumerate_lattice(L, beta)

    def state_q(sp):
        # an arbitrary positive proposal that depends on the state: strongly
        # prefers blocks whose spins agree with the lattice's majority
        s = sp[0]
        n = L // B
        blk = s.reshape(n, B, n, B).sum(axis=(1, 3)).ravel()
        return (1.5 * blk * np.sign(s.sum() + 0.5))[None]

    fn = None if kind == "uniform" else state_q
    chains = [_chain_bond_sums(fn, beta, 15000, 40 + c) for c in range(4)]
    series = [c[0] for c in chains]
    assert min(c[1] for c in chains) > 0.02  # moves are accepted
    for lev, p in zip(ex["bond_levels"], ex["bond_probs"]):
        if p < 0.03:
            continue
        ind = [(x == lev).astype(float) for x in series]
        f, err = stats.pooled_mean_and_error(ind)
        assert abs(f - p) < 4 * err + 1e-4, (lev, f, p, err)


def test_block_moves_with_the_network_keep_the_boltzmann_law():
    beta, L, B = 0.45, 4, 2
    theta = random_theta(7, 0.5)
    ex = exact.enumerate_lattice(L, beta)
    fn = lambda sp: ln.forward(theta, sp, B=B)  # noqa: E731
    chains = [_chain_bond_sums(fn, beta, 2500, 70 + c) for c in range(3)]
    series = [c[0] for c in chains]
    m, err = stats.pooled_mean_and_error([-x / 16.0 for x in series])
    assert abs(m - ex["e"]) < 4 * err, (m, err, ex["e"])
