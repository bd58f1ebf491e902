"""Parity of the learned block-proposal kernels with the float64 oracle.

Network forward and backward agree with oracle/learned.py (same
bfloat16-rounded weights, bfloat16 activations) within FP32 accumulation
error; the band pass for flipped states equals the full pass bit for bit; the
block energy
changes, the proposal draws, the acceptance decisions and the flipped planes
agree exactly, given the GPU's own logits; and a short training run on the
GPU makes network proposals accepted far more often than uniform ones.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1906_06297_gb300 as ising
from oracle import learned as ln

pytestmark = pytest.mark.gpu
BETA = 0.4406868


@pytest.fixture(scope="module", autouse=True)
def built():
    ising.build()
    oracle.build()


def chains(L, C, seed, sweeps=5):
    mv = ising.BlockMove(L, C, BETA)
    mv.batch.init(ising.ISING_INIT_RANDOM, seed)
    mv.batch.run(sweeps, seed)
    torch.cuda.synchronize()
    return mv


def host_spins(mv):
    return np.stack([oracle.from_planes_msc4(mv.L, *mv.batch.planes_numpy(c)) for c in range(mv.C)]).astype(np.float64)


def theta32(seed, scale=0.2):
    return np.random.default_rng(seed).normal(0.0, scale, ln.N_PARAMS).astype(np.float32)


def assert_logits_close(got, want):
    """Tolerance of the BF16 network.  The kernels accumulate in FP32 (about
    1e-6 relative against the oracle's float64), and where that decides a
    bfloat16 rounding of an activation differently, the activation moves by
    one bfloat16 step (<= 2^-8 relative).  On these sizes such flips move a
    logit by up to ~4e-4 on logits of size ~5 (measured by emulating FP32
    accumulation on the CPU); the bound is 1e-3 of the logit scale."""
    scale = max(1.0, float(np.abs(want).max()))
    np.testing.assert_allclose(got, want, rtol=1e-3, atol=1e-3 * scale)


def test_param_count_matches_oracle():
    assert ising.ising_net_param_count() == ln.N_PARAMS


# (L, C): one row spans 1/4, 1/2, 1 and 2 tiles of 128 pixels, a ragged
# 160-pixel row, 40 chains of 64^2 = 1280 tiles (several per CTA of the
# general kernel: both shared-memory stages and both barrier phases in use),
# and 40 chains of 128^2 = 320 units of 16 rows for the row-ring kernel (more
# units than CTAs; the ring of 10 rows and the 4 accumulators wrap)
@pytest.mark.parametrize("L,C", [(32, 3), (64, 2), (96, 2), (128, 2), (160, 1), (256, 1), (64, 40), (128, 40)])
def test_forward_matches_oracle(L, C):
    mv = chains(L, C, 11)
    th = theta32(1)
    params = torch.from_numpy(th).cuda()
    nb = (L // 8) ** 2
    logits = torch.zeros((C, nb), dtype=torch.float32, device="cuda")
    ising.ising_net_forward(L, C, mv.black, mv.white, None, params, logits, mv.work)
    flips = torch.tensor([(3 + 5 * c) % nb if c % 3 != 1 else -1 for c in range(C)], dtype=torch.int32,
                         device="cuda")
    logits_f = torch.zeros_like(logits)
    ising.ising_net_forward(L, C, mv.black, mv.white, flips, params, logits_f, mv.work)
    ising.ising_net_check()
    s = host_spins(mv)
    tb = ln.bf16_round(th)
    want = ln.forward(tb, s, B=8)
    want_f = ln.forward(tb, s, B=8, flip=flips.cpu().numpy())
    assert_logits_close(logits.cpu().numpy(), want)
    assert_logits_close(logits_f.cpu().numpy(), want_f)
    # the forward pass is deterministic
    again = torch.zeros_like(logits)
    ising.ising_net_forward(L, C, mv.black, mv.white, None, params, again, mv.work)
    torch.cuda.synchronize()
    assert torch.equal(again, logits)


def test_forward_at_full_size_on_sampled_chains():
    """The launch configuration of the benchmark's network leg: 1024 chains of
    128^2 after 20 sweeps.  Full forward and flipped-band forward of all
    chains on the GPU; chains 0, 517 and 1023 against the oracle."""
    L, C = 128, 1024
    mv = chains(L, C, 13, sweeps=20)
    th = theta32(2)
    params = torch.from_numpy(th).cuda()
    nb = (L // 8) ** 2
    logits = torch.zeros((C, nb), dtype=torch.float32, device="cuda")
    logits_f = torch.zeros_like(logits)
    flips = torch.tensor([(7 * c + 3) % nb for c in range(C)], dtype=torch.int32, device="cuda")
    ising.ising_net_forward(L, C, mv.black, mv.white, None, params, logits, mv.work)
    ising.ising_net_forward_flipped(L, C, mv.black, mv.white, flips, params, logits, logits_f, mv.work)
    ising.ising_net_check()
    torch.cuda.synchronize()
    sample = [0, 517, 1023]
    s = np.stack([oracle.from_planes_msc4(L, *mv.batch.planes_numpy(c)) for c in sample]).astype(np.float64)
    tb = ln.bf16_round(th)
    assert_logits_close(logits.cpu().numpy()[sample], ln.forward(tb, s, B=8))
    f = flips.cpu().numpy()[sample]
    assert_logits_close(logits_f.cpu().numpy()[sample], ln.forward(tb, s, B=8, flip=f))


@pytest.mark.parametrize("L,C", [(128, 6), (256, 3), (384, 2), (64, 3), (96, 2)])
def test_flipped_band_pass_equals_full_pass(L, C):
    """ising_net_forward_flipped recomputes a band of rows around each chain's
    flipped block (L a multiple of 128) and copies the other logits; it must
    equal the full forward of the flipped states bit for bit, including blocks
    in the first and last block rows (the band wraps around the torus)."""
    mv = chains(L, C, 17)
    params = torch.from_numpy(theta32(5, 0.25)).cuda()
    n1 = L // 8
    nb = n1 * n1
    picks = [0, nb - 1, n1 - 1, nb - n1, (n1 // 2) * n1 + 3, 5 * n1 + n1 // 3]
    flips = torch.tensor([picks[c % len(picks)] for c in range(C)], dtype=torch.int32, device="cuda")
    lx = torch.zeros((C, nb), dtype=torch.float32, device="cuda")
    ising.ising_net_forward(L, C, mv.black, mv.white, None, params, lx, mv.work)
    full = torch.zeros_like(lx)
    ising.ising_net_forward(L, C, mv.black, mv.white, flips, params, full, mv.work)
    band = torch.full_like(lx, float("nan"))
    ising.ising_net_forward_flipped(L, C, mv.black, mv.white, flips, params, lx, band, mv.work)
    ising.ising_net_check()
    assert torch.equal(band, full)
    # and the flip changed the logits near the block only
    changed = (full != lx).cpu().numpy()
    for c in range(C):
        by = int(flips[c]) // n1
        rows = {(by - 1) % n1, by, (by + 1) % n1}
        ch = changed[c].reshape(n1, n1)
        assert ch.any()
        assert not any(ch[r].any() for r in range(n1) if r not in rows)


def test_flipped_band_pass_rejects_bad_arguments():
    L, C = 128, 2
    mv = chains(L, C, 3, sweeps=1)
    params = torch.from_numpy(theta32(1)).cuda()
    lx = torch.zeros((C, (L // 8) ** 2), dtype=torch.float32, device="cuda")
    flips = torch.zeros(C, dtype=torch.int32, device="cuda")
    with pytest.raises(ising.IsingError):
        ising.ising_net_forward_flipped(L, C, mv.black, mv.white, flips, params, lx, lx, mv.work)
    with pytest.raises(ising.IsingError):
        ising.ising_net_forward_flipped(L, C, mv.black, mv.white, flips, params, lx, torch.zeros_like(lx),
                                        mv.work[:1024])


def test_bounded_wait_reports_timeout_and_device_stays_usable():
    """The first conv layer withholds one accumulator signal: its waits give up
    (about 2 s), ising_net_check reports ISING_ETIMEOUT, and a normal forward
    afterwards gives the same logits as before."""
    L, C = 128, 2
    mv = chains(L, C, 7)
    params = torch.from_numpy(theta32(3)).cuda()
    want = torch.zeros((C, (L // 8) ** 2), dtype=torch.float32, device="cuda")
    ising.ising_net_forward(L, C, mv.black, mv.white, None, params, want, mv.work)
    ising.ising_net_check()
    junk = torch.zeros_like(want)
    ising.ising_net_wait_selftest(L, C, mv.black, mv.white, params, junk, mv.work)
    with pytest.raises(ising.IsingError) as e:
        ising.ising_net_check()
    assert e.value.status == ising.ISING_ETIMEOUT
    ising.ising_net_check()  # the flag was cleared
    again = torch.zeros_like(want)
    ising.ising_net_forward(L, C, mv.black, mv.white, None, params, again, mv.work)
    ising.ising_net_check()
    assert torch.equal(again, want)


# (32, 2): CUDA-core weight gradients; (128, 2) and (256, 3): tensor-core
# weight gradients of the 32 -> 32 layers, one and two row segments, CTA
# ranges of one or two rows that run across chain boundaries, and of ~10 rows
@pytest.mark.parametrize("L,C", [(32, 2), (128, 2), (256, 3)])
def test_backward_and_loss_match_oracle(L, C):
    mv = chains(L, C, 5)
    th = theta32(2, 0.15)
    params = torch.from_numpy(th).cuda()
    work = torch.empty(ising.ising_net_workspace_bytes(L, C, True), dtype=torch.uint8, device="cuda")
    nb = (L // 8) ** 2
    logits = torch.zeros((C, nb), dtype=torch.float32, device="cuda")
    dlogits = torch.zeros_like(logits)
    chain_sq = torch.zeros(C, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    grad = torch.zeros(ln.N_PARAMS, dtype=torch.float32, device="cuda")
    ising.ising_net_forward(L, C, mv.black, mv.white, None, params, logits, work, train=True)
    ising.ising_net_targets_loss(L, C, mv.black, mv.white, BETA, logits, dlogits, chain_sq, loss)
    ising.ising_net_backward(L, C, mv.black, mv.white, params, dlogits, grad, work)
    torch.cuda.synchronize()
    s = host_spins(mv)
    tb = ln.bf16_round(th)
    want_loss, want_grad = ln.loss_and_grad(tb, s, BETA, B=8)
    assert abs(float(loss.item()) - want_loss) < 1e-4 * max(1.0, want_loss)
    g = grad.cpu().numpy().astype(np.float64)
    scale = np.abs(want_grad).max()
    np.testing.assert_allclose(g, want_grad, rtol=2e-3, atol=2e-5 * scale)
    # the reductions have a fixed order: a second backward pass is bit-identical
    again = torch.zeros_like(grad)
    ising.ising_net_backward(L, C, mv.black, mv.white, params, dlogits, again, work)
    ising.ising_net_check()
    assert torch.equal(again, grad)


def test_proposals_acceptances_and_flips_match_oracle():
    L, C, seed = 32, 8, 21
    mv = chains(L, C, seed, sweeps=20)
    th = theta32(4, 0.3)
    params = torch.from_numpy(th).cuda()
    s_before = host_spins(mv)
    for t in range(6):
        use_net = t % 2 == 0
        mv.move(params if use_net else None, seed, t)
        torch.cuda.synchronize()
        lx = mv.lx.cpu().numpy().astype(np.float64)
        lxp = mv.lxp.cpu().numpy().astype(np.float64)
        blocks = mv.block.cpu().numpy()
        acc = mv.accepted.cpu().numpy()
        dE = mv.dE.cpu().numpy()
        s_after = host_spins(mv)
        for c in range(C):
            u1 = oracle.draw_stream(seed, c, 0, t, 0, 3)
            u2 = oracle.draw_stream(seed, c, 1, t, 0, 3)
            b = ln.sample_block(lx[c], u1) if use_net else ln.sample_uniform(mv.nb, u1)
            assert blocks[c] == b
            assert dE[c] == ln.block_delta_E(s_before[c], b, 8)
            if use_net:
                lf = float(ln.log_softmax(lx[c])[b])
                lr = float(ln.log_softmax(lxp[c])[b])
                T = ln.accept_threshold(BETA, int(dE[c]), lf, lr)
            else:
                T = ln.accept_threshold(BETA, int(dE[c]))
            assert bool(acc[c]) == (u2 < T)
            want = ln.flip_blocks(s_before[c][None], [b], 8)[0] if acc[c] else s_before[c]
            np.testing.assert_array_equal(s_after[c], want)
        s_before = s_after


def test_training_on_a_side_stream_is_deterministic():
    """Training data, parameters and every kernel of a training run are
    ordered on the caller's stream: two runs on a side stream with the same
    seed give the same loss history and bit-identical parameters (the step-1
    loss comes before any update, so it depends on the data alone)."""
    runs = []
    for _ in range(2):
        s = torch.cuda.Stream()
        res = ising.train_block_proposer(32, BETA, n_configs=2048, batch=64, steps=6, lr=3e-3, seed=11,
                                         sweeps_between=2, equilibrate=5, log_every=1, stream=s)
        torch.cuda.synchronize()
        runs.append((res["loss"], res["params"].cpu()))
    assert runs[0][0] == runs[1][0]
    assert torch.equal(runs[0][1], runs[1][1])


def test_training_makes_proposals_accepted_more_often():
    """After a short GPU training run the network's proposals have a several
    times larger Metropolis-Hastings acceptance probability than uniform ones
    from the same states (at beta_c an 8x8 flip is rarely accepted at all:
    uniform proposals ~0.1%).  The mean acceptance probability min(1, e^x) of
    the proposals made is compared, which is far less noisy than counts."""
    L, C, steps = 32, 256, 30
    res = ising.train_block_proposer(L, BETA, n_configs=1024, batch=32, steps=300, lr=3e-3, seed=3)
    assert res["loss"][-1] < 0.5 * res["loss"][0]
    params = res["params"]
    mean_p, counts = {}, {}
    for name, p in (("net", params), ("uniform", None)):
        mv = chains(L, C, 99, sweeps=100)
        probs, acc = [], 0
        for t in range(steps):
            mv.batch.run(1, 99, 100 + t)
            mv.move(p, 99, t)
            dE = mv.dE.cpu().numpy().astype(np.float64)
            x = -BETA * dE
            if p is not None:
                lx = mv.lx.cpu().numpy().astype(np.float64)
                lxp = mv.lxp.cpu().numpy().astype(np.float64)
                b = mv.block.cpu().numpy()
                for c in range(C):
                    x[c] += ln.log_softmax(lxp[c])[b[c]] - ln.log_softmax(lx[c])[b[c]]
            probs.append(np.minimum(1.0, np.exp(x)))
            acc += int(mv.accepted.sum().item())
        mean_p[name] = float(np.mean(probs))
        counts[name] = acc
    assert mean_p["net"] > 3 * mean_p["uniform"], (mean_p, counts)
    assert counts["net"] > counts["uniform"], (mean_p, counts)
