"""Parity of the learned block-proposal kernels with the float64 oracle.

Network forward and backward agree with oracle/learned.py (same
bfloat16-rounded weights) within FP32 accumulation error; the block energy
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


def test_param_count_matches_oracle():
    assert ising.ising_net_param_count() == ln.N_PARAMS


@pytest.mark.parametrize("L,C", [(32, 3), (64, 2)])
def test_forward_matches_oracle(L, C):
    mv = chains(L, C, 11)
    th = theta32(1)
    params = torch.from_numpy(th).cuda()
    logits = torch.zeros((C, (L // 8) ** 2), dtype=torch.float32, device="cuda")
    ising.ising_net_forward(L, C, mv.black, mv.white, None, params, logits, mv.work)
    flips = torch.tensor([3, -1, 7][:C], dtype=torch.int32, device="cuda")
    logits_f = torch.zeros_like(logits)
    ising.ising_net_forward(L, C, mv.black, mv.white, flips, params, logits_f, mv.work)
    torch.cuda.synchronize()
    s = host_spins(mv)
    tb = ln.bf16_round(th)
    want = ln.forward(tb, s, B=8)
    want_f = ln.forward(tb, s, B=8, flip=flips.cpu().numpy())
    np.testing.assert_allclose(logits.cpu().numpy(), want, rtol=1e-4, atol=2e-5)
    np.testing.assert_allclose(logits_f.cpu().numpy(), want_f, rtol=1e-4, atol=2e-5)
    # the forward pass is deterministic
    again = torch.zeros_like(logits)
    ising.ising_net_forward(L, C, mv.black, mv.white, None, params, again, mv.work)
    torch.cuda.synchronize()
    assert torch.equal(again, logits)


def test_backward_and_loss_match_oracle():
    L, C = 32, 2
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
