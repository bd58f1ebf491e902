"""Oracle for the learned block-proposal move (float64 numpy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Not in the paper: a
Metropolis-Hastings move that flips one B x B block of spins, proposed by a
small convolutional network, interleaved with the checkerboard sweep.

Network f (all convolutions 3 x 3, periodic, cross-correlation,
z(y, x)[o] = b[o] + sum_{i, dy, dx} W[o][i][3(dy+1) + (dx+1)] a(y+dy, x+dx)[i]):
    a0 = spins (+1/-1), one channel
    a1 = r(gelu(conv(a0; W1, b1)))   1 -> 32 channels
    a2 = r(gelu(conv(a1; W2, b2)))  32 -> 32
    a3 = r(gelu(conv(a2; W3, b3)))  32 -> 32
    z4 = conv(a3; W4, b4)           32 -> 1
    l_b = mean of z4 over block b   (blocks of B x B, b = by * (L/B) + bx)
gelu(z) = z Phi(z) (Phi the standard normal CDF).  It is a BF16 network: the
caller passes bfloat16-valued weights, and r rounds each activation to the
nearest bfloat16 (via float32, ties to even); everything else is float64 here.
Gradients pass straight through r (the rounded activations enter the weight
gradients); in the same way the gradient entering each 32 -> 32 layer's data
gradient (dz3, dz2) is rounded to bfloat16 there, while the weight gradients
take it unrounded.  The proposal picks block b
with probability q_x(b) = softmax(l)_b; x' is x with block b flipped.

Move (exact Metropolis-Hastings): accept with min(1, exp(-beta dE) q_x'(b) /
q_x(b)), dE = E(x') - E(x) = 2 * sum over the bonds crossing the block
boundary of s_in * s_out.

Training target (regression of the block acceptance): t_b = min(0, -beta dE_b),
loss = mean over chains and blocks of (l_b - t_b)^2.

Parameters travel as one flat vector in the order W1 (32x9), b1 (32),
W2 (32x32x9), b2 (32), W3 (32x32x9), b3 (32), W4 (32x9), b4 (1).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

C1 = 32
SHAPES = [("W1", (C1, 1, 9)), ("b1", (C1,)), ("W2", (C1, C1, 9)), ("b2", (C1,)), ("W3", (C1, C1, 9)),
          ("b3", (C1,)), ("W4", (1, C1, 9)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
OFFSETS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]  # tap k = 3 (dy+1) + (dx+1)


def unflatten(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = theta[o:o + n].reshape(shape)
        o += n
    return out


def flatten(parts) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bf16_round(x) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(x, dtype=np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return z * 0.5 * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def conv(a, W, b):
    """a: (C, Cin, L, L); W: (Cout, Cin, 9); periodic 3x3 cross-correlation."""
    z = np.zeros((a.shape[0], W.shape[0], a.shape[2], a.shape[3]))
    for k, (dy, dx) in enumerate(OFFSETS):
        shifted = np.roll(a, shift=(-dy, -dx), axis=(2, 3))  # shifted[y, x] = a[y+dy, x+dx]
        z += np.einsum("oi,ciyx->coyx", W[:, :, k], shifted)
    return z + b[None, :, None, None]


def conv_backward(a, W, dz, dz_data=None):
    """Gradients of sum(dz * conv(a, W, b)) w.r.t. a, W and b; the gradient
    w.r.t. a uses dz_data in place of dz when it is given."""
    dW = np.zeros_like(W)
    da = np.zeros_like(a)
    dd = dz if dz_data is None else dz_data
    for k, (dy, dx) in enumerate(OFFSETS):
        shifted = np.roll(a, shift=(-dy, -dx), axis=(2, 3))
        dW[:, :, k] = np.einsum("coyx,ciyx->oi", dz, shifted)
        # z[y, x] uses a[y+dy, x+dx]: push dz back to those inputs
        back = np.einsum("oi,coyx->ciyx", W[:, :, k], dd)
        da += np.roll(back, shift=(dy, dx), axis=(2, 3))
    db = dz.sum(axis=(0, 2, 3))
    return da, dW, db


def block_pool(z4, B):
    C, _, L, _ = z4.shape
    n = L // B
    return z4[:, 0].reshape(C, n, B, n, B).mean(axis=(2, 4)).reshape(C, n * n)


def flip_blocks(spins, blocks, B):
    """Copy of spins (C, L, L) with block blocks[c] of chain c flipped (-1: none)."""
    s = np.array(spins, dtype=np.float64, copy=True)
    n = s.shape[1] // B
    for c, b in enumerate(blocks):
        if b < 0:
            continue
        by, bx = divmod(int(b), n)
        s[c, by * B:(by + 1) * B, bx * B:(bx + 1) * B] *= -1
    return s


def forward(theta, spins, B=8, flip=None, keep=False, round_act=True):
    """Logits (C, (L/B)^2) of the chains' spins (C, L, L); `flip` optionally
    flips one block per chain first.  round_act=False evaluates the same
    network without rounding the activations (a smooth function of the
    parameters, for finite-difference checks of the backward formulas)."""
    p = unflatten(theta)
    s = np.asarray(spins, dtype=np.float64)
    if flip is not None:
        s = flip_blocks(s, flip, B)
    r = bf16_round if round_act else (lambda v: v)
    a0 = s[:, None]
    z1 = conv(a0, p["W1"], p["b1"]); a1 = r(gelu(z1))
    z2 = conv(a1, p["W2"], p["b2"]); a2 = r(gelu(z2))
    z3 = conv(a2, p["W3"], p["b3"]); a3 = r(gelu(z3))
    z4 = conv(a3, p["W4"], p["b4"])
    logits = block_pool(z4, B)
    if keep:
        return logits, dict(a0=a0, z1=z1, a1=a1, z2=z2, a2=a2, z3=z3, a3=a3, B=B, round=round_act)
    return logits


def backward(theta, cache, dlogits):
    """Gradient (flat) of sum(dlogits * logits) w.r.t. the parameters, through
    the activations kept in `cache` (straight through their rounding)."""
    p = unflatten(theta)
    B = cache["B"]
    C, nb = dlogits.shape
    n = int(round(math.sqrt(nb)))
    L = n * B
    dz4 = np.repeat(np.repeat(dlogits.reshape(C, n, n), B, axis=1), B, axis=2)[:, None] / (B * B)
    r = bf16_round if cache.get("round", True) else (lambda v: v)
    da3, dW4, db4 = conv_backward(cache["a3"], p["W4"], dz4)
    dz3 = da3 * gelu_grad(cache["z3"])
    da2, dW3, db3 = conv_backward(cache["a2"], p["W3"], dz3, dz_data=r(dz3))
    dz2 = da2 * gelu_grad(cache["z2"])
    da1, dW2, db2 = conv_backward(cache["a1"], p["W2"], dz2, dz_data=r(dz2))
    dz1 = da1 * gelu_grad(cache["z1"])
    _, dW1, db1 = conv_backward(cache["a0"], p["W1"], dz1)
    assert L == cache["a0"].shape[2]
    return flatten(dict(W1=dW1, b1=db1, W2=dW2, b2=db2, W3=dW3, b3=db3, W4=dW4, b4=db4))


def block_delta_E(s, b, B):
    """E(x') - E(x) for flipping block b of one lattice s (L, L): twice the sum
    over bonds crossing the block boundary of s_in * s_out."""
    L = s.shape[0]
    n = L // B
    by, bx = divmod(int(b), n)
    y0, x0 = by * B, bx * B
    inside = lambda y, x: y0 <= y < y0 + B and x0 <= x < x0 + B  # noqa: E731
    d = 0
    for y in range(y0, y0 + B):
        for x in range(x0, x0 + B):
            for dy, dx in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                yy, xx = (y + dy) % L, (x + dx) % L
                if not inside(yy, xx):
                    d += int(s[y, x]) * int(s[yy, xx])
    return 2 * d


def targets(spins, beta, B=8):
    C, L, _ = spins.shape
    n = L // B
    t = np.zeros((C, n * n))
    for c in range(C):
        for b in range(n * n):
            t[c, b] = min(0.0, -beta * block_delta_E(spins[c], b, B))
    return t


def loss_and_grad(theta, spins, beta, B=8, round_act=True):
    logits, cache = forward(theta, spins, B, keep=True, round_act=round_act)
    t = targets(np.asarray(spins), beta, B)
    r = logits - t
    loss = float((r * r).mean())
    g = backward(theta, cache, 2.0 * r / r.size)
    return loss, g


def _seq_sum(values) -> float:
    acc = 0.0
    for v in values:
        acc += float(v)
    return acc


def log_softmax(l):
    """log softmax with the normaliser summed in block order (float64)."""
    l = np.asarray(l, dtype=np.float64)
    m = float(np.max(l))
    return l - (m + math.log(_seq_sum(np.exp(l - m))))


def sample_block(logits, u: int) -> int:
    """Inverse-CDF sample of softmax(logits) with the 32-bit draw u: the first
    block whose cumulative weight exceeds (u / 2^32) * total (float64, sums
    taken in block order)."""
    w = np.exp(np.asarray(logits, dtype=np.float64) - float(np.max(logits)))
    target = (u / 4294967296.0) * _seq_sum(w)
    acc = 0.0
    for b, x in enumerate(w):
        acc += float(x)
        if acc > target:
            return b
    return len(w) - 1


def sample_uniform(n_blocks: int, u: int) -> int:
    return int((u * n_blocks) >> 32)


def accept_threshold(beta, dE, logp_fwd=0.0, logp_rev=0.0) -> int:
    """floor(2^32 min(1, exp(-beta dE + logp_rev - logp_fwd)))."""
    x = -beta * dE + logp_rev - logp_fwd
    if x >= 0.0:
        return 1 << 32
    return int(math.floor(math.ldexp(math.exp(x), 32)))


def block_move(s, logits_fn, beta, B, u_prop: int, u_acc: int):
    """One Metropolis-Hastings block move of one lattice s (L, L) in place.
    logits_fn maps (1, L, L) spins to (1, nb) logits; None proposes blocks
    uniformly.  Returns (block, dE, accepted)."""
    L = s.shape[0]
    nb = (L // B) ** 2
    if logits_fn is None:
        b = sample_uniform(nb, u_prop)
        lf = lr = 0.0
    else:
        l = np.asarray(logits_fn(s[None]))[0]
        b = sample_block(l, u_prop)
        lf = float(log_softmax(l)[b])
    dE = block_delta_E(s, b, B)
    sp = flip_blocks(s[None], [b], B)[0]
    if logits_fn is not None:
        lr = float(log_softmax(np.asarray(logits_fn(sp[None]))[0])[b])
    T = accept_threshold(beta, dE, lf, lr)
    acc = u_acc < T
    if acc:
        s[...] = sp
    return b, dE, acc
