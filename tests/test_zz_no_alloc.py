"""The allocation-free batched entry point gives the same results as the
workspace-based one.

ising_batch_run_noalloc serves callers that may not allocate device memory
themselves (for example code running under another framework's memory
manager, or a latency-bound loop where an allocation could synchronise the
device): its scratch lives in a fixed array inside the library.  Here the
caller's planes and slot state are copies of a normally created batch, and
two calls in a row must leave planes, slots and traces identical to two
ising_batch_run calls with the same arguments.  The file sorts last so that
a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import paper_1906_06297_gb300 as ising

pytestmark = pytest.mark.gpu

L = [32] * 4 + [64] * 4 + [96] * 2 + [128] * 2
S = 2
BETA = [0.400, 0.403]


def test_noalloc_matches_batch_run_on_two_calls_in_a_row():
    ising.build()
    ref = ising.Batch(L, S, BETA)
    ref.init(ising.ISING_INIT_RANDOM, 7)
    torch.cuda.synchronize()
    words = int(ref.word_off[-1])
    # the caller's own buffers, holding the same initial state
    black = ref.ws[ref._black_off:ref._black_off + 8 * words].clone()
    white = ref.ws[ref._white_off:ref._white_off + 8 * words].clone()
    slot = ref.ws[ref._slot_off:ref._slot_off + 4 * len(L)].clone()
    at = ref.ws[ref._at_off:ref._at_off + 4 * len(L)].clone()
    offset = 0
    for n_sweeps in (13, 9):
        n_ev = ref.n_events(n_sweeps, offset, 4)
        tr_ref = torch.zeros((n_ev, len(L), 2), dtype=torch.int64, device="cuda")
        tr_na = torch.zeros_like(tr_ref)
        ref.run(n_sweeps, 7, offset, 4, True, tr_ref)
        ref.check()
        ising.ising_batch_run_noalloc(L, S, BETA, black, white, slot, at, n_sweeps, 7, offset, 4, True, tr_na)
        torch.cuda.synchronize()
        assert torch.equal(black, ref.ws[ref._black_off:ref._black_off + 8 * words])
        assert torch.equal(white, ref.ws[ref._white_off:ref._white_off + 8 * words])
        assert torch.equal(slot, ref.ws[ref._slot_off:ref._slot_off + 4 * len(L)])
        assert torch.equal(at, ref.ws[ref._at_off:ref._at_off + 4 * len(L)])
        np.testing.assert_array_equal(tr_na.cpu().numpy(), tr_ref.cpu().numpy())
        offset += n_sweeps
    assert not np.array_equal(ref.state_numpy()[0], np.arange(len(L)) % S)  # exchanges happened


def _caller_buffers(ref):
    words = int(ref.word_off[-1])
    black = ref.ws[ref._black_off:ref._black_off + 8 * words].clone()
    white = ref.ws[ref._white_off:ref._white_off + 8 * words].clone()
    slot = ref.ws[ref._slot_off:ref._slot_off + 4 * len(L)].clone()
    at = ref.ws[ref._at_off:ref._at_off + 4 * len(L)].clone()
    return black, white, slot, at


def test_noalloc_refuses_bad_caller_buffers_before_any_launch():
    """The caller's slot state and planes are checked on the host first: a
    slot outside the ladder, a slot array that is not the inverse of
    lattice_at, a misaligned plane and a tiny beta are each ISING_EINVAL, and
    the planes are left untouched."""
    ising.build()
    ref = ising.Batch(L, S, BETA)
    ref.init(ising.ISING_INIT_RANDOM, 3)
    torch.cuda.synchronize()
    black, white, slot, at = _caller_buffers(ref)
    black0 = black.clone()

    def refused(b, w, s_, a, beta=BETA):
        with pytest.raises(ising.IsingError) as e:
            ising.ising_batch_run_noalloc(L, S, beta, b, w, s_, a, 3, 7, 0, 0, False, None)
        assert e.value.status == ising.ISING_EINVAL

    bad = slot.view(torch.int32).clone()
    bad[5] = S  # a slot outside [0, S)
    refused(black, white, bad.view(torch.uint8), at)
    bad = slot.view(torch.int32).clone()
    bad[0], bad[1] = 0, 0  # two lattices of ladder 0 in one slot
    refused(black, white, bad.view(torch.uint8), at)
    bad = at.view(torch.int32).clone()
    bad[2] = 0  # ladder 1 pointing at a lattice of ladder 0
    refused(black, white, slot, bad.view(torch.uint8))
    wide = torch.zeros(black.numel() + 16, dtype=torch.uint8, device="cuda")
    refused(wide[8:8 + black.numel()], white, slot, at)  # plane 8 bytes off a 16-byte boundary
    refused(black, white, slot, at, beta=[1e-18, 0.4])
    torch.cuda.synchronize()
    assert torch.equal(black, black0)
