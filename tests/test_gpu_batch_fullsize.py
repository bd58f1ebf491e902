"""The 4096-lattice parallel-tempering batch the benchmark runs (ladders of
64 temperatures in [0.30, 0.60], sides 32..1024 in proportions 8:8:4:2:1:1),
checked ladder by ladder against the oracle after a short run."""
import numpy as np
import pytest
import torch

import oracle
import paper_1906_06297_gb300 as ising
from paper_1906_06297_gb300 import workloads

pytestmark = pytest.mark.gpu


def test_pt_batch_ladders_match_oracle():
    L, S, beta = workloads.pt_batch()
    assert len(L) == 4096 and S == 64
    g = ising.Batch(L, S, beta)
    g.init(ising.ISING_INIT_RANDOM, 1234)
    n, every = 20, 10
    tr = torch.zeros((2, len(L), 2), dtype=torch.int64, device="cuda")
    g.run(n, 1234, 0, every, True, tr)
    g.check()
    trace = tr.cpu().numpy()
    slot, at = g.state_numpy()
    for ladder in (0, 21, 42, 61, 63):  # L = 32, 64, 128, 1024 (first and last)
        lo = ladder * S
        o = oracle.Batch(L[lo:lo + S], S, beta, oracle.MODE_RANDOM, 1234, lattice_base=lo)
        tr_o = o.run(n, 1234, 0, every, True)
        np.testing.assert_array_equal(slot[lo:lo + S], o.slot_of)
        np.testing.assert_array_equal(at[lo:lo + S] - lo, o.lattice_at)
        np.testing.assert_array_equal(trace[:, lo:lo + S], tr_o)
        for i in (0, S // 2, S - 1):
            b, w = g.planes_numpy(lo + i)
            np.testing.assert_array_equal(oracle.from_planes_msc4(int(L[lo + i]), b, w), o.lattice(i))
