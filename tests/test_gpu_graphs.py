"""Davidson iterations captured into CUDA graphs (graph_iters > 0) give the
same energies, iteration counts and statuses as eager launches, bit for bit:
every kernel is deterministic and a problem that stops inside a block makes
the rest of the block a no-op for it."""
import numpy as np
import pytest
import torch

from synth import chain_24_uneven

import paper_2307_10675_gb300 as ifci

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.mark.parametrize("prec,hi", [("fp64e", "fp64e"), ("bf16", "fp64e"), ("fp64", "fp64")])
def test_graph_replay_equals_eager(prec, hi):
    chain = chain_24_uneven()
    sysa = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=DEV),
                             torch.tensor(chain.eri_packed(), device=DEV))
    with ifci.Handle(0, 0) as h:
        probs = []
        for X in [(0,), (3,), (0, 1), (5, 7), (8, 11, 12), (2, 9, 16)]:
            h1, eri, ec = ifci.ifci_frozen_core(h, sysa, X)
            probs.append(ifci.CIProblem(h1.shape[0], len(X), h1, eri, ec))
        e0, it0, st0 = ifci.ifci_davidson_batched(h, probs, ifci.davidson_opts(prec, hi_precision=hi, r_tol=1e-7))
        l0 = h.launches()
        e1, it1, st1 = ifci.ifci_davidson_batched(h, probs, ifci.davidson_opts(prec, hi_precision=hi, r_tol=1e-7,
                                                                             graph_iters=4))
        assert h.launches() > l0           # replayed launches are counted
    assert np.all(st0 == 0) and np.all(st1 == 0)
    np.testing.assert_array_equal(it0, it1)
    np.testing.assert_array_equal(e0, e1)


def test_graph_mode_increments_equal_eager():
    chain = chain_24_uneven()
    sysa = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=DEV),
                             torch.tensor(chain.eri_packed(), device=DEV))
    with ifci.Handle(0, 0) as h:
        a = ifci.ifci_increments(h, sysa, 2, ifci.davidson_opts("fp64e"))
        b = ifci.ifci_increments(h, sysa, 2, ifci.davidson_opts("fp64e", graph_iters=8))
    np.testing.assert_array_equal(a["e_x"], b["e_x"])
    assert a["e_total"] == b["e_total"]
