"""Failure detection without a GPU fault: a bounded device wait that runs out
returns IFCI_ERR_TIMEOUT and leaves the context usable; a Davidson batch cut
short by max_iter reports IFCI_ERR_NOT_CONVERGED per problem and can be
re-run to convergence."""
import numpy as np
import pytest
import torch

from oracle import fci
from synth import chain_4x2, chain_24_uneven, random_ci_vector

import paper_2307_10675_gb300 as ifci
from paper_2307_10675_gb300._capi import IFCI_ERR_NOT_CONVERGED, IFCI_ERR_TIMEOUT, IFCI_OK

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def handle():
    with ifci.Handle(0, 0) as h:
        yield h


def test_bounded_wait_times_out_and_context_survives(handle):
    assert ifci.ifci_wait_selftest(handle, 2_000_000) == IFCI_ERR_TIMEOUT     # ~1 ms at 2 GHz
    assert ifci.ifci_wait_selftest(handle, 0) != IFCI_OK                       # rejected limit
    # the same handle and context still compute correctly
    chain = chain_4x2()
    sysa = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=DEV),
                             torch.tensor(chain.eri_packed(), device=DEV))
    X = (0, 1, 2)
    h1, eri, ecore = ifci.ifci_frozen_core(handle, sysa, X)
    t = ifci.ifci_build_strings(handle, 6, 3)
    c = torch.tensor(random_ci_vector(t.nstr, t.nstr, seed=3), device=DEV)
    s = ifci.ifci_sigma(handle, t, h1, eri, c, precision=ifci.IFCI_FP64E)
    torch.cuda.synchronize()
    H = fci.Hamiltonian(fci.subsystem(chain, X))
    cn = c.cpu().numpy().reshape(-1)
    np.testing.assert_allclose(s.cpu().numpy().reshape(-1), H.matvec(cn) - ecore * cn, rtol=0, atol=1e-9)


def test_not_converged_is_reported_per_problem_and_rerun_converges(handle):
    chain = chain_24_uneven()
    sysa = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=DEV),
                             torch.tensor(chain.eri_packed(), device=DEV))
    probs = []
    for X in [(0,), (5, 7), (8, 11, 12)]:
        h1, eri, ec = ifci.ifci_frozen_core(handle, sysa, X)
        probs.append(ifci.CIProblem(h1.shape[0], len(X), h1, eri, ec))
    e, it, st = ifci.ifci_davidson_batched(handle, probs, ifci.davidson_opts("fp64e", max_iter=3),
                                           allow_unconverged=True)
    assert np.any(st == IFCI_ERR_NOT_CONVERGED)
    assert np.all(np.isfinite(e))
    with pytest.raises(ifci.IfciError):
        ifci.ifci_davidson_batched(handle, probs, ifci.davidson_opts("fp64e", max_iter=3))
    e2, it2, st2 = ifci.ifci_davidson_batched(handle, probs, ifci.davidson_opts("fp64e", max_iter=200))
    assert np.all(st2 == 0)
    # the cut-short energies are variational upper bounds of the converged ones
    assert np.all(e >= e2 - 1e-10)
