"""HBCI per CI space through the C ABI (ifci_hbci_batched; Methods, HBCI
paragraph) against the oracle (oracle/hbci.py).

* Body sets of the 4 x 2 and 24-body chains up to a few thousand
  determinants, at the paper's thresholds (eps1 = 1 mHa, eps2 = 1 µHa) and
  at eps1 = 0.1 mHa: the same selected space (size and number of variational
  steps), E_var to 1e-8 Eh and E_PT2 to 1e-9 Eh.  The GPU's vectors come from
  the FP64E Davidson at r_tol 1e-8 (coefficients good to ~1e-8), so a
  selection decision can only differ where a contribution lies within
  ~1e-8 Eh of eps1; cases whose oracle decisions all lie more than 2e-7 Eh
  from the threshold are compared (the test asserts there are such cases).
* eps1 = 0 on 3-body sets of adjacent bodies of the 24-body chain (tens of
  thousands of determinants, every determinant reachable from the
  reference): E_var equals the FCI energy of the Davidson solver, E_PT2 = 0.
* CAS(6e,18o) at the paper's thresholds: E_FCI <= E_var, a selection far
  smaller than the space, and E_var + E_PT2 closer to E_FCI than E_var.
"""
import numpy as np
import pytest
import torch

from oracle import hbci as ohbci
from synth import chain_4x2, chain_24_uneven

import paper_2307_10675_gb300 as ifci

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def handle():
    with ifci.Handle(0, 0) as h:
        yield h


def _problems(h, chain, sets):
    sysd = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=DEV),
                             torch.tensor(chain.eri_packed(), device=DEV))
    probs = []
    for X in sets:
        h1, eri, ec = ifci.ifci_frozen_core(h, sysd, X)
        probs.append(ifci.CIProblem(h1.shape[0], len(X), h1, eri, ec))
    return probs


CASES = [("4x2", (0,)), ("4x2", (0, 1)), ("4x2", (1, 2, 3)), ("4x2", (0, 1, 2, 3)),
         ("24", (0,)), ("24", (8,)), ("24", (0, 1)), ("24", (5, 7)), ("24", (2, 9)), ("24", (8, 11, 12)),
         ("24", (8, 9, 11)), ("24", (13, 16, 19))]


@pytest.mark.parametrize("eps1", [1e-3, 1e-4])
def test_hbci_matches_oracle(handle, eps1):
    eps2 = 1e-6
    compared = 0
    for which, X in CASES:
        chain = chain_4x2() if which == "4x2" else chain_24_uneven()
        ref = ohbci.hbci_subsystem(chain, X, eps1, eps2)
        if ref.margin1 < 2e-7:
            continue
        probs = _problems(handle, chain, [X])
        out = ifci.ifci_hbci_batched(handle, probs, [ifci.reference_determinant(chain.body_sizes, X)], eps1=eps1,
                                     eps2=eps2, opts=ifci.davidson_opts("fp64e", r_tol=1e-8, e_tol=1e-12,
                                                                         max_iter=300))
        assert out["status"][0] == 0
        assert out["nsel"][0] == ref.nsel, (which, X)
        assert out["rounds"][0] == ref.rounds, (which, X)
        assert out["e_var"][0] == pytest.approx(ref.e_var, abs=1e-8), (which, X)
        assert out["e_pt2"][0] == pytest.approx(ref.e_pt2, abs=1e-9), (which, X)
        compared += 1
    assert compared >= 6


def test_hbci_batch_equals_single_calls(handle):
    """Problems of different sizes and round counts in one call give what each gives alone."""
    chain = chain_24_uneven()
    sets = [(0,), (0, 1), (8, 11, 12), (5, 7)]
    starts = [ifci.reference_determinant(chain.body_sizes, X) for X in sets]
    opts = ifci.davidson_opts("fp64e", r_tol=1e-8, e_tol=1e-12, max_iter=300)
    allr = ifci.ifci_hbci_batched(handle, _problems(handle, chain, sets), starts, opts=opts)
    for i, X in enumerate(sets):
        one = ifci.ifci_hbci_batched(handle, _problems(handle, chain, [X]), [starts[i]], opts=opts)
        assert one["nsel"][0] == allr["nsel"][i]
        assert one["e_var"][0] == pytest.approx(allr["e_var"][i], abs=1e-10)
        assert one["e_pt2"][0] == pytest.approx(allr["e_pt2"][i], abs=1e-12)


@pytest.mark.parametrize("X", [(0, 1, 2), (3, 4, 5)])
def test_eps1_zero_reaches_fci(handle, X):
    chain = chain_24_uneven()
    probs = _problems(handle, chain, [X])
    opts = ifci.davidson_opts("fp64e", r_tol=1e-8, e_tol=1e-12, max_iter=300)
    e_fci, _, st = ifci.ifci_davidson_batched(handle, probs, opts)
    assert st[0] == 0
    out = ifci.ifci_hbci_batched(handle, probs, [ifci.reference_determinant(chain.body_sizes, X)], eps1=0.0,
                                 eps2=0.0, opts=opts)
    assert out["status"][0] == 0
    assert out["e_var"][0] == pytest.approx(e_fci[0], abs=1e-8)
    assert out["e_pt2"][0] == pytest.approx(0.0, abs=1e-12)


def test_cas_6e_18o_at_paper_thresholds(handle):
    chain = chain_24_uneven()
    X = tuple(b for b, s in enumerate(chain.body_sizes) if s == 6)[:3]
    probs = _problems(handle, chain, [X])
    opts = ifci.davidson_opts("fp64e", r_tol=1e-7, e_tol=1e-11, max_iter=300)
    e_fci, _, st = ifci.ifci_davidson_batched(handle, probs, opts)
    out = ifci.ifci_hbci_batched(handle, probs, [ifci.reference_determinant(chain.body_sizes, X)], eps1=1e-3,
                                 eps2=1e-6, opts=opts)
    assert st[0] == 0 and out["status"][0] == 0
    assert out["e_var"][0] >= e_fci[0] - 1e-9
    assert 1 < out["nsel"][0] < 816 ** 2 // 10
    assert out["rounds"][0] >= 2
    assert abs(out["e_hbci"][0] - e_fci[0]) < abs(out["e_var"][0] - e_fci[0])


def test_increments_with_hbci_match_the_oracle_expansion(handle):
    """ifci_increments with every E_X from HBCI (hbci_max_rounds > 0): the 4 x 2
    chain to 4 bodies (15 sets, every selection decision at least 3e-6 Eh
    from eps1) against the oracle's HBCI expansion, set by set and in total."""
    from oracle import fci
    s = chain_4x2()
    e0, ex, eps, total = ohbci.hbci_energies(s, 4, 1e-3, 1e-6)
    sysd = ifci.SystemArrays(s.body_offsets, torch.tensor(s.h, device=DEV), torch.tensor(s.eri_packed(), device=DEV))
    out = ifci.ifci_increments(handle, sysd, 4, ifci.davidson_opts("fp64e", r_tol=1e-8, e_tol=1e-12, max_iter=300,
                                                                    hbci_max_rounds=50))
    assert np.all(out["status"] == 0)
    for i, X in enumerate(fci.body_subsets(4, 4)):
        assert out["e_x"][i] == pytest.approx(ex[X], abs=1e-8), X
        assert out["eps"][i] == pytest.approx(eps[X], abs=1e-8), X
    assert out["e0"] == pytest.approx(e0, abs=1e-12)
    assert out["e_total"] == pytest.approx(total, abs=1e-8)
    with pytest.raises(ifci.IfciError):
        ifci.ifci_rdm_backward(handle, sysd, 4, 1.0, ifci.davidson_opts("fp64e", hbci_max_rounds=50))


def test_hbci_batch_matches_stored_oracle_energies(handle):
    """24 seeded 2-body sets of the 24-body chain in one batched call against
    the oracle's stored HBCI results at the paper's thresholds
    (tests/golden/chain24_hbci_oracle.json, written by
    make_chain24_hbci_golden.py; every selection decision there lies at least
    1e-6 Eh from eps1)."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "chain24_hbci_oracle.json")))
    chain = chain_24_uneven()
    keys = [k for k, g in gold["sets"].items() if g["margin1"] >= 2e-7]
    sets = [tuple(int(v) for v in k.split(",")) for k in keys]
    assert len(sets) >= 20
    out = ifci.ifci_hbci_batched(handle, _problems(handle, chain, sets),
                                 [ifci.reference_determinant(chain.body_sizes, X) for X in sets],
                                 eps1=gold["eps1"], eps2=gold["eps2"],
                                 opts=ifci.davidson_opts("fp64e", r_tol=1e-8, e_tol=1e-12, max_iter=300))
    assert np.all(out["status"] == 0)
    for i, k in enumerate(keys):
        g = gold["sets"][k]
        assert out["nsel"][i] == g["nsel"] and out["rounds"][i] == g["rounds"], k
        assert out["e_var"][i] == pytest.approx(g["e_var"], abs=1e-8), k
        assert out["e_pt2"][i] == pytest.approx(g["e_pt2"], abs=1e-9), k
