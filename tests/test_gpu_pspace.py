"""Single Hamiltonian elements (Slater–Condon on the GPU) and the Davidson start
vector built from them.

* Every element <I|H|J> of small frozen-core spaces equals the oracle's dense
  Hamiltonian (which applies the rules on spin-orbital bit strings with the
  core orbitals occupied, so its diagonal carries E_core).
* Body sets of the 40-body chain whose lowest singlet is hard to reach — two
  near-degenerate pairs and three states not led by the lowest-diagonal
  determinant — reach the oracle's lowest eigenvalue in every precision.
"""
import json
import os

import numpy as np
import pytest
import torch

from oracle import fci
from synth import chain_4x2, chain_24_uneven, chain_40_uneven

import paper_2307_10675_gb300 as ifci

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def handle():
    with ifci.Handle(0, 0) as h:
        yield h


def _small_sets():
    c24 = chain_24_uneven()
    sizes = c24.body_sizes
    tri = next((i, j, k) for i in range(24) for j in range(i + 1, 24) for k in range(j + 1, 24)
               if sizes[i] + sizes[j] + sizes[k] == 8)
    pair = next((i, j) for i in range(24) for j in range(i + 1, 24) if sizes[i] + sizes[j] == 12)
    return [("4x2", (0, 1, 2)), ("4x2", (0, 1, 2, 3)), ("24", (0, 1)), ("24", pair), ("24", tri)]


@pytest.mark.parametrize("which,X", _small_sets())
def test_h_elements_equal_oracle_dense(handle, which, X):
    """Every element of spaces of at most 4,900 determinants (all excitation
    levels, core contributions through h_eff), against the oracle's dense H."""
    chain = chain_4x2() if which == "4x2" else chain_24_uneven()
    sysa = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=DEV),
                             torch.tensor(chain.eri_packed(), device=DEV))
    h1, eri, ecore = ifci.ifci_frozen_core(handle, sysa, X)
    t = ifci.ifci_build_strings(handle, h1.shape[0], len(X))
    nd = t.nstr * t.nstr
    assert nd <= 5000
    ref = fci.Hamiltonian(fci.subsystem(chain, X)).dense()
    I, J = np.meshgrid(np.arange(nd), np.arange(nd), indexing="ij")
    I, J = I.reshape(-1), J.reshape(-1)
    got = ifci.ifci_h_elements(handle, t, h1, eri, torch.tensor(I, device=DEV), torch.tensor(J, device=DEV))
    got = got.cpu().numpy() + ecore * (I == J)
    np.testing.assert_allclose(got, ref[I, J], rtol=0, atol=1e-11)


@pytest.fixture(scope="module")
def hard_sets():
    gold = json.load(open(os.path.join(GOLDEN, "chain40_oracle.json")))
    sets = [(8, 20, 32), (12, 20, 27), (17, 21, 34), (7, 20, 21), (8, 14, 39)]
    return sets, [gold["energies"][",".join(map(str, X))]["energy"] for X in sets]


@pytest.mark.parametrize("prec,hi,tol", [("fp64", "fp64", 1e-8), ("fp64e", "fp64e", 1e-8),
                                         ("bf16", "fp64e", 1e-6)])
def test_hard_lowest_roots_reach_the_oracle(handle, hard_sets, prec, hi, tol):
    sets, ref = hard_sets
    chain = chain_40_uneven()
    sysa = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=DEV),
                             torch.tensor(chain.eri_packed(), device=DEV))
    probs = []
    for X in sets:
        h1, eri, ec = ifci.ifci_frozen_core(handle, sysa, X)
        probs.append(ifci.CIProblem(h1.shape[0], len(X), h1, eri, ec))
    e, it, st = ifci.ifci_davidson_batched(handle, probs, ifci.davidson_opts(prec, hi_precision=hi, r_tol=1e-7,
                                                                            e_tol=1e-11, max_iter=300))
    assert np.all(st == 0)
    np.testing.assert_allclose(e, ref, rtol=0, atol=tol)
