"""Exact blocks over decoupled orbital groups (decouple_tol, on by default).

A body set whose bodies fall into groups that no integral couples has an H
that conserves the alpha and beta electron counts of every group; the solver
then iterates every such block as its own Davidson problem (all blocks of a
space sharing one sigma per iteration) and polishes the lowest with the full
H, so that E_X, the lowest eigenvalue of the set's CI (Methods, definition
of E_c(X)), is found by construction rather than by a search over sectors.

* Sets of the 40-body chain whose lowest singlet is a charge-transfer state
  of decoupled bodies reach the oracle's energy in every precision.
* Turning the decomposition off (decouple_tol = 0) changes nothing where
  there are no decoupled groups (the 24-body chain to 2 bodies).
* Nesting at full size: E_{X u Y} <= E_X for every 3-body set of the
  40-body chain and each of its 2-body subsets, and every 2-body set and its
  1-body subsets (nested variational spaces); a set that missed a lower
  sector found by a subset breaks it.
"""
import itertools
import json
import os

import numpy as np
import pytest
import torch

from synth import chain_24_uneven, chain_40_uneven

import paper_2307_10675_gb300 as ifci

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _system(chain):
    return ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=DEV),
                             torch.tensor(chain.eri_packed(), device=DEV))


def _solve_sets(h, chain, sets, opts):
    sysd = _system(chain)
    probs = []
    for X in sets:
        h1, eri, ec = ifci.ifci_frozen_core(h, sysd, X)
        n = h1.shape[0]
        probs.append(ifci.CIProblem(n, len(X), h1, eri, ec))
    e, it, st = ifci.ifci_davidson_batched(h, probs, opts)
    return e, st


@pytest.mark.parametrize("prec,hi,tol", [("fp64", "fp64", 1e-8), ("fp64e", "fp64e", 1e-8), ("bf16", "fp64e", 1e-6)])
def test_decoupled_sets_reach_the_oracle(prec, hi, tol):
    """Every 2-body set of the 40-body chain whose bodies are more than 40
    orbitals apart (decoupled groups at the default tolerance), plus the
    golden 3-body sample, against the oracle."""
    chain = chain_40_uneven()
    gold2 = json.load(open(os.path.join(GOLDEN, "chain40_pairs_oracle.json")))["energies"]
    gold3 = json.load(open(os.path.join(GOLDEN, "chain40_oracle.json")))["energies"]
    off = chain.body_offsets
    far = [X for X in itertools.combinations(range(40), 2) if off[X[1]] - off[X[0] + 1] > 40]
    sets = far + [tuple(int(v) for v in k.split(",")) for k in gold3 if k.count(",") == 2]
    ref = [gold2[",".join(map(str, X))]["energy"] if len(X) == 2 else gold3[",".join(map(str, X))]["energy"]
           for X in sets]
    opts = ifci.davidson_opts(prec, hi_precision=hi, r_tol=1e-7, e_tol=1e-11, max_iter=300)
    with ifci.Handle(0, 0) as h:
        e, st = _solve_sets(h, chain, sets, opts)
    assert np.all(st == 0)
    bad = [(X, e[i] - r) for i, (X, r) in enumerate(zip(sets, ref)) if abs(e[i] - r) > tol]
    assert not bad, bad


def test_decomposition_off_changes_nothing_without_decoupled_groups():
    chain = chain_24_uneven()
    with ifci.Handle(0, 0) as h:
        sysd = _system(chain)
        a = ifci.ifci_increments(h, sysd, 2, ifci.davidson_opts("fp64e", r_tol=1e-7, e_tol=1e-11))
        b = ifci.ifci_increments(h, sysd, 2, ifci.davidson_opts("fp64e", r_tol=1e-7, e_tol=1e-11,
                                                                decouple_tol=0.0))
    np.testing.assert_allclose(a["e_x"], b["e_x"], rtol=0, atol=1e-9)


def test_c4_order3_nesting_invariant_every_set():
    """All 10,700 energies of the 40-body chain's 3-body expansion (FP64E):
    a body set's space contains each subset's space (the extra bodies'
    bonding orbitals doubly occupied), so its lowest eigenvalue is at most
    the subset's."""
    chain = chain_40_uneven()
    with ifci.Handle(0, 0) as h:
        out = ifci.ifci_increments(h, _system(chain), 3,
                                   ifci.davidson_opts("fp64e", r_tol=1e-7, e_tol=1e-11, max_iter=300))
    assert np.all(out["status"] == 0)
    subs = ifci.body_subsets(40, 3)
    e = {X: out["e_x"][i] for i, X in enumerate(subs)}
    bad = []
    for X in subs:
        for Y in itertools.combinations(X, len(X) - 1):
            if Y and e[X] > e[Y] + 1e-9:
                bad.append((X, Y, e[X] - e[Y]))
    assert not bad, bad[:20]


@pytest.mark.parametrize("prec,hi,tol", [("fp64", "fp64", 1e-8), ("fp64e", "fp64e", 1e-8), ("bf16", "fp64e", 1e-6)])
def test_weakly_coupled_and_cas6e18o_sets_against_the_oracle(prec, hi, tol):
    """Sets whose lowest singlet is a charge-transfer state between weakly
    coupled bodies (couplings 1e-9 .. 1e-6, where iterations started in the
    neutral sector reached different energies) and seeded CAS(6e,18o) sets
    (665,856 determinants), against the oracle's random-start Lanczos
    (tests/golden/chain40_sectors_oracle.json)."""
    chain = chain_40_uneven()
    gold = json.load(open(os.path.join(GOLDEN, "chain40_sectors_oracle.json")))["energies"]
    sets = [tuple(int(v) for v in k.split(",")) for k in gold]
    assert len(sets) >= 18 and sum(gold[k]["ndet"] == 665856 for k in gold) >= 5
    opts = ifci.davidson_opts(prec, hi_precision=hi, r_tol=1e-7, e_tol=1e-11, max_iter=300)
    with ifci.Handle(0, 0) as h:
        e, st = _solve_sets(h, chain, sets, opts)
    assert np.all(st == 0)
    bad = [(X, e[i] - gold[",".join(map(str, X))]["energy"]) for i, X in enumerate(sets)
           if abs(e[i] - gold[",".join(map(str, X))]["energy"]) > tol]
    assert not bad, bad
