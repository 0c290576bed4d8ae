"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (derived from the arithmetic):
* FP64 sigma: each output is a sum of at most 2*nexc*npair products of O(1)
  numbers, so rounding differences stay below ~1e-13 absolute; 1e-10 is used.
* FP32 sigma: inputs rounded to 2^-24 relative and FP32 accumulation over
  npair terms; bound 5e-5 relative to max|sigma|.
* Energies, FP64 path: 1e-8 Eh (the stated FP64 target); Davidson runs to
  residual 1e-7 so the actual error is ~1e-13.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import fci
from synth import chain_4x2, chain_24_uneven, random_ci_vector

import paper_2307_10675_gb300 as ifci

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def handle():
    with ifci.Handle(0, 0) as h:
        yield h


def _system(chain, on_host=False):
    if on_host:
        return ifci.SystemArrays(chain.body_offsets, chain.h, chain.eri_packed())
    return ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=DEV),
                             torch.tensor(chain.eri_packed(), device=DEV))


# ---------------------------------------------------------------- strings

@pytest.mark.parametrize("n,m", [(2, 1), (4, 2), (6, 3), (8, 4), (12, 2), (14, 7), (18, 3)])
def test_strings_and_excitation_table(handle, n, m):
    t = ifci.ifci_build_strings(handle, n, m)
    torch.cuda.synchronize()
    masks = t.strings.cpu().numpy().astype(np.uint64)
    ref = sorted(sum(1 << p for p in occ) for occ in itertools.combinations(range(n), m))
    assert [int(x) for x in masks] == ref                       # bit-exact
    exc = t.exc.cpu().numpy().reshape(t.nstr, t.nexc)
    rank = {v: i for i, v in enumerate(ref)}
    rows = range(t.nstr) if t.nstr <= 500 else np.random.default_rng(0).choice(t.nstr, 300, replace=False)
    for I in rows:
        mask = ref[I]
        seen = []
        for e in exc[I]:
            e = int(e) & 0xFFFFFFFF
            J, A, neg = e >> 10, (e >> 1) & 511, e & 1
            P = int((math.isqrt(8 * A + 1) - 1) // 2)
            Q = A - P * (P + 1) // 2
            seen.append(A)
            if P == Q:
                assert (mask >> P) & 1 and J == I and not neg
                continue
            # exactly one of P, Q occupied; the electron moves to the other
            src, dst = (Q, P) if (mask >> Q) & 1 else (P, Q)
            assert (mask >> src) & 1 and not (mask >> dst) & 1
            new = mask ^ (1 << src) ^ (1 << dst)
            lo, hi = min(P, Q), max(P, Q)
            between = bin(mask & ((1 << hi) - 1) & ~((1 << (lo + 1)) - 1)).count("1")
            assert J == rank[new] and neg == between % 2
        assert seen == sorted(seen) and len(set(seen)) == len(seen) == t.nexc


# ---------------------------------------------------------------- sigma / hdiag vs oracle

def _oracle_h(chain, X):
    return fci.Hamiltonian(fci.subsystem(chain, X))


SIGMA_CASES = [("4x2", (0, 1, 2, 3)), ("24", (0,)), ("24", (8,)), ("24", (0, 1)), ("24", (5, 7)),
               ("24", (8, 11, 12)), ("24", (2, 9, 16))]


@pytest.mark.parametrize("which,X", SIGMA_CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sigma_matches_oracle_matvec(handle, which, X, precision):
    chain = chain_4x2() if which == "4x2" else chain_24_uneven()
    sysa = _system(chain)
    h1, eri, ecore = ifci.ifci_frozen_core(handle, sysa, X)
    n = h1.shape[0]
    m = len(X)
    t = ifci.ifci_build_strings(handle, n, m)
    c = torch.tensor(random_ci_vector(t.nstr, t.nstr, seed=0), device=DEV)
    sig = ifci.ifci_sigma(handle, t, h1, eri, c, precision=ifci.PRECISIONS[precision])
    hd = ifci.ifci_hdiag(handle, t, h1, eri)
    torch.cuda.synchronize()
    H = _oracle_h(chain, X)
    cn = c.cpu().numpy().reshape(-1)
    ref = H.matvec(cn)
    got = sig.cpu().numpy().reshape(-1) + ecore * cn
    if precision == "fp64":
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10)
    else:
        assert np.max(np.abs(got - ref)) <= 5e-5 * max(1.0, np.max(np.abs(ref - ecore * cn)))
    # diagonal, sampled rows
    rows = np.unique(np.r_[0, H.ndet - 1, np.random.default_rng(1).integers(0, H.ndet, 20)])
    dref = np.array([H.element(int(i), int(i)) for i in rows])
    np.testing.assert_allclose(hd.cpu().numpy()[rows] + ecore, dref, rtol=0, atol=1e-10)


def test_sigma_full_size_cas_6e_18o_sampled(handle):
    """The largest 3-body space of the 24-body chain (three 6-orbital bodies), 665,856 dets."""
    chain = chain_24_uneven()
    six = [b for b, s in enumerate(chain.body_sizes) if s == 6][:3]
    X = tuple(six)
    sysa = _system(chain)
    h1, eri, ecore = ifci.ifci_frozen_core(handle, sysa, X)
    t = ifci.ifci_build_strings(handle, 18, 3)
    assert t.nstr == 816
    c = torch.tensor(random_ci_vector(816, 816, seed=3), device=DEV)
    sig = ifci.ifci_sigma(handle, t, h1, eri, c)
    torch.cuda.synchronize()
    H = _oracle_h(chain, X)
    rows = np.unique(np.r_[0, H.ndet - 1, np.random.default_rng(2).integers(0, H.ndet, 14)])
    cn = c.cpu().numpy().reshape(-1)
    ref = H.matvec_rows(cn, rows)
    got = sig.cpu().numpy().reshape(-1)[rows] + ecore * cn[rows]
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10)


# ---------------------------------------------------------------- Davidson and increments

def test_davidson_batched_matches_oracle(handle):
    chain = chain_24_uneven()
    sysa = _system(chain)
    sets = [(0,), (3,), (0, 1), (5, 7), (8, 11, 12)]
    probs = []
    for X in sets:
        h1, eri, ec = ifci.ifci_frozen_core(handle, sysa, X)
        n = h1.shape[0]
        nstr = math.comb(n, len(X))
        probs.append(ifci.CIProblem(n, len(X), h1, eri, ec,
                                    torch.empty(nstr * nstr, dtype=torch.float64, device=DEV)))
    e, it, st = ifci.ifci_davidson_batched(handle, probs, ifci.davidson_opts("fp64", r_tol=1e-7))
    assert all(s == 0 for s in st)
    for X, p, ei in zip(sets, probs, e):
        r = fci.solve_subsystem(chain, X, tol=1e-10)
        assert ei == pytest.approx(r.energy, abs=1e-8)
        H = _oracle_h(chain, X)
        v = p.c_out.cpu().numpy()
        assert np.linalg.norm(v) == pytest.approx(1.0, abs=1e-10)
        res = H.matvec(v) - ei * v
        assert np.linalg.norm(res) < 1e-6
        C = v.reshape(H.nstr, H.nstr)
        np.testing.assert_allclose(C, C.T, atol=1e-12)         # singlet sector


def test_davidson_empty_batch(handle):
    e, it, st = ifci.ifci_davidson_batched(handle, [])
    assert len(e) == 0


@pytest.mark.parametrize("order", [1, 2, 4])
def test_increments_chain_4x2_match_oracle(handle, order):
    chain = chain_4x2()
    out = ifci.ifci_increments(handle, _system(chain), order, ifci.davidson_opts("fp64", r_tol=1e-7))
    e0, ex, eps, total = fci.ifci_energies(chain, order, tol=1e-10)
    assert out["e0"] == pytest.approx(e0, abs=1e-12)
    subs = ifci.body_subsets(4, order)
    for i, X in enumerate(subs):
        assert out["e_x"][i] == pytest.approx(ex[X], abs=1e-8)
        assert out["eps"][i] == pytest.approx(eps[X], abs=1e-8)
    assert out["e_total"] == pytest.approx(total, abs=1e-8)
    if order == 4:
        full = fci.solve_subsystem(chain, (0, 1, 2, 3), tol=1e-10).energy
        assert out["e_total"] == pytest.approx(full, abs=1e-8)    # full-order identity, 4900 dets


def test_increments_host_buffers_equal_device_buffers(handle):
    chain = chain_4x2()
    a = ifci.ifci_increments(handle, _system(chain), 2)
    b = ifci.ifci_increments(handle, _system(chain, on_host=True), 2)
    np.testing.assert_array_equal(a["eps"], b["eps"])
    assert a["e_total"] == b["e_total"]


def test_chain24_all_increments_fp64_sampled_against_oracle(handle):
    """All 24 + 276 + 2024 body sets of the 24-body chain in one batched FP64
    run; the oracle's stored energies for a seeded sample decide parity."""
    chain = chain_24_uneven()
    gold = json.load(open(os.path.join(GOLDEN, "chain24_oracle.json")))
    out = ifci.ifci_increments(handle, _system(chain), 3, ifci.davidson_opts("fp64", r_tol=1e-7))
    assert np.all(out["status"] == 0)
    assert out["e0"] == pytest.approx(gold["e0"], abs=1e-11)
    subs = ifci.body_subsets(24, 3)
    index = {X: i for i, X in enumerate(subs)}
    for key, rec in gold["energies"].items():
        X = tuple(int(v) for v in key.split(","))
        assert out["e_x"][index[X]] == pytest.approx(rec["energy"], abs=1e-8), X
    # the increments are the Moebius inversion of the returned energies (Eqs. 2-5)
    ec = {X: out["e_x"][i] - out["e0"] for i, X in enumerate(subs)}
    eps = fci.increments_from_correlation(ec)
    got = out["eps"]
    np.testing.assert_allclose([eps[X] for X in subs], got, rtol=0, atol=1e-11)
    assert out["e_total"] == pytest.approx(out["e0"] + sum(got), abs=1e-10)


# ---------------------------------------------------------------- argument errors

def test_invalid_arguments_are_rejected(handle):
    chain = chain_4x2()
    sysa = _system(chain)
    with pytest.raises(ifci.IfciError):
        ifci.ifci_frozen_core(handle, sysa, [1, 1])
    with pytest.raises(ifci.IfciError):
        ifci.ifci_increments(handle, sysa, 5)
    with pytest.raises(ifci.IfciError):
        ifci.ifci_build_strings(handle, 32, 2)
