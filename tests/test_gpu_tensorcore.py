"""Tensor-core (tcgen05) BF16 / TF32 sigma and the mixed-precision Davidson.

Exactness test: with integrals and vectors on a coarse dyadic grid every
operand of the contraction is exactly representable in BF16 and every
partial sum in FP32, so the BF16 tensor-core sigma must equal the FP64 sigma
to FP64 rounding.  This pins the operand layouts (swizzle, descriptors,
instruction shape) exactly.  With random inputs the BF16 sigma differs from
the oracle by the BF16 input rounding (unit roundoff u = 2^-8): the test
bounds the relative norm error by 4u and the max error by 16u * max|sigma|.
TF32 (10 explicit mantissa bits, operands rounded with cvt.rna: u = 2^-11)
takes the same tests with its own u; its W streams through two shared-memory
stages, exercised up to npair 253 (n = 22).
"""
import math

import numpy as np
import pytest
import torch

from oracle import fci
from synth import chain_24_uneven, random_ci_vector

import paper_2307_10675_gb300 as ifci

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
U_BF16 = 2.0 ** -8
U_TF32 = 2.0 ** -11


@pytest.fixture(scope="module")
def handle():
    with ifci.Handle(0, 0) as h:
        yield h


def _dyadic_problem(n, seed):
    rng = np.random.default_rng(seed)
    npair = n * (n + 1) // 2
    h1 = rng.integers(-2, 3, size=(n, n)) / 2.0
    h1 = np.triu(h1) + np.triu(h1, 1).T
    V = rng.integers(-2, 3, size=(npair, npair)) / 4.0
    V = np.triu(V) + np.triu(V, 1).T
    return torch.tensor(h1, device=DEV), torch.tensor(V, device=DEV)


@pytest.mark.parametrize("n,m", [(6, 2), (10, 2), (14, 2), (18, 2), (8, 4)])
def test_bf16_sigma_exact_on_dyadic_inputs(handle, n, m):
    h1, V = _dyadic_problem(n, seed=n * 10 + m)
    t = ifci.ifci_build_strings(handle, n, m)
    rng = np.random.default_rng(n)
    c = torch.tensor(rng.integers(-3, 4, size=t.nstr * t.nstr) / 4.0, device=DEV)
    s64 = ifci.ifci_sigma(handle, t, h1, V, c, precision=ifci.IFCI_FP64)
    s16 = ifci.ifci_sigma(handle, t, h1, V, c, precision=ifci.IFCI_BF16)
    torch.cuda.synchronize()
    np.testing.assert_allclose(s16.cpu().numpy(), s64.cpu().numpy(), rtol=0, atol=1e-9)


@pytest.mark.parametrize("n,m", [(6, 2), (10, 2), (14, 2), (18, 2), (8, 4), (21, 2), (22, 2)])
def test_tf32_sigma_exact_on_dyadic_inputs(handle, n, m):
    h1, V = _dyadic_problem(n, seed=n * 10 + m + 5)
    t = ifci.ifci_build_strings(handle, n, m)
    rng = np.random.default_rng(n + 5)
    c = torch.tensor(rng.integers(-3, 4, size=t.nstr * t.nstr) / 4.0, device=DEV)
    s64 = ifci.ifci_sigma(handle, t, h1, V, c, precision=ifci.IFCI_FP64)
    s32 = ifci.ifci_sigma(handle, t, h1, V, c, precision=ifci.IFCI_TF32)
    torch.cuda.synchronize()
    np.testing.assert_allclose(s32.cpu().numpy(), s64.cpu().numpy(), rtol=0, atol=1e-9)


@pytest.mark.parametrize("X", [(0,), (0, 1), (5, 7), (8, 11, 12), (2, 9, 16), "six"])
def test_tf32_sigma_against_oracle(handle, X):
    chain = chain_24_uneven()
    if X == "six":
        X = tuple(b for b, s in enumerate(chain.body_sizes) if s == 6)[:3]
    sysa = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=DEV),
                             torch.tensor(chain.eri_packed(), device=DEV))
    h1, eri, ecore = ifci.ifci_frozen_core(handle, sysa, X)
    t = ifci.ifci_build_strings(handle, h1.shape[0], len(X))
    c = torch.tensor(random_ci_vector(t.nstr, t.nstr, seed=6), device=DEV)
    sig = ifci.ifci_sigma(handle, t, h1, eri, c, precision=ifci.IFCI_TF32)
    torch.cuda.synchronize()
    cn = c.cpu().numpy().reshape(-1)
    got = sig.cpu().numpy().reshape(-1)
    if t.nstr * t.nstr <= 40000:
        ref = fci.Hamiltonian(fci.subsystem(chain, X)).matvec(cn) - ecore * cn
    else:   # CAS(6e,18o): the FP64 path, itself checked against oracle rows
        ref = ifci.ifci_sigma(handle, t, h1, eri, c, precision=ifci.IFCI_FP64).cpu().numpy().reshape(-1)
    err = got - ref
    assert np.linalg.norm(err) <= 4 * U_TF32 * np.linalg.norm(ref)
    assert np.max(np.abs(err)) <= 16 * U_TF32 * np.max(np.abs(ref))


@pytest.mark.parametrize("X", [(0,), (0, 1), (5, 7), (8, 11, 12), (2, 9, 16)])
def test_bf16_sigma_against_oracle(handle, X):
    chain = chain_24_uneven()
    sysa = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=DEV),
                             torch.tensor(chain.eri_packed(), device=DEV))
    h1, eri, ecore = ifci.ifci_frozen_core(handle, sysa, X)
    t = ifci.ifci_build_strings(handle, h1.shape[0], len(X))
    c = torch.tensor(random_ci_vector(t.nstr, t.nstr, seed=4), device=DEV)
    sig = ifci.ifci_sigma(handle, t, h1, eri, c, precision=ifci.IFCI_BF16)
    torch.cuda.synchronize()
    H = fci.Hamiltonian(fci.subsystem(chain, X))
    cn = c.cpu().numpy().reshape(-1)
    ref = H.matvec(cn) - ecore * cn
    got = sig.cpu().numpy().reshape(-1)
    err = got - ref
    assert np.linalg.norm(err) <= 4 * U_BF16 * np.linalg.norm(ref)
    assert np.max(np.abs(err)) <= 16 * U_BF16 * np.max(np.abs(ref))


def test_bf16_sigma_full_size_matches_fp64_path(handle):
    """CAS(6e,18o), 665,856 dets: BF16 tensor-core sigma vs the FP64 path (oracle-checked)."""
    chain = chain_24_uneven()
    X = tuple(b for b, s in enumerate(chain.body_sizes) if s == 6)[:3]
    sysa = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=DEV),
                             torch.tensor(chain.eri_packed(), device=DEV))
    h1, eri, _ = ifci.ifci_frozen_core(handle, sysa, X)
    t = ifci.ifci_build_strings(handle, 18, 3)
    c = torch.tensor(random_ci_vector(816, 816, seed=8), device=DEV)
    s64 = ifci.ifci_sigma(handle, t, h1, eri, c, precision=ifci.IFCI_FP64)
    s16 = ifci.ifci_sigma(handle, t, h1, eri, c, precision=ifci.IFCI_BF16)
    torch.cuda.synchronize()
    err = (s16 - s64).cpu().numpy()
    ref = s64.cpu().numpy()
    assert np.linalg.norm(err) <= 4 * U_BF16 * np.linalg.norm(ref)


# ---------------------------------------------------------------- FP64-accurate tensor-core contraction

@pytest.mark.parametrize("n,m", [(6, 2), (14, 2), (18, 2), (8, 4), (21, 2), (24, 2)])
def test_fp64e_sigma_exact_on_dyadic_inputs(handle, n, m):
    """npair 231 and 300 (n = 21, 24) run in K chunks of 192 pairs whose int64
    partial sums are added into G: still exact."""
    h1, V = _dyadic_problem(n, seed=n * 10 + m + 1)
    t = ifci.ifci_build_strings(handle, n, m)
    rng = np.random.default_rng(n + 1)
    c = torch.tensor(rng.integers(-3, 4, size=t.nstr * t.nstr) / 4.0, device=DEV)
    s64 = ifci.ifci_sigma(handle, t, h1, V, c, precision=ifci.IFCI_FP64)
    s64e = ifci.ifci_sigma(handle, t, h1, V, c, precision=ifci.IFCI_FP64E)
    torch.cuda.synchronize()
    np.testing.assert_allclose(s64e.cpu().numpy(), s64.cpu().numpy(), rtol=0, atol=1e-12)


@pytest.mark.parametrize("X", [(0,), (0, 1), (5, 7), (8, 11, 12), (2, 9, 16), "six"])
def test_fp64e_sigma_matches_fp64(handle, X):
    """D is fixed point at 2^-38 dscale and W is sliced to 2^-40 of one scale
    per problem (max|W|), so one element of G is off by at most about
    npair (2^-38 + 2^-39) max|W| dscale, ~1e-9 of max|W| dscale at npair = 171,
    and by ~sqrt(npair) less in norm.  The test asks for 5e-10 relative in norm
    and 5e-9 of max|sigma| per element."""
    chain = chain_24_uneven()
    if X == "six":
        X = tuple(b for b, s in enumerate(chain.body_sizes) if s == 6)[:3]
    sysa = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=DEV),
                             torch.tensor(chain.eri_packed(), device=DEV))
    h1, eri, _ = ifci.ifci_frozen_core(handle, sysa, X)
    t = ifci.ifci_build_strings(handle, h1.shape[0], len(X))
    c = torch.tensor(random_ci_vector(t.nstr, t.nstr, seed=12), device=DEV)
    s64 = ifci.ifci_sigma(handle, t, h1, eri, c, precision=ifci.IFCI_FP64)
    s64e = ifci.ifci_sigma(handle, t, h1, eri, c, precision=ifci.IFCI_FP64E)
    torch.cuda.synchronize()
    a, b = s64e.cpu().numpy().reshape(-1), s64.cpu().numpy().reshape(-1)
    assert np.linalg.norm(a - b) <= 5e-10 * np.linalg.norm(b)
    assert np.max(np.abs(a - b)) <= 5e-9 * np.max(np.abs(b))


# ---------------------------------------------------------------- spin-flip-symmetric (alpha-only) gathers

def _symmetric(c, nstr):
    m = c.reshape(nstr, nstr)
    return ((m + m.T) / 2).reshape(-1).contiguous()


@pytest.mark.parametrize("prec,atol", [("fp64e", 1e-12), ("bf16", 1e-9), ("tf32", 1e-9)])
@pytest.mark.parametrize("n,m", [(6, 2), (14, 2), (18, 2), (8, 4), (12, 4)])
def test_symmetric_sigma_exact_on_dyadic_inputs(handle, prec, atol, n, m):
    """Alpha-only gather + S + S^T on a symmetric dyadic vector equals the FP64
    sigma of the full gather (tiles of several alpha rows at n = 6, one row
    split in column tiles at n = 18 and 12)."""
    h1, V = _dyadic_problem(n, seed=n * 10 + m + 2)
    t = ifci.ifci_build_strings(handle, n, m)
    rng = np.random.default_rng(n + 2)
    c = torch.tensor(rng.integers(-3, 4, size=t.nstr * t.nstr) / 8.0, device=DEV)
    c = _symmetric(c, t.nstr)          # multiples of 1/16: still exact
    s64 = ifci.ifci_sigma(handle, t, h1, V, c, precision=ifci.IFCI_FP64)
    ss = ifci.ifci_sigma(handle, t, h1, V, c, precision=ifci.PRECISIONS[prec], spin_symmetric=True)
    torch.cuda.synchronize()
    np.testing.assert_allclose(ss.cpu().numpy(), s64.cpu().numpy(), rtol=0, atol=atol)


@pytest.mark.parametrize("n,m", [(21, 2), (24, 2)])
def test_symmetric_fp64e_sigma_exact_beyond_204_pairs(handle, n, m):
    """The alpha-only FP64E path with K chunks (npair 231 and 300)."""
    h1, V = _dyadic_problem(n, seed=n * 10 + m + 3)
    t = ifci.ifci_build_strings(handle, n, m)
    rng = np.random.default_rng(n + 3)
    c = torch.tensor(rng.integers(-3, 4, size=t.nstr * t.nstr) / 8.0, device=DEV)
    c = _symmetric(c, t.nstr)
    s64 = ifci.ifci_sigma(handle, t, h1, V, c, precision=ifci.IFCI_FP64)
    ss = ifci.ifci_sigma(handle, t, h1, V, c, precision=ifci.IFCI_FP64E, spin_symmetric=True)
    torch.cuda.synchronize()
    np.testing.assert_allclose(ss.cpu().numpy(), s64.cpu().numpy(), rtol=0, atol=1e-12)


@pytest.mark.parametrize("X", [(0,), (0, 1), (5, 7), (8, 11, 12), "six"])
def test_symmetric_fp64e_sigma_matches_oracle(handle, X):
    """Same bound as the full-gather FP64E test, against the oracle's H c."""
    chain = chain_24_uneven()
    if X == "six":
        X = tuple(b for b, s in enumerate(chain.body_sizes) if s == 6)[:3]
    sysa = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=DEV),
                             torch.tensor(chain.eri_packed(), device=DEV))
    h1, eri, ecore = ifci.ifci_frozen_core(handle, sysa, X)
    t = ifci.ifci_build_strings(handle, h1.shape[0], len(X))
    c = _symmetric(torch.tensor(random_ci_vector(t.nstr, t.nstr, seed=13), device=DEV), t.nstr)
    s64e = ifci.ifci_sigma(handle, t, h1, eri, c, precision=ifci.IFCI_FP64E, spin_symmetric=True)
    torch.cuda.synchronize()
    cn = c.cpu().numpy()
    if t.nstr * t.nstr <= 40000:
        H = fci.Hamiltonian(fci.subsystem(chain, X))
        ref = H.matvec(cn) - ecore * cn
    else:   # CAS(6e,18o): 64 seeded rows of the oracle
        H = fci.Hamiltonian(fci.subsystem(chain, X))
        rows = np.random.default_rng(3).choice(t.nstr * t.nstr, size=64, replace=False)
        full = ifci.ifci_sigma(handle, t, h1, eri, c, precision=ifci.IFCI_FP64).cpu().numpy()
        ref_rows = H.matvec_rows(cn, rows) - ecore * cn[rows]
        np.testing.assert_allclose(full[rows], ref_rows, rtol=0, atol=1e-12 * np.max(np.abs(full)))
        ref = full
    a = s64e.cpu().numpy()
    assert np.linalg.norm(a - ref) <= 5e-10 * np.linalg.norm(ref)
    assert np.max(np.abs(a - ref)) <= 5e-9 * np.max(np.abs(ref))


@pytest.mark.parametrize("X", [(0, 1), (8, 11, 12)])
def test_symmetric_bf16_sigma_against_oracle(handle, X):
    chain = chain_24_uneven()
    sysa = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=DEV),
                             torch.tensor(chain.eri_packed(), device=DEV))
    h1, eri, ecore = ifci.ifci_frozen_core(handle, sysa, X)
    t = ifci.ifci_build_strings(handle, h1.shape[0], len(X))
    c = _symmetric(torch.tensor(random_ci_vector(t.nstr, t.nstr, seed=14), device=DEV), t.nstr)
    sig = ifci.ifci_sigma(handle, t, h1, eri, c, precision=ifci.IFCI_BF16, spin_symmetric=True)
    torch.cuda.synchronize()
    H = fci.Hamiltonian(fci.subsystem(chain, X))
    cn = c.cpu().numpy()
    ref = H.matvec(cn) - ecore * cn
    err = sig.cpu().numpy() - ref
    assert np.linalg.norm(err) <= 4 * U_BF16 * np.linalg.norm(ref)
    assert np.max(np.abs(err)) <= 16 * U_BF16 * np.max(np.abs(ref))


@pytest.mark.parametrize("prec,hi", [("fp64e", "fp64e"), ("bf16", "fp64e"), ("bf16", "fp64"), ("tf32", "fp64e")])
def test_tensor_core_davidson_reaches_fp64_accuracy(handle, prec, hi):
    chain = chain_24_uneven()
    sysa = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=DEV),
                             torch.tensor(chain.eri_packed(), device=DEV))
    sets = [(0,), (3,), (0, 1), (5, 7), (8, 11, 12)]
    probs = []
    for X in sets:
        h1, eri, ec = ifci.ifci_frozen_core(handle, sysa, X)
        probs.append(ifci.CIProblem(h1.shape[0], len(X), h1, eri, ec))
    e, it, st = ifci.ifci_davidson_batched(handle, probs, ifci.davidson_opts(prec, hi_precision=hi, r_tol=1e-7))
    assert all(s == 0 for s in st)
    for X, ei in zip(sets, e):
        ref = fci.solve_subsystem(chain, X, tol=1e-10).energy
        assert ei == pytest.approx(ref, abs=1e-8), X
