"""4-body spaces at full size: CAS(8e,24o) of the 24-body chain (four of its
6-orbital bodies; 10,626 strings, 112,911,876 determinants, 300 orbital
pairs), the largest term of the chain's n = 4 expansion (Methods, Eqs. 1-5
truncated at four bodies; Table 1 counts the n = 4 terms).

Their FP64-accurate sigma needs K chunks (300 pairs > the 204 whose level
sums stay exact; chunks of 192 pairs add int64 partial sums) and row slabs of
G (300 x 1.1e8 int64 elements do not fit beside the Davidson vectors; each
slab's scatter adds into an int64 accumulator).  Integer sums are exact in
any order, so neither split changes a bit of sigma.

* Row slabs change nothing: Davidson with a budget that splits every
  CAS(6e,18o)-sized space into slabs returns the same energies and iteration
  counts, bit for bit, as the unsplit run.
* sigma of CAS(8e,24o) (FP64E, spin-flip symmetric) on 64 seeded rows against
  the oracle's Slater-Condon rows.
* Davidson on CAS(8e,24o): the returned vector satisfies (H c)_I = E c_I on
  seeded rows of the oracle's H (to the residual tolerance), and E lies below
  the energy of each 3-body subset (nested variational spaces).
"""
import itertools

import numpy as np
import pytest
import torch

from oracle import fci
from synth import chain_24_uneven, random_ci_vector

import paper_2307_10675_gb300 as ifci

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def handle():
    with ifci.Handle(0, 0) as h:
        yield h


def _system(chain):
    return ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=DEV),
                             torch.tensor(chain.eri_packed(), device=DEV))


def _problems(h, chain, sets):
    sysd = _system(chain)
    probs = []
    for X in sets:
        h1, eri, ec = ifci.ifci_frozen_core(h, sysd, X)
        probs.append(ifci.CIProblem(h1.shape[0], len(X), h1, eri, ec))
    return probs


def _six(chain, k):
    return tuple(b for b, s in enumerate(chain.body_sizes) if s == 6)[:k]


def test_row_slabs_leave_davidson_bit_identical(handle):
    chain = chain_24_uneven()
    sets = [(0,), (0, 1), _six(chain, 3), (8, 11, 12), (2, 9, 16), (5, 7)]
    probs = _problems(handle, chain, sets)
    base = dict(r_tol=1e-7, e_tol=1e-11, max_iter=300)
    e0, it0, st0 = ifci.ifci_davidson_batched(handle, probs, ifci.davidson_opts("fp64e", **base))
    # 2^24 G elements per wave: CAS(6e,18o) (171 pairs x 665,856 determinants) runs in 7 row slabs
    e1, it1, st1 = ifci.ifci_davidson_batched(handle, probs, ifci.davidson_opts("fp64e", det_budget=1 << 24, **base))
    assert np.all(st0 == 0) and np.all(st1 == 0)
    assert np.array_equal(it0, it1)
    assert np.array_equal(e0, e1), e1 - e0


def test_sigma_cas_8e_24o_sampled_rows_against_oracle(handle):
    chain = chain_24_uneven()
    X = _six(chain, 4)
    sysd = _system(chain)
    h1, eri, ecore = ifci.ifci_frozen_core(handle, sysd, X)
    t = ifci.ifci_build_strings(handle, 24, 4)
    assert t.nstr == 10626
    c = torch.tensor(random_ci_vector(t.nstr, t.nstr, seed=24, symmetric=True), device=DEV)
    sig = ifci.ifci_sigma(handle, t, h1, eri, c, precision=ifci.IFCI_FP64E, spin_symmetric=True)
    torch.cuda.synchronize()
    H = fci.Hamiltonian(fci.subsystem(chain, X))
    assert H.ndet == 10626 ** 2
    rows = np.unique(np.r_[0, H.ndet - 1, np.random.default_rng(4).integers(0, H.ndet, 62)])
    cn = c.cpu().numpy().reshape(-1)
    ref = H.matvec_rows(cn, rows) - ecore * cn[rows]
    got = sig.cpu().numpy().reshape(-1)[rows]
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - ref)) <= 5e-9 * np.max(np.abs(ref)), np.max(np.abs(got - ref))


def test_davidson_cas_8e_24o_eigenpair_and_nesting(handle):
    chain = chain_24_uneven()
    X = _six(chain, 4)
    subs = list(itertools.combinations(X, 3))
    probs = _problems(handle, chain, [X] + subs)
    ndet = 10626 ** 2
    probs[0].c_out = torch.empty(ndet, dtype=torch.float64, device=DEV)
    r_tol = 1e-6
    e, it, st = ifci.ifci_davidson_batched(handle, probs, ifci.davidson_opts("fp64e", r_tol=r_tol, e_tol=1e-10,
                                                                            max_iter=300))
    torch.cuda.synchronize()
    assert np.all(st == 0)
    assert np.all(e[0] <= e[1:] + 1e-9), (e[0], e[1:])
    c = probs[0].c_out.cpu().numpy()
    assert abs(np.linalg.norm(c) - 1.0) < 1e-10
    H = fci.Hamiltonian(fci.subsystem(chain, X))
    ref_index = int(np.argmax(np.abs(c)))
    rows = np.unique(np.r_[ref_index, np.random.default_rng(5).integers(0, ndet, 31)])
    hc = H.matvec_rows(c, rows)
    # every residual component is bounded by the residual norm
    assert np.max(np.abs(hc - e[0] * c[rows])) <= 2 * r_tol, np.max(np.abs(hc - e[0] * c[rows]))
    # the dominant determinant carries the eigenvalue: E = (Hc)_I / c_I there
    assert abs(hc[list(rows).index(ref_index)] / c[ref_index] - e[0]) <= 4 * r_tol / abs(c[ref_index])
