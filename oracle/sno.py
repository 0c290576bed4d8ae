"""Summation natural orbitals (SNO) per increment — TEST INFRASTRUCTURE ONLY.

Methods, SNO paragraph: the virtual space of each n-body term is cut down
with summation natural orbitals.  A 1-body term's two electrons are treated
exactly (CISD is exact for two electrons), and the natural orbitals of its
one-body density span its virtual space; for a larger term the one-body
densities of its 1-body terms are summed (a 3-body term i, j, k takes
rho_i + rho_j + rho_k) and that sum's natural orbitals span the virtual
space; natural orbitals whose occupation is below 10^-eta are dropped (the
paper uses eta = 8.5).

Reading on the synthetic chains (the paper's orbitals are not available):
the occupied orbital of body b is its bonding orbital; the virtual space of
the system is every antibonding orbital; the 1-body term of b correlates
b's two electrons in {bonding_b} + every virtual, the other bonding orbitals
frozen (doubly occupied).  The SNO space of X has X's bonding orbitals and
the kept natural orbitals active, the other bonding orbitals as core.

The two-electron problem is solved here in its own formulation, independent
of the Slater–Condon code: a singlet pair function
Psi(1, 2) = sum_pq C_pq phi_p(1) phi_q(2), C symmetric, with
<pq|H|rs> = F_pr delta_qs + delta_pr F_qs + (pr|qs) over the active
orbitals, F = h + sum_core [2 (..|cc) - (.c|c.)], and energy E_core + the
lowest eigenvalue; its spin-summed one-body density is 2 C C^T (trace 2).
All arithmetic float64, dense (numpy); for the small chains of the tests.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

from . import fci


def _eri_full(system) -> np.ndarray:
    """(pq|rs) over all orbitals, (norb,)*4, from the packed supermatrix."""
    return fci._eri_from_packed(system.eri_packed(), list(range(system.norb)))


def _core_terms(h: np.ndarray, eri: np.ndarray, core: Sequence[int]):
    """E_core and the core-dressed one-electron matrix F = h + sum_c [2 (..|cc) - (.c|c.)]."""
    F = h.copy()
    e = 0.0
    for c in core:
        F += 2.0 * eri[:, :, c, c] - eri[:, c, c, :]
        e += 2.0 * h[c, c]
        for d in core:
            e += 2.0 * eri[c, c, d, d] - eri[c, d, d, c]
    return e, F


def two_electron_singlet(h: np.ndarray, eri: np.ndarray, core: Sequence[int], active: Sequence[int]
                         ) -> Tuple[float, np.ndarray]:
    """Lowest singlet of two electrons in `active` with `core` doubly occupied:
    (energy including the core, C over active x active, symmetric, sum C^2 = 1)."""
    ecore, F = _core_terms(h, eri, core)
    a = list(active)
    n = len(a)
    Fa = F[np.ix_(a, a)]
    Va = eri[np.ix_(a, a, a, a)]                 # (pr|qs) -> Va[p, r, q, s]
    # symmetric pair basis: (p, q) with p <= q, vector entries C_pq = C_qp
    pairs = [(p, q) for p in range(n) for q in range(p, n)]
    norm = np.array([1.0 if p == q else np.sqrt(2.0) for p, q in pairs])   # |pq>+|qp> normalisation
    m = len(pairs)
    Hm = np.empty((m, m))
    for i, (p, q) in enumerate(pairs):
        for j, (r, s) in enumerate(pairs):
            # <u_pq|H|u_rs>, u_pq = (|pq> + |qp>) / norm (|pp> itself)
            def el(p_, q_, r_, s_):
                return (Fa[p_, r_] * (q_ == s_) + (p_ == r_) * Fa[q_, s_] + Va[p_, r_, q_, s_])
            v = el(p, q, r, s)
            if r != s:
                v += el(p, q, s, r)
            if p != q:
                v += el(q, p, r, s)
                if r != s:
                    v += el(q, p, s, r)
            Hm[i, j] = v / (norm[i] * norm[j])
    w, y = np.linalg.eigh(Hm)
    C = np.zeros((n, n))
    for i, (p, q) in enumerate(pairs):
        C[p, q] = C[q, p] = y[i, 0] / norm[i]
    return ecore + float(w[0]), C


def one_body_density(system, b: int, h: np.ndarray = None, eri: np.ndarray = None) -> Tuple[List[int], np.ndarray]:
    """(virtual orbital list, spin-summed one-body density of body b's exact
    two-electron (CISD) problem over those virtuals)."""
    h = system.h if h is None else h
    eri = _eri_full(system) if eri is None else eri
    bond = [system.bonding_orbital(x) for x in range(system.nbody)]
    virt = [p for p in range(system.norb) if p not in bond]
    core = [bond[x] for x in range(system.nbody) if x != b]
    active = [bond[b]] + virt
    _, C = two_electron_singlet(h, eri, core, active)
    gamma = 2.0 * C @ C.T
    return virt, gamma[1:, 1:]


def summation_natural_orbitals(system, X: Sequence[int], eta: float, h: np.ndarray = None,
                               eri: np.ndarray = None) -> Tuple[np.ndarray, np.ndarray]:
    """(kept occupations, their natural orbitals as columns over the global
    orbital index) of rho_X = sum_{b in X} rho_b, occupations > 10^-eta."""
    h = system.h if h is None else h
    eri = _eri_full(system) if eri is None else eri
    rho = None
    virt = None
    for b in X:
        virt, g = one_body_density(system, b, h, eri)
        rho = g if rho is None else rho + g
    w, U = np.linalg.eigh(rho)
    order = np.argsort(-w)
    w, U = w[order], U[:, order]
    keep = w > 10.0 ** (-eta)
    T = np.zeros((system.norb, int(keep.sum())))
    T[virt, :] = U[:, keep]
    return w[keep], T


def sno_energy(system, X: Sequence[int], eta: float, h: np.ndarray = None, eri: np.ndarray = None) -> Tuple[float, int]:
    """(E_X in the SNO space of X, number of kept natural orbitals): lowest
    singlet of |X| alpha and |X| beta electrons in X's bonding orbitals plus
    the kept natural orbitals, the other bonding orbitals doubly occupied."""
    h = system.h if h is None else h
    eri = _eri_full(system) if eri is None else eri
    X = sorted(X)
    occ, Tv = summation_natural_orbitals(system, X, eta, h, eri)
    bond = [system.bonding_orbital(x) for x in range(system.nbody)]
    core = [bond[x] for x in range(system.nbody) if x not in X]
    cols = []
    for p in core + [bond[x] for x in X]:
        e = np.zeros(system.norb)
        e[p] = 1.0
        cols.append(e)
    T = np.column_stack(cols + [Tv[:, k] for k in range(Tv.shape[1])])
    ht = T.T @ h @ T
    et = np.einsum("pqrs,pa,qb,rc,sd->abcd", eri, T, T, T, T, optimize=True)
    ncore = len(core)
    n = T.shape[1]
    sub = fci.Subsystem(list(range(ncore)), list(range(ncore, n)), len(X), ht, et)
    H = fci.Hamiltonian(sub)
    e, _ = fci.lowest_singlet_dense(H)
    return e, Tv.shape[1]


def sno_energies(system, max_order: int, eta: float):
    """(E_0, {X: E_X}, {X: eps_X}, E_total) of the expansion with every E_X in
    the SNO space of X (Eqs. 1-5 unchanged; E_c(X) = E_X - E_0)."""
    eri = _eri_full(system)
    e0 = fci.reference_energy(system)
    ex = {X: sno_energy(system, X, eta, system.h, eri)[0] for X in fci.body_subsets(system.nbody, max_order)}
    eps = fci.increments_from_correlation({X: e - e0 for X, e in ex.items()})
    return e0, ex, eps, e0 + sum(eps.values())
