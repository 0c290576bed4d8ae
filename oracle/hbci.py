"""Heat-bath configuration interaction per increment — TEST INFRASTRUCTURE ONLY.

Methods, HBCI paragraph: the paper computes the correlation energy of every
increment with HBCI, a selected CI.  The determinants that matter most are
picked for a variational CI; the space is then widened and second-order
Epstein–Nesbet perturbation theory (EN-PT2) adds what the variational space
misses.  One threshold steers each selection: eps1 the variational one,
eps2 the perturbative one (1 mHa and 1 µHa in the paper).

The paper gives no more than that; the steps below are the heat-bath
criterion of the HBCI method it cites, in the order it applies them:

1. S = {reference determinant} (every bonding orbital of X doubly occupied).
2. Variational step: (E_var, c) = lowest eigenpair of H restricted to S, in
   the spin-flip-even sector c(Ia, Ib) = c(Ib, Ia) (the singlet-holding
   sector the FCI solver also works in; S is kept closed under the flip).
3. Selection: every determinant a outside S with max_{i in S} |H_ai c_i| >
   eps1 joins S, with its spin-flip image; back to 2 until none joins (or
   ``max_iter`` rounds).
4. EN-PT2 over the determinants outside S, each term screened by eps2:
   E_2 = sum_{a not in S} (sum_{i in S, |H_ai c_i| > eps2} H_ai c_i)^2 / (E_var - H_aa).
5. E_HBCI = E_var + E_2.

Determinants that no chain of couplings above eps1 joins to the reference
are never selected (for instance a charge-transfer sector between bodies no
integral couples): HBCI's E_var is the lowest state reachable from the
reference, a property of the method.

Everything is dense (numpy, float64) on the oracle's Slater–Condon matrix:
for spaces of a few thousand determinants at most.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from . import fci


@dataclass
class HBCIResult:
    e_var: float             # variational energy in S
    e_pt2: float             # EN-PT2 correction
    e_total: float           # e_var + e_pt2
    nsel: int                # |S|
    rounds: int              # variational steps taken
    selected: np.ndarray     # bool[ndet], S
    vector: np.ndarray       # float64[ndet], c (zero outside S)
    margin1: float = np.inf  # smallest | max_i |H_ai c_i| - eps1 | met in a selection (how
                             # far every decision was from the threshold)


def _flip_even_basis(idx: np.ndarray, flip: np.ndarray) -> np.ndarray:
    """Orthonormal basis (columns) of the flip-even vectors supported on the
    flip-closed determinant set idx (ascending), as rows over idx."""
    pos = {int(K): i for i, K in enumerate(idx)}
    cols = []
    for K in idx:
        F = int(flip[K])
        v = np.zeros(len(idx))
        if K < F:
            v[pos[int(K)]] = v[pos[F]] = np.sqrt(0.5)
            cols.append(v)
        elif K == F:
            v[pos[int(K)]] = 1.0
            cols.append(v)
    return np.array(cols).T


def hbci_dense(H: np.ndarray, flip: np.ndarray, start: int, eps1: float, eps2: float,
               max_iter: int = 100) -> HBCIResult:
    """Steps 1-5 on a dense symmetric H (ndet x ndet) with spin-flip
    permutation ``flip`` (an involution; the identity disables the sector
    restriction) from determinant ``start``."""
    ndet = H.shape[0]
    sel = np.zeros(ndet, dtype=bool)
    sel[start] = sel[flip[start]] = True
    diag = np.diag(H)
    rounds = 0
    margin1 = np.inf
    while True:
        rounds += 1
        idx = np.flatnonzero(sel)
        B = _flip_even_basis(idx, flip)
        w, y = np.linalg.eigh(B.T @ H[np.ix_(idx, idx)] @ B)
        e_var = float(w[0])
        c = np.zeros(ndet)
        c[idx] = B @ y[:, 0]
        if rounds >= max_iter:
            break
        # heat-bath criterion: the largest single contribution |H_ai c_i| over i in S
        contrib = np.abs(H[:, sel] * c[sel][None, :])
        best = contrib.max(axis=1)
        if (~sel).any():
            margin1 = min(margin1, float(np.min(np.abs(best[~sel] - eps1))))
        new = (best > eps1) & ~sel
        if not new.any():
            break
        new_idx = np.flatnonzero(new)
        sel[new_idx] = True
        sel[flip[new_idx]] = True
    out = ~sel
    terms = H[np.ix_(out, sel)] * c[sel][None, :]
    num = np.where(np.abs(terms) > eps2, terms, 0.0).sum(axis=1)
    e_pt2 = float(np.sum(num * num / (e_var - diag[out])))
    return HBCIResult(e_var, e_pt2, e_var + e_pt2, int(sel.sum()), rounds, sel, c, margin1)


def spin_flip_permutation(nstr: int) -> np.ndarray:
    """K = ia * nstr + ib  ->  ib * nstr + ia."""
    K = np.arange(nstr * nstr)
    return (K % nstr) * nstr + K // nstr


def hbci_subsystem(system, X: Sequence[int], eps1: float, eps2: float, max_iter: int = 100,
                   H: Optional[fci.Hamiltonian] = None) -> HBCIResult:
    """HBCI energy of body set X (frozen core, X's orbitals active), from the
    reference determinant of X; energies include the core (as fci.solve_subsystem)."""
    sub = fci.subsystem(system, X)
    if H is None:
        H = fci.Hamiltonian(sub)
    bonding_local = [sub.ncore + sub.active.index(system.bonding_orbital(b)) for b in sorted(X)]
    return hbci_dense(H.dense(), spin_flip_permutation(H.nstr), H.reference_index(bonding_local), eps1, eps2,
                      max_iter)


def hbci_energies(system, max_order: int, eps1: float, eps2: float):
    """(E_0, {X: E_X}, {X: eps_X}, E_total) of the expansion with every E_X
    from HBCI (Eqs. 1-5 unchanged; E_c(X) = E_X - E_0)."""
    e0 = fci.reference_energy(system)
    ex = {X: hbci_subsystem(system, X, eps1, eps2).e_total
          for X in fci.body_subsets(system.nbody, max_order)}
    eps = fci.increments_from_correlation({X: e - e0 for X, e in ex.items()})
    return e0, ex, eps, e0 + sum(eps.values())
