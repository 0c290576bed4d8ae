"""Seeded synthetic chain Hamiltonians that stand in for the paper's PFAS workloads.

The paper's molecules (TFA, PFBA, PFOA in cc-pVDZ, Results, Table 1) and their
geometries are not available, so every workload here is a chain of "bodies".
A body plays the role of one localized occupied orbital of the iFCI expansion
(Methods, Eq. 1) together with its own virtual orbitals.

Recipe (all draws from ``numpy.random.Generator(PCG64(seed))``, in this order):

1. Body order: if ``permute`` is set, ``rng.permutation(nbody)`` reorders the
   given list of body sizes.
2. Orbitals: body b owns ``size_b`` consecutive orbitals. The first is its
   bonding (reference-occupied) orbital, the rest are antibonding virtuals.
   Orbital p sits at x_p = 1.5 Angstrom * p on a line; d_pq = |x_p - x_q|.
3. One-electron integrals: ``z = rng.normal(size=norb)``;
   h_pp = -1 + 0.3 z_p (bonding) or +0.5 + 0.3 z_p (antibonding);
   h_pq = -0.3 exp(-d_pq / 2) for p != q.
4. Two-electron integrals: ``w = rng.normal(size=(16, npair))`` in pair order;
   B^L_pq = 0.1 w[L, pair(p,q)] exp(-d_pq / 2) for p <= q, mirrored;
   (pq|rs) = sum_L B^L_pq B^L_rs (8-fold symmetric, positive semidefinite as
   an npair x npair matrix).  The 0.1 is read as a standard deviation.

Pair index (interface layout shared by every consumer of these arrays):
pair(p, q) = P (P + 1) / 2 + Q with P = max(p, q), Q = min(p, q).
The packed ERI matrix is ``V[pair(p,q), pair(r,s)] = (pq|rs)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

SPACING_ANGSTROM = 1.5
NAUX = 16


def pair_index(p: int, q: int) -> int:
    """Packed index of the unordered orbital pair {p, q}."""
    P, Q = (p, q) if p >= q else (q, p)
    return P * (P + 1) // 2 + Q


@dataclass
class ChainSystem:
    """A seeded synthetic chain: bodies, integrals and the recipe that made them."""

    body_sizes: List[int]
    seed: int
    h: np.ndarray                 # (norb, norb) float64, symmetric
    bfac: np.ndarray              # (NAUX, npair) float64, B^L in pair order
    name: str = ""
    _eri_packed: Optional[np.ndarray] = field(default=None, repr=False)

    @property
    def nbody(self) -> int:
        return len(self.body_sizes)

    @property
    def norb(self) -> int:
        return int(sum(self.body_sizes))

    @property
    def npair(self) -> int:
        n = self.norb
        return n * (n + 1) // 2

    @property
    def body_offsets(self) -> List[int]:
        off = [0]
        for s in self.body_sizes:
            off.append(off[-1] + s)
        return off

    def body_orbitals(self, b: int) -> List[int]:
        off = self.body_offsets
        return list(range(off[b], off[b + 1]))

    def bonding_orbital(self, b: int) -> int:
        return self.body_offsets[b]

    def eri_packed(self) -> np.ndarray:
        """(npair, npair) float64 matrix V[pair(pq), pair(rs)] = (pq|rs)."""
        if self._eri_packed is None:
            self._eri_packed = self.bfac.T @ self.bfac
        return self._eri_packed

    def eri_sub(self, orbs: Sequence[int]) -> np.ndarray:
        """Dense (n, n, n, n) chemist-notation ERIs restricted to ``orbs`` (in that order)."""
        orbs = list(orbs)
        n = len(orbs)
        idx = np.empty((n, n), dtype=np.int64)
        for a, p in enumerate(orbs):
            for b, q in enumerate(orbs):
                idx[a, b] = pair_index(p, q)
        bsub = self.bfac[:, idx]                      # (L, n, n)
        return np.einsum("lpq,lrs->pqrs", bsub, bsub)

    def with_integrals(self, h: np.ndarray, eri_packed: np.ndarray) -> "ChainSystem":
        """A copy carrying replaced integrals (used for finite differences)."""
        out = ChainSystem(list(self.body_sizes), self.seed, np.array(h, dtype=np.float64),
                          self.bfac, name=self.name + "+perturbed")
        out._eri_packed = np.array(eri_packed, dtype=np.float64)
        return out


def make_chain(body_sizes: Sequence[int], seed: int, permute: bool = False,
               name: str = "") -> ChainSystem:
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = list(int(s) for s in body_sizes)
    if permute:
        perm = rng.permutation(len(sizes))
        sizes = [sizes[i] for i in perm]
    norb = sum(sizes)
    x = SPACING_ANGSTROM * np.arange(norb, dtype=np.float64)
    d = np.abs(x[:, None] - x[None, :])
    bonding = np.zeros(norb, dtype=bool)
    off = 0
    for s in sizes:
        bonding[off] = True
        off += s
    z = rng.normal(size=norb)
    h = -0.3 * np.exp(-d / 2.0)
    diag = np.where(bonding, -1.0, 0.5) + 0.3 * z
    h[np.arange(norb), np.arange(norb)] = diag
    npair = norb * (norb + 1) // 2
    w = rng.normal(size=(NAUX, npair))
    dpair = np.empty(npair)
    for P in range(norb):
        for Q in range(P + 1):
            dpair[P * (P + 1) // 2 + Q] = d[P, Q]
    bfac = 0.1 * w * np.exp(-dpair / 2.0)[None, :]
    return ChainSystem(sizes, seed, h, bfac, name=name)


def chain_4x2(seed: int = 2307) -> ChainSystem:
    """Four bodies of 2 orbitals (8e, 8o): the small plain-FP64 case."""
    return make_chain([2, 2, 2, 2], seed, name="chain-4x2")


def chain_24_uneven(seed: int = 2308) -> ChainSystem:
    """24 bodies of 2-6 orbitals (five each of 2, 3, 5, 6 and four of 4; 96 orbitals)."""
    sizes = [2] * 5 + [3] * 5 + [5] * 5 + [6] * 5 + [4] * 4
    return make_chain(sizes, seed, permute=True, name="chain-24-uneven")


def chain_7x2(seed: int = 2309) -> ChainSystem:
    """Seven bodies of 2 orbitals: one CAS(14e,14o) CI when all bodies are active."""
    return make_chain([2] * 7, seed, name="chain-7x2")


def chain_40_uneven(seed: int = 2310) -> ChainSystem:
    """40 bodies, eight each of sizes 2-6 (160 orbitals)."""
    sizes = [2] * 8 + [3] * 8 + [4] * 8 + [5] * 8 + [6] * 8
    return make_chain(sizes, seed, permute=True, name="chain-40-uneven")


def random_ci_vector(nstr_a: int, nstr_b: int, seed: int = 0,
                     symmetric: bool = False) -> np.ndarray:
    """A seeded unit-norm (nstr_a, nstr_b) float64 array of N(0,1) draws."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = rng.normal(size=(nstr_a, nstr_b))
    if symmetric:
        assert nstr_a == nstr_b
        c = 0.5 * (c + c.T)
    return c / np.linalg.norm(c)
