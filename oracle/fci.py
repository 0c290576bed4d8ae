"""Oracle FCI per iFCI increment — TEST INFRASTRUCTURE ONLY.

Follows the paper's Methods section ("Incremental Full Configuration
Interaction"):

* Eq. 1: E_c = sum_i eps_i + sum_{i>j} eps_ij + ...  over bodies (occupied
  localized orbitals and, here, their own virtuals).
* Eqs. 2-5: eps_X = E_c(X) - sum over the increments of every non-empty
  proper subset of X.
* E_c(X) is the correlation energy with only the orbitals of X correlated.
  Reading used here: the bonding orbitals of the other bodies stay doubly
  occupied (frozen at the reference) and their virtuals are deleted; the
  CI inside the orbitals of X is exact FCI (lowest singlet).
* E_0 is the energy of the single reference determinant (last paragraph of
  Methods): every body's bonding orbital doubly occupied.

All arithmetic in float64.  Matrix elements come from ``sc_fci.c``
(Slater–Condon on spin-orbital bit strings over the full local orbital set
core + active, so the frozen core enters through the full-space rules).
"""
from __future__ import annotations

import ctypes
import itertools
import math
from dataclasses import dataclass
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import build as _build

_LIB = None
DENSE_MAX = 2500          # dense eigh up to this many determinants, Lanczos above
SINGLET_S2_TOL = 1e-6


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        L.oracle_h_element.restype = ctypes.c_double
        L.oracle_h_element.argtypes = [ctypes.c_int, dp, dp] + [ctypes.c_uint64] * 4
        L.oracle_h_dense.restype = None
        L.oracle_h_dense.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, u64p, u64p, dp]
        L.oracle_matvec.restype = None
        L.oracle_matvec.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, u64p, i32p, dp, dp]
        L.oracle_matvec_rows.restype = None
        L.oracle_matvec_rows.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, u64p, i32p, dp, ctypes.c_int, i64p, dp]
        L.oracle_rdm12.restype = None
        L.oracle_rdm12.argtypes = [ctypes.c_int, ctypes.c_int64, u64p, u64p, dp, dp, dp]
        L.oracle_s_minus_s_plus.restype = ctypes.c_double
        L.oracle_s_minus_s_plus.argtypes = [ctypes.c_int, ctypes.c_int64, u64p, u64p, dp]
        L.oracle_num_threads.restype = ctypes.c_int
        L.oracle_num_threads.argtypes = []
        _LIB = L
    return _LIB


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def num_threads() -> int:
    return int(lib().oracle_num_threads())


# --------------------------------------------------------------------------
# Counting (Results, Table 1)
# --------------------------------------------------------------------------

def n_body_terms(n_occ: int, n: int) -> int:
    """Number of n-body terms over n_occ occupied orbitals (Table 1): the n-subsets."""
    return sum(1 for _ in itertools.combinations(range(n_occ), n)) if n_occ <= 24 else math.comb(n_occ, n)


def fci_determinants(n_elec: int, n_orb: int) -> int:
    """FCI determinant count with M_s = 0 (Table 1): C(n_orb, n_elec/2)^2."""
    return math.comb(n_orb, n_elec // 2) ** 2


def body_subsets(nbody: int, max_order: int) -> List[Tuple[int, ...]]:
    """All body sets of size 1..max_order: by size, then lexicographic."""
    out: List[Tuple[int, ...]] = []
    for k in range(1, max_order + 1):
        out.extend(itertools.combinations(range(nbody), k))
    return out


# --------------------------------------------------------------------------
# Frozen-body subsystem of a chain
# --------------------------------------------------------------------------

@dataclass
class Subsystem:
    """Local orbital set for body set X: core (other bodies' bonding) first, then active."""
    core: List[int]          # global orbital indices, ascending
    active: List[int]        # global orbital indices, ascending
    nelec_spin: int          # active electrons per spin = |X|
    h: np.ndarray            # local (n, n)
    eri: np.ndarray          # local (n, n, n, n)

    @property
    def local(self) -> List[int]:
        return self.core + self.active

    @property
    def ncore(self) -> int:
        return len(self.core)

    @property
    def nact(self) -> int:
        return len(self.active)


def subsystem(system, X: Sequence[int]) -> Subsystem:
    X = sorted(set(X))
    core = sorted(system.bonding_orbital(b) for b in range(system.nbody) if b not in X)
    active = sorted(p for b in X for p in system.body_orbitals(b))
    loc = core + active
    assert len(loc) <= 64, "oracle bit strings hold at most 64 local orbitals"
    h = system.h[np.ix_(loc, loc)].copy()
    eri = _eri_from_packed(system.eri_packed(), loc)
    return Subsystem(core, active, len(X), h, eri)


def _eri_from_packed(V: np.ndarray, loc: Sequence[int]) -> np.ndarray:
    n = len(loc)
    idx = np.empty((n, n), dtype=np.int64)
    for a, p in enumerate(loc):
        for b, q in enumerate(loc):
            P, Q = max(p, q), min(p, q)
            idx[a, b] = P * (P + 1) // 2 + Q
    return V[idx[:, :, None, None], idx[None, None, :, :]].copy()


def active_strings(nact: int, m: int, shift: int = 0) -> np.ndarray:
    """All m-electron occupation masks of nact orbitals, ascending as integers."""
    masks = sorted(sum(1 << (shift + p) for p in occ)
                   for occ in itertools.combinations(range(nact), m))
    return np.array(masks, dtype=np.uint64)


def determinant_list(sub: Subsystem) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(alpha masks, beta masks, active strings) with the core bits set; index = ia*nstr+ib."""
    strings = active_strings(sub.nact, sub.nelec_spin, shift=sub.ncore)
    core = np.uint64((1 << sub.ncore) - 1)
    nstr = len(strings)
    da = np.repeat(strings, nstr) | core
    db = np.tile(strings, nstr) | core
    return da, db, strings


def _rank_table(strings: np.ndarray, ncore: int, nact: int) -> np.ndarray:
    tab = np.full(1 << nact, -1, dtype=np.int32)
    for i, s in enumerate(strings):
        tab[int(s) >> ncore] = i
    return tab


class Hamiltonian:
    """H over the determinant list of a subsystem (dense or matrix-free)."""

    def __init__(self, sub: Subsystem):
        self.sub = sub
        self.n = sub.ncore + sub.nact
        self.h = np.ascontiguousarray(sub.h, dtype=np.float64)
        self.eri = np.ascontiguousarray(sub.eri, dtype=np.float64)
        self.da, self.db, self.strings = determinant_list(sub)
        self.nstr = len(self.strings)
        self.ndet = self.nstr * self.nstr
        self.rank = _rank_table(self.strings, sub.ncore, sub.nact)

    def element(self, I: int, J: int) -> float:
        return lib().oracle_h_element(self.n, _p(self.h, ctypes.c_double), _p(self.eri, ctypes.c_double),
                                      int(self.da[I]), int(self.db[I]), int(self.da[J]), int(self.db[J]))

    def dense(self) -> np.ndarray:
        H = np.empty((self.ndet, self.ndet))
        lib().oracle_h_dense(self.n, _p(self.h, ctypes.c_double), _p(self.eri, ctypes.c_double),
                             self.ndet, _p(self.da, ctypes.c_uint64), _p(self.db, ctypes.c_uint64),
                             _p(H, ctypes.c_double))
        return H

    def matvec(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        y = np.empty_like(x)
        lib().oracle_matvec(self.n, _p(self.h, ctypes.c_double), _p(self.eri, ctypes.c_double),
                            self.sub.ncore, self.sub.nact, self.nstr,
                            _p(self.strings, ctypes.c_uint64), _p(self.rank, ctypes.c_int32),
                            _p(x, ctypes.c_double), _p(y, ctypes.c_double))
        return y

    def matvec_rows(self, x: np.ndarray, rows: Sequence[int]) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        r = np.ascontiguousarray(rows, dtype=np.int64)
        y = np.empty(len(r))
        lib().oracle_matvec_rows(self.n, _p(self.h, ctypes.c_double), _p(self.eri, ctypes.c_double),
                                 self.sub.ncore, self.sub.nact, self.nstr,
                                 _p(self.strings, ctypes.c_uint64), _p(self.rank, ctypes.c_int32),
                                 _p(x, ctypes.c_double), len(r), _p(r, ctypes.c_int64),
                                 _p(y, ctypes.c_double))
        return y

    def reference_index(self, bonding_local: Sequence[int]) -> int:
        m = sum(1 << p for p in bonding_local)
        i = int(self.rank[m >> self.sub.ncore])
        return i * self.nstr + i

    def s_squared(self, c: np.ndarray) -> float:
        """<S^2> = <S- S+> + S_z(S_z+1); S_z = 0 in this space."""
        c = np.ascontiguousarray(c, dtype=np.float64).reshape(-1)
        return float(lib().oracle_s_minus_s_plus(self.n, self.ndet, _p(self.da, ctypes.c_uint64),
                                                 _p(self.db, ctypes.c_uint64), _p(c, ctypes.c_double)))

    def rdm12(self, c: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
        c = np.ascontiguousarray(c, dtype=np.float64).reshape(-1)
        n = self.n
        g1 = np.empty((n, n))
        g2 = np.empty((n, n, n, n))
        lib().oracle_rdm12(n, self.ndet, _p(self.da, ctypes.c_uint64), _p(self.db, ctypes.c_uint64),
                           _p(c, ctypes.c_double), _p(g1, ctypes.c_double), _p(g2, ctypes.c_double))
        return g1, g2


# --------------------------------------------------------------------------
# Eigen-solvers
# --------------------------------------------------------------------------

DEGENERATE_TOL = 1e-8      # eigenvalues closer than this form one eigenspace


def lowest_singlet_dense(H: Hamiltonian) -> Tuple[float, np.ndarray]:
    """Dense eigh; the lowest eigenvalue whose eigenspace holds a singlet.

    S^2 commutes with H, so every eigenspace has a basis of spin eigenstates,
    but eigh returns an arbitrary basis of a degenerate eigenspace (e.g. the
    exactly degenerate singlet and triplet of two unpaired electrons on bodies
    that do not couple): S^2 is diagonalised inside each eigenspace, from its
    matrix elements <v_i|S^2|v_j> (by polarisation of the expectation values),
    and the eigenspace counts as singlet when S^2 has an eigenvalue below
    SINGLET_S2_TOL there."""
    w, v = np.linalg.eigh(H.dense())
    k = 0
    while k < len(w):
        m = k + 1
        while m < len(w) and w[m] - w[k] < DEGENERATE_TOL:
            m += 1
        V = v[:, k:m]
        d = m - k
        S = np.empty((d, d))
        for i in range(d):
            S[i, i] = H.s_squared(V[:, i])
            for j in range(i):
                S[i, j] = S[j, i] = 0.25 * (H.s_squared(V[:, i] + V[:, j]) - H.s_squared(V[:, i] - V[:, j]))
        sw, sv = np.linalg.eigh(S)
        if abs(sw[0]) < SINGLET_S2_TOL:
            c = V @ sv[:, 0]
            return float(w[k]), c / np.linalg.norm(c)
        k = m
    raise RuntimeError("no singlet root found")


def lanczos_lowest(H: Hamiltonian, v0: np.ndarray, tol: float = 1e-9, max_iter: int = 300,
                   project=None) -> Tuple[float, np.ndarray, int]:
    """Lanczos with full reorthogonalisation for the lowest eigenpair.

    Stops when the Ritz residual estimate beta_j |y_j| is below ``tol`` (the
    energy error is then of order tol^2 / gap).  ``project`` (optional) is
    applied to every new Krylov vector, e.g. the spin-flip symmetriser.
    """
    v = v0 / np.linalg.norm(v0)
    V = [v]
    alphas: List[float] = []
    betas: List[float] = []
    theta_prev = None
    for j in range(max_iter):
        w = H.matvec(V[j])
        if project is not None:
            w = project(w)
        a = float(V[j] @ w)
        alphas.append(a)
        w = w - a * V[j] - (betas[-1] * V[j - 1] if j > 0 else 0.0)
        Vm = np.array(V)
        for _ in range(2):
            w = w - Vm.T @ (Vm @ w)
        b = float(np.linalg.norm(w))
        T = np.diag(alphas) + np.diag(betas, 1) + np.diag(betas, -1)
        tw, tv = np.linalg.eigh(T)
        theta, y = float(tw[0]), tv[:, 0]
        res = b * abs(y[-1])
        if res < tol or b < 1e-14 or len(V) >= H.ndet:
            x = Vm.T @ y
            return theta, x / np.linalg.norm(x), j + 1
        theta_prev = theta
        betas.append(b)
        V.append(w / b)
    raise RuntimeError(f"Lanczos did not converge in {max_iter} iterations (last {theta_prev})")


def spin_flip_symmetrize(nstr: int):
    """Projector onto C = C^T (alpha <-> beta exchange even), which holds S = 0, 2, ..."""
    def proj(x):
        C = x.reshape(nstr, nstr)
        return (0.5 * (C + C.T)).reshape(-1)
    return proj


@dataclass
class CIResult:
    energy: float
    vector: np.ndarray
    s2: float
    ndet: int
    method: str
    iterations: int = 0


def random_symmetric_start(nstr: int, seed: int) -> np.ndarray:
    """Seeded N(0,1) vector projected on C = C^T: it overlaps every state of the
    spin-flip-even sector (with probability one), unlike a single determinant,
    which can be orthogonal to a charge-transfer ground state."""
    rng = np.random.Generator(np.random.PCG64(seed))
    C = rng.normal(size=(nstr, nstr))
    return (0.5 * (C + C.T)).reshape(-1)


def solve_subsystem(system, X: Sequence[int], method: str = "auto", tol: float = 1e-9,
                    start: str = "random") -> CIResult:
    """Lowest singlet CI energy E_X of body set X (core frozen, FCI in X's orbitals).

    E_X is the lowest eigenvalue (Methods, definition of E_c(X)); the dense
    path sees every root, the Lanczos path starts from a seeded random vector
    of the singlet-containing sector (``start="reference"`` starts from the
    reference determinant instead, which finds the lowest state only when
    that state overlaps the reference).
    """
    sub = subsystem(system, X)
    H = Hamiltonian(sub)
    if method == "auto":
        method = "dense" if H.ndet <= DENSE_MAX else "lanczos"
    if method == "dense":
        e, c = lowest_singlet_dense(H)
        return CIResult(e, c, H.s_squared(c), H.ndet, "dense")
    if start == "reference":
        bonding_local = [sub.ncore + sub.active.index(system.bonding_orbital(b)) for b in sorted(X)]
        v0 = np.zeros(H.ndet)
        v0[H.reference_index(bonding_local)] = 1.0
    else:
        v0 = random_symmetric_start(H.nstr, seed=1000003 * len(X) + sum(31 ** i * b for i, b in enumerate(sorted(X))))
    e, c, it = lanczos_lowest(H, v0, tol=tol, project=spin_flip_symmetrize(H.nstr))
    return CIResult(e, c, H.s_squared(c), H.ndet, "lanczos", it)


# --------------------------------------------------------------------------
# Reference energy and increments (Methods, Eqs. 1-5)
# --------------------------------------------------------------------------

def reference_energy(system) -> float:
    """E_0: energy of the single determinant with every bonding orbital doubly occupied."""
    bond = [system.bonding_orbital(b) for b in range(system.nbody)]
    h = np.ascontiguousarray(system.h[np.ix_(bond, bond)])
    eri = np.ascontiguousarray(_eri_from_packed(system.eri_packed(), bond))
    m = (1 << len(bond)) - 1
    return float(lib().oracle_h_element(len(bond), _p(h, ctypes.c_double), _p(eri, ctypes.c_double),
                                        m, m, m, m))


def increments_from_correlation(ec: Dict[Tuple[int, ...], float]) -> Dict[Tuple[int, ...], float]:
    """Eqs. 2-5 in general form: eps_X = E_c(X) - sum_{Y proper, non-empty subset of X} eps_Y.

    ``ec`` maps sorted body tuples to E_c(X); every non-empty subset of every
    key must be present.  Processes sets in order of size.
    """
    eps: Dict[Tuple[int, ...], float] = {}
    for X in sorted(ec, key=lambda t: (len(t), t)):
        val = ec[X]
        for k in range(1, len(X)):
            for Y in itertools.combinations(X, k):
                val -= eps[Y]
        eps[X] = val
    return eps


def ifci_energies(system, max_order: int, method: str = "auto", tol: float = 1e-9,
                  subsets: Optional[List[Tuple[int, ...]]] = None, cnb: float = 0.0):
    """E_0, {X: E_X}, {X: eps_X} and E_iFCI = E_0 + sum eps (Eq. 1 truncated at max_order).

    ``cnb`` > 0 applies the connected n-body screening to the sets of three
    or more bodies (Methods, screening paragraph; see ``cnb_connected``):
    a screened set is not solved, has no entry in the E_X map, and its
    increment is 0 in the recursion of Eqs. 2-5 and in the total."""
    e0 = reference_energy(system)
    subs = subsets if subsets is not None else body_subsets(system.nbody, max_order)
    if cnb <= 0.0:
        ex = {X: solve_subsystem(system, X, method, tol).energy for X in subs}
        ec = {X: ex[X] - e0 for X in subs}
        eps = increments_from_correlation(ec)
        total = e0 + sum(eps.values())
        return e0, ex, eps, total
    ex: Dict[Tuple[int, ...], float] = {}
    eps: Dict[Tuple[int, ...], float] = {}
    for k in sorted({len(X) for X in subs}):
        for X in [Y for Y in subs if len(Y) == k]:
            if k >= 3 and not cnb_connected(X, eps, cnb):
                eps[X] = 0.0
                continue
            ex[X] = solve_subsystem(system, X, method, tol).energy
            val = ex[X] - e0
            for j in range(1, k):
                for Y in itertools.combinations(X, j):
                    val -= eps[Y]
            eps[X] = val
    total = e0 + sum(eps.values())
    return e0, ex, eps, total


def cnb_connected(X: Tuple[int, ...], eps: Dict[Tuple[int, ...], float], C: float) -> bool:
    """Connected n-body screening (Methods, screening paragraph: terms with
    n >= 3 are kept by a connectivity argument with threshold C; the exact rule
    is in the paper's Supplementary Information, which is not available).
    Reading used here: the bodies of X are the vertices of a graph whose
    edges are the pairs {a, b} of X with |eps_ab| >= C; X is kept when that
    graph is connected (for three bodies: at least two of the three pairs)."""
    X = tuple(sorted(X))
    seen = {X[0]}
    stack = [X[0]]
    while stack:
        a = stack.pop()
        for b in X:
            if b not in seen and abs(eps[tuple(sorted((a, b)))]) >= C:
                seen.add(b)
                stack.append(b)
    return len(seen) == len(X)


# --------------------------------------------------------------------------
# Gradient (Hellmann–Feynman through the increment expansion)
# --------------------------------------------------------------------------

def expansion_weight(Y: Tuple[int, ...], nbody: int, max_order: int) -> int:
    """w_Y = sum over supersets X of Y with |X| <= max_order of (-1)^(|X|-|Y|).

    E_iFCI = E_0 + sum_{|X|<=n} eps_X = (1 - sum_Y w_Y) E_0 + sum_Y w_Y E_Y.
    """
    others = [b for b in range(nbody) if b not in Y]
    w = 0
    for k in range(0, max_order - len(Y) + 1):
        for _ in itertools.combinations(others, k):
            w += (-1) ** k
    return w


def subsystem_rdm_global(system, X: Sequence[int], c: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Full-space spin-summed gamma (norb^2) and Gamma (norb^4) of the state c of body set X."""
    sub = subsystem(system, X)
    H = Hamiltonian(sub)
    g1l, g2l = H.rdm12(c)
    n = system.norb
    loc = np.array(sub.local)
    g1 = np.zeros((n, n))
    g2 = np.zeros((n, n, n, n))
    g1[np.ix_(loc, loc)] = g1l
    g2[np.ix_(loc, loc, loc, loc)] = g2l
    return g1, g2


def reference_rdm_global(system) -> Tuple[np.ndarray, np.ndarray]:
    """gamma, Gamma of the single reference determinant (brute force over a one-det list)."""
    bond = [system.bonding_orbital(b) for b in range(system.nbody)]
    nb = len(bond)
    m = np.array([(1 << nb) - 1], dtype=np.uint64)
    g1l = np.empty((nb, nb))
    g2l = np.empty((nb, nb, nb, nb))
    one = np.ones(1)
    lib().oracle_rdm12(nb, 1, _p(m, ctypes.c_uint64), _p(m.copy(), ctypes.c_uint64), _p(one, ctypes.c_double),
                       _p(g1l, ctypes.c_double), _p(g2l, ctypes.c_double))
    n = system.norb
    g1 = np.zeros((n, n))
    g2 = np.zeros((n, n, n, n))
    g1[np.ix_(bond, bond)] = g1l
    g2[np.ix_(bond, bond, bond, bond)] = g2l
    return g1, g2


def fold_gamma2_packed(g2: np.ndarray) -> np.ndarray:
    """dE/dV[A,B] = 1/2 sum over ordered (p,q) in A and (r,s) in B of Gamma[p,q,r,s].

    V[pair(pq), pair(rs)] = (pq|rs) is the packed ERI matrix; each packed entry
    is one independent input of H = sum h E + 1/2 sum V[pq,rs] (E_pq E_rs - d_qr E_ps).
    """
    n = g2.shape[0]
    npair = n * (n + 1) // 2
    P = np.empty((n, n), dtype=np.int64)
    for p in range(n):
        for q in range(n):
            a, b = max(p, q), min(p, q)
            P[p, q] = a * (a + 1) // 2 + b
    flat = P.reshape(-1)
    G = 0.5 * g2.reshape(n * n, n * n)
    rows = np.zeros((npair, n * n))
    np.add.at(rows, flat, G)                 # fold (p,q) -> A
    out = np.zeros((npair, npair))
    np.add.at(out.T, flat, rows.T)           # fold (r,s) -> B
    return out


def ifci_gradient(system, max_order: int, method: str = "auto", tol: float = 1e-10):
    """(E_iFCI, dE/dh (norb^2), dE/dV (npair^2)) by Hellmann–Feynman on every E_Y."""
    e0 = reference_energy(system)
    subs = body_subsets(system.nbody, max_order)
    n = system.norb
    dh = np.zeros((n, n))
    dg2 = np.zeros((n, n, n, n))
    wsum = 0
    ex = {}
    for Y in subs:
        r = solve_subsystem(system, Y, method, tol)
        ex[Y] = r.energy
        w = expansion_weight(Y, system.nbody, max_order)
        wsum += w
        if w == 0:
            continue
        g1, g2 = subsystem_rdm_global(system, Y, r.vector)
        dh += w * g1
        dg2 += w * g2
    g1, g2 = reference_rdm_global(system)
    dh += (1 - wsum) * g1
    dg2 += (1 - wsum) * g2
    eps = increments_from_correlation({X: ex[X] - e0 for X in subs})
    total = e0 + sum(eps.values())
    return total, dh, fold_gamma2_packed(dg2)
