"""Pins of the CPU oracle against things other than itself.

Each test fixes the oracle to a closed form, a brute-force construction that
shares none of its code, an invariant, or a number printed in the paper.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fci
from synth import chain_4x2, chain_24_uneven, make_chain, pair_index

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Table 1

def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_counts.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, ne, no, dets, *terms = line.split()
            rows.append((name, int(ne), int(no), float(dets), [int(t) for t in terms]))
    return rows


@pytest.mark.parametrize("row", _table1(), ids=lambda r: r[0])
def test_table1_term_and_determinant_counts(row):
    """Results, Table 1: n-body term counts over N_occ = electrons/2 orbitals; FCI dets."""
    name, ne, no, dets, terms = row
    nocc = ne // 2
    for n, t in enumerate(terms, start=1):
        assert fci.n_body_terms(nocc, n) == t
    got = fci.fci_determinants(ne, no)
    mant, exp = f"{got:.1e}".split("e")
    assert float(f"{mant}e{exp}") == pytest.approx(dets, rel=1e-12)


def test_body_subset_enumeration_counts_and_order():
    subs = fci.body_subsets(24, 3)
    assert len(subs) == 24 + 276 + 2024
    assert subs[:3] == [(0,), (1,), (2,)]
    assert subs[24] == (0, 1) and subs[-1] == (21, 22, 23)
    assert len(set(subs)) == len(subs)


# ---------------------------------------------------------------- Fock-space brute force

def _annihilator(nmodes, j):
    """a_j on the 2^nmodes Fock space; basis state k has mode i occupied iff bit i of k."""
    dim = 1 << nmodes
    rows, cols, vals = [], [], []
    for k in range(dim):
        if (k >> j) & 1:
            sign = -1.0 if bin(k & ((1 << j) - 1)).count("1") % 2 else 1.0
            rows.append(k ^ (1 << j))
            cols.append(k)
            vals.append(sign)
    return sp.csr_matrix((vals, (rows, cols)), shape=(dim, dim))


def _fock_hamiltonian(h, eri):
    """H = sum h_pq a+_ps a_qs + 1/2 sum (pq|rs) a+_ps a+_rt a_st a_qs as explicit matrices.

    Mode order: alpha orbitals 0..n-1, then beta orbitals n..2n-1.
    """
    n = h.shape[0]
    nm = 2 * n
    a = [_annihilator(nm, j) for j in range(nm)]
    ad = [x.T.tocsr() for x in a]
    H = sp.csr_matrix((1 << nm, 1 << nm))
    for s in range(2):
        for p in range(n):
            for q in range(n):
                if h[p, q] != 0.0:
                    H = H + h[p, q] * (ad[p + s * n] @ a[q + s * n])
    for s in range(2):
        for t in range(2):
            for p in range(n):
                for q in range(n):
                    left = ad[p + s * n]
                    right = a[q + s * n]
                    for r in range(n):
                        for ss in range(n):
                            v = eri[p, q, r, ss]
                            if v != 0.0:
                                H = H + 0.5 * v * (left @ ad[r + t * n] @ a[ss + t * n] @ right)
    return H.toarray()


def _random_integrals(n, seed):
    rng = np.random.default_rng(seed)
    h = rng.normal(size=(n, n))
    h = 0.5 * (h + h.T)
    B = rng.normal(size=(5, n, n))
    B = 0.5 * (B + B.transpose(0, 2, 1))
    eri = np.einsum("lpq,lrs->pqrs", B, B)
    return h, eri


@pytest.mark.parametrize("ncore,nact,m", [(0, 3, 1), (1, 3, 2), (2, 2, 1), (0, 4, 2)])
def test_slater_condon_matches_fock_space(ncore, nact, m):
    """Every Slater–Condon element equals the second-quantized H built from explicit matrices."""
    n = ncore + nact
    h, eri = _random_integrals(n, seed=10 * n + m)
    sub = fci.Subsystem(list(range(ncore)), list(range(ncore, n)), m, h, eri)
    H = fci.Hamiltonian(sub)
    Hsc = H.dense()
    F = _fock_hamiltonian(h, eri)
    idx = [int(a) | (int(b) << n) for a, b in zip(H.da, H.db)]
    Hfock = F[np.ix_(idx, idx)]
    np.testing.assert_allclose(Hsc, Hfock, atol=1e-12, rtol=0)
    # the matrix-free matvec is the same operator
    x = np.random.default_rng(1).normal(size=H.ndet)
    np.testing.assert_allclose(H.matvec(x), Hfock @ x, atol=1e-11, rtol=0)
    rows = [0, H.ndet // 2, H.ndet - 1]
    np.testing.assert_allclose(H.matvec_rows(x, rows), (Hfock @ x)[rows], atol=1e-11, rtol=0)


# ---------------------------------------------------------------- closed forms

def test_h2_minimal_basis_closed_form():
    """2 orbitals (g, u), 2 electrons: singlet 2x2 CI [[E_g, K], [K, E_u]]."""
    hgg, huu, Jgg, Juu, Jgu, K = -1.25, -0.47, 0.67, 0.70, 0.66, 0.18
    h = np.diag([hgg, huu])
    eri = np.zeros((2, 2, 2, 2))
    eri[0, 0, 0, 0] = Jgg
    eri[1, 1, 1, 1] = Juu
    eri[0, 0, 1, 1] = eri[1, 1, 0, 0] = Jgu
    for p, q, r, s in itertools.permutations([0, 1, 0, 1]):
        if p != q and r != s:
            eri[p, q, r, s] = K
    sub = fci.Subsystem([], [0, 1], 1, h, eri)
    e, c = fci.lowest_singlet_dense(fci.Hamiltonian(sub))
    Eg, Eu = 2 * hgg + Jgg, 2 * huu + Juu
    exact = 0.5 * (Eg + Eu) - math.sqrt(0.25 * (Eg - Eu) ** 2 + K ** 2)
    assert e == pytest.approx(exact, abs=1e-13)
    w = np.linalg.eigvalsh(fci.Hamiltonian(sub).dense())
    # open-shell singlet and triplet: h_gg + h_uu + J_gu +/- K
    for val in (hgg + huu + Jgu + K, hgg + huu + Jgu - K, 0.5 * (Eg + Eu) + math.sqrt(0.25 * (Eg - Eu) ** 2 + K ** 2)):
        assert np.min(np.abs(w - val)) < 1e-12


def _h2_eigenpairs():
    """The 4 x 4 M_s = 0 CI of the H2-like model above: eigenpairs of the dense H."""
    hgg, huu, Jgg, Juu, Jgu, K = -1.25, -0.47, 0.67, 0.70, 0.66, 0.18
    h = np.diag([hgg, huu])
    eri = np.zeros((2, 2, 2, 2))
    eri[0, 0, 0, 0] = Jgg
    eri[1, 1, 1, 1] = Juu
    eri[0, 0, 1, 1] = eri[1, 1, 0, 0] = Jgu
    for p, q, r, s in itertools.permutations([0, 1, 0, 1]):
        if p != q and r != s:
            eri[p, q, r, s] = K
    H = fci.Hamiltonian(fci.Subsystem([], [0, 1], 1, h, eri))
    w, v = np.linalg.eigh(H.dense())
    return H, w, v, (hgg, huu, Jgu, K)


def test_s_squared_h2_triplet_and_open_shell_singlet():
    """<S^2> of the H2 eigenvectors: the level h_gg + h_uu + J_gu - K is the
    M_s = 0 component of the triplet (S(S+1) = 2); the open-shell level
    h_gg + h_uu + J_gu + K and both closed-shell mixtures are singlets (0).
    A phase error in S- S+ (or an S^2 that returns 0 for every vector) fails
    the triplet value."""
    H, w, v, (hgg, huu, Jgu, K) = _h2_eigenpairs()
    trip = int(np.argmin(np.abs(w - (hgg + huu + Jgu - K))))
    sing = int(np.argmin(np.abs(w - (hgg + huu + Jgu + K))))
    assert abs(w[trip] - (hgg + huu + Jgu - K)) < 1e-12
    assert H.s_squared(v[:, trip]) == pytest.approx(2.0, abs=1e-12)
    assert H.s_squared(v[:, sing]) == pytest.approx(0.0, abs=1e-12)
    for k in range(4):
        if k not in (trip, sing):
            assert H.s_squared(v[:, k]) == pytest.approx(0.0, abs=1e-12)
    # the triplet is spin-flip odd (C = -C^T), the singlets even (C = C^T)
    C = v[:, trip].reshape(2, 2)
    np.testing.assert_allclose(C, -C.T, atol=1e-12)


def _fock_s_squared(n):
    """S^2 = S- S+ + S_z (S_z + 1) from explicit Jordan–Wigner matrices on the
    2^(2n) Fock space (alpha modes 0..n-1, beta modes n..2n-1), with
    S+ = sum_p a+_{p alpha} a_{p beta} and S_z = (N_alpha - N_beta) / 2."""
    nm = 2 * n
    a = [_annihilator(nm, j) for j in range(nm)]
    ad = [x.T.tocsr() for x in a]
    dim = 1 << nm
    Sp = sp.csr_matrix((dim, dim))
    Sz = sp.csr_matrix((dim, dim))
    for p in range(n):
        Sp = Sp + ad[p] @ a[p + n]
        Sz = Sz + 0.5 * (ad[p] @ a[p] - ad[p + n] @ a[p + n])
    S2 = Sp.T @ Sp + Sz @ Sz + Sz
    return S2.toarray()


@pytest.mark.parametrize("ncore,nact,m", [(0, 3, 1), (1, 3, 2), (2, 2, 1), (0, 4, 2)])
def test_s_squared_matches_fock_space_operator(ncore, nact, m):
    """The oracle's <c|S^2|c> equals c^T S^2 c with S^2 built from explicit
    fermion matrices (independent of the oracle's string code), for random
    vectors c of the CI space, core orbitals included: a quadratic form that
    agrees on random vectors is the same form.  Its polarisation
    <u|S^2|v> = (<u+v|S^2|u+v> - <u-v|S^2|u-v>) / 4, used by the dense
    solver inside degenerate eigenspaces, then agrees too."""
    n = ncore + nact
    h, eri = _random_integrals(n, seed=7 * n + m)
    H = fci.Hamiltonian(fci.Subsystem(list(range(ncore)), list(range(ncore, n)), m, h, eri))
    S2 = _fock_s_squared(n)
    idx = [int(x) | (int(y) << n) for x, y in zip(H.da, H.db)]
    S2sub = S2[np.ix_(idx, idx)]
    # the CI space is closed under S^2 (no weight leaks out of it)
    assert np.abs(S2[:, idx]).sum() == pytest.approx(np.abs(S2sub).sum(), abs=1e-12)
    rng = np.random.default_rng(100 + n)
    for _ in range(3):
        c = rng.normal(size=H.ndet)
        u = rng.normal(size=H.ndet)
        assert H.s_squared(c) == pytest.approx(c @ S2sub @ c, abs=1e-10)
        pol = 0.25 * (H.s_squared(c + u) - H.s_squared(c - u))
        assert pol == pytest.approx(u @ S2sub @ c, abs=1e-10)


def test_degenerate_eigenspace_spin_matches_fock_space():
    """Two bodies with no coupling that moves charge between them and one
    unpaired electron on each (body 0: bonding and antibonding orbitals
    degenerate in h, no pair hopping): the lowest levels form a degenerate
    singlet/triplet space.  Inside each degenerate eigenspace the matrix
    <v_i|S^2|v_j> from the oracle equals the Fock-space S^2 projected on it,
    and the dense solver's pick has S^2 = 0."""
    n = 4
    h = np.diag([-1.0, -1.0, -0.2, 0.9])
    eri = np.zeros((n, n, n, n))
    body = [0, 0, 1, 1]
    for p, q, r, s in itertools.product(range(n), repeat=4):
        if p == q and r == s:
            eri[p, q, r, s] = 0.5 if body[p] == body[r] else 0.1
    for p in range(n):                       # on-site exchange of body 1 only
        for q in range(n):
            if p != q and body[p] == body[q] == 1:
                eri[p, q, q, p] = eri[p, q, p, q] = 0.05
    H = fci.Hamiltonian(fci.Subsystem([], list(range(n)), 2, h, eri))
    w, v = np.linalg.eigh(H.dense())
    S2 = _fock_s_squared(n)
    idx = [int(x) | (int(y) << n) for x, y in zip(H.da, H.db)]
    S2sub = S2[np.ix_(idx, idx)]
    k = 0
    checked = 0
    while k < len(w):
        m = k + 1
        while m < len(w) and w[m] - w[k] < fci.DEGENERATE_TOL:
            m += 1
        V = v[:, k:m]
        for i in range(m - k):
            for j in range(m - k):
                pol = 0.25 * (H.s_squared(V[:, i] + V[:, j]) - H.s_squared(V[:, i] - V[:, j]))
                assert pol == pytest.approx(V[:, i] @ S2sub @ V[:, j], abs=1e-10)
        checked += (m - k) > 1
        k = m
    assert checked >= 1                      # at least one degenerate level was examined
    e, c = fci.lowest_singlet_dense(H)
    assert c @ S2sub @ c == pytest.approx(0.0, abs=1e-10)


@pytest.mark.parametrize("t,U", [(1.0, 4.0), (0.3, 0.1), (1.0, 0.0)])
def test_two_site_hubbard_closed_form(t, U):
    h = np.array([[0.0, -t], [-t, 0.0]])
    eri = np.zeros((2, 2, 2, 2))
    eri[0, 0, 0, 0] = eri[1, 1, 1, 1] = U
    sub = fci.Subsystem([], [0, 1], 1, h, eri)
    e, _ = fci.lowest_singlet_dense(fci.Hamiltonian(sub))
    assert e == pytest.approx(0.5 * (U - math.sqrt(U * U + 16 * t * t)), abs=1e-13)


def test_reference_energy_closed_form():
    """E_0 = sum_c 2 h_cc + sum_{c,d} [2 (cc|dd) - (cd|dc)] over bonding orbitals."""
    s = chain_4x2()
    bond = [s.bonding_orbital(b) for b in range(s.nbody)]
    V = s.eri_packed()
    e = sum(2 * s.h[c, c] for c in bond)
    for c in bond:
        for d in bond:
            e += 2 * V[pair_index(c, c), pair_index(d, d)] - V[pair_index(c, d), pair_index(d, c)]
    assert fci.reference_energy(s) == pytest.approx(e, abs=1e-12)


# ---------------------------------------------------------------- solvers and invariants

def test_dense_and_lanczos_agree():
    s = chain_24_uneven()
    for X in [(0, 1), (8, 11, 12)]:
        rd = fci.solve_subsystem(s, X, "dense")
        rl = fci.solve_subsystem(s, X, "lanczos", tol=1e-10)
        assert rd.energy == pytest.approx(rl.energy, abs=1e-10)
        assert abs(abs(rd.vector @ rl.vector) - 1.0) < 1e-8


def test_degenerate_singlet_triplet_level_is_resolved():
    """Bodies 0 and 13 of the 40-body chain sit 70 A apart (couplings
    ~exp(-35)): the lowest level of the pair is an exactly degenerate singlet
    and triplet (one electron moved between the bodies).  The dense solver
    must resolve S^2 inside that eigenspace and report the level as a singlet,
    as the Lanczos of the spin-flip-even sector does (that sector excludes
    the triplet), and the returned vector must be a pure singlet."""
    from synth import chain_40_uneven
    s = chain_40_uneven()
    H = fci.Hamiltonian(fci.subsystem(s, (0, 13)))
    w = np.linalg.eigvalsh(H.dense())
    assert w[1] - w[0] < 1e-8                      # the degenerate pair
    dense = fci.solve_subsystem(s, (0, 13), "dense")
    lan = fci.solve_subsystem(s, (0, 13), "lanczos", tol=1e-10)
    assert dense.energy == pytest.approx(w[0], abs=1e-10)
    assert lan.energy == pytest.approx(dense.energy, abs=1e-9)
    assert abs(dense.s2) < 1e-8


def test_lanczos_finds_a_charge_transfer_ground_state():
    """Two bodies with no inter-body hopping: each body's electron count is
    conserved, and the ground state lies in the charge-transfer sector (0, 4)
    where the reference determinant (2, 2) has exactly zero weight.  The
    random-start Lanczos must reach the dense lowest singlet; a reference
    start stays in the (2, 2) sector above it."""
    s = chain_4x2()
    n = s.norb
    h = np.zeros((n, n))
    h[0, 0], h[1, 1] = -0.2, 2.0            # body 0: bonding high, antibonding far up
    h[2, 2], h[3, 3] = -1.0, -0.9           # body 1: both orbitals low
    h[4, 4], h[5, 5], h[6, 6], h[7, 7] = -1.0, 0.5, -1.0, 0.5
    h[0, 1] = h[1, 0] = -0.1
    h[2, 3] = h[3, 2] = -0.1
    body = [0, 0, 1, 1, 2, 2, 3, 3]
    V = np.zeros((s.npair, s.npair))
    for p in range(n):
        for q in range(p + 1):
            for r in range(n):
                for t in range(r + 1):
                    A, B = pair_index(p, q), pair_index(r, t)
                    if body[p] == body[q] and body[r] == body[t]:
                        V[A, B] = 0.3 if (p == q and r == t) else 0.02
    s2 = s.with_integrals(h, V)
    dense = fci.solve_subsystem(s2, (0, 1), "dense")
    lan = fci.solve_subsystem(s2, (0, 1), "lanczos", tol=1e-10)
    ref = fci.solve_subsystem(s2, (0, 1), "lanczos", tol=1e-10, start="reference")
    assert lan.energy == pytest.approx(dense.energy, abs=1e-10)
    assert ref.energy > dense.energy + 0.1
    sub = fci.subsystem(s2, (0, 1))
    H = fci.Hamiltonian(sub)
    bl = [sub.ncore + sub.active.index(s2.bonding_orbital(b)) for b in (0, 1)]
    assert abs(dense.vector[H.reference_index(bl)]) < 1e-12


def test_lowest_singlet_is_spin_flip_symmetric_and_lowest_overall():
    """C[Ia, Ib] = C[Ib, Ia] for the singlet (alpha-major string order), and for
    these seeds the lowest M_s = 0 root is that singlet."""
    s = chain_4x2()
    for X in [(0, 1), (1, 2, 3)]:
        H = fci.Hamiltonian(fci.subsystem(s, X))
        e, c = fci.lowest_singlet_dense(H)
        C = c.reshape(H.nstr, H.nstr)
        np.testing.assert_allclose(C, C.T, atol=1e-10)
        assert e == pytest.approx(np.linalg.eigvalsh(H.dense())[0], abs=1e-12)


def test_particle_number_and_spin():
    s = chain_4x2()
    for X in [(0,), (1, 3), (0, 1, 2)]:
        r = fci.solve_subsystem(s, X)
        g1, g2 = fci.subsystem_rdm_global(s, X, r.vector)
        N = 2 * s.nbody                       # every body brings 2 electrons
        assert np.trace(g1) == pytest.approx(N, abs=1e-10)
        assert np.einsum("pprr->", g2) == pytest.approx(N * (N - 1), abs=1e-9)
        assert abs(r.s2) < 1e-8


def test_rdm_reconstructs_energy():
    s = chain_4x2()
    V = s.eri_packed()
    n = s.norb
    eri = np.empty((n, n, n, n))
    for p, q, r, t in itertools.product(range(n), repeat=4):
        eri[p, q, r, t] = V[pair_index(p, q), pair_index(r, t)]
    for X in [(2,), (0, 3)]:
        r = fci.solve_subsystem(s, X)
        g1, g2 = fci.subsystem_rdm_global(s, X, r.vector)
        e = np.sum(s.h * g1) + 0.5 * np.sum(eri * g2)
        assert e == pytest.approx(r.energy, abs=1e-11)


def test_variational_bounds_and_nesting():
    """E_X <= E_0 (the reference determinant is in every space) and E_{X u Y} <= E_X."""
    s = chain_4x2()
    e0, ex, _, _ = fci.ifci_energies(s, 3)
    for X, e in ex.items():
        assert e <= e0 + 1e-12
        for Y in ex:
            if set(X) < set(Y):
                assert ex[Y] <= e + 1e-12


def test_separability_zeroes_cross_increments():
    """Integrals coupling bodies {0,1} with {2,3} set to zero: every increment spanning both groups is 0."""
    s = chain_4x2()
    g1 = set(s.body_orbitals(0) + s.body_orbitals(1))
    n = s.norb
    h = s.h.copy()
    V = s.eri_packed().copy()
    for p in range(n):
        for q in range(n):
            if (p in g1) != (q in g1):
                h[p, q] = 0.0
    grp = np.array([p in g1 for p in range(n)])
    pairs = [(P, Q) for P in range(n) for Q in range(P + 1)]
    for A, (p, q) in enumerate(pairs):
        for B, (r, t) in enumerate(pairs):
            g = {bool(grp[p]), bool(grp[q]), bool(grp[r]), bool(grp[t])}
            if len(g) > 1:
                V[A, B] = 0.0
    s2 = s.with_integrals(h, V)
    _, _, eps, _ = fci.ifci_energies(s2, 4)
    for X, e in eps.items():
        bodies_in_g1 = {b for b in X if b in (0, 1)}
        if bodies_in_g1 and len(bodies_in_g1) < len(X):
            assert abs(e) < 1e-12, (X, e)


def test_full_order_expansion_equals_fci():
    """Eq. 1 taken to n = number of bodies telescopes to the full FCI energy (8e, 8o)."""
    s = chain_4x2()
    e0, ex, eps, total = fci.ifci_energies(s, 4)
    assert len(eps) == 15
    full = fci.solve_subsystem(s, (0, 1, 2, 3), "lanczos", tol=1e-10)
    dense = fci.solve_subsystem(s, (0, 1, 2, 3), "dense")
    assert full.ndet == 4900
    assert total == pytest.approx(dense.energy, abs=1e-10)
    assert full.energy == pytest.approx(dense.energy, abs=1e-10)


# ---------------------------------------------------------------- increment algebra

def _random_ec(nbody, order, seed):
    rng = np.random.default_rng(seed)
    return {X: float(rng.normal()) for X in fci.body_subsets(nbody, order)}


def test_increments_match_eqs_2_to_5_written_out():
    ec = _random_ec(5, 4, 3)
    eps = fci.increments_from_correlation(ec)
    i, j, k, l = 0, 2, 3, 4
    e = lambda *X: eps[tuple(sorted(X))]
    E = lambda *X: ec[tuple(sorted(X))]
    assert e(i) == E(i)                                                          # Eq. 2
    assert e(i, j) == pytest.approx(E(i, j) - e(i) - e(j), abs=1e-14)            # Eq. 3
    assert e(i, j, k) == pytest.approx(E(i, j, k) - e(i, j) - e(i, k) - e(j, k)
                                       - e(i) - e(j) - e(k), abs=1e-14)          # Eq. 4
    assert e(i, j, k, l) == pytest.approx(
        E(i, j, k, l) - e(i, j, k) - e(i, j, l) - e(i, k, l) - e(j, k, l)
        - e(i, j) - e(i, k) - e(i, l) - e(j, k) - e(j, l) - e(k, l)
        - e(i) - e(j) - e(k) - e(l), abs=1e-14)                                   # Eq. 5


def test_increments_equal_inclusion_exclusion():
    ec = _random_ec(6, 3, 4)
    eps = fci.increments_from_correlation(ec)
    for X in ec:
        mob = sum((-1) ** (len(X) - k) * ec[Y] for k in range(1, len(X) + 1)
                  for Y in itertools.combinations(X, k))
        assert eps[X] == pytest.approx(mob, abs=1e-13)


@pytest.mark.parametrize("N,n", [(6, 2), (7, 3), (24, 3), (5, 4)])
def test_expansion_weights_closed_form(N, n):
    for Y in [tuple(range(k)) for k in range(1, n + 1)]:
        w = fci.expansion_weight(Y, N, n) if N <= 8 else None
        closed = (-1) ** (n - len(Y)) * math.comb(N - len(Y) - 1, n - len(Y))
        if w is not None:
            assert w == closed
    if N <= 8:
        ec = _random_ec(N, n, 5)
        eps = fci.increments_from_correlation(ec)
        e0 = 0.37
        lhs = e0 + sum(eps.values())
        ws = {Y: fci.expansion_weight(Y, N, n) for Y in ec}
        rhs = (1 - sum(ws.values())) * e0 + sum(ws[Y] * (ec[Y] + e0) for Y in ec)
        assert lhs == pytest.approx(rhs, abs=1e-12)


# ---------------------------------------------------------------- gradient

def test_oracle_gradient_matches_central_differences():
    """dE_iFCI/dh and dE_iFCI/dV (n=2 on the 4x2 chain) against central differences, step 1e-5."""
    s = chain_4x2()
    order = 2
    total, dh, dV = fci.ifci_gradient(s, order, method="dense")
    rng = np.random.default_rng(7)
    n = s.norb
    step = 1e-5
    checks = 0
    for _ in range(6):
        p, q = sorted(rng.integers(0, n, size=2))
        hp, hm = s.h.copy(), s.h.copy()
        hp[p, q] += step; hm[p, q] -= step
        if p != q:
            hp[q, p] += step; hm[q, p] -= step
        ep = fci.ifci_energies(s.with_integrals(hp, s.eri_packed()), order, "dense")[3]
        em = fci.ifci_energies(s.with_integrals(hm, s.eri_packed()), order, "dense")[3]
        fd = (ep - em) / (2 * step)
        an = dh[p, q] + (dh[q, p] if p != q else 0.0)
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-9)
        checks += 1
    npair = s.npair
    for _ in range(6):
        A, B = sorted(rng.integers(0, npair, size=2))
        Vp, Vm = s.eri_packed().copy(), s.eri_packed().copy()
        Vp[A, B] += step; Vm[A, B] -= step
        if A != B:
            Vp[B, A] += step; Vm[B, A] -= step
        ep = fci.ifci_energies(s.with_integrals(s.h, Vp), order, "dense")[3]
        em = fci.ifci_energies(s.with_integrals(s.h, Vm), order, "dense")[3]
        fd = (ep - em) / (2 * step)
        an = dV[A, B] + (dV[B, A] if A != B else 0.0)
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-9)
        checks += 1
    assert checks == 12


@pytest.mark.parametrize("order", [1, 2, 3])
def test_oracle_gradient_obeys_euler_identity(order):
    """E_iFCI(lambda h, lambda V) = lambda E_iFCI (every E_Y, E_core and E_0 is
    an eigenvalue or energy of a Hamiltonian linear in the integrals), so
    sum h dE/dh + sum V dE/dV = E_iFCI exactly for Hellmann–Feynman
    derivatives: a dropped core term, a wrong expansion weight or a wrong
    factor on the two-electron part breaks it."""
    s = chain_4x2()
    e, dh, dV = fci.ifci_gradient(s, order, method="dense")
    euler = float(np.sum(s.h * dh) + np.sum(s.eri_packed() * dV))
    assert euler == pytest.approx(e, abs=1e-10)


# ---------------------------------------------------------------- connected n-body screening

@pytest.fixture(scope="module")
def chain4x2_order4():
    s = chain_4x2()
    return s, fci.ifci_energies(s, 4)


def test_cnb_screening_off_equals_the_full_expansion(chain4x2_order4):
    s, full = chain4x2_order4
    pair_min = min(abs(v) for X, v in full[2].items() if len(X) == 2)
    b = fci.ifci_energies(s, 4, cnb=0.5 * pair_min)       # every pair is an edge: nothing screened
    assert b[3] == pytest.approx(full[3], abs=1e-10)
    assert set(b[1]) == set(full[1])


def test_cnb_screening_keeps_exactly_the_connected_sets(chain4x2_order4):
    """The kept 3- and 4-body sets are the sets whose graph of pair increments
    at or above C is connected, checked with networkx on the pair table;
    screened increments are zero and the others follow Eqs. 2-5 with them."""
    nx = pytest.importorskip("networkx")
    s, full = chain4x2_order4
    eps_full = full[2]
    pair_mags = sorted(abs(v) for X, v in eps_full.items() if len(X) == 2)
    C = 0.5 * (pair_mags[2] + pair_mags[3])          # keeps the three largest pairs
    e0, ex, eps, total = fci.ifci_energies(s, 4, cnb=C)
    kept = 0
    for X in fci.body_subsets(4, 4):
        if len(X) < 3:
            assert X in ex
            continue
        g = nx.Graph()
        g.add_nodes_from(X)
        g.add_edges_from(p for p in itertools.combinations(X, 2) if abs(eps_full[p]) >= C)
        assert (X in ex) == nx.is_connected(g), X
        if X in ex:
            kept += 1
            rec = ex[X] - e0 - sum(eps[Y] for j in range(1, len(X)) for Y in itertools.combinations(X, j))
            assert eps[X] == pytest.approx(rec, abs=1e-13)
            assert ex[X] == pytest.approx(full[1][X], abs=1e-9)   # a kept set is solved as before
        else:
            assert eps[X] == 0.0
    assert 0 < kept < 5
    assert total == pytest.approx(e0 + sum(eps.values()), abs=1e-13)


def test_cnb_screening_everything_above_two_bodies_gives_the_order_2_total(chain4x2_order4):
    s, _ = chain4x2_order4
    two = fci.ifci_energies(s, 2)[3]
    scr = fci.ifci_energies(s, 4, cnb=1e3)
    assert scr[3] == pytest.approx(two, abs=1e-13)
    assert all(len(X) <= 2 for X in scr[1])
