"""Pins of the oracle's HBCI (oracle/hbci.py; Methods, HBCI paragraph).

* Toy matrices whose selection rounds and energies follow by hand: the
  heat-bath rule takes the largest single contribution |H_ai c_i| (a
  determinant whose contributions cancel in the sum is still selected; one
  whose coupling |H_ai| is large but whose |H_ai c_i| is not, is not), the
  threshold is strict, EN-PT2 has the numerator (sum of the kept H_ai c_i)^2
  over E_var - H_aa, and eps2 drops the terms at or below it.
* H2 in a minimal basis: from the reference |g g>, eps1 above the coupling K
  gives E_var = E_g and E_2 = K^2 / (E_g - E_u) (second-order perturbation
  theory of the 2 x 2 CI, whose singles do not couple by symmetry); eps1
  below K gives the exact 2 x 2 root and E_2 = 0.
* eps1 = 0 on body sets of the 4 x 2 chain selects the whole connected
  space: E_var equals the FCI lowest singlet (itself pinned) and E_2 = 0.
* E_var is variational (>= E_FCI) at every eps1, and at the paper's
  thresholds E_var + E_2 lies closer to E_FCI than E_var alone.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import fci, hbci
from synth import chain_4x2


def _identity(n):
    return np.arange(n)


def test_toy_selection_rounds_and_pt2():
    H = np.array([[-1.0, 0.01, 0.0], [0.01, 0.0, 0.2], [0.0, 0.2, 0.5]])
    E2x2 = -0.5 - math.sqrt(0.25 + 0.01 ** 2)
    # eigenvector of [[-1, 0.01], [0.01, 0]] for E2x2: c1 / c0 = (1 + E) / 0.01
    r = (1.0 + E2x2) / 0.01
    c0, c1 = 1.0 / math.sqrt(1.0 + r * r), r / math.sqrt(1.0 + r * r)
    res = hbci.hbci_dense(H, _identity(3), 0, eps1=0.005, eps2=0.0)
    # round 1 adds state 1 (|0.01 * 1| > 0.005); round 2 finds |0.2 c1| ~ 0.002 < 0.005: stop
    assert res.rounds == 2 and res.nsel == 2
    assert res.e_var == pytest.approx(E2x2, abs=1e-14)
    assert res.e_pt2 == pytest.approx((0.2 * c1) ** 2 / (E2x2 - 0.5), rel=1e-12)
    assert abs(res.vector[0]) == pytest.approx(abs(c0), abs=1e-12)
    # eps2 above |H_21 c_1| drops the only PT2 term
    res = hbci.hbci_dense(H, _identity(3), 0, eps1=0.005, eps2=0.003)
    assert res.e_pt2 == 0.0
    # eps1 below |H_21 c_1| selects everything: the exact lowest eigenvalue, no PT2
    res = hbci.hbci_dense(H, _identity(3), 0, eps1=0.001, eps2=0.0)
    assert res.nsel == 3 and res.rounds == 3 and res.e_pt2 == 0.0
    assert res.e_var == pytest.approx(np.linalg.eigvalsh(H)[0], abs=1e-14)
    # the threshold is strict: eps1 equal to the largest contribution selects nothing
    res = hbci.hbci_dense(H, _identity(3), 0, eps1=0.01, eps2=0.0)
    assert res.nsel == 1 and res.e_var == -1.0
    assert res.e_pt2 == pytest.approx(0.01 ** 2 / (-1.0 - 0.0), rel=1e-14)


def test_toy_largest_contribution_not_the_sum():
    """State 3 couples to 1 and 2 with opposite signs; by symmetry c1 = c2, so
    its summed coupling vanishes, but each single contribution is |0.2 c1|."""
    a, b = 0.1, 0.2
    H = np.array([[-1.0, a, a, 0.0], [a, 0.0, 0.0, b], [a, 0.0, 0.0, -b], [0.0, b, -b, 1.0]])
    res = hbci.hbci_dense(H, _identity(4), 0, eps1=0.005, eps2=0.0)
    assert res.nsel == 4 and res.rounds == 3
    # state 3 decouples from the ground state by the same symmetry: exact energy
    assert res.e_var == pytest.approx(np.linalg.eigvalsh(H)[0], abs=1e-13)
    # a coupling |H_ai| above eps1 alone does not select: H_30 = 0, and at eps1 = 0.05
    # round 2 sees |b c1| < 0.05 although |b| = 0.2 > 0.05
    res = hbci.hbci_dense(H, _identity(4), 0, eps1=0.05, eps2=0.0)
    w3 = np.linalg.eigvalsh(H[:3, :3])[0]
    assert res.nsel == 3 and res.e_var == pytest.approx(w3, abs=1e-13)
    # PT2 of state 3: the two contributions cancel exactly (num = b c1 - b c2 = 0)
    assert res.e_pt2 == pytest.approx(0.0, abs=1e-15)


def _h2():
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
    return H, 2 * hgg + Jgg, 2 * huu + Juu, K


def test_h2_minimal_basis_hbci_closed_forms():
    H, Eg, Eu, K = _h2()
    ref = H.reference_index([0])
    flip = hbci.spin_flip_permutation(H.nstr)
    res = hbci.hbci_dense(H.dense(), flip, ref, eps1=0.5, eps2=0.0)
    assert res.nsel == 1
    assert res.e_var == pytest.approx(Eg, abs=1e-14)
    assert res.e_pt2 == pytest.approx(K * K / (Eg - Eu), rel=1e-12)
    res = hbci.hbci_dense(H.dense(), flip, ref, eps1=0.1, eps2=0.0)
    assert res.nsel == 2
    assert res.e_var == pytest.approx(0.5 * (Eg + Eu) - math.sqrt(0.25 * (Eg - Eu) ** 2 + K * K), abs=1e-13)
    assert res.e_pt2 == pytest.approx(0.0, abs=1e-15)


@pytest.mark.parametrize("X", [(0,), (1, 2), (0, 1, 3)])
def test_eps1_zero_is_fci(X):
    s = chain_4x2()
    res = hbci.hbci_subsystem(s, X, eps1=0.0, eps2=0.0)
    exact = fci.solve_subsystem(s, X, method="dense").energy
    assert res.e_var == pytest.approx(exact, abs=1e-11)
    assert res.e_pt2 == pytest.approx(0.0, abs=1e-14)


@pytest.mark.parametrize("X", [(0, 1), (1, 2, 3), (0, 2, 3)])
def test_variational_bound_and_pt2_at_paper_thresholds(X):
    s = chain_4x2()
    exact = fci.solve_subsystem(s, X, method="dense").energy
    last = None
    for eps1 in (1e-1, 1e-2, 1e-3, 1e-4):
        res = hbci.hbci_subsystem(s, X, eps1=eps1, eps2=1e-6)
        assert res.e_var >= exact - 1e-12
        if last is not None:
            assert res.nsel >= last
        last = res.nsel
    res = hbci.hbci_subsystem(s, X, eps1=1e-3, eps2=1e-6)
    if res.e_var - exact > 1e-8:
        assert abs(res.e_total - exact) < abs(res.e_var - exact)


def test_charge_transfer_ground_state_outside_the_selection():
    """The 24-body chain's set (15, 17): its lowest singlet (FCI) lies 0.41 Eh
    below the lowest state reachable from the reference through contributions
    above 1 mHa, so HBCI at the paper's thresholds stays there; eps1 = 0
    selects every determinant and reaches FCI.  A property of the method that
    the GPU path must share (it is compared set by set with this oracle)."""
    from synth import chain_24_uneven
    c = chain_24_uneven()
    X = (15, 17)
    exact = fci.solve_subsystem(c, X, method="dense").energy
    paper = hbci.hbci_subsystem(c, X, 1e-3, 1e-6)
    full = hbci.hbci_subsystem(c, X, 0.0, 0.0)
    assert paper.e_total - exact > 0.4
    assert paper.nsel < full.nsel == 2025
    assert full.e_var == pytest.approx(exact, abs=1e-10)


def test_reference_determinant_index_matches_the_oracle():
    """The package's host helper for HBCI start determinants (rank of the
    string of bonding orbitals) against the oracle's own reference index."""
    import paper_2307_10675_gb300 as ifci
    from synth import chain_24_uneven
    c = chain_24_uneven()
    for X in [(0,), (0, 1), (5, 7), (8, 11, 12), (2, 9, 16), (1, 3, 5, 7)]:
        sub = fci.subsystem(c, X)
        H = fci.Hamiltonian(sub)
        bonding_local = [sub.ncore + sub.active.index(c.bonding_orbital(b)) for b in X]
        assert ifci.reference_determinant(c.body_sizes, X) == H.reference_index(bonding_local), X
