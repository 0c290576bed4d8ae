"""Pins of the oracle's summation natural orbitals (oracle/sno.py; Methods,
SNO paragraph).

* The two-electron singlet solver (pair functions, its own formulation)
  equals the Slater–Condon FCI of the same orbitals and core.
* A 1-body density is symmetric, has trace 2 and occupations in [0, 2].
* Keeping every natural orbital, the SNO energy equals the CI of X's bonding
  orbitals plus all virtuals in the original basis (CI is invariant under a
  rotation of its active orbitals): a wrong transformation of h or of the
  integrals fails it.
* Energies do not rise as eta grows (the kept spaces are nested) and the
  kept count does not fall.
* A random rotation of the system's virtual orbitals changes no SNO energy
  (the construction depends only on the densities, not on the basis).
"""
import numpy as np
import pytest

from oracle import fci, sno
from synth import chain_4x2, make_chain


def _loc_integrals(system, loc):
    h = system.h[np.ix_(loc, loc)].copy()
    return h, fci._eri_from_packed(system.eri_packed(), loc)


@pytest.mark.parametrize("b", [0, 2])
def test_two_electron_solver_equals_slater_condon(b):
    s = chain_4x2()
    bond = [s.bonding_orbital(x) for x in range(s.nbody)]
    virt = [p for p in range(s.norb) if p not in bond]
    core = [bond[x] for x in range(s.nbody) if x != b]
    active = [bond[b]] + virt
    e2, C = sno.two_electron_singlet(s.h, sno._eri_full(s), core, active)
    h, eri = _loc_integrals(s, core + active)
    sub = fci.Subsystem(core, active, 1, h, eri)
    e_sc, _ = fci.lowest_singlet_dense(fci.Hamiltonian(sub))
    assert e2 == pytest.approx(e_sc, abs=1e-10)
    assert np.allclose(C, C.T) and np.sum(C * C) == pytest.approx(1.0, abs=1e-12)


def test_one_body_density_invariants():
    s = make_chain([2, 3, 2, 3], seed=77)
    for b in range(s.nbody):
        virt, g = sno.one_body_density(s, b)
        w = np.linalg.eigvalsh(g)
        assert np.allclose(g, g.T)
        assert w.min() > -1e-12 and w.max() < 2.0
        # the virtual block's trace is what the bonding orbital lost: below 2
        assert 0.0 < np.trace(g) < 2.0


@pytest.mark.parametrize("X", [(0,), (0, 1), (1, 3), (0, 2, 3)])
def test_keeping_every_natural_orbital_equals_the_full_virtual_ci(X):
    s = chain_4x2()
    e_sno, nkept = sno.sno_energy(s, X, eta=300.0)
    bond = [s.bonding_orbital(x) for x in range(s.nbody)]
    virt = [p for p in range(s.norb) if p not in bond]
    core = [bond[x] for x in range(s.nbody) if x not in X]
    active = sorted([bond[x] for x in X] + virt)
    h, eri = _loc_integrals(s, core + active)
    e_ref, _ = fci.lowest_singlet_dense(fci.Hamiltonian(fci.Subsystem(core, active, len(X), h, eri)))
    assert nkept == len(virt)
    assert e_sno == pytest.approx(e_ref, abs=1e-9)


@pytest.mark.parametrize("X", [(0, 1), (1, 2)])
def test_energy_does_not_rise_with_eta(X):
    s = make_chain([2, 3, 2, 3], seed=77)
    last_e, last_n = None, -1
    for eta in (1.0, 2.0, 4.0, 8.5):
        e, n = sno.sno_energy(s, X, eta)
        assert n >= last_n
        if last_e is not None:
            assert e <= last_e + 1e-10
        last_e, last_n = e, n


def test_rotation_of_the_virtuals_changes_nothing():
    s = make_chain([2, 3, 2, 3], seed=77)
    eri = sno._eri_full(s)
    bond = [s.bonding_orbital(x) for x in range(s.nbody)]
    virt = [p for p in range(s.norb) if p not in bond]
    Q, _ = np.linalg.qr(np.random.default_rng(5).normal(size=(len(virt), len(virt))))
    R = np.eye(s.norb)
    R[np.ix_(virt, virt)] = Q
    h2 = R.T @ s.h @ R
    eri2 = np.einsum("pqrs,pa,qb,rc,sd->abcd", eri, R, R, R, R, optimize=True)
    for X in [(0, 1), (2, 3)]:
        rho = sum(sno.one_body_density(s, b)[1] for b in X)
        occ = np.clip(np.linalg.eigvalsh(rho), 1e-300, None)
        assert np.min(np.abs(np.log10(occ) + 4.0)) > 0.05      # no occupation at the threshold
        e1, n1 = sno.sno_energy(s, X, 4.0)
        e2, n2 = sno.sno_energy(s, X, 4.0, h2, eri2)
        assert n1 == n2
        assert e1 == pytest.approx(e2, abs=1e-9)


def test_full_order_sno_expansion_keeping_everything_is_fci():
    """At full order the expansion telescopes to E of the set of all bodies;
    keeping every natural orbital that set's space is every orbital: the
    total equals FCI(8e,8o) of the 4 x 2 chain (Slater–Condon, dense)."""
    s = chain_4x2()
    _, _, _, total = sno.sno_energies(s, 4, eta=300.0)
    h, eri = _loc_integrals(s, list(range(s.norb)))
    e_fci, _ = fci.lowest_singlet_dense(fci.Hamiltonian(fci.Subsystem([], list(range(s.norb)), 4, h, eri)))
    assert total == pytest.approx(e_fci, abs=1e-9)
    # a truncated space at full order is variational
    _, _, _, total_cut = sno.sno_energies(s, 4, eta=2.0)
    assert total_cut >= e_fci - 1e-10
