"""The seeded synthetic inputs follow their stated recipe: sizes of the four
chains, the integral symmetries, positive semidefinite ERIs, the decay with
distance, reproducibility from the seed, and the CI sizes quoted for each
configuration (2324 and 10,700 body sets, CAS(6e,18o) = 665,856 determinants,
CAS(14e,14o) = 11,778,624)."""
import itertools
import math

import numpy as np
import pytest

from synth import chain_4x2, chain_7x2, chain_24_uneven, chain_40_uneven, pair_index


@pytest.mark.parametrize("make,nbody,norb,sizes", [
    (chain_4x2, 4, 8, {2: 4}),
    (chain_7x2, 7, 14, {2: 7}),
    (chain_24_uneven, 24, 96, {2: 5, 3: 5, 4: 4, 5: 5, 6: 5}),
    (chain_40_uneven, 40, 160, {2: 8, 3: 8, 4: 8, 5: 8, 6: 8}),
])
def test_chain_shapes(make, nbody, norb, sizes):
    c = make()
    assert c.nbody == nbody and c.norb == norb
    assert {s: c.body_sizes.count(s) for s in set(c.body_sizes)} == sizes
    assert c.body_offsets[0] == 0 and c.body_offsets[-1] == norb


def test_integral_symmetries_and_psd():
    c = chain_4x2()
    h, V = c.h, c.eri_packed()
    np.testing.assert_array_equal(h, h.T)
    np.testing.assert_array_equal(V, V.T)                                   # (pq|rs) = (rs|pq)
    assert np.linalg.eigvalsh(V).min() > -1e-12                            # sum_L B B^T is PSD
    n = c.norb
    for p, q, r, s in itertools.product(range(n), repeat=4):               # (pq|rs) = (qp|rs) by packing
        assert V[pair_index(p, q), pair_index(r, s)] == V[pair_index(q, p), pair_index(s, r)]


def test_one_electron_recipe_and_decay():
    c = chain_24_uneven()
    h = c.h
    bonding = {c.bonding_orbital(b) for b in range(c.nbody)}
    diag = np.diag(h)
    # bonding around -1, antibonding around +0.5 (standard deviation 0.3)
    assert abs(np.mean([diag[p] for p in bonding]) + 1.0) < 0.3
    assert abs(np.mean([diag[p] for p in range(c.norb) if p not in bonding]) - 0.5) < 0.15
    # off-diagonal h_pq = -0.3 exp(-d/2), d = 1.5 A |p - q|
    for p, q in [(0, 1), (3, 7), (10, 40)]:
        assert h[p, q] == pytest.approx(-0.3 * math.exp(-0.75 * abs(p - q)), rel=1e-12)
    # exchange-type integrals between distant orbitals vanish, Coulomb-type do not
    V = c.eri_packed()
    far = V[pair_index(0, 80), pair_index(0, 80)]
    coul = V[pair_index(0, 0), pair_index(80, 80)]
    assert abs(far) < 1e-40 and abs(coul) > 1e-6


def test_reproducible_from_seed():
    a, b = chain_24_uneven(), chain_24_uneven()
    np.testing.assert_array_equal(a.h, b.h)
    np.testing.assert_array_equal(a.eri_packed(), b.eri_packed())
    c = chain_24_uneven(seed=2309)
    assert not np.array_equal(a.h, c.h)


def test_configuration_sizes():
    c24, c40 = chain_24_uneven(), chain_40_uneven()
    assert sum(math.comb(24, k) for k in (1, 2, 3)) == 2324
    assert sum(math.comb(40, k) for k in (1, 2, 3)) == 10700
    big = max(itertools.combinations(range(24), 3), key=lambda X: sum(c24.body_sizes[b] for b in X))
    n = sum(c24.body_sizes[b] for b in big)
    assert n == 18 and math.comb(n, 3) ** 2 == 665856
    assert max(sum(c40.body_sizes[b] for b in X) for X in itertools.combinations(range(40), 3)) == 18
    assert math.comb(14, 7) ** 2 == 11778624
