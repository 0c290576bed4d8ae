"""Writes chain40_oracle.json: oracle energies of a seeded sample of body sets
of the 40-body uneven chain (seed 2310), used by the GPU parity tests of the
production-scale 3-body expansion (10,700 body sets in all).

Calls only ``oracle/`` (and the seeded ``synth`` inputs).  Sample: 8 seeded
1-body sets, 20 seeded 2-body sets plus the largest one, 40 seeded 3-body
sets with at most 30,000 determinants, and five 3-body sets with hard lowest
roots: (8, 20, 32) and (12, 20, 27), whose two lowest singlets are 2.8e-5 and
5.0e-4 Eh apart, and (17, 21, 34), (7, 20, 21), (8, 14, 39), whose lowest
singlet is not led by the lowest-diagonal determinant.  Run from the
repository root:
    python tests/golden/make_chain40_golden.py
"""
import itertools
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fci  # noqa: E402
from synth import chain_40_uneven  # noqa: E402


def main():
    s = chain_40_uneven()
    sizes = s.body_sizes
    N = s.nbody
    rng = np.random.default_rng(20231031)
    ones = [(int(b),) for b in sorted(rng.choice(N, 8, replace=False))]
    pairs = list(itertools.combinations(range(N), 2))
    two = [pairs[i] for i in sorted(rng.choice(len(pairs), 20, replace=False))]
    big2 = max(pairs, key=lambda X: sum(sizes[b] for b in X))
    if big2 not in two:
        two.append(big2)
    triples = [X for X in itertools.combinations(range(N), 3)
               if math.comb(sum(sizes[b] for b in X), 3) ** 2 <= 30000]
    three = [triples[i] for i in sorted(rng.choice(len(triples), 40, replace=False))]
    hard = [(8, 20, 32), (12, 20, 27), (17, 21, 34), (7, 20, 21), (8, 14, 39)]
    out = {"system": "chain-40-uneven", "seed": s.seed, "body_sizes": sizes,
           "e0": fci.reference_energy(s), "energies": {}}
    t0 = time.time()
    for X in ones + two + three + hard:
        r = fci.solve_subsystem(s, X, tol=1e-10)
        out["energies"][",".join(map(str, X))] = {"energy": r.energy, "ndet": r.ndet, "s2": r.s2,
                                                   "method": r.method}
        print(X, r.ndet, r.energy, f"{time.time() - t0:.1f}s", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "chain40_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
