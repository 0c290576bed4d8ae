"""Writes chain24_oracle.json: oracle energies of sampled body sets of the
24-body uneven chain (seed 2308), used by the GPU parity tests.

Calls only ``oracle/`` (and the seeded ``synth`` inputs).  Sample: every
1-body set, 30 seeded 2-body sets plus the largest one, 10 seeded 3-body
sets with at most 30,000 determinants, and two 3-body sets (132,496
determinants each) whose lowest singlet is a charge-transfer state with
almost no weight on the reference determinant.  Run from the repository root:
    python tests/golden/make_chain24_golden.py
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
from synth import chain_24_uneven  # noqa: E402


def main():
    s = chain_24_uneven()
    sizes = s.body_sizes
    rng = np.random.default_rng(20230719)
    ones = [(b,) for b in range(24)]
    pairs = list(itertools.combinations(range(24), 2))
    two = [pairs[i] for i in sorted(rng.choice(len(pairs), 30, replace=False))]
    big2 = max(pairs, key=lambda X: sum(sizes[b] for b in X))
    if big2 not in two:
        two.append(big2)
    triples = [X for X in itertools.combinations(range(24), 3)
               if math.comb(sum(sizes[b] for b in X), 3) ** 2 <= 30000]
    three = [triples[i] for i in sorted(rng.choice(len(triples), 10, replace=False))]
    hard = [(5, 11, 15), (5, 14, 15)]
    out = {"system": "chain-24-uneven", "seed": s.seed, "body_sizes": sizes,
           "e0": fci.reference_energy(s), "energies": {}}
    t0 = time.time()
    for X in ones + two + three + hard:
        r = fci.solve_subsystem(s, X, tol=1e-10)
        out["energies"][",".join(map(str, X))] = {"energy": r.energy, "ndet": r.ndet, "s2": r.s2,
                                                   "method": r.method}
        print(X, r.ndet, r.energy, f"{time.time() - t0:.1f}s", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "chain24_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
