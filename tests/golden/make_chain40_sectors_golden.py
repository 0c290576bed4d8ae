"""Writes chain40_sectors_oracle.json: oracle energies of body sets of the
40-body uneven chain (seed 2310) whose lowest singlet lies in a
charge-transfer sector between weakly coupled bodies, and of seeded
CAS(6e,18o) sets (three 6-orbital bodies, 665,856 determinants).

Calls only ``oracle/`` (and the seeded ``synth`` inputs).

* Weakly coupled sets: 3-body sets with a body pair whose largest coupling
  integral (|h_pq| or |(pq|rs)| over p in one body, q in the other) lies
  between 1e-9 and 1e-6, so that a charge-transfer sector between them is
  all but invisible to an iteration started in another sector (the sets
  where iterations started from the lowest-diagonal determinants reached
  different energies).
* CAS(6e,18o) sets: five of the C(8, 3) = 56 sets of three 6-orbital
  bodies, drawn with a seeded generator; the Lanczos runs take about half
  an hour each on 8 cores, so the file also serves as their cache: sets
  already present are skipped.  Run from the repository root:
    python tests/golden/make_chain40_sectors_golden.py
"""
import itertools
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fci  # noqa: E402
from synth import chain_40_uneven  # noqa: E402

WEAK = [(0, 7, 17), (0, 7, 18), (0, 7, 21), (0, 7, 31), (0, 7, 36), (2, 34, 39), (6, 20, 29), (6, 29, 39),
        (6, 33, 39), (8, 21, 27), (11, 20, 23), (21, 27, 34), (27, 29, 34)]
PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "chain40_sectors_oracle.json")


def cas6e18o_sets(s):
    six = [b for b in range(s.nbody) if s.body_sizes[b] == 6]
    allx = list(itertools.combinations(six, 3))
    rng = np.random.default_rng(20261203)
    return [allx[i] for i in sorted(rng.choice(len(allx), 5, replace=False))]


def main():
    s = chain_40_uneven()
    out = {"system": "chain-40-uneven", "seed": s.seed, "e0": fci.reference_energy(s), "energies": {}}
    if os.path.exists(PATH):
        out["energies"] = json.load(open(PATH))["energies"]
    sets = sorted(WEAK, key=lambda X: sum(s.body_sizes[b] for b in X)) + cas6e18o_sets(s)
    t0 = time.time()
    for X in sets:
        key = ",".join(map(str, X))
        if key in out["energies"]:
            continue
        r = fci.solve_subsystem(s, X, tol=1e-8)
        out["energies"][key] = {"energy": r.energy, "ndet": r.ndet, "s2": r.s2, "method": r.method,
                                "iterations": r.iterations}
        print(X, r.ndet, r.energy, r.s2, f"{time.time() - t0:.1f}s", flush=True)
        with open(PATH, "w") as f:
            json.dump(out, f, indent=1)
    print("wrote", PATH)


if __name__ == "__main__":
    main()
