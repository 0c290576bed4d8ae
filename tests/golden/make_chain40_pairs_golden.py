"""Writes chain40_pairs_oracle.json: oracle energies of every 2-body set of the
40-body uneven chain (seed 2310), 780 sets of at most 4,356 determinants, for
the set-by-set parity of the order-2 expansion.

Calls only ``oracle/`` (and the seeded ``synth`` inputs).  Run from the
repository root:
    python tests/golden/make_chain40_pairs_golden.py
"""
import itertools
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fci  # noqa: E402
from synth import chain_40_uneven  # noqa: E402


def main():
    s = chain_40_uneven()
    out = {"system": "chain-40-uneven", "seed": s.seed, "e0": fci.reference_energy(s), "energies": {}}
    t0 = time.time()
    for X in itertools.combinations(range(s.nbody), 2):
        r = fci.solve_subsystem(s, X, tol=1e-10)
        out["energies"][",".join(map(str, X))] = {"energy": r.energy, "ndet": r.ndet, "s2": r.s2}
    print(f"{len(out['energies'])} sets in {time.time() - t0:.0f} s", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "chain40_pairs_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print("wrote", path)


if __name__ == "__main__":
    main()
