"""Writes chain24_hbci_oracle.json: the oracle's HBCI energies (oracle/hbci.py,
eps1 = 1 mHa, eps2 = 1 µHa: the paper's thresholds) of seeded 2-body sets
of the 24-body uneven chain (seed 2308) up to 4,356 determinants, with the
selection margin of each (how far every selection decision lay from eps1).
Calls only ``oracle/`` (and the seeded ``synth`` inputs).  Run from the
repository root:  python tests/golden/make_chain24_hbci_golden.py
"""
import itertools
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fci, hbci  # noqa: E402
from synth import chain_24_uneven  # noqa: E402

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "chain24_hbci_oracle.json")
EPS1, EPS2 = 1e-3, 1e-6


def main():
    s = chain_24_uneven()
    pairs = list(itertools.combinations(range(s.nbody), 2))
    rng = np.random.default_rng(20261203)
    chosen = [pairs[i] for i in sorted(rng.choice(len(pairs), 24, replace=False))]
    out = {"system": "chain-24-uneven", "seed": s.seed, "eps1": EPS1, "eps2": EPS2, "sets": {}}
    for X in chosen:
        r = hbci.hbci_subsystem(s, X, EPS1, EPS2)
        out["sets"][",".join(map(str, X))] = {"e_var": r.e_var, "e_pt2": r.e_pt2, "nsel": r.nsel,
                                               "rounds": r.rounds, "margin1": r.margin1,
                                               "ndet": int(len(r.selected))}
        print(X, r.nsel, r.e_var, r.e_pt2, r.margin1, flush=True)
    with open(PATH, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", PATH)


if __name__ == "__main__":
    main()
