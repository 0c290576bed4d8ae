"""Autotuner of the batched solver's launch parameters.

The kernels' tile shapes are fixed by the hardware they are written for (128
TMEM lanes per tile, five 96-column level accumulators in the 512 TMEM
columns, 64-pair K atoms in shared memory), so what is left to choose per
workload and GPU are the parameters of the batched solve itself:

* ``max_space``: Davidson subspace size before a thick restart (fewer
  restarts and iterations against more vector traffic per iteration; on a
  sample too small to fill the GPU a small subspace looks cheaper than it is
  at full scale, where the extra sigma builds dominate, so the grid starts at
  10);
* ``det_budget``: D elements per sigma wave (how many problems one sigma
  launch covers: larger waves fill the GPU better, smaller ones keep the
  intermediates in L2);
* ``graph_iters``: Davidson iterations captured per CUDA graph (0 = launched
  one by one), which removes launch latency for batches of small problems.

Every candidate is timed on the same seeded sample of the workload's CI
problems (their frozen-body Hamiltonians, one ``ifci_davidson_batched`` call
each, after one untimed call); a candidate whose energies differ from the
first candidate's by more than ``tol`` is rejected.  The choice is cached in
a JSON file keyed by the GPU name and a signature of the workload, and the
search is coordinate-wise (one parameter at a time, the others at their
best so far).  All arithmetic runs in the library; this module only times
calls and chooses among them.
"""
from __future__ import annotations

import hashlib
import json
import os
import time
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import api

DEFAULT_GRID = {
    "max_space": [12, 10, 16],
    "det_budget": [1 << 31, 1 << 30],
    "graph_iters": [0, 4],
}


def workload_signature(system: api.SystemArrays, sets: Sequence[Sequence[int]], precision: str, r_tol: float) -> str:
    sizes = [int(system.body_offset[b + 1] - system.body_offset[b]) for b in range(system.nbody)]
    key = json.dumps({"sizes": sizes, "sets": [list(X) for X in sets], "precision": precision, "r_tol": r_tol},
                     sort_keys=True)
    return hashlib.sha1(key.encode()).hexdigest()[:16]


def _problems(handle: api.Handle, system: api.SystemArrays, sets):
    probs = []
    for X in sets:
        h1, eri, ec = api.ifci_frozen_core(handle, system, X)
        probs.append(api.CIProblem(h1.shape[0], len(X), h1, eri, ec))
    return probs


def _time(handle, probs, opts, repeats=1, warm=True):
    if warm:
        api.ifci_davidson_batched(handle, probs, opts, allow_unconverged=True)   # set-up (workspace growth)
        torch.cuda.synchronize()
    best = float("inf")
    e = None
    for _ in range(repeats):
        t0 = time.perf_counter()
        e, _, st = api.ifci_davidson_batched(handle, probs, opts, allow_unconverged=True)
        torch.cuda.synchronize()
        best = min(best, time.perf_counter() - t0)
        if np.any(st != 0):
            return float("inf"), e
    return best, e


def autotune(handle: api.Handle, system: api.SystemArrays, sets: Sequence[Sequence[int]], precision: str = "fp64e",
             r_tol: float = 1e-6, e_tol: float = 1e-10, tol: float = 1e-8, grid: Optional[Dict[str, List]] = None,
             cache: Optional[str] = None, **fixed) -> Dict:
    """Chooses max_space, det_budget and graph_iters for solving ``sets`` of
    ``system`` (body index tuples).  Returns {"params": {...}, "table": [...],
    "cached": bool}; ``table`` lists every timed candidate (seconds, energy
    deviation from the first candidate)."""
    grid = dict(DEFAULT_GRID if grid is None else grid)
    dev_name = torch.cuda.get_device_name(handle.device)
    sig = workload_signature(system, sets, precision, r_tol)
    key = f"{dev_name}|{sig}"
    if cache and os.path.exists(cache):
        try:
            data = json.load(open(cache))
            if key in data:
                return {"params": data[key]["params"], "table": data[key]["table"], "cached": True}
        except (OSError, ValueError):
            pass
    probs = _problems(handle, system, sets)
    best = {k: v[0] for k, v in grid.items()}   # the first value of each list is the starting point
    table = []
    ref_e = None
    best_t = float("inf")
    seen = {}
    for name, values in grid.items():
        for val in values:
            cand = dict(best, **{name: val})
            key_c = tuple(sorted(cand.items()))
            if key_c in seen:          # the incumbent, already timed
                continue
            opts = api.davidson_opts(precision, r_tol=r_tol, e_tol=e_tol, max_iter=300, **cand, **fixed)
            t, e = _time(handle, probs, opts, warm=not seen)
            seen[key_c] = t
            if ref_e is None:
                ref_e = e
            dev = float(np.max(np.abs(e - ref_e))) if e is not None else float("inf")
            ok = t < float("inf") and dev <= tol
            table.append({"params": cand, "seconds": t, "max_abs_energy_deviation": dev, "accepted": ok})
            if ok and t < best_t:
                best_t = t
                best = cand
    out = {"params": best, "table": table, "cached": False}
    if cache:
        try:
            data = json.load(open(cache)) if os.path.exists(cache) else {}
        except (OSError, ValueError):
            data = {}
        data[key] = {"params": best, "table": table}
        with open(cache, "w") as f:
            json.dump(data, f, indent=1)
    return out
