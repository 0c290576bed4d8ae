#!/usr/bin/env python
"""Benchmark of the iFCI increment CI solve on one GB300 (or N, one rank each).

One step = the whole hot path over one synthetic workload, through
``ifci_increments`` with device-resident integrals: every body set of the
40-body uneven chain (seed 2310; eight bodies each of 2-6 orbitals, 160
orbitals) up to 3 bodies (40 + 780 + 9880 = 10,700 CI problems, largest
CAS(6e,18o) with 665,856 determinants), frozen-body Hamiltonians, the exact
blocks of decoupled bodies, batched Davidson to convergence, and the FP64
increments with their sum.  ``--workload c1`` takes the 24-body chain (2324
problems) instead.

Default path ("fp64e"): every sigma contraction FP64-accurate on the FP16
tensor cores (digit slices, exact level sums), all Davidson arithmetic FP64.
The timed steps run without per-kernel profiling; one more step with the
library's per-kernel CUDA-event profiling gives the kernel-class times and
the roofline.  The plain FP64 path and the mixed BF16 path are timed against
FP64E on a seeded sample of the same body sets (``paths_sample``).

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "iFCI increments/s & sigma TFLOP/s, 1 GB300, batched+mixed vs plain FP64 @1µEh"
# dram__bytes_read.sum + dram__bytes_write.sum of one oz_contract_kernel launch
# on CAS(6e,18o) (45.65 + 850.18 MB, 171 x 665,856 G elements; ncu capture of
# `bench.py --case sigma --precision fp64e`); set to None whenever that kernel
# changes until it is captured again
OZ_DRAM_BYTES_PER_G_ELEMENT = (45.652992e6 + 850.175232e6) / (171 * 665856)
UNIT = "increments/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c4", choices=["c4", "c1"],
                    help="c4: 40-body chain (10,700 CI problems); c1: 24-body chain (2324)")
    ap.add_argument("--precision", default="fp64e", choices=["fp64", "fp32", "tf32", "bf16", "fp64e"])
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64 and mixed comparison on the sample")
    ap.add_argument("--compare-fraction", type=float, default=0.05,
                    help="seeded fraction of the 3-body sets in the path comparison (all 1- and 2-body sets)")
    ap.add_argument("--max-order", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--sample-seconds", type=float, default=20.0)
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the autotuner (max_space, det_budget, graph_iters) and use the library defaults")
    ap.add_argument("--autotune-fraction", type=float, default=0.25,
                    help="seeded fraction of the largest body sets in the autotuner's sample")
    ap.add_argument("--dump", default="", help="--case c4: directory for per-set energies")
    ap.add_argument("--det-budget", type=int, default=0,
                    help="determinants per sigma wave (0: library default)")
    ap.add_argument("--case", default="increments", choices=["increments", "sigma", "c2", "c4", "hbci", "fourbody"],
                    help="sigma: time ifci_sigma alone on the workload's largest problem, CAS(6e,18o) "
                         "(the small case for kernel profiles); c2: one CAS(14e,14o) CI per precision; "
                         "c4: 3-body iFCI of the 40-body chain in every precision on all 10,700 sets "
                         "(totals and per-set differences), plus the RDM backward; hbci: the workload's "
                         "expansion with HBCI increments at the paper's thresholds against exact CI; "
                         "fourbody: sigma and Davidson of CAS(8e,24o), the largest 4-body space")
    return ap.parse_args()


# ---------------------------------------------------------------- workload

R_TOL, E_TOL = 1e-6, 1e-10
WORKLOAD_NAMES = {
    "c4": "chain-40-uneven, iFCI to 3 bodies, 10,700 CI problems, max CAS(6e,18o)",
    "c1": "chain-24-uneven, iFCI to 3 bodies, 2324 CI problems, max CAS(6e,18o)",
}


def max_over_ranks(value: float, dist, device) -> float:
    """The slowest rank's time (every rank returns it); ``dist`` None = one rank."""
    if not dist:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(rank: int = 0, name: str = "c4"):
    """Weak scaling: rank r solves its own chain (base seed + r) of the same shape."""
    from synth import chain_24_uneven, chain_40_uneven
    if name == "c1":
        return chain_24_uneven(seed=2308 + rank)
    return chain_40_uneven(seed=2310 + rank)


def cost_of(n: int, m: int):
    """(determinants, sigma contraction FLOPs 2*ndet*npair^2) of one CI problem."""
    nd = math.comb(n, m) ** 2
    npair = n * (n + 1) // 2
    return nd, 2.0 * nd * npair * npair


def subset_sizes(chain, max_order):
    import itertools
    out = []
    for k in range(1, max_order + 1):
        for X in itertools.combinations(range(chain.nbody), k):
            out.append((X, sum(chain.body_sizes[b] for b in X), k))
    return out


def body_coupling(chain):
    """(nbody, nbody) largest integral joining two bodies: |h_pq| and
    max_rs |(pq|rs)| over p in one body and q in the other."""
    V = np.abs(chain.eri_packed())
    vmax = V.max(axis=1)
    off = chain.body_offsets
    nb = chain.nbody
    C = np.zeros((nb, nb))
    for a in range(nb):
        for b in range(a + 1, nb):
            m = 0.0
            for p in range(off[a], off[a + 1]):
                for q in range(off[b], off[b + 1]):
                    P, Q = max(p, q), min(p, q)
                    m = max(m, abs(chain.h[p, q]), vmax[P * (P + 1) // 2 + Q])
            C[a, b] = C[b, a] = m
    return C


def contracted_pairs(X, sizes, C, tau=1e-5):
    """Pairs the FP64E contraction of body set X runs over: the pairs within
    one group of bodies that the library splits apart (integrals joining two
    groups all below tau; its H' has no others).  An accounting estimate from
    the chain's integrals: the library decides on the frozen-body integrals."""
    grp = {b: b for b in X}

    def find(b):
        while grp[b] != b:
            b = grp[b]
        return b
    for i, a in enumerate(X):
        for b in X[i + 1:]:
            if C[a, b] > tau:
                grp[find(a)] = find(b)
    tot = {}
    for b in X:
        r = find(b)
        tot[r] = tot.get(r, 0) + sizes[b]
    return sum(m * (m + 1) // 2 for m in tot.values())


def compare_sample(chain, max_order, fraction, seed=7):
    """Seeded sample of the workload's body sets for the path comparison:
    every set of size < max_order and a fraction of the largest ones."""
    subs = subset_sizes(chain, max_order)
    top = [i for i, (_, _, k) in enumerate(subs) if k == max_order]
    rng = np.random.default_rng(seed)
    pick = {top[j] for j in rng.choice(len(top), max(1, int(round(fraction * len(top)))), replace=False)}
    return [s for i, s in enumerate(subs) if s[2] < max_order or i in pick]


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle baseline

def oracle_conn(n, m):
    """Determinants connected to one determinant (itself included) by H."""
    s1 = m * (n - m)
    s2 = math.comb(m, 2) * math.comb(n - m, 2)
    return 1 + 2 * (s1 + s2) + s1 * s1


def oracle_baseline(chain, max_order, seconds, seed=11, check_large=True, prior_check=None):
    """Times the oracle on a seeded sample of the workload's body sets for about
    ``seconds`` and extrapolates the whole workload's time.  Two regimes, as
    the oracle solves them: dense eigh (ndet <= oracle DENSE_MAX), every such
    set timed or its mean taken; Lanczos (matrix-free Slater–Condon matvecs),
    calibrated on the sampled sets up to 30,000 determinants with the model
    t = a * ndet * (determinants connected per row).  ``check_large``: one
    matvec of the workload's largest space and one of the largest sampled
    set are timed as well; the ratio of their cost per ndet * connection
    rescales the model for the sets above the calibration range (their
    Lanczos iteration count is taken equal to the sampled sets' mean);
    ``prior_check`` reuses the ratio of an earlier call."""
    from oracle import fci
    subs = subset_sizes(chain, max_order)
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(subs))
    fci.lib()                       # build/load before timing
    dense = [i for i in order if math.comb(subs[i][1], subs[i][2]) ** 2 <= fci.DENSE_MAX]
    lanc = [i for i in order if fci.DENSE_MAX < math.comb(subs[i][1], subs[i][2]) ** 2 <= 30000]
    t_dense, n_dense, t_lanc, m_lanc, n_lanc, it_lanc = 0.0, 0, 0.0, 0.0, 0, 0
    for i in dense:
        X, n, k = subs[i]
        t0 = time.perf_counter()
        fci.solve_subsystem(chain, X)
        t_dense += time.perf_counter() - t0
        n_dense += 1
        if t_dense > 0.25 * seconds:
            break
    biggest = None
    for i in lanc:
        X, n, k = subs[i]
        t0 = time.perf_counter()
        r = fci.solve_subsystem(chain, X)
        t_lanc += time.perf_counter() - t0
        m_lanc += math.comb(n, k) ** 2 * oracle_conn(n, k)
        n_lanc += 1
        it_lanc += r.iterations
        if biggest is None or math.comb(n, k) > math.comb(biggest[1], biggest[2]):
            biggest = subs[i]
        if t_lanc > 0.75 * seconds:
            break
    unit = t_lanc / max(m_lanc, 1.0)
    scale_large, check = 1.0, None
    large = max(subs, key=lambda t: math.comb(t[1], t[2]))
    if prior_check:
        scale_large, check = prior_check["matvec_unit_cost_ratio"], prior_check
    elif check_large and biggest is not None and math.comb(large[1], large[2]) ** 2 > 30000:
        def matvec_unit(t):
            X, n, k = t
            H = fci.Hamiltonian(fci.subsystem(chain, X))
            x = np.random.default_rng(3).normal(size=H.ndet)
            t0 = time.perf_counter()
            H.matvec(x)
            return (time.perf_counter() - t0) / (H.ndet * oracle_conn(n, k))
        u_small, u_large = matvec_unit(biggest), matvec_unit(large)
        scale_large = u_large / u_small
        check = {"matvec_unit_cost_ratio": scale_large, "large_set": list(large[0]),
                 "large_ndet": math.comb(large[1], large[2]) ** 2, "calibration_set": list(biggest[0]),
                 "calibration_ndet": math.comb(biggest[1], biggest[2]) ** 2,
                 "sampled_lanczos_iterations_mean": it_lanc / max(n_lanc, 1),
                 "predicted_seconds_largest_set": unit * scale_large * math.comb(large[1], large[2]) ** 2 *
                                                  oracle_conn(large[1], large[2])}
    nd_dense = sum(1 for _, n, k in subs if math.comb(n, k) ** 2 <= fci.DENSE_MAX)
    model_mid = sum(math.comb(n, k) ** 2 * oracle_conn(n, k) for _, n, k in subs
                    if fci.DENSE_MAX < math.comb(n, k) ** 2 <= 30000)
    model_big = sum(math.comb(n, k) ** 2 * oracle_conn(n, k) for _, n, k in subs if math.comb(n, k) ** 2 > 30000)
    t_total = t_dense / max(n_dense, 1) * nd_dense + unit * (model_mid + scale_large * model_big)
    out = {"value": len(subs) / t_total, "unit": UNIT, "cores": fci.num_threads(), "kind": "oracle",
           "sample": (f"{n_dense} dense and {n_lanc} Lanczos body sets (<= 30,000 determinants) of the workload, "
                      f"seeded, timed in {t_dense + t_lanc:.1f} s; whole-workload time extrapolated per regime "
                      f"(dense: mean per set; Lanczos: ndet x connected determinants per row, the cost per unit "
                      f"above 30,000 determinants rescaled by a timed matvec of the largest space), "
                      f"{t_total:.0f} s for {len(subs)} sets")}
    if check:
        out["model_check"] = check
    return out


# ---------------------------------------------------------------- main

def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        steps = args.steps if args.steps is not None else 1
        chain = workload(0, args.workload)
        per = max(3.0, args.sample_seconds / 2)
        prior = None
        for _ in range(args.warmup):
            w = oracle_baseline(chain, args.max_order, per, prior_check=prior)
            prior = w.get("model_check")
        vals = []
        t0 = time.perf_counter()
        for _ in range(steps):
            r = oracle_baseline(chain, args.max_order, per, prior_check=prior)
            prior = r.get("model_check")
            vals.append(r["value"])
        el = time.perf_counter() - t0
        v = float(np.mean(vals))
        line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0, "steps": steps, "warmup": args.warmup,
                "ms_per_step": 1000 * el / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": {"workload": WORKLOAD_NAMES[args.workload], "seed": chain.seed,
                           "sample": "bounded oracle sample per step"},
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                                 "sample": r["sample"], "model_check": r.get("model_check")},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0

    import torch
    import paper_2307_10675_gb300 as ifci

    if args.case == "sigma":
        return sigma_case(args, torch, ifci)
    if args.case == "c2":
        return c2_case(args, torch, ifci)
    if args.case == "c4":
        return c4_case(args, torch, ifci)
    if args.case == "hbci":
        return hbci_case(args, torch, ifci)
    if args.case == "fourbody":
        return fourbody_case(args, torch, ifci)

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    steps = args.steps if args.steps is not None else 3
    warmup = max(3, args.warmup)

    chain = workload(rank, args.workload)
    sysd = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=dev),
                             torch.tensor(chain.eri_packed(), device=dev))
    subs = subset_sizes(chain, args.max_order)
    nsub = len(subs)
    handle = ifci.Handle(0, local)

    tuned = {"max_space": 12, "det_budget": args.det_budget, "graph_iters": 0}
    tune_info = None
    if not args.no_autotune:
        from paper_2307_10675_gb300 import autotune
        # the largest body sets carry nearly all of the cost: the sample is a seeded fraction of them
        sample = [X for X, _, k in compare_sample(chain, args.max_order, args.autotune_fraction, seed=5)
                  if k == args.max_order]
        t0 = time.perf_counter()
        res = autotune.autotune(handle, sysd, sample, args.precision, r_tol=R_TOL, e_tol=E_TOL)
        tuned = res["params"]
        tune_info = {"params": tuned, "sample_sets": len(sample), "seconds": time.perf_counter() - t0,
                     "table": [[c["params"], round(c["seconds"], 4), c["accepted"]] for c in res["table"]]}

    def opts_for(prec):
        return ifci.davidson_opts(prec, r_tol=R_TOL, e_tol=E_TOL, max_iter=300, **tuned)

    stream = torch.cuda.current_stream(dev)
    for _ in range(warmup):
        ifci.ifci_increments(handle, sysd, args.max_order, opts_for(args.precision))
    torch.cuda.synchronize(dev)

    # ---- timed steps: no per-kernel profiling
    clocks = ClockSampler(local)
    clocks.start()
    l0 = handle.launches()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        out = ifci.ifci_increments(handle, sysd, args.max_order, opts_for(args.precision))
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    launches = handle.launches() - l0
    clk = clocks.stop()
    ms_step = max_over_ranks(ev0.elapsed_time(ev1), dist, dev) / steps
    value = world * nsub / (ms_step / 1000.0)

    # ---- one profiled step: kernel-class times (CUDA events around every launch)
    handle.profile_enable(True)
    outp = ifci.ifci_increments(handle, sysd, args.max_order, opts_for(args.precision))
    torch.cuda.synchronize(dev)
    prof = handle.profile_read()
    handle.profile_enable(False)

    # sigma FLOPs of a step: sigma builds per problem x 2 ndet npair^2 (the
    # algorithmic count of the Knowles–Handy contraction), and the same over the pairs the FP64E
    # contraction runs over (a set whose bodies split into decoupled groups
    # contracts only the pairs within each group: its H' has no others)
    its = outp["iters"]
    Cb = body_coupling(chain)
    flops_full = 0.0
    flops_step = 0.0
    exec_step = 0.0
    gelems_step = 0.0
    for (X, n, k), it in zip(subs, its):
        nd, fl = cost_of(n, k)
        npc = contracted_pairs(X, chain.body_sizes, Cb) if k > 1 else n * (n + 1) // 2
        it = float(it)
        flops_full += it * fl
        flops_step += it * 2.0 * nd * npc * npc
        exec_step += it * executed_oz_flops(n, k, npc)
        gelems_step += it * nd * npc
    sig_ms = sum(prof[k][0] for k in ("gather", "contract", "contract_hi", "scatter"))
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    bf = peaks.get("bf16_tflops_sustained")
    bf_src = "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)" if bf else \
        "fallback 1700 TFLOP/s sustained (of fallback)"
    bf = bf or 1700.0
    fp64_peak_tf, fp64_how = _dgemm_peak(dev)
    if args.precision == "fp64":
        c_ms = prof["contract"][0]
        ach = flops_step / (c_ms / 1000.0) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": fp64_peak_tf, "unit": "TFLOP/s",
                "frac": ach / fp64_peak_tf, "traffic": None, "kernel": "contract_simt_kernel<double>",
                "peak_source": fp64_how}
        dtype = "f64"
    elif args.precision == "fp64e":
        c_ms = prof["contract_hi"][0]
        nlaunch = max(1, prof["contract_hi"][1])
        ach = flops_step / (c_ms / 1000.0) / 1e12
        roof = {"bound": "tensor", "achieved": ach, "peak": bf, "unit": "TFLOP/s", "frac": ach / bf,
                "traffic": (OZ_DRAM_BYTES_PER_G_ELEMENT * gelems_step / nlaunch
                            if OZ_DRAM_BYTES_PER_G_ELEMENT else None),
                "kernel": "oz_contract_kernel", "peak_source": bf_src,
                "achieved_note": "FP64-equivalent FLOPs of the contraction (2 ndet npc^2 per sigma, npc the pairs "
                                 "contracted: all pairs, or the intra-group pairs of a set of decoupled body "
                                 "groups) / event-timed oz_contract_kernel time of one profiled step",
                "achieved_full_npair": flops_full / (c_ms / 1000.0) / 1e12,
                "full_npair_note": "2 ndet npair^2 per sigma over every pair (the contraction without the "
                                   "block structure of decoupled groups)",
                "launches_per_step": nlaunch,
                "emulation": {"fp16_products_per_fp64_product": 15, "ceiling": bf / 15.0,
                              "frac_of_ceiling": ach / (bf / 15.0),
                              "executed_fp16_tflops": exec_step / (c_ms / 1000.0) / 1e12}}
        dtype = "f64 (FP16 tensor-core emulation)"
    else:
        lo_ms = prof["contract"][0]
        hi_ms = prof["contract_hi"][0]
        ach = flops_step / ((lo_ms + hi_ms) / 1000.0) / 1e12
        roof = {"bound": "tensor", "achieved": ach, "peak": bf, "unit": "TFLOP/s", "frac": ach / bf,
                "traffic": None, "kernel": "tc_contract_bf16_kernel + oz_contract_kernel", "peak_source": bf_src}
        dtype = args.precision + "+f64"

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": dtype, "data": "synthetic",
        "config": {"workload": WORKLOAD_NAMES[args.workload], "seed": chain.seed, "bodies": chain.nbody,
                   "orbitals": chain.norb, "max_order": args.max_order, "precision": args.precision,
                   "davidson": dict(r_tol=R_TOL, e_tol=E_TOL, decouple_tol=1e-5, **tuned),
                   "l2": "inputs larger than L2: Davidson vectors of one step are tens of GB",
                   "parallelism": f"{world} independent chains (one per GPU)"},
        "roofline": roof,
        "autotune": tune_info,
        "gpu_launches": int(launches),
        "clocks": clk,
        "e_total": out["e_total"],
        "profiled_step": {"ms": sum(v[0] for v in prof.values()),
                          "kernel_ms": {k: v[0] for k, v in prof.items()},
                          "sigma_tflops": flops_step / (sig_ms / 1000.0) / 1e12 if sig_ms > 0 else None,
                          "class_rooflines": class_rooflines(subs, its, {k: v[0] for k, v in prof.items()}, 1,
                                                             float(peaks.get("hbm_gbs", 6800.0)), fp64_peak_tf),
                          "e_total": outp["e_total"]},
    }
    if not args.no_compare and world == 1:
        line["paths_sample"] = paths_sample(ifci, torch, handle, chain, sysd, args, dev)
    if not args.no_e2e:
        line["e2e"] = _e2e(ifci, handle, chain, args.max_order, opts_for(args.precision), world, nsub, dist, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_baseline(workload(0, args.workload), args.max_order, args.sample_seconds)
    handle.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def paths_sample(ifci, torch, handle, chain, sysd, args, dev):
    """FP64E, plain FP64 and mixed BF16 and TF32 (+FP64E restarts) on the same seeded
    sample of body sets (their frozen-body CI problems through
    ifci_davidson_batched, one batch per path): increments/s of each path and
    the largest energy difference from the plain FP64 path."""
    sample = compare_sample(chain, args.max_order, args.compare_fraction)
    probs = []
    for X, n, k in sample:
        h1, eri, ec = ifci.ifci_frozen_core(handle, sysd, X)
        probs.append(ifci.CIProblem(n, k, h1, eri, ec))
    res = {}
    for name, prec, hi in (("fp64e", "fp64e", "fp64e"), ("fp64", "fp64", "fp64"), ("bf16_mixed", "bf16", "fp64e"),
                           ("tf32_mixed", "tf32", "fp64e")):
        o = ifci.davidson_opts(prec, hi_precision=hi, r_tol=R_TOL, e_tol=E_TOL, max_iter=300)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        e, it, st = ifci.ifci_davidson_batched(handle, probs, o, allow_unconverged=True)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        res[name] = {"increments_per_s": len(probs) / wall, "seconds": wall, "iters_mean": float(np.mean(it)),
                     "unconverged": int(np.sum(st != 0)), "_e": e}
    e64 = res["fp64"]["_e"]
    for name in res:
        d = res[name].pop("_e") - e64
        res[name]["max_abs_minus_fp64_eh"] = float(np.max(np.abs(d)))
        res[name]["speedup_vs_fp64"] = res[name]["increments_per_s"] / res["fp64"]["increments_per_s"]
    nk = [sum(1 for s in sample if s[2] == k) for k in range(1, args.max_order + 1)]
    return {"sample": f"{len(sample)} body sets ({' + '.join(map(str, nk))} of sizes 1..{args.max_order}; "
                      f"a seeded {args.compare_fraction:.0%} of the largest), each path timed once, set-up included",
            "r_tol": R_TOL, "runs": res}


def class_rooflines(subs, iters, kernel_ms, steps, hbm_gbs, fp64_tflops, max_space=12):
    """Achieved rates of the per-step kernel classes other than the contraction,
    from their CUDA-event times and algorithmic work:

    * scatter (+ quantise, symmetrisation): per determinant and sigma, the G
      values its alpha and beta lists read (2 nexc x 8 B), the quantised
      copy read and written (16 B) and sigma read and written (16 B); HBM-bound.
    * Davidson vector kernels: per determinant and iteration ~(5k + 8) x 8 B
      and ~9k FP64 FMAs at an average subspace size k = (max_space + 4) / 2
      (thick restarts keep 4 vectors); bound by the FP64 ALU on this GPU."""
    sbytes = 0.0
    vbytes = 0.0
    vflops = 0.0
    kbar = (max_space + 4) / 2.0
    for (X, n, k), it in zip(subs, iters):
        nd = math.comb(n, k) ** 2
        nexc = k * (n - k + 1)
        it = float(it)
        sbytes += it * nd * (16.0 * nexc + 32.0)
        vbytes += it * nd * (5.0 * kbar + 8.0) * 8.0
        vflops += it * nd * 9.0 * kbar * 2.0
    out = {}
    sc_ms = (kernel_ms.get("scatter", 0.0) + kernel_ms.get("gather", 0.0)) / steps
    if sc_ms > 0:
        gbs = sbytes / (sc_ms / 1000.0) / 1e9
        out["scatter"] = {"bound": "hbm", "achieved": gbs, "peak": hbm_gbs, "unit": "GB/s", "frac": gbs / hbm_gbs}
    v_ms = kernel_ms.get("vector", 0.0) / steps
    if v_ms > 0:
        tf = vflops / (v_ms / 1000.0) / 1e12
        gbs = vbytes / (v_ms / 1000.0) / 1e9
        out["davidson_vectors"] = {"bound": "fp64_alu", "achieved": tf, "peak": fp64_tflops, "unit": "TFLOP/s",
                                   "frac": tf / fp64_tflops if fp64_tflops else None,
                                   "hbm_gbs": gbs, "hbm_frac": gbs / hbm_gbs,
                                   "note": "estimated k = (max_space + 4) / 2 for the subspace size"}
    return out


def sigma_case(args, torch, ifci):
    """One sigma = H c of the workload's largest CI problem (three 6-orbital
    bodies: CAS(6e,18o), 665,856 determinants, 171 pairs) on a spin-flip
    symmetric vector, repeated; the kernel-level small case.  Prints one JSON
    line with the per-call time."""
    from synth import chain_24_uneven, random_ci_vector
    dev = torch.device("cuda", 0)
    chain = chain_24_uneven()
    sysd = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=dev),
                             torch.tensor(chain.eri_packed(), device=dev))
    X = tuple(b for b, sz in enumerate(chain.body_sizes) if sz == 6)[:3]
    n, m = 18, 3
    steps = args.steps if args.steps is not None else 20
    prec = ifci.PRECISIONS[args.precision]
    with ifci.Handle(0, 0) as h:
        h1, eri, _ = ifci.ifci_frozen_core(h, sysd, X)
        t = ifci.ifci_build_strings(h, n, m)
        nstr = math.comb(n, m)
        c = torch.tensor(random_ci_vector(nstr, nstr, seed=1), device=dev).reshape(nstr, nstr)
        c = (c + c.T).reshape(-1).contiguous()     # spin-flip symmetric, as every Davidson vector
        c /= c.norm()
        for _ in range(max(3, args.warmup)):
            ifci.ifci_sigma(h, t, h1, eri, c, precision=prec, spin_symmetric=True)
        torch.cuda.synchronize(dev)
        h.profile_enable(True)
        l0 = h.launches()
        stream = torch.cuda.current_stream(dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            ifci.ifci_sigma(h, t, h1, eri, c, precision=prec, spin_symmetric=True)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        prof = h.profile_read()
        h.profile_enable(False)
        launches = h.launches() - l0
    ms = ev0.elapsed_time(ev1) / steps
    nd, fl = cost_of(n, m)
    line = {"case": "sigma", "workload": "CAS(6e,18o) of chain-24-uneven (bodies %s), 665,856 determinants" % (X,),
            "precision": args.precision, "steps": steps, "ms_per_sigma": ms,
            "algorithmic_tflops": fl / (ms / 1000.0) / 1e12,
            "kernel_ms_per_sigma": {k: v[0] / steps for k, v in prof.items()},
            "gpu_launches": int(launches)}
    if args.precision == "fp64e":
        c_ms = prof["contract_hi"][0] / steps
        line["contract_hi_tflops_algorithmic"] = fl / (c_ms / 1000.0) / 1e12
        line["contract_hi_executed_fp16_tflops"] = executed_oz_flops(n, m) / (c_ms / 1000.0) / 1e12
    print(json.dumps(line), flush=True)
    return 0


def c2_case(args, torch, ifci):
    """One large CI: CAS(14e,14o) of the seven-body chain (seed 2309), 11,778,624
    determinants, lowest singlet, solved once per sigma precision (after one
    untimed warm-up solve each); prints energies, their differences from the
    FP64 path, iterations, wall time and sigma kernel time per precision."""
    from synth import chain_7x2
    dev = torch.device("cuda", 0)
    chain = chain_7x2()
    X = tuple(range(7))
    runs = [("fp64", "fp64", "fp64"), ("fp32+fp64", "fp32", "fp64"), ("tf32+fp64", "tf32", "fp64"),
            ("bf16+fp64", "bf16", "fp64"), ("tf32+fp64e", "tf32", "fp64e"), ("bf16+fp64e", "bf16", "fp64e"),
            ("fp64e", "fp64e", "fp64e")]
    res = {}
    with ifci.Handle(0, 0) as h:
        sysd = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=dev),
                                 torch.tensor(chain.eri_packed(), device=dev))
        h1, eri, ecore = ifci.ifci_frozen_core(h, sysd, X)
        for name, prec, hi in runs:
            opts = ifci.davidson_opts(prec, hi_precision=hi, r_tol=1e-7, e_tol=1e-11, max_iter=200)
            prob = ifci.CIProblem(14, 7, h1, eri, ecore)
            ifci.ifci_davidson_batched(h, [prob], opts)
            torch.cuda.synchronize(dev)
            h.profile_enable(True)
            t0 = time.perf_counter()
            e, it, st = ifci.ifci_davidson_batched(h, [prob], opts)
            torch.cuda.synchronize(dev)
            wall = time.perf_counter() - t0
            prof = h.profile_read()
            h.profile_enable(False)
            res[name] = {"energy": float(e[0]), "iters": int(it[0]), "status": int(st[0]), "seconds": wall,
                         "sigma_ms": {k: v[0] for k, v in prof.items() if k != "vector" and v[0] > 0},
                         "vector_ms": prof["vector"][0]}
    e64 = res["fp64"]["energy"]
    for name in res:
        res[name]["minus_fp64_eh"] = res[name]["energy"] - e64
    nd, fl = cost_of(14, 7)
    print(json.dumps({"case": "c2", "workload": "CAS(14e,14o) of chain-7x2 (seed 2309), 11,778,624 determinants",
                      "sigma_flops": fl, "davidson": {"r_tol": 1e-7, "e_tol": 1e-11}, "runs": res}), flush=True)
    return 0


def c4_case(args, torch, ifci):
    """Production-scale 3-body iFCI of the 40-body uneven chain (seed 2310):
    10,700 body sets up to CAS(6e,18o), one timed ifci_increments per path
    (FP64E, mixed BF16 + FP64E, plain FP64; no warm-up: each run builds its
    own tables and plans), then the RDM backward of the FP64E run.  Prints
    E_total per path, its difference from the plain FP64 path, the largest
    per-set energy difference, and increments/s; with ``--dump DIR`` the
    per-set energies go to DIR/c4_<path>.npz."""
    from synth import chain_40_uneven
    dev = torch.device("cuda", 0)
    chain = chain_40_uneven()
    sysd = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=dev),
                             torch.tensor(chain.eri_packed(), device=dev))
    nsub = len(subset_sizes(chain, 3))
    paths = [("fp64e", "fp64e", "fp64e"), ("bf16+fp64e", "bf16", "fp64e"), ("tf32+fp64e", "tf32", "fp64e"),
             ("fp64", "fp64", "fp64")]
    res, ex = {}, {}
    with ifci.Handle(0, 0) as h:
        for name, prec, hi in paths:
            opts = ifci.davidson_opts(prec, hi_precision=hi, r_tol=R_TOL, e_tol=E_TOL, max_iter=300)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            out = ifci.ifci_increments(h, sysd, 3, opts, allow_unconverged=True)
            torch.cuda.synchronize(dev)
            wall = time.perf_counter() - t0
            ex[name] = out["e_x"]
            res[name] = {"e_total": out["e_total"], "seconds": wall, "increments_per_s": nsub / wall,
                         "unconverged": int(np.sum(out["status"] != 0)), "iters_mean": float(np.mean(out["iters"]))}
            if args.dump:
                os.makedirs(args.dump, exist_ok=True)
                np.savez(os.path.join(args.dump, f"c4_{name}.npz"), e_x=out["e_x"], iters=out["iters"],
                         status=out["status"], e0=out["e0"], e_total=out["e_total"])
            if name == "fp64e":
                t0 = time.perf_counter()
                dh, dV = ifci.ifci_rdm_backward(h, sysd, 3, 1.0, opts)
                torch.cuda.synchronize(dev)
                res[name]["rdm_backward_seconds"] = time.perf_counter() - t0
                res[name]["euler_identity_minus_e_total"] = float(
                    (torch.sum(sysd.h * dh) + torch.sum(sysd.eri * dV)).item() - out["e_total"])
                del dh, dV
    for name in res:
        res[name]["minus_fp64_eh"] = res[name]["e_total"] - res["fp64"]["e_total"]
        res[name]["max_set_minus_fp64_eh"] = float(np.max(np.abs(ex[name] - ex["fp64"])))
        res[name]["speedup_vs_fp64"] = res[name]["increments_per_s"] / res["fp64"]["increments_per_s"]
    print(json.dumps({"case": "c4", "workload": WORKLOAD_NAMES["c4"], "davidson": {"r_tol": R_TOL, "e_tol": E_TOL},
                      "runs": res}), flush=True)
    return 0


def hbci_case(args, torch, ifci):
    """The workload's expansion (default 40-body chain to 3 bodies) with every
    E_X from HBCI at the paper's thresholds (eps1 = 1 mHa, eps2 = 1 µHa) and
    with exact CI (FP64E), each timed once after one untimed run; prints
    increments/s of both, the totals and the largest per-set difference."""
    dev = torch.device("cuda", 0)
    chain = workload(0, args.workload)
    res = {}
    with ifci.Handle(0, 0) as h:
        sysd = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=dev),
                                 torch.tensor(chain.eri_packed(), device=dev))
        for name, extra in (("fci", {}), ("hbci", {"hbci_max_rounds": 50, "hbci_eps1": 1e-3, "hbci_eps2": 1e-6})):
            opts = ifci.davidson_opts("fp64e", r_tol=R_TOL, e_tol=E_TOL, max_iter=300, **extra)
            ifci.ifci_increments(h, sysd, args.max_order, opts)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            out = ifci.ifci_increments(h, sysd, args.max_order, opts)
            torch.cuda.synchronize(dev)
            res[name] = (time.perf_counter() - t0, out)
    nsub = len(res["fci"][1]["eps"])
    d = res["hbci"][1]["e_x"] - res["fci"][1]["e_x"]
    line = {"case": "hbci", "workload": WORKLOAD_NAMES[args.workload], "eps1": 1e-3, "eps2": 1e-6,
            "fci": {"seconds": res["fci"][0], "increments_per_s": nsub / res["fci"][0],
                    "e_total": res["fci"][1]["e_total"]},
            "hbci": {"seconds": res["hbci"][0], "increments_per_s": nsub / res["hbci"][0],
                     "e_total": res["hbci"][1]["e_total"],
                     "mean_variational_steps": float(np.mean(res["hbci"][1]["iters"]))},
            "e_total_hbci_minus_fci": res["hbci"][1]["e_total"] - res["fci"][1]["e_total"],
            "max_abs_e_x_difference": float(np.max(np.abs(d))),
            "largest_e_x_differences": [[list(ifci.body_subsets(chain.nbody, args.max_order)[i]), float(d[i])]
                                        for i in np.argsort(-np.abs(d))[:5]],
            "min_e_x_difference": float(np.min(d)),
            "note": "HBCI's variational step runs the FCI sigma over the whole space (selection kept by a mask): "
                    "it reproduces the paper's approximation, not its savings"}
    print(json.dumps(line), flush=True)
    return 0


def fourbody_case(args, torch, ifci):
    """CAS(8e,24o) of the 24-body chain (four 6-orbital bodies; 10,626 strings,
    112,911,876 determinants, 300 pairs): the FP64E sigma (K chunks and row
    slabs of G) timed over a few calls, then one Davidson solve of the space."""
    from synth import chain_24_uneven, random_ci_vector
    dev = torch.device("cuda", 0)
    chain = chain_24_uneven()
    X = tuple(b for b, sz in enumerate(chain.body_sizes) if sz == 6)[:4]
    n, m = 24, 4
    steps = args.steps if args.steps is not None else 3
    with ifci.Handle(0, 0) as h:
        sysd = ifci.SystemArrays(chain.body_offsets, torch.tensor(chain.h, device=dev),
                                 torch.tensor(chain.eri_packed(), device=dev))
        h1, eri, ecore = ifci.ifci_frozen_core(h, sysd, X)
        t = ifci.ifci_build_strings(h, n, m)
        nstr = math.comb(n, m)
        c = torch.tensor(random_ci_vector(nstr, nstr, seed=1, symmetric=True), device=dev).reshape(-1)
        ifci.ifci_sigma(h, t, h1, eri, c, precision=ifci.IFCI_FP64E, spin_symmetric=True)
        torch.cuda.synchronize(dev)
        h.profile_enable(True)
        stream = torch.cuda.current_stream(dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            ifci.ifci_sigma(h, t, h1, eri, c, precision=ifci.IFCI_FP64E, spin_symmetric=True)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        prof = h.profile_read()
        h.profile_enable(False)
        ms = ev0.elapsed_time(ev1) / steps
        del c
        prob = ifci.CIProblem(n, m, h1, eri, ecore)
        t0 = time.perf_counter()
        e, it, st = ifci.ifci_davidson_batched(h, [prob], ifci.davidson_opts("fp64e", r_tol=R_TOL, e_tol=E_TOL,
                                                                             max_iter=300))
        torch.cuda.synchronize(dev)
        dav_s = time.perf_counter() - t0
    nd, fl = cost_of(n, m)
    c_ms = prof["contract_hi"][0] / steps
    line = {"case": "fourbody", "workload": "CAS(8e,24o) of chain-24-uneven (bodies %s), %d determinants" % (X, nd),
            "sigma_ms": ms, "sigma_algorithmic_tflops": fl / (ms / 1000.0) / 1e12,
            "contract_hi_ms": c_ms, "contract_hi_tflops_algorithmic": fl / (c_ms / 1000.0) / 1e12,
            "kernel_ms_per_sigma": {k: v[0] / steps for k, v in prof.items()},
            "davidson": {"seconds": dav_s, "energy": float(e[0]), "sigma_builds": int(it[0]), "status": int(st[0])}}
    print(json.dumps(line), flush=True)
    return 0


def executed_oz_flops(n: int, m: int, npc: int = 0) -> float:
    """FP16 MMA FLOPs the FP64-emulating contraction issues for one sigma of one
    problem: row-aligned tiles of 128 determinants x 96-pair output tiles x
    the contracted pairs (npc, default all) rounded to 16, 15 slice products."""
    nstr = math.comb(n, m)
    np_ = npc if npc else n * (n + 1) // 2
    if nstr >= 128:
        tiles = nstr * ((nstr + 127) // 128)
    else:
        r = min(16, 128 // nstr)
        tiles = (nstr + r - 1) // r
    kpad = (np_ + 15) // 16 * 16
    npad = 0
    for n0 in range(0, np_, 96):
        npad += (min(96, np_ - n0) + 15) // 16 * 16
    return 15.0 * 2.0 * tiles * 128 * npad * kpad


def _dgemm_peak(dev):
    """cuBLAS DGEMM throughput on this GPU (best of 5, 4096^3) as the FP64 peak."""
    import torch
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    for _ in range(2):
        torch.matmul(a, b)
    torch.cuda.synchronize(dev)
    best = 1e9
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize(dev)
        best = min(best, e0.elapsed_time(e1))
    tf = 2.0 * n ** 3 / (best / 1000.0) / 1e12
    return tf, "measured in this run: cuBLAS DGEMM 4096^3 (torch.matmul float64), best of 5"


def _e2e(ifci, handle, chain, max_order, opts, world, nsub, dist, dev):
    """Same metric through the public call with host buffers: the integrals are
    copied in from pinned host memory and all results come back inside the call."""
    import torch
    h_pin = torch.tensor(chain.h).pin_memory()
    v_pin = torch.tensor(chain.eri_packed()).pin_memory()
    sysh = ifci.SystemArrays(chain.body_offsets, h_pin.numpy(), v_pin.numpy())
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    out = ifci.ifci_increments(handle, sysh, max_order, opts)
    torch.cuda.synchronize(dev)
    el = time.perf_counter() - t0
    el = max_over_ranks(el, dist, dev)
    h2d = h_pin.numel() * 8 + v_pin.numel() * 8
    d2h = (2 * nsub + 2) * 8 + nsub * 4
    return {"value": world * nsub / el, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "e_total": out["e_total"]}


if __name__ == "__main__":
    sys.exit(main())
