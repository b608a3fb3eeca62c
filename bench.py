#!/usr/bin/env python3
"""Benchmark of the EPSR hot path on GB300: Monte Carlo moves/s and g(r) pair distances/s
at 100k atoms.

Workload (one step): the paper-scale water box (33,333 rigid 3-site molecules, 99,999
atoms, 0.1 atoms/A^3, seed 1): 10,000 Metropolis moves (each with dU of the moved
molecule against all atoms), then one full all-pair partial histogram g_ab(r) (333 x
0.03 A bins) and S(Q) on 1000 Q points by Eq. (1). This is one "g(r)/S(Q) every 10,000
moves" cycle of the 1e6-move run. Inputs are synthetic (seeded random sequential
addition), resident in HBM when the timed region starts.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU (torchrun): every rank advances its own replica box (seed 1 + rank), no
data-path collective (weak scaling); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MOVES_PER_STEP = 10_000
METRIC = "MC moves/s and g(r) pair-distances/s at 100k atoms on 1 GB300, % of roofline"
OPS_PER_PAIR_EVAL = 26     # algorithmic FP32+INT32 lane operations per (moved atom, partner, position)
OPS_PER_PAIR_DIST = 12     # algorithmic INT32 lane operations per g(r) pair distance
LANES_PER_SM = 128


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_name(system, moves: int) -> str:
    m = int(system.mol_start[1] - system.mol_start[0])
    kind = ((f"{system.n_mol} flexible {m}-site molecules" if getattr(system, "flexible", False)
             else f"{system.n_mol} rigid {m}-site molecules") if m > 1 else "single-atom moves")
    cut = f", LJ cut at {system.r_lj:g} A" if getattr(system, "r_lj", 0.0) > 0 else ""
    return (f"paper-scale {system.name}, {system.n_atoms:,} atoms ({kind}{cut}), {moves:,} MC moves + full "
            f"g_ab(r) ({system.n_bins} x {system.dr:g} A) + S(Q) ({len(system.Q)} Q) per step")


# ------------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ------------------------------------------------------------------------------------------

def oracle_full_step(system, moves_per_step: int = MOVES_PER_STEP, seed: int = 1):
    """The FP64 oracle on one whole step of the workload, measured, not extrapolated: the
    Monte Carlo chain of `moves_per_step` moves on one host core (a Markov chain is
    sequential), then one full all-pair histogram on every host core (the oracle's OpenMP
    pair scan), then S(Q). Returns a dict of the measured times and rates."""
    import oracle
    ob = oracle.Box(system)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    ob.mc_sweep(moves_per_step, seed=seed, move0=0)
    t_mc = time.perf_counter() - t0
    t0 = time.perf_counter()
    H = ob.histogram(threads=threads)
    t_gr = time.perf_counter() - t0
    g = ob.normalize_g(H)
    t0 = time.perf_counter()
    oracle.sq_of_box(ob, g)
    t_sq = time.perf_counter() - t0
    N = system.n_atoms
    pairs = N * (N - 1) // 2
    # beside it: the pair scan on one core, over the first rows (about 10 s of work)
    rows = max(1, min(N - 1, int(3.0e8 / N)))
    t0 = time.perf_counter()
    ob.histogram(0, rows)
    t_rows = time.perf_counter() - t0
    pairs_rows = rows * (N - 1) - rows * (rows - 1) // 2
    return {"t_mc": t_mc, "t_gr": t_gr, "t_sq": t_sq, "threads": threads, "pairs": pairs,
            "pairs_1core_per_s": pairs_rows / t_rows, "rows_1core": rows,
            "pairs_1core_sample": pairs_rows}


def oracle_sample_step(ob, system, frac: float, move0: int, seed: int = 1):
    """One step of the reference arm: the fraction `frac` of the step's work done by the
    oracle on one host core -- frac x 10,000 moves of the chain, the first rows of the pair
    scan holding frac x N(N-1)/2 pair distances, and one S(Q). Returns (seconds, moves, pairs)."""
    import oracle
    N = system.n_atoms
    moves = max(1, int(round(frac * MOVES_PER_STEP)))
    target = frac * (N * (N - 1) // 2)
    rows, pairs = 0, 0
    while rows < N - 1 and pairs < target:
        pairs += N - 1 - rows
        rows += 1
    t0 = time.perf_counter()
    ob.mc_sweep(moves, seed=seed, move0=move0)
    H = ob.histogram(0, rows)
    oracle.sq_of_box(ob, ob.normalize_g(H))
    return time.perf_counter() - t0, moves, pairs


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on one host core. Each step is the
    fraction 1/100 of the benchmarked step (100 moves, 5.0e7 of the 5.0e9 pair distances, one
    S(Q)), timed as it runs; the rate of that sample is the line's value and its measured
    time the line's ms_per_step, so the steps printed are the steps that ran."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1904_08756_gb300 import synth
    system = synth.paper_water()
    ob = oracle.Box(system)
    frac = 0.01
    times, moves_done, pairs_done = [], 0, 0
    for i in range(args.warmup + args.steps):
        t, m, p = oracle_sample_step(ob, system, frac, move0=i * 1000)
        if i >= args.warmup:
            times.append(t)
            moves_done += m
            pairs_done += p
    t = sum(times)
    v = moves_done / t
    N = system.n_atoms
    desc = (f"each step 1/100 of the benchmarked step, measured: {moves_done // args.steps} moves of "
            f"the chain + the first rows of the pair scan ({pairs_done / args.steps:.3g} of "
            f"{N * (N - 1) // 2:.3g} pair distances) + one S(Q); value = moves done / time taken")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "moves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(system, MOVES_PER_STEP),
                       "n_atoms": system.n_atoms, "moves_per_step": MOVES_PER_STEP},
            "cpu_baseline": {"value": v, "unit": "moves/s", "cores": 1, "kind": "oracle",
                             "sample": desc},
            "sample_fraction_of_step": frac,
            "e2e": {"value": v, "unit": "moves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# Replicas: 64 boxes of uneven size advanced together, each step captured as a CUDA graph
# ------------------------------------------------------------------------------------------

def time_sq_modes(Q, g, ws, flats, S_like, nb, stream, flush, reps: int = 20, autotune: bool = True):
    """S(Q) of the same resident g(r) columns in every contraction mode: mean time of one
    epsr_sq_exec (CUDA events on the launching stream, L2 flushed before each, the GPU kept
    busy ahead of the events so that no host latency falls between them) and the largest
    difference from the FP32 mode's result."""
    import torch
    from paper_1904_08756_gb300 import epsr
    peaks, peak_kind = measured_peaks()
    names = {epsr.SQ_FP32: "fp32", epsr.SQ_TF32X3: "tf32x3", epsr.SQ_BF16X3: "bf16x3",
             epsr.SQ_BF16X6: "bf16x6"}
    products = {epsr.SQ_TF32X3: 3, epsr.SQ_BF16X3: 3, epsr.SQ_BF16X6: 6}
    n_q, n_bins, n_cols = len(Q), g.shape[1], g.shape[0]
    out = {}
    S_fp32 = None
    with torch.cuda.stream(stream):
        for mode, name in names.items():
            plan = epsr.SqPlan(Q, n_bins, 0.02, mode, max_cols=n_cols)
            S = torch.zeros_like(S_like)
            if autotune:
                plan.epsr_sq_plan_autotune(g, ws, 3, flats, None, S)
            for _ in range(3):
                plan.epsr_sq_exec(g, ws, 3, flats, None, S, stream=stream.cuda_stream)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(reps)]
            for a, b in evs:
                # a device-side delay ahead of the flush keeps the GPU behind the host, so the
                # events bracket the contraction alone and not the host's enqueue latency
                torch.cuda._sleep(400_000)
                flush.fill_(1.0)
                a.record(stream)
                plan.epsr_sq_exec(g, ws, 3, flats, None, S, stream=stream.cuda_stream)
                b.record(stream)
            stream.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in evs) / reps
            flops = 2.0 * n_q * n_bins * n_cols
            if mode == epsr.SQ_FP32:
                S_fp32 = S.clone()
            rec = {"ms": ms, "algorithmic_tflops": flops / (ms * 1e-3) / 1e12,
                   "max_abs_diff_vs_fp32": float((S - S_fp32).abs().max())}
            if mode != epsr.SQ_FP32:
                rec["tiles"] = dict(zip(("cols_per_cta", "k_split"), plan.epsr_sq_plan_get_tiles(n_cols, 3)))
            if mode in products and peaks.get("bf16_tflops"):
                issued = flops * products[mode] / (ms * 1e-3) / 1e12
                peak = peaks["bf16_tflops"] * (0.5 if mode == epsr.SQ_TF32X3 else 1.0)
                rec.update({"tensor_tflops_issued": issued, "tensor_peak_tflops": peak,
                            "tensor_frac": issued / peak,
                            "peak_source": f"{peak_kind} bf16 burst" + (" x 1/2 (tf32 nominal ratio)"
                                                                   if mode == epsr.SQ_TF32X3 else "")})
            out[name] = rec
            plan.close()
    return out


# the paper's Table 1: simulation speed of its GPU code (V100), steps/s, by atom count
PAPER_TABLE1_GPU = {3000: 1562.0, 30000: 9507.0, 100000: 12412.0, 250000: 10189.0,
                    1200000: 3917.0, 3000000: 1963.0, 10000000: 757.0, 30000000: 340.3}


def run_sweep(args):
    """Monte Carlo moves/s of rigid water at the atom counts of the paper's Table 1 (3e3 to
    3e7 atoms, lattice-placed boxes at 0.1 atoms/A^3), each timed over about half a second of
    sweeps after a warm-up; boxes whose partner slices exceed shared memory run the
    global-memory variant of the sweep."""
    import torch
    from paper_1904_08756_gb300 import build, epsr, synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    if not os.path.exists(epsr.LIB_PATH):
        build.build()
    sizes = sorted(PAPER_TABLE1_GPU)
    if args.max_atoms:
        sizes = [n for n in sizes if n <= args.max_atoms]
    rows = []
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    with ClockSampler(0) as clk:
        for n_atoms in sizes:
            s = synth.water_lattice(n_atoms // 3, seed=11)
            box = epsr.Box(s)
            move0 = 0
            t0 = time.perf_counter()
            box.epsr_mc_sweep(512, 5, move0)
            move0 += 512
            est = 512 / max(time.perf_counter() - t0, 1e-6)
            n_timed = int(min(200000, max(1024, 0.5 * est)))
            for _ in range(args.warmup):
                box.epsr_mc_sweep(256, 5, move0)
                move0 += 256
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            stats = box.epsr_mc_sweep(n_timed, 5, move0)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            mps = n_timed / (ms * 1e-3)
            rows.append({"atoms": s.n_atoms, "moves": n_timed, "ms": ms, "moves_per_s": mps,
                         "pair_evals_per_s": mps * 6 * (s.n_atoms - 3),
                         "acceptance": stats[0][1] / max(1, stats[0][0]),
                         "paper_v100_steps_per_s": PAPER_TABLE1_GPU[n_atoms],
                         "ratio_to_paper": mps / PAPER_TABLE1_GPU[n_atoms]})
            box.close()
            del s
    ref = next((r for r in rows if r["atoms"] == 99999), rows[-1])
    line = {"metric": METRIC + " (atom-count sweep, MC only)", "value": ref["moves_per_s"],
            "unit": "moves/s", "n_gpus": 1, "steps": len(rows), "warmup": args.warmup,
            "ms_per_step": ref["ms"], "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "fp32+int64", "data": "synthetic",
            "config": {"workload": "rigid 3-site water on a simple cubic lattice of molecules, "
                                   "0.1 atoms/A^3, at the atom counts of the paper's Table 1; "
                                   "value = the 99,999-atom box",
                       "l2": "flushed before each timed sweep"},
            "sweep": rows, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_smeared(args):
    """The differentiable form on the 99,999-atom water box (seed 4): chi^2 of the smeared
    g(r) against a target S(Q) (a seed-5 box plus N(0, 0.005^2) noise) and its gradients with
    respect to every coordinate and the EP coefficients, timed forward and backward, beside
    the exact histogram of the same box."""
    import torch
    from paper_1904_08756_gb300 import build, epsr, synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    if not os.path.exists(epsr.LIB_PATH):
        build.build()
    s = synth.paper_water(seed=4)
    t = synth.paper_water(seed=5)
    sigma, P = 0.05, 3
    box, tbox = epsr.Box(s), epsr.Box(t)
    w_cols, flat = box.epsr_sq_weights(0)
    rho = s.n_atoms / s.L ** 3
    W = np.asarray(w_cols) / (4.0 * np.pi * rho)
    plan = epsr.SqPlan(s.Q, s.n_bins, s.dr, epsr.SQ_FP32, max_cols=P)
    H = torch.zeros(tbox.hist_len, dtype=torch.int64, device=dev)
    g = torch.zeros(tbox.hist_len, dtype=torch.float32, device=dev)
    tbox.epsr_partial_gr(H, g, 1)
    St = torch.zeros((1, len(s.Q)), dtype=torch.float32, device=dev)
    plan.epsr_sq_exec(g.view(P, -1), w_cols, P, np.array([flat]), None, St)
    noise = torch.from_numpy(np.random.default_rng(5).normal(size=len(s.Q)) * 0.005).float().to(dev)
    target = St[0] + noise
    F = epsr.smeared_chi2_function()
    C_ = torch.tensor(np.random.default_rng(6).normal(size=(P, 20)) * 0.001, dtype=torch.float64,
                      device=dev, requires_grad=True)
    pos = torch.zeros((s.n_atoms, 3), dtype=torch.float32, device=dev, requires_grad=True)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def once(ev=None):
        pos.grad = None
        C_.grad = None
        if ev:
            ev[0].record(stream)
        chi2 = F.apply(pos, C_, box, plan, sigma, W, w_cols, flat, target, 0.5, rho)
        if ev:
            ev[1].record(stream)
        chi2.backward()
        if ev:
            ev[2].record(stream)
        return chi2

    launches0 = epsr.epsr_launch_count()
    for _ in range(args.warmup):
        once()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    launches0 = epsr.epsr_launch_count()
    with ClockSampler(0) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            chi2 = once(evs[k])
        torch.cuda.synchronize()
    launches = epsr.epsr_launch_count() - launches0
    t_f = sum(e[0].elapsed_time(e[1]) for e in evs) / args.steps
    t_b = sum(e[1].elapsed_time(e[2]) for e in evs) / args.steps
    Hx = torch.zeros(box.hist_len, dtype=torch.int64, device=dev)
    ge = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a_ev, b_ev in ge:
        Hx.zero_()
        flush.fill_(3.0)
        a_ev.record(stream)
        box.epsr_partial_gr(Hx)
        b_ev.record(stream)
    torch.cuda.synchronize()
    t_h = sum(a.elapsed_time(b) for a, b in ge) / len(ge)
    pairs = s.n_atoms * (s.n_atoms - 1) // 2
    line = {"metric": "chi^2 and dchi^2/dx evaluations/s (differentiable form) at 100k atoms", "value": 1e3 / (t_f + t_b),
            "unit": "evaluations/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_f + t_b, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "fp32 (fixed-point 2^-20 accumulation, fp64 chi^2)", "data": "synthetic",
            "config": {"workload": "99,999-atom water (seed 4), sigma 0.05 A Gaussian-smeared g(r) (333 x 0.03 A), "
                                   "S(Q) on 1000 Q, chi^2 against a seed-5 target + noise, gradients for all "
                                   "coordinates and 60 EP coefficients via torch.autograd",
                       "l2": "flushed before every evaluation outside the timed events"},
            "ms_breakdown": {"forward": t_f, "backward": t_b, "exact_histogram_same_box": t_h},
            "pair_distances_per_s_forward": pairs / (t_f * 1e-3),
            "chi2": float(chi2.item()), "gpu_launches": launches, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_sq(args):
    """The batched S(Q) of the 64-replica workload alone: [2000 Q x 600 r] x [600 r x 192]
    (3 partial g(r) of 64 boxes, g-like synthetic columns: an excluded core, a first shell,
    decaying oscillations), every contraction mode, L2 flushed before each call."""
    import torch
    from paper_1904_08756_gb300 import build, epsr

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    if not os.path.exists(epsr.LIB_PATH):
        build.build()
    nb, n_bins, dr = 64, 600, 0.02
    Q = 0.3 + np.arange(2000) * (39.7 / 1999.0)
    rng = np.random.default_rng(3)
    r = (np.arange(n_bins) + 0.5) * dr
    r0 = rng.uniform(2.4, 3.2, (3 * nb, 1))
    g = (1 + 1.5 * np.exp(-((r - r0) / 0.25) ** 2) - np.exp(-(r / 1.8) ** 8)
         + 0.3 * np.sin(2 * np.pi * r / r0) * np.exp(-r / 4)).astype(np.float32)
    gd = torch.from_numpy(g).to(dev)
    ws = rng.uniform(0.05, 0.4, 3 * nb)
    flats = rng.uniform(0.2, 0.6, nb)
    S = torch.zeros((nb, len(Q)), dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    with ClockSampler(0) as clk:
        modes = time_sq_modes(Q, gd, ws, flats, S, nb, stream, flush, reps=max(args.steps, 5),
                              autotune=not args.no_autotune)
    b = modes["bf16x3"]
    line = {"metric": "batched S(Q) contraction time (Eq. (1), 64 replicas)", "value": b["ms"] * 1e3,
            "unit": "us", "n_gpus": 1, "steps": max(args.steps, 5), "warmup": 3, "ms_per_step": b["ms"],
            "higher_is_better": False, "scaling": "strong", "vs_baseline": None, "dtype": "bf16x3 (fp32 accumulate)",
            "data": "synthetic",
            "config": {"workload": "[2000 Q x 600 r] x [600 r x 192 columns] (cfg-3 batched S(Q))",
                       "l2": "flushed before every call outside the timed events"},
            "sq_modes": modes, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_replicas(args):
    import torch
    from paper_1904_08756_gb300 import build, epsr, synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    if not os.path.exists(epsr.LIB_PATH):
        build.build()
    systems = synth.replica_batch()
    nb = len(systems)
    box = epsr.Box(systems)
    tuning = None if args.no_autotune else box.epsr_autotune()
    ws = np.concatenate([box.epsr_sq_weights(b)[0] for b in range(nb)])
    flats = np.array([box.epsr_sq_weights(b)[1] for b in range(nb)])
    # the batched S(Q): all 3 x 64 columns in one BF16 split-precision tensor-core contraction
    plan = epsr.SqPlan(systems[0].Q, 600, 0.02, epsr.SQ_BF16X3, max_cols=3 * nb)
    H = torch.zeros(box.hist_len, dtype=torch.int64, device=dev)
    g = torch.zeros(box.hist_len, dtype=torch.float32, device=dev)
    S = torch.zeros((nb, len(systems[0].Q)), dtype=torch.float32, device=dev)
    box.epsr_partial_gr(H, g, 1)
    sq_tuning = None if args.no_autotune else plan.epsr_sq_plan_autotune(g.view(-1, 600), ws, 3, flats, None, S)
    H.zero_()
    stream = torch.cuda.Stream()
    moves = args.moves

    def enqueue(k, st):
        box.epsr_mc_sweep_async(moves, 3, k * moves, stream=st)
        H.zero_()
        box.epsr_partial_gr(H, g, 1, stream=st)
        plan.epsr_sq_exec(g.view(-1, 600), ws, 3, flats, None, S, stream=st)

    with torch.cuda.stream(stream):
        for k in range(args.warmup):
            enqueue(k, stream.cuda_stream)
    torch.cuda.synchronize()
    graphs = []
    launches0 = epsr.epsr_launch_count()
    for k in range(args.steps):
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr, stream=stream):
            enqueue(args.warmup + k, torch.cuda.current_stream().cuda_stream)
        graphs.append(gr)
    launches = epsr.epsr_launch_count() - launches0     # each captured graph is replayed once
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        for k, gr in enumerate(graphs):
            flush.fill_(float(k))
            evs[k][0].record()
            gr.replay()
            evs[k][1].record()
        torch.cuda.synchronize()
    status = box.epsr_mc_status()
    t = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    sq_modes = time_sq_modes(systems[0].Q, g.view(-1, 600), ws, flats, S, nb, stream, flush,
                             autotune=not args.no_autotune)
    n_atoms = [s.n_atoms for s in systems]
    line = {"metric": METRIC + " (replica batch)", "value": nb * moves / (t * 1e-3),
            "unit": "moves/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "fp32+int64", "data": "synthetic",
            "config": {"workload": f"{nb} replica boxes (log-uniform 2k-60k atoms, half water, half "
                                   f"silica, {sum(n_atoms)} atoms), {moves} moves per box + g(r) + "
                                   f"S(Q) [2000 x 600] x [600 x {3 * nb}] in BF16x3 per step, one CUDA graph per step",
                       "l2": "flushed before every step outside the timed events"},
            "pair_distances_per_step": sum(n * (n - 1) // 2 for n in n_atoms),
            "status": status, "clocks": clk.summary(), "gpu_launches": launches,
            "tuning": tuning and {k: tuning[k] for k in ("mc_batch", "mc_ctas", "gr_ctas_per_sm", "from_cache")},
            "sq_step_mode": "bf16x3", "sq_tuning": sq_tuning,
            "sq_modes": sq_modes}
    print(json.dumps(line), flush=True)
    box.close()
    plan.close()
    return 0


# ------------------------------------------------------------------------------------------
# Side workloads of the default line (each its own process and JSON line, summarised)
# ------------------------------------------------------------------------------------------

SIDE_KEYS = ("metric", "value", "unit", "ms_per_step", "steps", "ms_breakdown", "roofline", "roofline_gr",
             "gr_pair_distances_per_s", "mc_moves_per_s_kernel", "mc_pair_evals_per_s_kernel", "mc_lj_cutoff",
             "tuning", "sq_tuning", "sq_modes", "clocks", "gpu_launches", "status", "sweep", "e2e", "config")


def run_side_workloads():
    """The other paper-shaped workloads, run in child processes on the same GPU after the main
    measurement (so that the default run records them too): the silica step, the 64-replica
    step under CUDA graphs, the batched S(Q) alone, the differentiable form, and the atom-count
    sweep up to 2.5e5 atoms. Each entry is the child's own JSON line (selected keys) and its
    wall time; a child that fails is recorded with its exit status."""
    side = {}
    runs = {"silica": ["--workload", "silica", "--steps", "10", "--no-cpu-baseline"],
            "replicas": ["--workload", "replicas", "--steps", "5"],
            "sq": ["--workload", "sq", "--steps", "10"],
            "smeared": ["--workload", "smeared", "--steps", "5"],
            "sweep": ["--workload", "sweep", "--max-atoms", "250000"]}
    for name, extra in runs.items():
        t0 = time.perf_counter()
        r = subprocess.run([sys.executable, os.path.abspath(__file__), *extra], capture_output=True, text=True,
                           cwd=ROOT, timeout=900)
        rec = {"wall_s": time.perf_counter() - t0, "args": " ".join(extra)}
        lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
        if r.returncode != 0 or not lines:
            rec.update({"status": "failed", "returncode": r.returncode, "stderr_tail": r.stderr[-400:]})
        else:
            d = json.loads(lines[-1])
            rec.update({k: d[k] for k in SIDE_KEYS if k in d})
        side[name] = rec
    return side


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-side", action="store_true",
                    help="water line: skip the side workloads (silica step, 64 replicas, batched S(Q), "
                         "differentiable form, atom-count sweep to 2.5e5 atoms) run as subprocesses")
    ap.add_argument("--no-autotune", action="store_true",
                    help="profiling runs only: keep the built-in launch rules (no tuning launches)")
    ap.add_argument("--workload", default="water", choices=["water", "silica", "flexible", "replicas", "sweep", "smeared", "sq"],
                    help="water: the paper-scale water box (default line); silica: the paper-scale "
                         "SiO2 box with single-atom moves; flexible: the water box with flexible "
                         "molecules (springs, three kinds of moves); replicas: 64 uneven boxes; sweep: MC "
                         "moves/s at the paper's Table 1 atom counts; smeared: chi^2 and gradients of "
                         "the differentiable form; sq: the batched S(Q) contraction alone")
    ap.add_argument("--max-atoms", type=int, default=0, help="sweep: largest atom count (0: all)")
    ap.add_argument("--r-lj", type=float, default=0.0,
                    help="water / silica / flexible: Lennard-Jones cutoff (A) of the stepped box (0: every pair, "
                         "the paper's form)")
    ap.add_argument("--moves", type=int, default=MOVES_PER_STEP,
                    help="moves per step (profiling runs only; the benchmark uses 10,000)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "replicas":
        return run_replicas(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "smeared":
        return run_smeared(args)
    if args.workload == "sq":
        return run_sq(args)

    import torch
    from paper_1904_08756_gb300 import build, epsr, shard, synth

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if not os.path.exists(epsr.LIB_PATH):
        build.build()

    if args.workload == "silica":
        system = synth.paper_silica(seed=2 + rank)
    elif args.workload == "flexible":
        system = synth.flexible_water_box(33333, seed=1 + rank)
    else:
        system = synth.paper_water(seed=1 + rank)
    if args.r_lj > 0:
        system.r_lj = args.r_lj
    N = system.n_atoms
    m_atoms = int(system.mol_start[1] - system.mol_start[0])
    moves = args.moves
    stream = torch.cuda.current_stream(dev)
    box = epsr.Box(system)
    tuning = None if args.no_autotune else box.epsr_autotune()   # launch shapes timed on this handle
    P = 3
    H = torch.zeros(box.hist_len, dtype=torch.int64, device=dev)
    g = torch.zeros(box.hist_len, dtype=torch.float32, device=dev)
    S_t = torch.zeros((1, len(system.Q)), dtype=torch.float32, device=dev)
    w, flat = box.epsr_sq_weights(0)
    plan = epsr.SqPlan(system.Q, system.n_bins, system.dr, epsr.SQ_FP32, max_cols=P)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    n_cfg = [0]
    move0 = [0]

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        box.epsr_mc_sweep(moves, shard.replica_seed(2024, rank), move0[0])
        move0[0] += moves
        if ev is not None:
            ev[1].record(stream)
        n_cfg[0] += 1
        box.epsr_partial_gr(H, g, n_cfg[0])
        if ev is not None:
            ev[2].record(stream)
        plan.epsr_sq_exec(g.view(P, -1), w, P, np.array([flat]), None, S_t)
        if ev is not None:
            ev[3].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = epsr.epsr_launch_count()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))                 # L2 flush, outside the events
            step(evs[k])
        torch.cuda.synchronize()
    launches = epsr.epsr_launch_count() - launches0
    if ws > 1:
        torch.distributed.barrier()
    t_mc = sum(e[0].elapsed_time(e[1]) for e in evs) / args.steps
    t_gr = sum(e[1].elapsed_time(e[2]) for e in evs) / args.steps
    t_sq = sum(e[2].elapsed_time(e[3]) for e in evs) / args.steps
    t_step = t_mc + t_gr + t_sq
    if ws > 1:
        tt = torch.tensor([t_step, t_mc, t_gr, t_sq], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_step, t_mc, t_gr, t_sq = tt.tolist()
    moves_per_s = ws * moves / (t_step * 1e-3)
    pairs = N * (N - 1) // 2
    gr_pairs_per_s = pairs / (t_gr * 1e-3)

    # ---- end to end through the public API with host buffers --------------------------------
    # host wall clock around: coordinates from (pinned) host memory into the box by the
    # library's host entry, the step, S(Q) back to host memory, synchronise
    xyz_pin = torch.from_numpy(np.ascontiguousarray(box.epsr_box_get_coords())).pin_memory()
    xyz_host = xyz_pin.numpy()
    S_host = torch.empty((1, len(system.Q)), dtype=torch.float32).pin_memory()
    t_e2e_s = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        box.epsr_box_set_coords(xyz_host)
        step()
        S_host.copy_(S_t, non_blocking=True)
        torch.cuda.synchronize()
        t_e2e_s.append(time.perf_counter() - t0)
    t_e2e = 1e3 * sum(t_e2e_s) / args.steps
    if ws > 1:
        tt = torch.tensor([t_e2e], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_e2e = tt.item()

    # ---- the same histogram over cell lists (O(N), reported beside the O(N^2) scan) -----------
    Hc = torch.zeros_like(H)
    for _ in range(3):
        box.epsr_partial_gr_cells(Hc)
    gc_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a_ev, b_ev in gc_ev:
        Hc.zero_()
        flush.fill_(2.0)
        a_ev.record(stream)
        box.epsr_partial_gr_cells(Hc)
        b_ev.record(stream)
    torch.cuda.synchronize()
    t_gc = sum(a_ev.elapsed_time(b_ev) for a_ev, b_ev in gc_ev) / len(gc_ev)
    in_range = int(Hc.sum().item())

    # ---- the cutoff form of dU (LJ truncated at 9 A, partners by cell queries), beside --------
    cut_sys = synth.System(**{**system.__dict__, "r_lj": 9.0})
    cbox = epsr.Box(cut_sys)
    cbox.epsr_mc_sweep(moves, 77, 0)
    c_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for k, (a_ev, b_ev) in enumerate(c_ev):
        flush.fill_(4.0)
        a_ev.record(stream)
        cbox.epsr_mc_sweep(moves, 77, moves * (k + 1))
        b_ev.record(stream)
    torch.cuda.synchronize()
    t_cut = sum(a_ev.elapsed_time(b_ev) for a_ev, b_ev in c_ev) / len(c_ev)
    cbox.close()

    # ---- bounds of the sweep measured on this GPU: grid-barrier floor, issue rates ------------
    sms_dev = torch.cuda.get_device_properties(dev).multi_processor_count
    barrier_ns = epsr.epsr_bench_barrier_floor(sms_dev, 4000)
    int_rate = epsr.epsr_bench_alu_rate(0)
    fma_rate = epsr.epsr_bench_alu_rate(1)

    if rank == 0:
        peaks, src = measured_peaks()
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        clock = clk.summary()
        alu_peak = sms * LANES_PER_SM * peaks.get("sm_max_mhz", 2070.0) * 1e6   # lane-ops/s
        evals_per_move = 2 * m_atoms * (N - m_atoms)
        mc_ops = moves * evals_per_move * OPS_PER_PAIR_EVAL
        mc_achieved = mc_ops / (t_mc * 1e-3)
        gr_achieved = pairs * OPS_PER_PAIR_DIST / (t_gr * 1e-3)
        traffic_file = os.path.join(ROOT, "profiles", "traffic.json")
        traffic = traffic_gr = None
        if os.path.exists(traffic_file):
            tj = json.load(open(traffic_file))
            traffic = tj.get("mc_sweep_kernel_bytes_per_launch")
            traffic_gr = tj.get("partial_gr_kernel_bytes_per_launch")
        if args.workload != "water" or moves != MOVES_PER_STEP or args.r_lj > 0:
            traffic = traffic_gr = None          # the counters were taken on the water step
        line = {
            "metric": METRIC, "value": moves_per_s, "unit": "moves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "fp32+int64", "data": "synthetic",
            "config": {"workload": workload_name(system, moves),
                       "n_atoms": N, "moves_per_step": moves,
                       "l2": "flushed before every step by a 256 MiB write outside the timed events",
                       "parallelism": f"replicas x{ws}"},
            "gr_pair_distances_per_s": gr_pairs_per_s,
            "mc_moves_per_s_kernel": moves / (t_mc * 1e-3),
            "mc_pair_evals_per_s_kernel": moves * evals_per_move / (t_mc * 1e-3),
            "ms_breakdown": {"mc_sweep": t_mc, "partial_gr": t_gr, "sq": t_sq},
            "roofline": {"bound": "alu", "achieved": mc_achieved / 1e12, "peak": alu_peak / 1e12,
                         "unit": "Tops/s", "frac": mc_achieved / alu_peak, "traffic": traffic,
                         "kernel": "mc_sweep_kernel",
                         "peak_source": f"{sms} SMs x {LANES_PER_SM} lanes x {peaks.get('sm_max_mhz', 2070.0):.0f} MHz ({src} max clock)"},
            "roofline_gr": {"bound": "alu", "achieved": gr_achieved / 1e12, "peak": alu_peak / 1e12,
                            "unit": "Tops/s", "frac": gr_achieved / alu_peak, "traffic": traffic_gr,
                            "kernel": "partial_gr_kernel"},
            "measured_bounds": {
                "grid_barrier_floor_us": barrier_ns * 1e-3,
                "mc_ceiling_moves_per_s_at_64_per_barrier": 64.0 / (barrier_ns * 1e-9),
                "int32_xor_add_lane_ops_per_s": int_rate, "fp32_fma_lane_ops_per_s": fma_rate,
                "note": "epsr_bench_barrier_floor (152 CTAs, the sweep's exchange alone) and "
                        "epsr_bench_alu_rate (independent xor+add / FMA chains); the roofline peak stays "
                        "the unit-count figure"},
            "mc_lj_cutoff": {"r_lj_A": 9.0, "ms_per_sweep": t_cut, "moves_per_s": moves / (t_cut * 1e-3),
                             "speedup_vs_all_pairs": t_mc / t_cut,
                             "note": "dU with Lennard-Jones truncated at 9 A (epsr_box_desc.r_lj), every "
                                     "partner row by cell queries; not the paper's all-pairs dU, not in the step"},
            "gr_cell_list": {"ms": t_gc, "pairs_in_range": in_range,
                             "pairs_in_range_per_s": in_range / (t_gc * 1e-3),
                             "speedup_vs_all_pairs": t_gr / t_gc,
                             "note": "epsr_partial_gr_cells, same integer counts, not part of the step"},
            "clocks": {"sm_mhz": clock["sm_mhz"], "sm_max_mhz": clock["sm_max_mhz"],
                       "reasons": clock["reasons"]},
            "e2e": {"value": ws * moves / (t_e2e * 1e-3), "unit": "moves/s",
                    "h2d_bytes_per_step": N * 3 * 4, "d2h_bytes_per_step": len(system.Q) * 4,
                    "timing": "host wall clock: epsr_box_set_coords from pinned host memory, the step, "
                              "S(Q) to host, synchronise"},
            "gpu_launches": launches,
            "tuning": tuning and {k: tuning[k] for k in ("mc_batch", "mc_ctas", "gr_ctas_per_sm", "from_cache")},
        }
        if args.workload == "water" and ws == 1 and not args.no_side and moves == MOVES_PER_STEP:
            line["side_workloads"] = run_side_workloads()
        if not args.no_cpu_baseline and ws == 1:
            o = oracle_full_step(system, moves_per_step=moves)
            t_cpu = o["t_mc"] + o["t_gr"] + o["t_sq"]
            line["cpu_baseline"] = {
                "value": moves / t_cpu, "unit": "moves/s", "cores": o["threads"], "kind": "oracle",
                "sample": (f"full step, measured: {moves} moves of the chain on 1 core "
                           f"({o['t_mc']:.1f} s) + the full pair scan ({o['pairs']:.4g} pair "
                           f"distances) on {o['threads']} cores ({o['t_gr']:.1f} s) + S(Q) "
                           f"({o['t_sq']:.2f} s)"),
                "moves_per_s_1core": moves / o["t_mc"],
                "pair_distances_per_s_all_cores": o["pairs"] / o["t_gr"],
                "pair_distances_per_s_1core": o["pairs_1core_per_s"],
                "pair_distances_1core_sample": (f"the first {o['rows_1core']} rows of the pair scan "
                                                f"({o['pairs_1core_sample']:.3g} pair distances)")}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    box.close()
    plan.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
