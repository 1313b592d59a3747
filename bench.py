#!/usr/bin/env python
"""Pair-Poisson solves per second of the exact-exchange hot path on one GB300.

One step = one exx_compute call over the water-64-scale workload (L = 23.5 bohr,
120^3 grid, 256 orbitals in 64 clusters of 4, R_pair = 10 bohr, R_PE/R_ME =
24/32 grid points, l_max = 6, relative residual 1e-8): pair list, gather,
multipoles, shell potential, CG solves, E_xx reduction and D_xx scatter.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl exx|reference]

Under torchrun (N > 1) every rank runs an independent replica of the workload
on its own GPU (the path has no exchange step on one node: replicas only) and
rank 0 prints one JSON line with the whole-job rate.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pair-Poisson solves/s at fixed E_xx error"
UNIT = "pair solves/s"
SMEM_BYTES_PER_CLK_SM = 128  # shared-memory bandwidth of one SM (32 banks x 4 B per clock)
# the quad-map stencil's shared-memory traffic per point and iteration: 15
# loads of 16 bytes per quad of 4 points plus the store of p (context only;
# the roofline's algorithmic bytes are the CG state's)
SMEM_MODEL_BYTES_PER_POINT_ITER = 15 * 16 / 4 + 4
# The multigrid PCG's algorithmic bytes per fine-level point and iteration
# (FP32, every vector read or written once per sweep): A p (8), the d and r
# updates (24), the V-cycle's level-0 sweeps: Jacobi (8), residual (12),
# restriction (4), prolongation (8), smoothing (12); r.z (8) and the p update
# (12): 96 B; the coarse levels add their share of the V-cycle (44 B x 1/7)
MG_BYTES_PER_POINT_ITER = 96 + 44 / 7


def _peaks():
    """HBM GB/s and the maximum SM clock (MHz) with their source."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), float(d.get("sm_max_mhz", 2070.0)), "measured"
    return 6800.0, 2070.0, "fallback"


# the sources that decide the pair kernels' code and launch layout (DRAM
# traffic): a change to any of them invalidates the committed ncu figures
KERNEL_SOURCES = ("exx_cluster.cu", "exx_phases.cuh", "exx_kernels.cuh", "exx_internal.h", "exx_geometry.cpp",
                  "exx_geometry.h", "exx_solve.cu", "exx_mg.cuh")


def _kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1911_10630_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel source changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(f"{kernel}|{workload}")
    if not e or e.get("kernel_hash") != _kernel_hash():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over the ranks of the default process group (any backend)."""
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws: int, units_per_rank: int, steps: int, max_ms: float) -> float:
    """Whole-job units per second: every rank processed units_per_rank per step
    (replicas), timed by the slowest rank."""
    return ws * units_per_rank * steps / (max_ms / 1e3)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _algorithmic(pairs, stats, n_pe, n_me, precision):
    """Algorithmic bytes and FLOPs of one pair-kernel launch: per-unit figures
    times the units the launch processed (the design notes derive each).

    cg: each point-iteration must read and write the CG state x, r and p
      once: 6 words, 24 B in FP32 (the fast path keeps them on chip) and
      48 B in FP64.
    hbm: per pair, the gather of phi_i, phi_j on the ME ball (16 B per point),
      the D_xx read-modify-write of one or two orbitals on the ME ball
      (16 or 32 B per point) and one more read of phi_i, phi_j for the scatter.
    flops: 38 per point-iteration (19-point stencil and the CG updates)."""
    it = pairs["iters"].astype(np.float64)
    point_iters = float(stats.get("point_iters") or n_pe * it.sum())
    two = (pairs["i"] != pairs["j"]).astype(np.float64)
    hbm = float(np.sum((16.0 + 16.0 + 16.0 * (1.0 + two)) * n_me))
    s = 4 if precision == 1 else 8
    return dict(cg=6.0 * s * point_iters, hbm=hbm, flops=38.0 * point_iters, point_iters=point_iters)


def batched_uneven_leg(dev, stream, steps=3, plain_steps=1):
    """Config 2 (batched uneven): 512 orbitals in 128 clusters on 150^3, per-pair
    radii 12..32 from the orbital exponents, tol 1e-8. The mixed-precision
    cluster solver in radius classes (one launch per R_PE, the largest first,
    one captured graph) and the multigrid CG against the pure-FP64 GPU solve of
    the same pairs; all from inputs resident on the device, CUDA events on the
    stream."""
    import torch
    from paper_1911_10630_gb300 import synth
    from paper_1911_10630_gb300.exx import Exx
    w = synth.config2()
    phi = synth.orbitals_torch(w, device=dev)
    cen = torch.from_numpy(np.ascontiguousarray(w.centers)).to(dev)
    al = torch.from_numpy(np.ascontiguousarray(w.alphas)).to(dev)
    D = torch.empty_like(phi)
    out = {"workload": w.name, "n_orbitals": w.n, "grid": int(w.grid[0]), "tol": w.tol}

    def timed(n, **opt):
        ex = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, radii_mode=1, **opt)
        e = ex.compute(phi, cen, D, alphas=al, stream=stream)  # warm-up (graph capture)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(n):
            e = ex.compute(phi, cen, D, alphas=al, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / n
        st = ex.stats()
        cls = ex.radius_classes()
        ex.close()
        return e, ms, st, cls

    e1, ms1, st1, cls = timed(steps, precision=1)
    em, msm, stm, _ = timed(steps, precision=1, preconditioner=1)
    e0, ms0, st0, _ = timed(plain_steps, precision=0)
    n_pair = st1["n_pair"]
    out.update({"n_pair": n_pair, "value": n_pair / (ms1 / 1e3), "unit": UNIT, "ms_per_step": ms1,
                "iters_p50": st1["iters_p50"], "iters_max": st1["iters_max"], "n_nonconv": st1["n_nonconv"],
                "radius_classes": [{"r_pe": r, "ctas_per_pair": c, "resident": k} for r, c, k in cls],
                "pure_fp64_gpu": {"value": n_pair / (ms0 / 1e3), "ms_per_step": ms0, "iters_p50": st0["iters_p50"]},
                "speedup_vs_pure_fp64_gpu": ms0 / ms1, "dE_vs_fp64_per_orbital": abs(e1 - e0) / w.n,
                # the multigrid CG, one CTA per pair, all radius classes in one largest-first launch
                "multigrid_pcg": {"value": n_pair / (msm / 1e3), "ms_per_step": msm, "iters_p50": stm["iters_p50"],
                                  "iters_max": stm["iters_max"], "n_nonconv": stm["n_nonconv"],
                                  "speedup_vs_pure_fp64_gpu": ms0 / msm,
                                  "dE_vs_fp64_per_orbital": abs(em - e0) / w.n}})
    del phi, D
    torch.cuda.empty_cache()
    return out


def learned_leg(w, dphi, dcen, dD, stream, zero_ms, plain_ms, steps=2, train_workloads=8, per_workload=400,
                epochs=6):
    """The workload solved from the learned warm start (warm_start = 2): the
    R_PE 24 network (cube 48) trained on the GPU by the library's own kernels
    on solver samples of other seeds of the same form (train_workloads x
    per_workload pairs), then the batched mixed-precision solve from its guess.
    Reports pair solves/s with the network's time included, CG iterations per
    pair against the zero start, and the ratios to the zero start and to the
    plain FP64 CG of the main line."""
    import time as _t
    import torch
    from paper_1911_10630_gb300 import guess_train, synth
    from paper_1911_10630_gb300.exx import Exx, guess_model_blob
    t0 = _t.time()
    inp, tgt = guess_train.solve_and_export(range(3000, 3000 + train_workloads), S=guess_train.CUBE_R24,
                                            torch=torch, workload=synth.config1, per_workload=per_workload)
    net, hist = guess_train.train(inp, tgt, S=guess_train.CUBE_R24, epochs=epochs, batch=32, lr=1e-3)
    blob = guess_model_blob(guess_train.CUBE_R24, net.get_params())
    net.close()
    del inp, tgt
    torch.cuda.empty_cache()
    train_s = _t.time() - t0
    ex = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, precision=1, warm_start=2)
    ex.load_guess_model(blob)
    e = ex.compute(dphi, dcen, dD, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    its, gms = [], []
    for _ in range(steps):
        e = ex.compute(dphi, dcen, dD, stream=stream)
        st = ex.stats()
        its.append(st["iters_total"] / st["n_pair"])
        gms.append(st["guess_ms"])
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    n_pair = st["n_pair"]
    ex.close()
    return {"value": n_pair / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "guess_ms_per_step": float(np.mean(gms)),
            "iters_per_pair": float(np.mean(its)), "E_xx": e, "n_nonconv": st["n_nonconv"],
            "training": {"samples": train_workloads * per_workload, "epochs": epochs, "seconds": train_s,
                         "loss_first_last": [hist[0], hist[-1]]},
            "vs_zero_start": zero_ms / ms, "speedup_vs_plain_fp64_cg": plain_ms / ms if plain_ms else None}


def run_oracle_sample(w, phi, pairs_all, seconds=12.0, seed=0):
    """Times the oracle on a bounded random sample of the workload's pairs."""
    import oracle
    rng = np.random.default_rng(seed)
    nthr = oracle.num_threads()
    npair = len(pairs_all[0])
    order = rng.permutation(npair)
    done, t_used, k = 0, 0.0, 0
    chunk = max(2 * nthr, 8)
    while t_used < seconds and k < npair:
        idx = np.sort(order[k:k + chunk])
        sub = tuple(a[idx] for a in pairs_all)
        t0 = time.perf_counter()
        oracle.exx(w.cell, w.grid, phi, sub, w.r_pe, w.r_me, w.l_max, tol=w.tol, want_d=True)
        t_used += time.perf_counter() - t0
        done += len(idx)
        k += chunk
    return done / t_used, done, t_used, nthr


def reference_arm(args, w):
    """The oracle (FP64 C, OpenMP over pairs) on the host cores: each step a
    bounded sample of the workload's pairs."""
    import oracle
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    phi = w.orbitals()
    pairs_all = oracle.pair_list(w.centers, w.cell, w.grid, w.r_pair)
    nthr = oracle.num_threads()
    per_step = max(2 * nthr, 8)
    rng = np.random.default_rng(123)
    times = []
    for s in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(len(pairs_all[0]), per_step, replace=False))
        sub = tuple(a[idx] for a in pairs_all)
        t0 = time.perf_counter()
        oracle.exx(w.cell, w.grid, phi, sub, w.r_pe, w.r_me, w.l_max, tol=w.tol, want_d=True)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = per_step * len(times) / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n_orbitals": w.n, "grid": int(w.grid[0]), "r_pair_bohr": w.r_pair,
                   "r_pe": w.r_pe, "r_me": w.r_me, "l_max": w.l_max, "tol": w.tol,
                   "n_pair_total": int(len(pairs_all[0]))},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthr, "kind": "oracle",
                         "sample": f"{per_step} random pairs of the workload per step (of {len(pairs_all[0])}), "
                                   f"FP64 CG to the workload tol, D_xx scatter included"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="exx", choices=["exx", "reference"])
    ap.add_argument("--precision", type=int, default=1, help="1: FP32 inner + FP64 refinement, 0: FP64 CG")
    ap.add_argument("--preconditioner", type=int, default=1,
                    help="1: multigrid-preconditioned CG (the fastest form; FP32 inside FP64 refinement at "
                         "precision 1), 0: plain CG (the cluster solver at precision 1)")
    ap.add_argument("--plain-steps", type=int, default=1, help="timed steps of the plain FP64 CG comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--solver-kind", type=int, default=0, help="0 auto, 1 one CTA per pair, 2 cluster per pair")
    ap.add_argument("--cluster-size", type=int, default=0)
    ap.add_argument("--lane-map", type=int, default=0)
    ap.add_argument("--update-drop", type=float, default=1e-4)
    ap.add_argument("--autotune", type=int, default=1)
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the batched-uneven (config 2) and learned-guess legs")
    ap.add_argument("--orbitals", type=int, default=0,
                    help="keep only the first N orbitals of the workload (small cases for profiling)")
    args = ap.parse_args()
    if args.precision == 0:
        args.preconditioner = 0  # the FP64 bench line is the plain FP64 CG (the speed-ups' denominator)

    from paper_1911_10630_gb300 import synth
    w = synth.config1()
    if args.orbitals:
        w.centers, w.alphas, w.pvecs = w.centers[:args.orbitals], w.alphas[:args.orbitals], w.pvecs[:args.orbitals]
        w.name = w.name + "-first%d" % args.orbitals
    if args.impl == "reference":
        return reference_arm(args, w)

    import torch
    import torch.distributed as dist
    ws, rank, local = _dist()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_1911_10630_gb300 import build as _build
    _build.build(quiet=True)
    from paper_1911_10630_gb300 import exx as exx_mod
    from paper_1911_10630_gb300.exx import Exx

    phi = w.orbitals()
    centers = np.ascontiguousarray(w.centers)
    dphi = torch.from_numpy(phi).to(dev)
    dcen = torch.from_numpy(centers).to(dev)
    dD = torch.empty_like(dphi)
    stream = torch.cuda.current_stream(dev)
    ex = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, precision=args.precision,
             threads=args.threads, ctas_per_sm=args.ctas_per_sm, solver_kind=args.solver_kind,
             cluster_size=args.cluster_size, lane_map=args.lane_map, update_drop=args.update_drop,
             autotune=args.autotune, preconditioner=args.preconditioner)

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        ex.compute(dphi, dcen, dD, stream=stream)
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    solve_ms, exx_vals = [], []
    with ClockSampler(dev.index) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            exx_vals.append(ex.compute(dphi, dcen, dD, stream=stream))
            solve_ms.append(ex.stats()["solve_ms"])
        ev1.record(stream)
        barrier()
    total_ms = ev0.elapsed_time(ev1)
    if ws > 1:
        total_ms = max_over_ranks(total_ms, dist, dev)
    st = ex.stats()
    pairs = ex.pairs()
    n_pair = st["n_pair"]
    value = job_rate(ws, n_pair, args.steps, total_ms)
    n_pe, n_me = ex.ball_size()
    alg = _algorithmic(pairs, st, n_pe, n_me, args.precision)
    kern_ms = statistics.mean(solve_ms)
    hbm_peak, sm_mhz_max, peak_src = _peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    workload_key = f"{w.name}|p{args.precision}" + ("m" if args.preconditioner == 1 else "")
    fp64_peak = exx_mod.probe_fp64_rate(stream)  # the FP64 pipe's FMA rate, measured on this GPU
    def cg_roofline(st_, alg_, kms):
        """The plain FP32 CG's roofline: the cluster solver keeps the CG state in
        shared memory, so the bound is shared-memory bandwidth."""
        kname = "cluster_pair_kernel" if st_["solver_kind"] == 2 else "pair_kernel"
        smem_peak = n_sm * SMEM_BYTES_PER_CLK_SM * sm_mhz_max * 1e6 / 1e9
        achieved = alg_["cg"] / (kms / 1e3) / 1e9
        return {"kernel": kname, "bound": "smem", "achieved": achieved, "peak": smem_peak, "unit": "GB/s",
                "frac": achieved / smem_peak,
                "peak_source": f"{n_sm} SMs x {SMEM_BYTES_PER_CLK_SM} B/clk x {sm_mhz_max:.0f} MHz "
                               f"(max SM clock, {peak_src})",
                "algorithmic_bytes_per_launch": alg_["cg"], "bytes_per_point_iteration": 24,
                "traffic": _traffic(kname, f"{w.name}|p1"),
                "smem_model": {"bytes_per_point_iteration": SMEM_MODEL_BYTES_PER_POINT_ITER,
                               "frac": SMEM_MODEL_BYTES_PER_POINT_ITER / 24 * achieved / smem_peak},
                "hbm": {"algorithmic_bytes_per_launch": alg_["hbm"],
                        "achieved": alg_["hbm"] / (kms / 1e3) / 1e9, "peak": hbm_peak, "peak_source": peak_src},
                "kernel_ms": kms}

    if args.precision == 1 and args.preconditioner == 1:
        # one CTA per pair, every vector in the pair's workspace: the sweeps
        # stream from HBM (the pairs in flight hold far more than L2)
        mg_bytes = MG_BYTES_PER_POINT_ITER * alg["point_iters"]
        achieved = mg_bytes / (kern_ms / 1e3) / 1e9
        roofline = {"kernel": "pair_kernel", "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "peak_source": peak_src,
                    "algorithmic_bytes_per_launch": mg_bytes, "bytes_per_point_iteration": MG_BYTES_PER_POINT_ITER,
                    "traffic": _traffic("pair_kernel", workload_key), "kernel_ms": kern_ms}
    elif args.precision == 1:
        roofline = cg_roofline(st, alg, kern_ms)
    else:
        fl = alg["flops"] / (kern_ms / 1e3) / 1e12
        roofline = {"kernel": "pair_kernel", "bound": "alu", "achieved": fl, "peak": fp64_peak,
                    "unit": "TFLOP/s", "frac": fl / fp64_peak,
                    "peak_source": "FP64 FMA rate measured on this GPU (exx_probe_fp64_rate)",
                    "flops_per_point_iteration": 38, "traffic": _traffic("pair_kernel", workload_key),
                    "kernel_ms": kern_ms}

    # the host-buffer leg runs first, before the comparison contexts below
    # allocate and free their workspaces (measured: copies into freshly
    # allocated device buffers run at about 200 GB/s, after much allocation
    # churn far slower)
    e2e = None
    if not args.no_e2e:
        hphi = torch.from_numpy(phi).pin_memory()
        hD = torch.empty(phi.shape, dtype=torch.float64).pin_memory()
        hc = torch.from_numpy(centers).pin_memory()
        exh = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, precision=args.precision,
                  preconditioner=args.preconditioner)
        exh.compute_host(hphi, hc, hD, stream=stream)  # warm-up (allocates the device copies)
        barrier()
        t0 = time.perf_counter()
        nrep = max(1, min(args.steps, 3))
        for _ in range(nrep):
            exh.compute_host(hphi, hc, hD, stream=stream)
        barrier()
        dt = (time.perf_counter() - t0) / nrep
        e2e = {"value": ws * n_pair / dt, "unit": UNIT, "h2d_bytes_per_step": int(phi.nbytes + centers.nbytes),
               "d2h_bytes_per_step": int(phi.nbytes + 8), "ms_per_step": dt * 1e3}
        exh.close()
        del hphi, hD

    extra = {}
    if rank == 0 and args.precision == 1 and args.plain_steps > 0:
        ex0 = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, precision=0)
        ex0.compute(dphi, dcen, dD, stream=stream)
        torch.cuda.synchronize(dev)
        t = []
        for _ in range(args.plain_steps):
            ev0.record(stream)
            e0 = ex0.compute(dphi, dcen, dD, stream=stream)
            ev1.record(stream)
            torch.cuda.synchronize(dev)
            t.append(ev0.elapsed_time(ev1))
        st0 = ex0.stats()
        alg0 = _algorithmic(ex0.pairs(), st0, n_pe, n_me, 0)
        fl0 = alg0["flops"] / (st0["solve_ms"] / 1e3) / 1e12
        extra["plain_fp64_cg"] = {"value": n_pair / (statistics.mean(t) / 1e3), "unit": UNIT,
                                  "ms_per_step": statistics.mean(t), "E_xx": e0,
                                  "dE_vs_fast_per_orbital": abs(e0 - exx_vals[-1]) / w.n,
                                  "iters_p50": st0["iters_p50"], "iters_max": st0["iters_max"],
                                  "roofline": {"kernel": "pair_kernel", "bound": "alu", "achieved": fl0,
                                               "peak": fp64_peak, "unit": "TFLOP/s", "frac": fl0 / fp64_peak,
                                               "peak_source": "FP64 FMA rate measured on this GPU "
                                                              "(exx_probe_fp64_rate)",
                                               "flops_per_point_iteration": 38,
                                               "kernel_ms": st0["solve_ms"]}}
        extra["speedup_vs_plain_fp64_cg"] = value / ws / extra["plain_fp64_cg"]["value"]
        ex0.close()
        if args.preconditioner == 1:
            # the unpreconditioned FP32 CG on the cluster solver (autotuned launch shape)
            exc = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, precision=1)
            exc.compute(dphi, dcen, dD, stream=stream)
            torch.cuda.synchronize(dev)
            tc, sc = [], []
            for _ in range(max(1, min(args.steps, 3))):
                ev0.record(stream)
                ec = exc.compute(dphi, dcen, dD, stream=stream)
                ev1.record(stream)
                torch.cuda.synchronize(dev)
                tc.append(ev0.elapsed_time(ev1))
                sc.append(exc.stats()["solve_ms"])
            stc = exc.stats()
            algc = _algorithmic(exc.pairs(), stc, n_pe, n_me, 1)
            extra["cluster_cg"] = {
                "value": n_pair / (statistics.mean(tc) / 1e3), "unit": UNIT, "ms_per_step": statistics.mean(tc),
                "E_xx": ec, "dE_vs_headline_per_orbital": abs(ec - exx_vals[-1]) / w.n,
                "iters_p50": stc["iters_p50"], "iters_max": stc["iters_max"],
                "iters_per_pair": stc["iters_total"] / stc["n_pair"],
                "solver": f"{stc['solver_kind']}x{stc['cluster_size']} ctas={stc['grid_ctas']} "
                          f"threads={stc['threads']} lane_map={stc['lane_map']} "
                          f"autotuned_from={stc['n_candidates']}",
                "roofline": cg_roofline(stc, algc, statistics.mean(sc)),
                "phase_ms_per_cluster": {"setup": stc["phase_ms"][0], "fp64_residuals": stc["phase_ms"][1],
                                         "fp32_cg": stc["phase_ms"][2], "finish": stc["phase_ms"][3]},
                "speedup_vs_plain_fp64_cg": statistics.mean(t) / statistics.mean(tc)}
            exc.close()
        # the same FP64 solve with the multigrid-preconditioned CG (one V-cycle per iteration)
        exm = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, precision=0, preconditioner=1)
        exm.compute(dphi, dcen, dD, stream=stream)
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        em = exm.compute(dphi, dcen, dD, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        tm = ev0.elapsed_time(ev1)
        stm = exm.stats()
        extra["fp64_multigrid_pcg"] = {"value": n_pair / (tm / 1e3), "unit": UNIT, "ms_per_step": tm, "E_xx": em,
                                       "dE_vs_plain_per_orbital": abs(em - e0) / w.n,
                                       "iters_p50": stm["iters_p50"], "iters_max": stm["iters_max"],
                                       "speedup_vs_plain_fp64_cg": statistics.mean(t) / tm}
        exm.close()

    if rank == 0 and ws == 1 and not args.no_legs and not args.orbitals:
        extra["batched_uneven"] = batched_uneven_leg(dev, stream)
        plain_ms = extra.get("plain_fp64_cg", {}).get("ms_per_step")
        # the learned start runs on the unpreconditioned cluster solver: compare it with that solver's zero start
        zc = extra.get("cluster_cg")
        zero_ms = zc["ms_per_step"] if zc else total_ms / args.steps
        extra["learned_guess"] = learned_leg(w, dphi, dcen, dD, stream, zero_ms, plain_ms)
        extra["learned_guess"]["iters_per_pair_zero_start"] = (zc["iters_per_pair"] if zc
                                                               else st["iters_total"] / st["n_pair"])

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        pairs_all = (pairs["i"], pairs["j"], pairs["g"])
        v, done, used, nthr = run_oracle_sample(w, phi, pairs_all)
        cpu = {"value": v, "unit": UNIT, "cores": nthr, "kind": "oracle",
               "sample": f"{done} random pairs of the workload ({used:.1f} s), FP64 CG to tol {w.tol}, "
                         f"D_xx scatter included"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == 1 else "f64", "data": "synthetic",
            "config": {"workload": w.name, "n_orbitals": w.n, "grid": int(w.grid[0]), "cell_bohr": float(w.cell[0]),
                       "r_pair_bohr": w.r_pair, "r_pe": w.r_pe, "r_me": w.r_me, "l_max": w.l_max, "tol": w.tol,
                       "n_pair": n_pair,
                       "precision": ("fp32 multigrid-preconditioned CG + fp64 refinement" if args.preconditioner == 1
                                     else "fp32 inner CG + fp64 refinement") if args.precision == 1 else "fp64 CG",
                       "l2": "inputs larger than L2 (orbitals 3.5 GB, D_xx 3.5 GB)",
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "solver": f"{st['solver_kind']}x{st['cluster_size']} ctas={st['grid_ctas']} "
                                 f"threads={st['threads']} lane_map={st['lane_map']} "
                                 f"autotuned_from={st['n_candidates']}"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": 6 * args.steps,
            "clocks": clk.summary(),
            "E_xx": exx_vals[-1],
            "cg": {"iters_p50": st["iters_p50"], "iters_p99": st["iters_p99"], "iters_max": st["iters_max"],
                   "refine_max": st["refine_max"], "point_iters": st["point_iters"], "n_nonconv": st["n_nonconv"],
                   # the kernel time split by the CTAs' (clusters') cycle counts
                   "phase_ms": {"setup": st["phase_ms"][0], "fp64_residuals": st["phase_ms"][1],
                                "cg_iterations": st["phase_ms"][2], "finish": st["phase_ms"][3]}},
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
