"""MD-like sequences: drifting orbitals solved step after step with a warm start.

Each step of the sequence is the molecular-dynamics-like workload (1024
Gaussian orbitals in 256 clusters of 4, a 37.3-bohr cell on 190^3 points,
R_pair 10 bohr, R_PE / R_ME = 24 / 32, tol 1e-8) after ``step`` independent
drifts of the centres (N(0, 0.02^2) bohr per component) and 1 % perturbations
of the exponents; the orbitals are rebuilt on the device between steps
(untimed). The solver runs the batched mixed-precision path with one of the
warm starts of exx_options.warm_start: 0 (zero), 1 (the previous step's
potential of each pair kept from the previous step), 2 (a learned guess) or 3
(polynomial extrapolation from the last two or three steps). With
--preconditioner 1 each step is solved from zero by the multigrid-
preconditioned CG instead (exx_options.preconditioner; it takes no warm start).

    python -m paper_1911_10630_gb300.md_sequence --steps 20 --warm 1
    python -m paper_1911_10630_gb300.md_sequence --steps 20 --warm 0 --preconditioner 1
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import synth
from .exx import Exx


def pair_energies(ex, subset):
    """E_ij of the last call for the (i, j) pairs of subset (NaN for a pair
    that left the list)."""
    pairs = ex.pairs()
    key = {(int(i), int(j)): k for k, (i, j) in enumerate(zip(pairs["i"], pairs["j"]))}
    return np.array([pairs["e_pair"][key[p]] if p in key else np.nan for p in subset])


def run(steps: int = 20, warm: int = 0, model_blob: bytes = None, seed: int = 0, on_step=None, subset=None,
        preconditioner: int = 0):
    """Runs the sequence; returns one dict per step (E_xx, pairs, timings, CG
    iterations; with subset, a list of (i, j), also their E_ij as e_sub).
    on_step(step, workload, orbitals, d_xx, exx) is called after each step
    (for checks on the step's outputs)."""
    import torch
    w0 = synth.config4(seed, 0)
    ex = Exx(w0.cell, w0.grid, w0.r_pair, w0.r_pe, w0.r_me, w0.l_max, w0.tol, precision=1, warm_start=warm,
             preconditioner=preconditioner)
    if warm == 2:
        ex.load_guess_model(model_blob)
    phi = torch.empty((w0.n, int(w0.grid[0]), int(w0.grid[1]), int(w0.grid[2])), dtype=torch.float64, device="cuda")
    D = torch.empty_like(phi)
    out = []
    for s in range(steps):
        w = synth.config4(seed, s)
        synth.orbitals_torch(w, out=phi)
        cen = torch.from_numpy(np.ascontiguousarray(w.centers)).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e = ex.compute(phi, cen, D)
        wall = time.perf_counter() - t0
        st = ex.stats()
        rec = dict(step=s, E_xx=e, n_pair=st["n_pair"], total_ms=st["total_ms"], solve_ms=st["solve_ms"],
                   guess_ms=st["guess_ms"], wall_ms=1e3 * wall, iters_p50=st["iters_p50"],
                   iters_p99=st["iters_p99"], iters_total=st["iters_total"], n_nonconv=st["n_nonconv"],
                   pair_solves_per_s=st["n_pair"] / (st["total_ms"] / 1e3))
        if subset is not None:
            rec["e_sub"] = pair_energies(ex, subset).tolist()
        out.append(rec)
        if on_step:
            on_step(s, w, phi, D, ex)
    ex.close()
    return out


def step_time_percentiles(recs):
    """p50 and p99 of the device time per step over the sequence (ms)."""
    t = np.array([r["total_ms"] for r in recs])
    return float(np.percentile(t, 50)), float(np.percentile(t, 99))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warm", type=int, default=1, choices=[0, 1, 2, 3])
    ap.add_argument("--model", default=None, help="model blob for --warm 2")
    ap.add_argument("--preconditioner", type=int, default=0, choices=[0, 1],
                    help="1: the multigrid-preconditioned CG (with --warm 0)")
    args = ap.parse_args()
    blob = open(args.model, "rb").read() if args.model else None
    recs = run(args.steps, args.warm, blob, preconditioner=args.preconditioner)
    for r in recs:
        print(json.dumps(r), flush=True)
    t = np.array([r["total_ms"] for r in recs[1:]] or [recs[0]["total_ms"]])
    print(json.dumps({"warm": args.warm, "preconditioner": args.preconditioner, "p50_ms": float(np.percentile(t, 50)), "p99_ms": float(np.percentile(t, 99)),
                      "pair_solves_per_s": float(np.mean([r["pair_solves_per_s"] for r in recs[1:]] or [0]))}))


if __name__ == "__main__":
    main()
