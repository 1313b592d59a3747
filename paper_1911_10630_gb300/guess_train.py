"""Training of the learned CG warm start (include/exx_guess.h).

Samples come from the solver itself: each seeded workload of the tiny form
(8 Gaussian orbitals in a 9-bohr cell on 48^3 points, R_PE = 16, R_ME = 20,
every pair, CG to 1e-10) is solved with warm_start = 1, and
exx_export_samples turns every pair's converged v_ij and its density into
one (input, target) cube of side 32. The network then trains with Adam on the
GPU through exx_guess_train_step; every step runs in the library's kernels.

    python -m paper_1911_10630_gb300.guess_train --out guess_r16.bin

With --workload water64 the samples come from water-64-form workloads
(R_PE = 24, cube side 48; a subset of each workload's pairs), for the solver
at the radii of the water-64 and MD-like workloads.

The model blob is what exx_load_guess_model (warm_start = 2) expects.
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np

from . import synth
from .exx import GUESS_CHANNELS, Exx, GuessNet, guess_model_blob

CUBE = 32      # network input side for R_PE = 16 (the ball's +16 poles fall outside)
CUBE_R24 = 48  # and for R_PE = 24


def init_params(n_params: int, seed: int) -> np.ndarray:
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases, layer table of exx_guess.h."""
    cin = (GUESS_CHANNELS, 16, 16, 32, 32, 64, 64, 128, 192, 64, 96, 32, 48, 16, 16)
    cout = (16, 16, 32, 32, 64, 64, 128, 128, 64, 64, 32, 32, 16, 16, 1)
    rng = np.random.default_rng(seed)
    parts = []
    for l, (a, b) in enumerate(zip(cin, cout)):
        fan = a if l == len(cin) - 1 else 27 * a
        parts.append(rng.uniform(-math.sqrt(6.0 / fan), math.sqrt(6.0 / fan), fan * b))
        parts.append(np.zeros(b))
    p = np.concatenate(parts).astype(np.float32)
    if p.size != n_params:
        raise RuntimeError("layer table does not match the library's network")
    return p


def solve_and_export(seeds, S: int = CUBE, torch=None, workload=None, per_workload: int = 0):
    """Solves each seeded workload (default: the tiny form, synth.config0) and
    returns the samples of its pairs as device tensors (input [n][S^3][3],
    target [n][S^3]); per_workload > 0 keeps that many pairs, spread evenly
    over the list, of each workload."""
    import torch as _t
    torch = torch or _t
    make = workload or synth.config0
    ins, tgts = [], []
    ex = None
    for seed in seeds:
        w = make(seed)
        if ex is None:  # one fixed launch shape: the samples do not depend on a timing-based choice
            ex = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, precision=1, warm_start=1,
                     autotune=0)
        phi = synth.orbitals_torch(w)
        cen = torch.from_numpy(np.ascontiguousarray(w.centers)).cuda()
        D = torch.empty_like(phi)
        ex.compute(phi, cen, D)
        del D
        cap = ex.stats()["n_pair"]
        inp = torch.empty((cap, S, S, S, GUESS_CHANNELS), dtype=torch.float32, device="cuda")
        tgt = torch.empty((cap, S, S, S), dtype=torch.float32, device="cuda")
        n = ex.export_samples(phi, S, inp, tgt, cap)
        keep = torch.arange(n, device="cuda")
        if per_workload and per_workload < n:
            keep = torch.linspace(0, n - 1, per_workload, device="cuda").round().long()
        ins.append(inp.index_select(0, keep))
        tgts.append(tgt.index_select(0, keep))
        del inp, tgt, phi
    ex.close()
    return torch.cat(ins), torch.cat(tgts)


def train(inp, tgt, S: int = CUBE, epochs: int = 20, batch: int = 32, lr: float = 2e-3, seed: int = 0,
          time_limit: float = 1e30, log=None):
    """Adam on the samples (cosine-decayed learning rate); returns the net and the
    per-epoch mean loss. Initialisation and batch order come from seed, and every
    gradient reduction of the library runs in a fixed order, so the same samples
    and arguments give bitwise the same parameters."""
    import torch
    n = inp.shape[0]
    net = GuessNet(S, batch)
    net.set_params(init_params(net.n_params, seed))
    rng = np.random.default_rng(seed + 1)
    steps_per_epoch = max(1, n // batch)
    total = epochs * steps_per_epoch
    hist = []
    t0 = time.time()
    k = 0
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)).cuda()
        acc = 0.0
        for s in range(steps_per_epoch):
            idx = perm[s * batch:(s + 1) * batch]
            bi = inp.index_select(0, idx).contiguous()
            bt = tgt.index_select(0, idx).contiguous()
            a = lr * 0.5 * (1.0 + math.cos(math.pi * k / total))
            acc += net.train_step(bi, bt, batch, max(a, 1e-3 * lr))
            k += 1
        hist.append(acc / steps_per_epoch)
        if log:
            log(f"epoch {ep} loss {hist[-1]:.4e} ({time.time() - t0:.1f} s)")
        if time.time() - t0 > time_limit:
            break
    return net, hist


def conv_macs(S: int) -> int:
    """Multiply-adds of one forward pass at cube side S (3x3x3 layers)."""
    cin = (GUESS_CHANNELS, 16, 16, 32, 32, 64, 64, 128, 192, 64, 96, 32, 48, 16)
    cout = (16, 16, 32, 32, 64, 64, 128, 128, 64, 64, 32, 32, 16, 16)
    lvl = (0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0)
    return sum(27 * a * b * (S >> l) ** 3 for a, b, l in zip(cin, cout, lvl))


def time_forward(S: int, B: int, reps: int = 5) -> dict:
    """CUDA-event time of the network's forward pass on B random samples."""
    import torch
    net = GuessNet(S, B)
    net.set_params(init_params(net.n_params, 0))
    inp = torch.rand((B, S, S, S, GUESS_CHANNELS), device="cuda", dtype=torch.float32)
    out = torch.empty((B, S, S, S), device="cuda", dtype=torch.float32)
    net.forward(inp, out, B)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        net.forward(inp, out, B)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    net.close()
    return {"S": S, "batch": B, "ms": ms, "us_per_sample": 1e3 * ms / B,
            "tflops": 2.0 * conv_macs(S) * B / (ms / 1e3) / 1e12}


def evaluate(model_blob: bytes, seeds, tol: float = 1e-8, log=None) -> dict:
    """CG iterations to tol from zero and from the learned guess on every pair
    of the seeded tiny-form workloads (each solved twice, warm_start 0 and 2)."""
    import torch
    it0 = it2 = pairs = 0
    de = 0.0
    guess_ms = solve0 = solve2 = 0.0
    ex0 = ex2 = None
    for seed in seeds:
        w = synth.config0(seed)
        if ex0 is None:
            ex0 = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, tol, precision=1, warm_start=0)
            ex2 = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, tol, precision=1, warm_start=2)
            ex2.load_guess_model(model_blob)
        phi = torch.from_numpy(w.orbitals()).cuda()
        cen = torch.from_numpy(np.ascontiguousarray(w.centers)).cuda()
        D = torch.empty_like(phi)
        e0 = ex0.compute(phi, cen, D)
        s0 = ex0.stats()
        e2 = ex2.compute(phi, cen, D)
        s2 = ex2.stats()
        it0 += s0["iters_total"]
        it2 += s2["iters_total"]
        pairs += s0["n_pair"]
        de = max(de, abs(e2 - e0) / w.n)
        guess_ms += s2["guess_ms"]
        solve0 += s0["solve_ms"]
        solve2 += s2["solve_ms"]
    ex0.close()
    ex2.close()
    out = {"pairs": pairs, "tol": tol, "iters_per_pair_zero": it0 / pairs, "iters_per_pair_learned": it2 / pairs,
           "iteration_ratio": it2 / it0, "max_dE_per_orbital": de, "guess_us_per_pair": 1e3 * guess_ms / pairs,
           "solve_ms_zero": solve0, "solve_ms_learned": solve2}
    if log:
        log(str(out))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--train-seeds", type=int, default=140)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--workload", default="tiny", choices=["tiny", "water64"])
    ap.add_argument("--per-workload", type=int, default=400, help="water64: pairs kept per workload")
    ap.add_argument("--eval-seeds", type=int, default=0, help="held-out tiny-form workloads to evaluate on")
    ap.add_argument("--eval-tol", type=float, default=1e-8)
    ap.add_argument("--time-forward", type=int, nargs=2, metavar=("S", "B"), default=None,
                    help="only time the forward pass on B random samples of side S (He-initialised weights)")
    args = ap.parse_args()
    import torch
    if args.time_forward:
        print(time_forward(*args.time_forward))
        return
    t0 = time.time()
    if args.workload == "tiny":
        S = CUBE
        inp, tgt = solve_and_export(range(1000, 1000 + args.train_seeds), torch=torch)
    else:
        S = CUBE_R24
        inp, tgt = solve_and_export(range(1000, 1000 + args.train_seeds), S=S, torch=torch, workload=synth.config1,
                                    per_workload=args.per_workload)
    print(f"{inp.shape[0]} samples in {time.time() - t0:.1f} s", flush=True)
    net, hist = train(inp, tgt, S=S, epochs=args.epochs, batch=args.batch, lr=args.lr, log=print)
    blob = guess_model_blob(S, net.get_params())
    if args.out:
        with open(args.out, "wb") as f:
            f.write(blob)
    print("loss", hist[0], "->", hist[-1], flush=True)
    if args.eval_seeds and args.workload == "tiny":
        del inp, tgt
        net.close()
        torch.cuda.empty_cache()
        evaluate(blob, range(5000, 5000 + args.eval_seeds), tol=args.eval_tol, log=print)


if __name__ == "__main__":
    main()
