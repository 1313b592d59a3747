"""Seeded synthetic inputs: Gaussian orbital clusters that stand in for MLWFs.

The paper measures on liquid-water MLWFs from PBE0 Car-Parrinello runs
((H2O)64/128/256, Sec. IV.A and IV.B). Those orbitals cannot be regenerated
without a full DFT code, so every workload here is synthetic: real orbitals

    phi_i(g) = N_i * exp(-alpha_i |d|^2) * (1 + p_i . d),   d = minimg(r_g - C_i)

sampled on the periodic grid r_g = g * delta (grid points numbered 0..N-1,
Eq. l2g), with N_i fixed by the discrete normalisation sum_g phi_i^2 dV = 1.

This module holds none of the exact-exchange arithmetic: it only draws random
numbers and evaluates the input orbitals. Both the CUDA path and the CPU
oracle consume what it returns; neither is imported here.

Draw order (fixed, numpy PCG64 ``default_rng(seed)``):
  1. centers (independent: rejection in the cell with a minimum min-image
     separation; clustered: cluster centres by the same rejection, then per
     orbital an offset uniform in a ball of radius ``spread``, drawn by
     rejection from the enclosing cube),
  2. alpha_i ~ U(alpha_lo, alpha_hi), one per orbital,
  3. p_i ~ N(0, p_sigma^2) per component, three per orbital.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

__all__ = [
    "Workload",
    "orbitals",
    "orbital",
    "config0",
    "config1",
    "config2",
    "config4",
    "orbitals_torch",
    "tiny",
    "CONFIGS",
]


@dataclasses.dataclass
class Workload:
    """One synthetic exact-exchange problem (inputs plus solver parameters)."""

    name: str
    cell: np.ndarray          # (3,) orthorhombic cell lengths L_a, bohr
    grid: np.ndarray          # (3,) grid points N_a per axis
    centers: np.ndarray       # (n, 3) orbital centres C_i in [0, L), bohr
    alphas: np.ndarray        # (n,) Gaussian exponents, bohr^-2
    pvecs: np.ndarray         # (n, 3) linear factors p_i, bohr^-1
    r_pair: float             # pair cutoff, bohr (strict <); inf = all pairs
    r_pe: int                 # PE ball radius, grid points
    r_me: int                 # ME ball radius, grid points
    l_max: int                # multipole order
    tol: float                # relative CG residual ||r|| / ||b||
    seed: int
    radii_mode: int = 0       # 0 fixed radii, 1 per-pair radii from alpha
    note: str = ""

    @property
    def n(self) -> int:
        return int(self.centers.shape[0])

    @property
    def delta(self) -> np.ndarray:
        return self.cell / self.grid

    def orbitals(self, dtype=np.float64) -> np.ndarray:
        return orbitals(self.cell, self.grid, self.centers, self.alphas, self.pvecs, dtype=dtype)

    def centers_flat(self) -> np.ndarray:
        return np.ascontiguousarray(self.centers, dtype=np.float64)


def _minimg(x: np.ndarray, length: float) -> np.ndarray:
    return x - length * np.floor(x / length + 0.5)


def orbital(cell, grid, center, alpha, pvec, out: Optional[np.ndarray] = None) -> np.ndarray:
    """Evaluate one normalised orbital on the full periodic grid (C order)."""
    cell = np.asarray(cell, dtype=np.float64)
    grid = np.asarray(grid, dtype=np.int64)
    axes = []
    for a in range(3):
        r = np.arange(grid[a], dtype=np.float64) * (cell[a] / grid[a])
        axes.append(_minimg(r - center[a], cell[a]))
    dx, dy, dz = axes
    ex, ey, ez = (np.exp(-alpha * d * d) for d in axes)
    if out is None:
        out = np.empty((int(grid[0]), int(grid[1]), int(grid[2])), dtype=np.float64)
    # exp(-a|d|^2)(1 + p.d) is a sum of separable terms; evaluate it plane by plane
    exy = ex[:, None] * ey[None, :]
    lin_xy = 1.0 + pvec[0] * dx[:, None] + pvec[1] * dy[None, :]
    out[...] = (exy * lin_xy)[:, :, None] * ez[None, None, :]
    out += (exy * pvec[2])[:, :, None] * (ez * dz)[None, None, :]
    dv = float(np.prod(cell / grid))
    norm = math.sqrt(float(np.einsum("ijk,ijk->", out, out)) * dv)
    out /= norm
    return out


def orbitals(cell, grid, centers, alphas, pvecs, dtype=np.float64) -> np.ndarray:
    """All orbitals as one (n, N0, N1, N2) C-contiguous array."""
    n = len(centers)
    grid = np.asarray(grid, dtype=np.int64)
    phi = np.empty((n, int(grid[0]), int(grid[1]), int(grid[2])), dtype=np.float64)
    for i in range(n):
        orbital(cell, grid, centers[i], float(alphas[i]), pvecs[i], out=phi[i])
    return phi if dtype == np.float64 else phi.astype(dtype)


def orbitals_torch(w: "Workload", device="cuda", chunk: int = 16, out=None):
    """The workload's orbitals evaluated on a torch device, same formula and
    normalisation as :func:`orbital` (float64, [n][N0][N1][N2]); for inputs too
    large to build in host memory. Values agree with the NumPy path to
    rounding; tests that compare against the oracle copy the device arrays
    back rather than rebuilding them."""
    import torch
    cell = np.asarray(w.cell, dtype=np.float64)
    grid = [int(g) for g in w.grid]
    n = w.n
    if out is None:
        out = torch.empty((n, grid[0], grid[1], grid[2]), dtype=torch.float64, device=device)
    axes = [torch.arange(grid[a], dtype=torch.float64, device=device) * (cell[a] / grid[a]) for a in range(3)]
    dv = float(np.prod(cell / np.asarray(grid)))
    cen = torch.as_tensor(np.asarray(w.centers, dtype=np.float64), device=device)
    alp = torch.as_tensor(np.asarray(w.alphas, dtype=np.float64), device=device)
    pv = torch.as_tensor(np.asarray(w.pvecs, dtype=np.float64), device=device)
    for i0 in range(0, n, chunk):
        i1 = min(n, i0 + chunk)
        d = []
        e = []
        for a in range(3):
            x = axes[a][None, :] - cen[i0:i1, a:a + 1]
            x = x - cell[a] * torch.floor(x / cell[a] + 0.5)
            d.append(x)
            e.append(torch.exp(-alp[i0:i1, None] * x * x))
        exy = e[0][:, :, None] * e[1][:, None, :]
        lin = 1.0 + pv[i0:i1, 0, None, None] * d[0][:, :, None] + pv[i0:i1, 1, None, None] * d[1][:, None, :]
        blk = out[i0:i1]
        blk.copy_((exy * lin)[:, :, :, None] * e[2][:, None, None, :])
        blk.add_((exy * pv[i0:i1, 2, None, None])[:, :, :, None] * (e[2] * d[2])[:, None, None, :])
        norm = torch.sqrt(torch.einsum("bxyz,bxyz->b", blk, blk) * dv)
        blk.div_(norm[:, None, None, None])
    return out


def _minimg_dist(a: np.ndarray, b: np.ndarray, cell: np.ndarray) -> np.ndarray:
    d = _minimg(b - a, cell)
    return np.sqrt(np.sum(d * d, axis=-1))


def _reject_points(rng, count: int, cell: np.ndarray, min_sep: float, max_tries: int = 200000):
    pts = []
    tries = 0
    while len(pts) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("rejection sampling of centres did not finish")
        c = rng.uniform(0.0, 1.0, size=3) * cell
        if pts and np.min(_minimg_dist(np.asarray(pts), c[None, :], cell)) < min_sep:
            continue
        pts.append(c)
    return np.asarray(pts)


def _ball_offsets(rng, count: int, radius: float) -> np.ndarray:
    out = np.empty((count, 3))
    for i in range(count):
        while True:
            v = rng.uniform(-radius, radius, size=3)
            if v @ v <= radius * radius:
                out[i] = v
                break
    return out


def _clustered(rng, n_clusters, per, cell, min_sep, spread):
    cc = _reject_points(rng, n_clusters, cell, min_sep)
    offs = _ball_offsets(rng, n_clusters * per, spread)
    centers = np.repeat(cc, per, axis=0) + offs
    return np.mod(centers, cell)


def config0(seed: int = 0) -> Workload:
    """Plain method, tiny: L = 9 bohr, 48^3, 8 independent orbitals, all 36 pairs."""
    rng = np.random.default_rng(seed)
    cell = np.full(3, 9.0)
    grid = np.full(3, 48, dtype=np.int64)
    centers = _reject_points(rng, 8, cell, 1.5)
    alphas = rng.uniform(0.8, 1.5, size=8)
    pvecs = rng.normal(0.0, 0.3, size=(8, 3))
    return Workload("tiny-8orb-48^3", cell, grid, centers, alphas, pvecs,
                    r_pair=math.inf, r_pe=16, r_me=20, l_max=6, tol=1e-10, seed=seed)


def config1(seed: int = 0, r_pair: float = 10.0) -> Workload:
    """Water-64 scale: L = 23.5 bohr, 120^3, 64 clusters x 4 orbitals, R_pair = 10 bohr."""
    rng = np.random.default_rng(seed)
    cell = np.full(3, 23.5)
    grid = np.full(3, 120, dtype=np.int64)
    centers = _clustered(rng, 64, 4, cell, 4.5, 0.7)
    alphas = rng.uniform(0.8, 1.5, size=256)
    pvecs = rng.normal(0.0, 0.3, size=(256, 3))
    return Workload("water64-256orb-120^3", cell, grid, centers, alphas, pvecs,
                    r_pair=r_pair, r_pe=24, r_me=32, l_max=6, tol=1e-8, seed=seed)


def config2(seed: int = 0) -> Workload:
    """Batched uneven: L = 29.6 bohr, 150^3, 128 clusters x 4, alpha ~ U(0.5, 2)."""
    rng = np.random.default_rng(seed)
    cell = np.full(3, 29.6)
    grid = np.full(3, 150, dtype=np.int64)
    centers = _clustered(rng, 128, 4, cell, 4.5, 0.7)
    alphas = rng.uniform(0.5, 2.0, size=512)
    pvecs = rng.normal(0.0, 0.3, size=(512, 3))
    return Workload("batched128-512orb-150^3", cell, grid, centers, alphas, pvecs,
                    r_pair=10.0, r_pe=32, r_me=43, l_max=6, tol=1e-8, seed=seed,
                    radii_mode=1)


def config4(seed: int = 0, step: int = 0) -> Workload:
    """MD-like sequence: L = 37.3 bohr, 190^3, 256 clusters x 4; ``step`` drifts the inputs.

    Step s applies s independent draws of C += N(0, 0.02^2) and
    alpha <- alpha (1 + 0.01 xi), xi ~ N(0, 1), from a second stream seeded
    with (seed, 4); p stays fixed.
    """
    rng = np.random.default_rng(seed)
    cell = np.full(3, 37.3)
    grid = np.full(3, 190, dtype=np.int64)
    centers = _clustered(rng, 256, 4, cell, 4.5, 0.7)
    alphas = rng.uniform(0.8, 1.5, size=1024)
    pvecs = rng.normal(0.0, 0.3, size=(1024, 3))
    drift = np.random.default_rng([seed, 4])
    for _ in range(step):
        centers = np.mod(centers + drift.normal(0.0, 0.02, size=centers.shape), cell)
        alphas = alphas * (1.0 + 0.01 * drift.normal(0.0, 1.0, size=alphas.shape))
    return Workload(f"md256-1024orb-190^3-step{step}", cell, grid, centers, alphas, pvecs,
                    r_pair=10.0, r_pe=24, r_me=32, l_max=6, tol=1e-8, seed=seed)


def tiny(seed: int = 0, n: int = 4, npts: int = 24, length: float = 6.0, r_pe: int = 6,
         r_me: int = 9, r_pair: float = math.inf, tol: float = 1e-10,
         alpha=(0.8, 1.5), p_sigma: float = 0.3, min_sep: float = 1.0) -> Workload:
    """Small independent-orbital case for pins and quick parity checks."""
    rng = np.random.default_rng(seed)
    cell = np.full(3, float(length))
    grid = np.full(3, int(npts), dtype=np.int64)
    centers = _reject_points(rng, n, cell, min_sep)
    alphas = rng.uniform(alpha[0], alpha[1], size=n)
    pvecs = rng.normal(0.0, p_sigma, size=(n, 3))
    return Workload(f"tiny-{n}orb-{npts}^3", cell, grid, centers, alphas, pvecs,
                    r_pair=r_pair, r_pe=r_pe, r_me=r_me, l_max=6, tol=tol, seed=seed)


CONFIGS = {"cfg0": config0, "cfg1": config1, "cfg2": config2, "cfg4": config4}
