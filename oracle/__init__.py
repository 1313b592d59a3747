"""FP64 CPU oracle for the pair-Poisson exact exchange (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg
may import this package. The CUDA library never imports, links or calls it.

The arithmetic lives in ``oracle_exx.c`` (plain C, FP64, OpenMP over pairs);
this module only builds it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle_exx.c")
_LIB = os.path.join(_HERE, "liboracle_exx.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_i = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile oracle_exx.c into liboracle_exx.so next to it (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-std=c11", "-shared", "-fPIC",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.oracle_version.restype = ctypes.c_int
            L.oracle_num_threads.restype = ctypes.c_int
            L.oracle_pair_list.restype = ctypes.c_int
            L.oracle_pair_list.argtypes = [ctypes.c_int, _d, _d, _i, ctypes.c_double, ctypes.c_int, _i, _i, _i]
            L.oracle_proto_subdomain.restype = ctypes.c_int
            L.oracle_proto_subdomain.argtypes = [ctypes.c_int, ctypes.c_int, _i, _i, _i]
            L.oracle_real_ylm.restype = None
            L.oracle_real_ylm.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, _d]
            L.oracle_laplacian_box.restype = None
            L.oracle_laplacian_box.argtypes = [_d, _i, _d, _d]
            L.oracle_laplacian_periodic.restype = None
            L.oracle_laplacian_periodic.argtypes = [_d, _i, _d, _d]
            L.oracle_cg_periodic.restype = ctypes.c_int
            L.oracle_cg_periodic.argtypes = [_d, _i, _d, _d, ctypes.c_double, ctypes.c_int]
            L.oracle_ball_cg.restype = ctypes.c_int
            L.oracle_ball_cg.argtypes = [ctypes.c_int, ctypes.c_int, _d, _d, _d, ctypes.c_double, ctypes.c_int]
            L.oracle_ball_apply.restype = ctypes.c_int
            L.oracle_ball_apply.argtypes = [ctypes.c_int, ctypes.c_int, _d, _d, _d]
            L.oracle_pair_solve.restype = ctypes.c_double
            L.oracle_pair_solve.argtypes = [_d, _i, _d, ctypes.c_int, ctypes.c_int, _i, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_int, _d, _d, _d, _d, _d, _i]
            L.oracle_pair_radius.restype = ctypes.c_int
            L.oracle_pair_radius.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int, ctypes.c_int, _i]
            L.oracle_pair_list_radii.restype = ctypes.c_int
            L.oracle_pair_list_radii.argtypes = [ctypes.c_int, _d, _d, _i, ctypes.c_double, _d, ctypes.c_double,
                                                 ctypes.c_int, ctypes.c_int, ctypes.c_int, _i, _i, _i, _i, _i]
            L.oracle_exx_pairs_radii.restype = ctypes.c_double
            L.oracle_exx_pairs_radii.argtypes = [_d, _i, _d, ctypes.c_int, ctypes.c_int, _i, _i, _i, _i, _i,
                                                 ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_int, _d, _i, _d, _i, ctypes.c_int]
            L.oracle_exx_pairs.restype = ctypes.c_double
            L.oracle_exx_pairs.argtypes = [_d, _i, _d, ctypes.c_int, ctypes.c_int, _i, _i, _i, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int, _d, _i, _d, _i, ctypes.c_int]
            _lib = L
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(_d)


def _ip(a):
    return None if a is None else a.ctypes.data_as(_i)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def pair_list(centers, cell, grid, r_pair):
    """Step II pair list: returns (i, j, g_ij) as int32 arrays, i-major, j ascending."""
    centers = _f64(centers).reshape(-1, 3)
    n = centers.shape[0]
    cap = n * (n + 1) // 2
    pi = np.empty(cap, np.int32)
    pj = np.empty(cap, np.int32)
    g = np.empty((cap, 3), np.int32)
    r = float(r_pair) if math.isfinite(r_pair) else 1e300
    cnt = lib().oracle_pair_list(n, _dp(centers), _dp(_f64(cell)), _ip(_i32(grid)), r, cap,
                                 _ip(pi), _ip(pj), _ip(g))
    if cnt < 0:
        raise RuntimeError("pair list overflow")
    return pi[:cnt].copy(), pj[:cnt].copy(), g[:cnt].copy()


LN_INV_EPS = math.log(1e14)  # ln(1/eps) of the per-pair radius rule, eps = 1e-14


def pair_radius(ai, aj, d2, delta, r_min=12, r_max=32):
    """Per-pair (R_PE, R_ME) of the spread-dependent subdomain rule."""
    rme = ctypes.c_int()
    r = lib().oracle_pair_radius(float(ai), float(aj), float(d2), float(delta), LN_INV_EPS, int(r_min), int(r_max),
                                 ctypes.byref(rme))
    return r, rme.value


def pair_list_radii(centers, cell, grid, r_pair, alphas, r_min=12, r_max=32):
    """Pair list plus per-pair radii: (i, j, g, r_pe, r_me)."""
    centers = _f64(centers).reshape(-1, 3)
    n = centers.shape[0]
    cap = n * (n + 1) // 2
    pi = np.empty(cap, np.int32)
    pj = np.empty(cap, np.int32)
    g = np.empty((cap, 3), np.int32)
    rpe = np.empty(cap, np.int32)
    rme = np.empty(cap, np.int32)
    r = float(r_pair) if math.isfinite(r_pair) else 1e300
    cnt = lib().oracle_pair_list_radii(n, _dp(centers), _dp(_f64(cell)), _ip(_i32(grid)), r, _dp(_f64(alphas)),
                                       LN_INV_EPS, int(r_min), int(r_max), cap, _ip(pi), _ip(pj), _ip(g),
                                       _ip(rpe), _ip(rme))
    if cnt < 0:
        raise RuntimeError("pair list overflow")
    return tuple(a[:cnt].copy() for a in (pi, pj, g, rpe, rme))


def proto_subdomain(r_pe, r_me):
    """Algorithm 2: (offsets (N_ME, 3) PE-first, N_PE)."""
    npe = ctypes.c_int()
    nme = ctypes.c_int()
    lib().oracle_proto_subdomain(r_pe, r_me, None, ctypes.byref(npe), ctypes.byref(nme))
    off = np.empty((nme.value, 3), np.int32)
    lib().oracle_proto_subdomain(r_pe, r_me, _ip(off), None, None)
    return off, npe.value


def real_ylm(lmax, x, y, z):
    out = np.zeros((lmax + 1) ** 2)
    lib().oracle_real_ylm(lmax, float(x), float(y), float(z), _dp(out))
    return out


def laplacian_box(f, delta):
    f = _f64(f)
    out = np.empty_like(f)
    lib().oracle_laplacian_box(_dp(f), _ip(_i32(f.shape)), _dp(_f64(delta)), _dp(out))
    return out


def laplacian_periodic(f, delta):
    f = _f64(f)
    out = np.empty_like(f)
    lib().oracle_laplacian_periodic(_dp(f), _ip(_i32(f.shape)), _dp(_f64(delta)), _dp(out))
    return out


def cg_periodic(b, delta, tol=1e-13, maxit=100000):
    b = _f64(b)
    v = np.empty_like(b)
    it = lib().oracle_cg_periodic(_dp(b), _ip(_i32(b.shape)), _dp(_f64(delta)), _dp(v), tol, maxit)
    return v, it


def ball_cg(r_pe, r_me, delta, b, x0=None, tol=1e-13, maxit=100000):
    b = _f64(b)
    x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
    it = lib().oracle_ball_cg(r_pe, r_me, _dp(_f64(delta)), _dp(b), _dp(x), tol, maxit)
    return x, it


def ball_apply(r_pe, r_me, delta, p):
    p = _f64(p)
    out = np.empty_like(p)
    lib().oracle_ball_apply(r_pe, r_me, _dp(_f64(delta)), _dp(p), _dp(out))
    return out


def pair_solve(cell, grid, orbitals, i, j, gij, r_pe, r_me, lmax=6, tol=1e-13, tol_report=None,
               maxit=100000, x0=None):
    """Steps III-V for one pair. Returns dict(E, rho, Q, v, b, iters, rep_iters)."""
    orbitals = _f64(orbitals)
    off, npe = proto_subdomain(r_pe, r_me)
    nme = off.shape[0]
    rho = np.empty(nme)
    Q = np.empty((lmax + 1) ** 2)
    v = np.empty(nme)
    b = np.empty(npe)
    iters = np.empty(2, np.int32)
    e = lib().oracle_pair_solve(_dp(_f64(cell)), _ip(_i32(grid)), _dp(orbitals), int(i), int(j),
                                _ip(_i32(gij)), r_pe, r_me, lmax, tol,
                                tol if tol_report is None else tol_report, maxit,
                                None if x0 is None else _dp(_f64(x0)),
                                _dp(rho), _dp(Q), _dp(v), _dp(b), _ip(iters))
    return dict(E=e, rho=rho, Q=Q, v=v, b=b, iters=int(iters[0]), rep_iters=int(iters[1]),
                off=off, n_pe=npe)


def exx(cell, grid, orbitals, pairs, r_pe, r_me, lmax=6, tol=1e-13, tol_report=None, maxit=100000,
        want_d=True, dmask=None, solve_all=True):
    """Step V over a pair list (i, j, g) or (i, j, g, r_pe, r_me) with per-pair
    radii. Returns dict(E_xx, E_pair, iters, rep_iters, D)."""
    orbitals = _f64(orbitals)
    pi, pj, g = (_i32(a) for a in pairs[:3])
    rpe = _i32(pairs[3]) if len(pairs) > 3 else None
    rme = _i32(pairs[4]) if len(pairs) > 4 else None
    npair = len(pi)
    n_orb = orbitals.shape[0]
    e_pair = np.empty(npair)
    iters = np.empty((npair, 2), np.int32)
    D = np.empty_like(orbitals) if want_d else None
    mask = None if dmask is None else _i32(dmask)
    exx_v = lib().oracle_exx_pairs_radii(_dp(_f64(cell)), _ip(_i32(grid)), _dp(orbitals), n_orb, npair,
                                         _ip(pi), _ip(pj), _ip(g), _ip(rpe), _ip(rme), r_pe, r_me, lmax, tol,
                                         tol if tol_report is None else tol_report, maxit, _dp(e_pair),
                                         _ip(iters), _dp(D), _ip(mask), 1 if solve_all else 0)
    return dict(E_xx=exx_v, E_pair=e_pair, iters=iters[:, 0].copy(), rep_iters=iters[:, 1].copy(), D=D)


def exx_workload(w, tol=1e-13, tol_report=None, want_d=True, orbitals=None):
    """Full pipeline for a synth.Workload (per-pair radii when w.radii_mode == 1)."""
    phi = w.orbitals() if orbitals is None else orbitals
    if getattr(w, "radii_mode", 0) == 1:
        pairs = pair_list_radii(w.centers, w.cell, w.grid, w.r_pair, w.alphas, 12, w.r_pe)
    else:
        pairs = pair_list(w.centers, w.cell, w.grid, w.r_pair)
    out = exx(w.cell, w.grid, phi, pairs, w.r_pe, w.r_me, w.l_max, tol=tol,
              tol_report=w.tol if tol_report is None else tol_report, want_d=want_d)
    out["pairs"] = pairs
    return out
