"""Thin ctypes binding of the C ABI in include/exx.h (same names, marshalling only).

Every computation runs in the CUDA library ``libexx_gb300.so``; this module
only converts arguments. Device arrays are torch CUDA tensors (their
``data_ptr()`` is passed through); host arrays are numpy arrays. Loading fails
loudly when the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libexx_gb300.so")

EXX_OK, EXX_EINVAL, EXX_ENOMEM, EXX_ECUDA, EXX_ENOCONV, EXX_ENOPAIR, EXX_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
_STATUS = {0: "EXX_OK", -1: "EXX_EINVAL", -2: "EXX_ENOMEM", -3: "EXX_ECUDA", -4: "EXX_ENOCONV",
           -5: "EXX_ENOPAIR", -6: "EXX_ETIMEOUT"}


class ExxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class exx_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("batched", ctypes.c_int), ("warm_start", ctypes.c_int),
                ("radii_mode", ctypes.c_int), ("max_iter", ctypes.c_int), ("inner_max_iter", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("threads", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("solver_kind", ctypes.c_int), ("cluster_size", ctypes.c_int), ("update_drop", ctypes.c_double),
                ("lane_map", ctypes.c_int), ("autotune", ctypes.c_int), ("r_pe_nonself", ctypes.c_int),
                ("r_me_nonself", ctypes.c_int), ("fixed_residual", ctypes.c_int),
                ("deterministic", ctypes.c_int), ("preconditioner", ctypes.c_int),
                ("inject_wait_timeout", ctypes.c_int)]


class exx_stats(ctypes.Structure):
    _fields_ = [("n_pair", ctypes.c_int), ("n_nonconv", ctypes.c_int), ("iters_max", ctypes.c_int),
                ("iters_p50", ctypes.c_int), ("iters_p99", ctypes.c_int), ("iters_total", ctypes.c_longlong),
                ("point_iters", ctypes.c_longlong), ("refine_max", ctypes.c_int), ("solve_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("n_pe", ctypes.c_int), ("n_me", ctypes.c_int),
                ("solver_kind", ctypes.c_int), ("cluster_size", ctypes.c_int), ("grid_ctas", ctypes.c_int),
                ("threads", ctypes.c_int), ("phase_ms", ctypes.c_double * 4), ("lane_map", ctypes.c_int),
                ("n_candidates", ctypes.c_int), ("tune_ms", ctypes.c_double),
                ("guess_ms", ctypes.c_double), ("n_timeouts", ctypes.c_int), ("n_nonfinite", ctypes.c_int),
                ("n_clipped", ctypes.c_int), ("n_dropped", ctypes.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["phase_ms"] = list(self.phase_ms)
        return d


_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_d = ctypes.POINTER(ctypes.c_double)
_i = ctypes.POINTER(ctypes.c_int)
_f = ctypes.POINTER(ctypes.c_float)
_ctx_p = ctypes.c_void_p

# (name, restype, argtypes): every function declared in include/exx.h
SIGNATURES = [
    ("exx_default_options", exx_options, []),
    ("exx_init", ctypes.c_int, [ctypes.POINTER(_ctx_p), _d, _i, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, ctypes.c_double, ctypes.POINTER(exx_options)]),
    ("exx_compute", ctypes.c_int, [_ctx_p, _vp, _vp, ctypes.c_int, _vp, _d, _vp, _vp]),
    ("exx_compute_async", ctypes.c_int, [_ctx_p, _vp, _vp, ctypes.c_int, _vp, _vp, _vp, _vp]),
    ("exx_compute_host", ctypes.c_int, [_ctx_p, _vp, _vp, ctypes.c_int, _vp, _d, _vp, _vp]),
    ("exx_compute_boxes", ctypes.c_int, [_ctx_p, _vp, _vp, _i, _vp, ctypes.c_int, _vp, _d, _vp, _vp]),
    ("exx_get_stats", ctypes.c_int, [_ctx_p, ctypes.POINTER(exx_stats)]),
    ("exx_get_pairs", ctypes.c_int, [_ctx_p, _i, _i, _i, _i, _d, _i, ctypes.c_int, _i]),
    ("exx_debug_pair", ctypes.c_int, [_ctx_p, _vp, ctypes.c_int, _d, _d, _d, _vp]),
    ("exx_apply_operator", ctypes.c_int, [_ctx_p, _vp, _vp, _vp]),
    ("exx_apply_preconditioner", ctypes.c_int, [_ctx_p, _vp, _vp, _vp]),
    ("exx_ball_size", ctypes.c_int, [_ctx_p, _i, _i]),
    ("exx_radius_classes", ctypes.c_int, [_ctx_p, _i, _i, _i, ctypes.c_int, _i]),
    ("exx_quad_map", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    ("exx_ball_tables", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _i, _i, _i, ctypes.c_size_t, _i, _i]),
    ("exx_mg_levels", ctypes.c_int, [ctypes.c_int, _d, _i, _i, _i, ctypes.c_int, _i, _d, ctypes.c_size_t]),
    ("exx_load_guess_model", ctypes.c_int, [_ctx_p, _vp, ctypes.c_size_t]),
    ("exx_pair_list_static", ctypes.c_int, [_vp, ctypes.c_int, _d, _i, ctypes.c_double, _vp, ctypes.c_int, _i,
                                            _vp]),
    ("exx_probe_fp64_rate", ctypes.c_int, [_d, _vp]),
    ("exx_last_error", ctypes.c_char_p, [_ctx_p]),
    ("exx_destroy", None, [_ctx_p]),
    # include/exx_guess.h
    ("exx_guess_param_count", ctypes.c_size_t, []),
    ("exx_guess_create", ctypes.c_int, [ctypes.POINTER(_ctx_p), ctypes.c_int, ctypes.c_int]),
    ("exx_guess_set_params", ctypes.c_int, [_ctx_p, _f, ctypes.c_size_t]),
    ("exx_guess_get_params", ctypes.c_int, [_ctx_p, _f, ctypes.c_size_t]),
    ("exx_guess_forward", ctypes.c_int, [_ctx_p, _vp, _vp, ctypes.c_int, _vp]),
    ("exx_guess_gradient", ctypes.c_int, [_ctx_p, _vp, _vp, ctypes.c_int, _f, _f, _vp]),
    ("exx_guess_train_step", ctypes.c_int, [_ctx_p, _vp, _vp, ctypes.c_int, ctypes.c_float, _f, _vp]),
    ("exx_guess_destroy", None, [_ctx_p]),
    ("exx_export_samples", ctypes.c_int, [_ctx_p, _vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _i, _vp]),
    ("exx_unet_conv3d", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp]),
]


def load(path: Optional[str] = None):
    """Loads libexx_gb300.so (raises OSError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise OSError(f"{p} is missing: build it with paper_1911_10630_gb300.build.build()")
            L = ctypes.CDLL(p)
            for name, res, args in SIGNATURES:
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def exx_default_options() -> exx_options:
    return load().exx_default_options()


def exx_last_error(ctx=None) -> str:
    s = load().exx_last_error(ctx)
    return s.decode() if s else ""


def probe_fp64_rate(stream=None) -> float:
    """Measured FP64 FMA rate of the current device in TFLOP/s (exx_probe_fp64_rate)."""
    out = ctypes.c_double(0.0)
    _check(load().exx_probe_fp64_rate(ctypes.byref(out), _stream_handle(stream)))
    return float(out.value)


def _check(status: int, ctx=None):
    if status != EXX_OK:
        raise ExxError(status, exx_last_error(ctx))


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return int(t)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:  # pragma: no cover
            return None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class Exx:
    """Owns one exx_ctx (exx_init ... exx_destroy)."""

    def __init__(self, cell, grid, r_pair, r_pe, r_me, l_max=6, tol=1e-8, **opts):
        L = load()
        o = L.exx_default_options()
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        self.options = o
        cell = np.ascontiguousarray(cell, np.float64)
        grid = np.ascontiguousarray(grid, np.int32)
        self.cell, self.grid = cell, grid
        self.r_pe, self.r_me = int(r_pe), int(r_me)
        ctx = _ctx_p()
        rp = float(r_pair) if math.isfinite(r_pair) else float("inf")
        st = L.exx_init(ctypes.byref(ctx), cell.ctypes.data_as(_d), grid.ctypes.data_as(_i), rp, int(r_pe),
                        int(r_me), int(l_max), float(tol), ctypes.byref(o))
        _check(st, None)
        self._ctx = ctx
        self.last_status = EXX_OK

    @property
    def ctx(self):
        return self._ctx

    def close(self):
        if getattr(self, "_ctx", None):
            load().exx_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def compute(self, orbitals, centers, d_xx, alphas=None, stream=None, allow_noconv=False,
                allow_timeout=False) -> float:
        """exx_compute on device tensors; returns E_xx, fills d_xx."""
        e = ctypes.c_double()
        st = load().exx_compute(self._ctx, _ptr(orbitals), _ptr(centers), int(centers.shape[0]), _ptr(alphas),
                                ctypes.byref(e), _ptr(d_xx), _stream_handle(stream))
        self.last_status = st
        if not (st == EXX_OK or (allow_noconv and st == EXX_ENOCONV) or (allow_timeout and st == EXX_ETIMEOUT)):
            _check(st, self._ctx)
        return e.value

    def compute_async(self, orbitals, centers, d_xx, e_xx_dev, alphas=None, stream=None) -> None:
        """exx_compute_async: E_xx into e_xx_dev (a float64 device tensor of one element), no host wait;
        the outcome is in stats()."""
        st = load().exx_compute_async(self._ctx, _ptr(orbitals), _ptr(centers), int(centers.shape[0]), _ptr(alphas),
                                      _ptr(e_xx_dev), _ptr(d_xx), _stream_handle(stream))
        self.last_status = st
        _check(st, self._ctx)

    def compute_boxes(self, boxes, origin, centers, d_boxes, alphas=None, stream=None, allow_noconv=False) -> float:
        """exx_compute_boxes on device tensors: boxes [n][B0][B1][B2], origin [n][3] int32; returns E_xx."""
        e = ctypes.c_double()
        bd = np.ascontiguousarray(boxes.shape[1:], np.int32)
        st = load().exx_compute_boxes(self._ctx, _ptr(boxes), _ptr(origin), bd.ctypes.data_as(_i), _ptr(centers),
                                      int(centers.shape[0]), _ptr(alphas), ctypes.byref(e), _ptr(d_boxes),
                                      _stream_handle(stream))
        self.last_status = st
        if not (st == EXX_OK or (allow_noconv and st == EXX_ENOCONV)):
            _check(st, self._ctx)
        return e.value

    def compute_host(self, orbitals, centers, d_xx, alphas=None, stream=None, allow_noconv=False) -> float:
        """exx_compute_host on numpy arrays; returns E_xx, fills d_xx (numpy)."""
        e = ctypes.c_double()
        st = load().exx_compute_host(self._ctx, _ptr(orbitals), _ptr(centers), int(centers.shape[0]),
                                     _ptr(alphas), ctypes.byref(e), _ptr(d_xx), _stream_handle(stream))
        self.last_status = st
        if not (st == EXX_OK or (allow_noconv and st == EXX_ENOCONV)):
            _check(st, self._ctx)
        return e.value

    def load_guess_model(self, blob: bytes):
        """exx_load_guess_model: the learned warm start used by warm_start = 2."""
        b = ctypes.create_string_buffer(bytes(blob), len(blob))
        _check(load().exx_load_guess_model(self._ctx, b, len(blob)), self._ctx)

    def export_samples(self, orbitals, S: int, inp, target, cap: int, stream=None) -> int:
        """exx_export_samples after a warm_start = 1 call; returns the call's pair count."""
        n = ctypes.c_int()
        _check(load().exx_export_samples(self._ctx, _ptr(orbitals), int(S), _ptr(inp), _ptr(target), int(cap),
                                         ctypes.byref(n), _stream_handle(stream)), self._ctx)
        return n.value

    def stats(self) -> dict:
        s = exx_stats()
        _check(load().exx_get_stats(self._ctx, ctypes.byref(s)), self._ctx)
        return s.as_dict()

    def pairs(self):
        n = ctypes.c_int()
        _check(load().exx_get_pairs(self._ctx, None, None, None, None, None, None, 0, ctypes.byref(n)), self._ctx)
        m = n.value
        pi = np.empty(m, np.int32)
        pj = np.empty(m, np.int32)
        g = np.empty((m, 3), np.int32)
        radii = np.empty((m, 2), np.int32)
        e = np.empty(m)
        it = np.empty(m, np.int32)
        _check(load().exx_get_pairs(self._ctx, pi.ctypes.data_as(_i), pj.ctypes.data_as(_i), g.ctypes.data_as(_i),
                                    radii.ctypes.data_as(_i), e.ctypes.data_as(_d), it.ctypes.data_as(_i), m,
                                    ctypes.byref(n)), self._ctx)
        return dict(i=pi, j=pj, g=g, radii=radii, e_pair=e, iters=it)

    def radius_classes(self):
        """exx_radius_classes: (R_PE, CTAs per pair or 0, resident clusters) per class."""
        n = ctypes.c_int()
        _check(load().exx_radius_classes(self._ctx, None, None, None, 0, ctypes.byref(n)), self._ctx)
        r, c, k = (np.zeros(n.value, np.int32) for _ in range(3))
        _check(load().exx_radius_classes(self._ctx, r.ctypes.data_as(_i), c.ctypes.data_as(_i), k.ctypes.data_as(_i),
                                         n.value, ctypes.byref(n)), self._ctx)
        return [(int(a), int(b), int(x)) for a, b, x in zip(r, c, k)]

    def ball_size(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(load().exx_ball_size(self._ctx, ctypes.byref(a), ctypes.byref(b)), self._ctx)
        return a.value, b.value

    def debug_pair(self, orbitals, index, stream=None):
        n_pe, n_me = self.ball_size()
        rho = np.empty(n_me)
        v = np.empty(n_me)
        b = np.empty(n_pe)
        _check(load().exx_debug_pair(self._ctx, _ptr(orbitals), int(index), rho.ctypes.data_as(_d),
                                     v.ctypes.data_as(_d), b.ctypes.data_as(_d), _stream_handle(stream)), self._ctx)
        return dict(rho=rho, v=v, b=b)

    def apply_operator(self, p, ap, stream=None):
        _check(load().exx_apply_operator(self._ctx, _ptr(p), _ptr(ap), _stream_handle(stream)), self._ctx)

    def apply_preconditioner(self, r, z, stream=None):
        _check(load().exx_apply_preconditioner(self._ctx, _ptr(r), _ptr(z), _stream_handle(stream)), self._ctx)


class GuessNet:
    """Owns one exx_guess (the learned warm start's U-Net; include/exx_guess.h)."""

    def __init__(self, S: int, batch_max: int):
        L = load()
        h = ctypes.c_void_p()
        _check(L.exx_guess_create(ctypes.byref(h), int(S), int(batch_max)))
        self._h = h
        self.S = int(S)
        self.batch_max = int(batch_max)
        self.n_params = int(L.exx_guess_param_count())

    def set_params(self, params: np.ndarray):
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(load().exx_guess_set_params(self._h, p.ctypes.data_as(_f), p.size))

    def get_params(self) -> np.ndarray:
        p = np.empty(self.n_params, np.float32)
        _check(load().exx_guess_get_params(self._h, p.ctypes.data_as(_f), p.size))
        return p

    def forward(self, inp, out, batch: int, stream=None):
        _check(load().exx_guess_forward(self._h, _ptr(inp), _ptr(out), int(batch), _stream_handle(stream)))

    def gradient(self, inp, target, batch: int, want_grad: bool = True, stream=None):
        loss = ctypes.c_float()
        g = np.empty(self.n_params, np.float32) if want_grad else None
        _check(load().exx_guess_gradient(self._h, _ptr(inp), _ptr(target), int(batch), ctypes.byref(loss),
                                         g.ctypes.data_as(_f) if g is not None else None, _stream_handle(stream)))
        return float(loss.value), g

    def train_step(self, inp, target, batch: int, lr: float, stream=None) -> float:
        loss = ctypes.c_float()
        _check(load().exx_guess_train_step(self._h, _ptr(inp), _ptr(target), int(batch), float(lr),
                                           ctypes.byref(loss), _stream_handle(stream)))
        return float(loss.value)

    def close(self):
        if getattr(self, "_h", None):
            load().exx_guess_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # pragma: no cover
            pass


def unet_conv3d(x, w, bias, mask, y, batch, D, H, W, cin, cout, mode, stream=None):
    """One tensor-core 3x3x3 convolution (exx_unet_conv3d); device tensors."""
    _check(load().exx_unet_conv3d(_ptr(x), _ptr(w), _ptr(bias), _ptr(mask), _ptr(y), int(batch), int(D), int(H),
                                  int(W), int(cin), int(cout), int(mode), _stream_handle(stream)))


GUESS_MAGIC = 0x47585845
GUESS_CHANNELS = 3  # network input: rho / s, multipole boundary values, ball mask


def quad_map(r_pe: int, cluster_size: int, threads: int, quads: int, bank_aware: int = 0):
    """exx_quad_map: the cluster solver's quad thread map built on the host.
    Returns (quad_pk, quad_k) as int32 arrays [cluster_size][quads][threads]
    and the info vector (see include/exx.h)."""
    n = cluster_size * quads * threads
    pk = np.zeros(n, np.int32)
    kk = np.zeros(n, np.int32)
    info = np.zeros(4 + 4 * cluster_size, np.int32)
    _check(load().exx_quad_map(int(r_pe), int(cluster_size), int(threads), int(quads), int(bank_aware),
                               pk.ctypes.data, kk.ctypes.data, n, info.ctypes.data))
    shape = (cluster_size, quads, threads)
    return pk.reshape(shape), kk.reshape(shape), info


def ball_tables(r_pe: int, r_me: int):
    """exx_ball_tables: the proto-subdomain tables built on the host. Returns a
    dict with int32 arrays off (packed), cube and near (one entry per ME ball
    point, PE ball first) and the counts n_pe, n_me."""
    n_pe, n_me = ctypes.c_int(0), ctypes.c_int(0)
    lib = load()
    status = lib.exx_ball_tables(int(r_pe), int(r_me), (ctypes.c_int * 1)(), None, None, 0, ctypes.byref(n_pe),
                                 ctypes.byref(n_me))
    if n_me.value == 0:
        _check(status)
    n = n_me.value
    off, cube, near = (np.zeros(n, np.int32) for _ in range(3))
    _check(lib.exx_ball_tables(int(r_pe), int(r_me), off.ctypes.data_as(_i), cube.ctypes.data_as(_i),
                               near.ctypes.data_as(_i), n, ctypes.byref(n_pe), ctypes.byref(n_me)))
    return dict(off=off, cube=cube, near=near, n_pe=n_pe.value, n_me=n_me.value)


def mg_levels(r_pe: int, delta, want_minv: bool = False):
    """exx_mg_levels: the multigrid hierarchy of a PE ball, built on the host.
    Returns a dict with int32 arrays radius, points, side (levels 1..L) and,
    with want_minv, the coarsest level's inverse operator [n][n]."""
    d = np.ascontiguousarray(delta, dtype=np.float64)
    cap = 8
    radius, points, side = (np.zeros(cap, np.int32) for _ in range(3))
    levels = ctypes.c_int(0)
    lib = load()
    _check(lib.exx_mg_levels(int(r_pe), d.ctypes.data_as(_d), radius.ctypes.data_as(_i), points.ctypes.data_as(_i),
                             side.ctypes.data_as(_i), cap, ctypes.byref(levels), None, 0))
    L = levels.value
    out = dict(radius=radius[:L].copy(), points=points[:L].copy(), side=side[:L].copy())
    if want_minv:
        n = int(points[L - 1])
        m = np.zeros(n * n, np.float64)
        _check(lib.exx_mg_levels(int(r_pe), d.ctypes.data_as(_d), radius.ctypes.data_as(_i),
                                 points.ctypes.data_as(_i), side.ctypes.data_as(_i), cap, ctypes.byref(levels),
                                 m.ctypes.data_as(_d), m.size))
        out["minv"] = m.reshape(n, n)
    return out


def guess_model_blob(S: int, params: np.ndarray) -> bytes:
    """Model blob of exx_load_guess_model: {magic, 2, S, count} then the FP32 parameters."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    return np.array([GUESS_MAGIC, 2, int(S), p.size], dtype=np.int32).tobytes() + p.tobytes()
