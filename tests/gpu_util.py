"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare with the oracle under the accuracy gates of the method."""
import math

import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1911_10630_gb300 import build, exx
    build.build(quiet=True)  # raises if nvcc fails: no silent fallback
    exx.load()
    return torch


def run_gpu(w, phi=None, torch=None, allow_noconv=False, **opts):
    """One exx_compute call on the workload; returns E_xx, D (numpy), pairs, stats."""
    import torch as _t
    torch = torch or _t
    from paper_1911_10630_gb300.exx import Exx
    phi = w.orbitals() if phi is None else phi
    dphi = torch.from_numpy(phi).cuda()
    dcen = torch.from_numpy(np.ascontiguousarray(w.centers)).cuda()
    dD = torch.empty_like(dphi)
    dal = None
    if getattr(w, "radii_mode", 0) == 1:
        opts.setdefault("radii_mode", 1)
        dal = torch.from_numpy(np.ascontiguousarray(w.alphas, dtype=np.float64)).cuda()
    expect = opts.pop("expect_status", None)
    ex = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, opts.pop("tol", w.tol), **opts)
    if expect is not None:  # a call expected to fail: report its status and message
        from paper_1911_10630_gb300.exx import ExxError
        try:
            e = ex.compute(dphi, dcen, dD, alphas=dal, allow_noconv=allow_noconv)
            err = ""
        except ExxError as x:
            e, err = float("nan"), str(x)
        torch.cuda.synchronize()
        return dict(E_xx=e, status=ex.last_status, error=err, ex=ex)
    e = ex.compute(dphi, dcen, dD, alphas=dal, allow_noconv=allow_noconv)
    torch.cuda.synchronize()
    out = dict(E_xx=e, D=dD.cpu().numpy(), pairs=ex.pairs(), stats=ex.stats(), ex=ex, dphi=dphi,
               status=ex.last_status)
    return out


def d_maxrel(D, Dref):
    """max_i ||D^i - Dref^i||_inf / ||Dref^i||_inf over orbitals with a nonzero reference."""
    n = D.shape[0]
    worst = 0.0
    for i in range(n):
        den = np.max(np.abs(Dref[i]))
        if den == 0.0:
            continue
        worst = max(worst, float(np.max(np.abs(D[i] - Dref[i])) / den))
    return worst


def gamma_xx(D, Dref):
    """Relative L1 force error averaged over orbitals (Eqs. gammaxx_i, gammaxx)."""
    vals = [np.sum(np.abs(Dref[i] - D[i])) / np.sum(np.abs(Dref[i])) for i in range(D.shape[0])]
    return float(np.mean(vals))


E_GATE_PER_ORBITAL = 1e-7   # |E_GPU - E_oracle| / N_o, Ha
D_GATE_MAXREL = 1e-6        # max_i ||dD^i||_inf / ||D^i||_inf

finite = math.isfinite
