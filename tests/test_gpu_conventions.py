"""The C ABI's failure conventions on the GPU.

- A bounded device wait that runs out is reported as EXX_ETIMEOUT with its
  own count, and the context stays usable. The test makes one wait run out
  through the test-only option inject_wait_timeout: thread 0 of every CTA of
  the cluster solver polls an mbarrier that nothing arrives on and no copy or
  store targets, so the launch still completes every exchange and cluster
  barrier it would have run; its results stay those of a normal call.
- NaN inputs propagate and exx_get_stats counts them (n_nonfinite); the call
  itself completes (no solve spins on a NaN).
- The FP64-pipe probe behind the plain CG's roofline returns a plausible rate.
"""
import numpy as np
import pytest

import oracle
from paper_1911_10630_gb300 import synth
from tests.gpu_util import D_GATE_MAXREL, E_GATE_PER_ORBITAL, d_maxrel, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


@pytest.fixture(scope="module")
def tiny():
    w = synth.tiny(seed=0, n=4, npts=24, length=6.0, r_pe=6, r_me=9, tol=1e-10)
    phi = w.orbitals()
    return w, phi, oracle.exx_workload(w, tol=1e-13, orbitals=phi)


@pytest.mark.parametrize("warm_start", [0, 1])
def test_injected_wait_timeout_then_clean_call(torch, tiny, warm_start):
    from paper_1911_10630_gb300.exx import EXX_ETIMEOUT, EXX_OK, Exx
    w, phi, ref = tiny
    dphi = torch.from_numpy(phi).cuda()
    dcen = torch.from_numpy(np.ascontiguousarray(w.centers)).cuda()
    dD = torch.empty_like(dphi)
    ex = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, precision=1, solver_kind=2,
             warm_start=warm_start, inject_wait_timeout=1)
    e1 = ex.compute(dphi, dcen, dD, allow_timeout=True)
    st1 = ex.stats()
    assert ex.last_status == EXX_ETIMEOUT
    assert st1["n_timeouts"] == st1["grid_ctas"]  # one run-out wait per CTA
    # the injected wait changes nothing else: the results meet the gates
    assert abs(e1 - ref["E_xx"]) / w.n <= E_GATE_PER_ORBITAL
    assert d_maxrel(dD.cpu().numpy(), ref["D"]) <= D_GATE_MAXREL
    # the next call on the same context is clean
    e2 = ex.compute(dphi, dcen, dD)
    st2 = ex.stats()
    assert ex.last_status == EXX_OK and st2["n_timeouts"] == 0
    assert abs(e2 - ref["E_xx"]) / w.n <= E_GATE_PER_ORBITAL
    ex.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_orbital_propagates_and_is_counted(torch, tiny, precision):
    from paper_1911_10630_gb300.exx import EXX_OK, Exx
    w, phi, _ = tiny
    bad = phi.copy()
    g = np.floor(w.centers[2] / w.delta + 0.5).astype(int) % w.grid
    bad[2, g[0], g[1], g[2]] = np.nan  # on the PE ball of every pair of orbital 2
    dphi = torch.from_numpy(bad).cuda()
    dcen = torch.from_numpy(np.ascontiguousarray(w.centers)).cuda()
    dD = torch.empty_like(dphi)
    ex = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, precision=precision)
    e = ex.compute(dphi, dcen, dD, allow_noconv=True)
    st = ex.stats()
    pairs = ex.pairs()
    with_2 = int(np.sum((pairs["i"] == 2) | (pairs["j"] == 2)))
    assert with_2 > 0 and st["n_nonfinite"] >= 1
    assert st["n_nonfinite"] <= with_2
    assert np.isnan(e)
    # the pairs without orbital 2 are untouched: finite energies
    keep = (pairs["i"] != 2) & (pairs["j"] != 2)
    assert np.all(np.isfinite(pairs["e_pair"][keep]))
    ex.close()
    # a clean call after it on a fresh context is unaffected
    ex = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, precision=precision)
    e = ex.compute(torch.from_numpy(phi).cuda(), dcen, dD)
    assert ex.last_status == EXX_OK and ex.stats()["n_nonfinite"] == 0 and np.isfinite(e)
    ex.close()


def test_nan_centre_is_counted(torch, tiny):
    from paper_1911_10630_gb300.exx import Exx
    w, phi, _ = tiny
    cen = np.ascontiguousarray(w.centers).copy()
    cen[1, 0] = np.nan
    dphi = torch.from_numpy(phi).cuda()
    dD = torch.empty_like(dphi)
    ex = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, precision=1)
    ex.compute(dphi, torch.from_numpy(cen).cuda(), dD, allow_noconv=True)
    st = ex.stats()
    assert st["n_nonfinite"] >= 1
    pairs = ex.pairs()
    # a NaN distance fails the strict R_pair test: orbital 1 takes part in no pair
    assert not np.any((pairs["i"] == 1) | (pairs["j"] == 1))
    ex.close()


def test_fp64_probe_rate_is_plausible(torch):
    from paper_1911_10630_gb300 import exx
    r = exx.probe_fp64_rate()
    # GB300 issues FP64 at a small fraction of its FP32 rate: about 1.2 TFLOP/s
    assert 0.3 < r < 20.0, r
