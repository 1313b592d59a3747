"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Integer work (the pair list, the grid centres) is compared bit for bit;
floating-point results against the accuracy gates of the method:
|E_xx(GPU) - E_xx(oracle)| / N_o <= 1e-7 Ha and
max_i ||D^i(GPU) - D^i(oracle)||_inf / ||D^i(oracle)||_inf <= 1e-6, with the
oracle's CG converged to 1e-13. Intermediates of single pairs (rho, the shell
potential, the right-hand side, the operator) are compared element by element.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1911_10630_gb300 import synth
from tests.gpu_util import D_GATE_MAXREL, E_GATE_PER_ORBITAL, d_maxrel, gamma_xx, require_gpu, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


@pytest.fixture(scope="module")
def cfg0():
    w = synth.config0()
    phi = w.orbitals()
    ref = oracle.exx_workload(w, tol=1e-13, orbitals=phi)
    return w, phi, ref


def _pairs_equal(gpu_pairs, ref_pairs):
    pi, pj, g = ref_pairs
    np.testing.assert_array_equal(gpu_pairs["i"], pi)
    np.testing.assert_array_equal(gpu_pairs["j"], pj)
    np.testing.assert_array_equal(gpu_pairs["g"], g)


@pytest.mark.parametrize("precision,solver_kind,cluster_size,lane_map", [
    (0, 1, 0, None), (1, 1, 0, None), (1, 2, 9, None), (1, 2, 8, None), (1, 2, 4, None), (1, 2, 2, None),
    (1, 2, 8, 0), (1, 2, 4, 2), (1, 2, 9, 3), (1, 2, 4, 3), (1, 2, 9, 4), (1, 2, 9, 5)])
def test_cfg0_end_to_end(torch, cfg0, precision, solver_kind, cluster_size, lane_map):
    w, phi, ref = cfg0
    extra = {} if lane_map is None else dict(lane_map=lane_map, autotune=0)
    out = run_gpu(w, phi, torch=torch, precision=precision, solver_kind=solver_kind, cluster_size=cluster_size,
                  **extra)
    assert out["stats"]["solver_kind"] == solver_kind
    if cluster_size:
        assert out["stats"]["cluster_size"] == cluster_size
    if lane_map is not None:
        assert out["stats"]["lane_map"] == lane_map
    _pairs_equal(out["pairs"], ref["pairs"])
    assert out["stats"]["n_pair"] == 36 and out["stats"]["n_nonconv"] == 0
    assert abs(out["E_xx"] - ref["E_xx"]) / w.n <= E_GATE_PER_ORBITAL
    assert d_maxrel(out["D"], ref["D"]) <= D_GATE_MAXREL
    assert gamma_xx(out["D"], ref["D"]) <= D_GATE_MAXREL
    np.testing.assert_allclose(out["pairs"]["e_pair"], ref["E_pair"], rtol=1e-8, atol=1e-12)
    # E_xx is the fixed-multiplicity sum of the per-pair energies
    m = np.where(out["pairs"]["i"] == out["pairs"]["j"], 1.0, 2.0)
    assert abs(out["E_xx"] + np.sum(m * out["pairs"]["e_pair"])) <= 1e-12 * abs(out["E_xx"])
    if precision == 0:
        # FP64 CG to the same tolerance takes the oracle's iteration count (+-2)
        assert np.max(np.abs(out["pairs"]["iters"] - ref["rep_iters"])) <= 2


@pytest.mark.parametrize("solver_kind", [1, 2])
def test_cfg0_deterministic_d_xx(torch, cfg0, solver_kind):
    """deterministic = 1: D_xx from fixed-point integer atomics meets the gates
    and repeats bit for bit (the FP64-atomic default need not)."""
    w, phi, ref = cfg0
    from paper_1911_10630_gb300.exx import Exx
    dphi = torch.from_numpy(phi).cuda()
    dcen = torch.from_numpy(np.ascontiguousarray(w.centers)).cuda()
    ex = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, precision=1, solver_kind=solver_kind,
             deterministic=1)
    outs = []
    for _ in range(2):
        D = torch.empty_like(dphi)
        e = ex.compute(dphi, dcen, D)
        outs.append((e, D.cpu().numpy()))
    ex.close()
    (e0, D0), (e1, D1) = outs
    assert e0 == e1 and np.array_equal(D0, D1)
    assert abs(e0 - ref["E_xx"]) / w.n <= E_GATE_PER_ORBITAL
    assert d_maxrel(D0, ref["D"]) <= D_GATE_MAXREL


@pytest.mark.parametrize("fixed_residual", [1, 2])
def test_cfg0_residual_paths(torch, cfg0, fixed_residual):
    """The quad map with halo planes with the FP64 stencil for the refinement
    residuals (1) and with the fixed-point copy forced past its bound on every
    pair (2), which must fall back to the FP64 stencil: both meet the gates."""
    w, phi, ref = cfg0
    out = run_gpu(w, phi, torch=torch, precision=1, solver_kind=2, cluster_size=9, lane_map=5, autotune=0,
                  fixed_residual=fixed_residual)
    assert out["stats"]["lane_map"] == 5 and out["stats"]["n_nonconv"] == 0
    assert abs(out["E_xx"] - ref["E_xx"]) / w.n <= E_GATE_PER_ORBITAL
    assert d_maxrel(out["D"], ref["D"]) <= D_GATE_MAXREL
    np.testing.assert_allclose(out["pairs"]["e_pair"], ref["E_pair"], rtol=1e-8, atol=1e-12)


@pytest.mark.parametrize("scale", [1e3, 1e-3])
def test_fixed_point_residuals_at_large_and_small_potentials(torch, cfg0, scale):
    """The fixed-point residual stencil (the exponent of its scale chosen per
    pair from a bound on |v|) against the FP64 stencil on orbitals scaled by
    1e3 and 1e-3 (rho and v by 1e6 and 1e-6): the same energies to the solve's
    tolerance, both within the gates of the oracle scaled alike."""
    w, phi, ref = cfg0
    outs = {}
    for fixed in (0, 1):
        outs[fixed] = run_gpu(w, phi * scale, torch=torch, precision=1, solver_kind=2, cluster_size=9, lane_map=5,
                              autotune=0, fixed_residual=fixed)
        assert outs[fixed]["stats"]["n_nonconv"] == 0
    e_ref = ref["E_xx"] * scale ** 4
    for fixed in (0, 1):
        assert abs(outs[fixed]["E_xx"] - e_ref) / w.n <= E_GATE_PER_ORBITAL * scale ** 4
    np.testing.assert_allclose(outs[0]["pairs"]["e_pair"], outs[1]["pairs"]["e_pair"], rtol=1e-8,
                               atol=1e-12 * scale ** 4)


def test_deterministic_d_xx_range_is_guarded(torch, cfg0):
    """deterministic = 1 keeps D_xx as integers at scale 2^40: contributions
    |v phi| >= 2^22 cannot be represented; they are dropped and counted, and
    the call fails instead of returning a wrapped sum."""
    from paper_1911_10630_gb300.exx import EXX_EINVAL
    w, phi, _ = cfg0
    out = run_gpu(w, phi * 400.0, torch=torch, precision=1, deterministic=1, allow_noconv=False,
                  expect_status=EXX_EINVAL)
    assert out["status"] == EXX_EINVAL
    assert "2^22" in out["error"]


@pytest.mark.parametrize("precision", [0, 1])
def test_cfg0_pair_intermediates(torch, cfg0, precision):
    w, phi, ref = cfg0
    out = run_gpu(w, phi, torch=torch, precision=precision)
    pi, pj, g = ref["pairs"]
    for k in (0, 1, 9, 35):
        got = out["ex"].debug_pair(out["dphi"], k)
        orc = oracle.pair_solve(w.cell, w.grid, phi, pi[k], pj[k], g[k], w.r_pe, w.r_me, w.l_max, tol=1e-13)
        npe = orc["n_pe"]
        np.testing.assert_array_equal(got["rho"][:npe], orc["rho"][:npe])  # one IEEE product per point
        sh_scale = np.max(np.abs(orc["v"][npe:]))
        layer = _boundary_layer(orc["off"], npe)
        dv = np.abs(got["v"][npe:] - orc["v"][npe:])
        # Eq. me on the shell: FP64 where the stencil legs of the PE ball read it,
        # FP32 on the rest (only the D_xx scatter reads it)
        assert np.max(dv[layer]) <= 1e-12 * sh_scale
        assert np.max(dv) <= 1e-6 * sh_scale
        assert np.max(np.abs(got["b"] - orc["b"])) <= 1e-11 * np.max(np.abs(orc["b"]))
        assert np.max(np.abs(got["v"][:npe] - orc["v"][:npe])) <= 1e-8 * np.max(np.abs(orc["v"][:npe]))


def _boundary_layer(off, npe):
    """Shell points within three axial steps of a PE point."""
    pe = {tuple(o) for o in off[:npe]}
    out = np.zeros(len(off) - npe, bool)
    for t, o in enumerate(off[npe:]):
        for a in range(3):
            for q in (1, 2, 3):
                for sg in (-1, 1):
                    u = list(o)
                    u[a] += sg * q
                    if tuple(u) in pe:
                        out[t] = True
    return out


def test_operator_matches_oracle(torch):
    from paper_1911_10630_gb300.exx import Exx
    cell, grid = np.array([7.0, 7.5, 8.0]), np.array([40, 42, 44])
    ex = Exx(cell, grid, math.inf, 9, 13, 6, 1e-8)
    n_pe, _ = ex.ball_size()
    p = np.random.default_rng(0).normal(size=n_pe)
    dp = torch.from_numpy(p).cuda()
    dap = torch.empty_like(dp)
    ex.apply_operator(dp, dap)
    ref = oracle.ball_apply(9, 13, cell / grid, p)
    assert np.max(np.abs(dap.cpu().numpy() - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("precision,solver_kind,lane_map", [(0, 1, None), (1, 1, None), (1, 2, None), (1, 2, 3), (1, 2, 4), (1, 2, 5)])
def test_small_anisotropic_ragged(torch, precision, solver_kind, lane_map):
    # non-cubic grid and cell, small balls, finite R_pair, pairs across faces
    w = synth.tiny(seed=3, n=6, npts=28, length=6.5, r_pe=5, r_me=9, r_pair=3.0, tol=1e-10)
    w.grid = np.array([28, 30, 26])
    w.cell = np.array([6.5, 7.1, 6.2])
    w.centers = np.mod(w.centers, w.cell)
    w.centers[0] = [0.05, 3.0, 6.1]
    w.centers[1] = [6.3, 3.2, 0.2]
    phi = w.orbitals()
    ref = oracle.exx_workload(w, tol=1e-13, orbitals=phi)
    extra = {} if lane_map is None else dict(lane_map=lane_map, autotune=0)
    out = run_gpu(w, phi, torch=torch, precision=precision, solver_kind=solver_kind, **extra)
    assert out["stats"]["solver_kind"] == solver_kind
    if lane_map is not None:
        assert out["stats"]["lane_map"] == lane_map
    _pairs_equal(out["pairs"], ref["pairs"])
    assert abs(out["E_xx"] - ref["E_xx"]) / w.n <= E_GATE_PER_ORBITAL
    assert d_maxrel(out["D"], ref["D"]) <= D_GATE_MAXREL


def test_single_orbital_and_self_pairs_only(torch):
    w = synth.tiny(seed=4, n=1, npts=32, length=8.0, r_pe=8, r_me=12)
    phi = w.orbitals()
    ref = oracle.exx_workload(w, tol=1e-13, orbitals=phi)
    out = run_gpu(w, phi, torch=torch)
    assert out["stats"]["n_pair"] == 1
    assert abs(out["E_xx"] - ref["E_xx"]) <= E_GATE_PER_ORBITAL
    w2 = synth.tiny(seed=5, n=5, npts=32, length=8.0, r_pe=8, r_me=12, r_pair=0.5, min_sep=1.0)
    phi2 = w2.orbitals()
    ref2 = oracle.exx_workload(w2, tol=1e-13, orbitals=phi2)
    out2 = run_gpu(w2, phi2, torch=torch)
    assert out2["stats"]["n_pair"] == 5
    assert abs(out2["E_xx"] - ref2["E_xx"]) / 5 <= E_GATE_PER_ORBITAL
    assert d_maxrel(out2["D"], ref2["D"]) <= D_GATE_MAXREL


def test_deterministic_energy_and_graph_replay(torch, cfg0):
    w, phi, _ = cfg0
    from paper_1911_10630_gb300.exx import Exx
    dphi = torch.from_numpy(phi).cuda()
    dc = torch.from_numpy(np.ascontiguousarray(w.centers)).cuda()
    dD = torch.empty_like(dphi)
    a = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, 6, w.tol, batched=1)
    b = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, 6, w.tol, batched=0)
    e1 = a.compute(dphi, dc, dD)
    e2 = a.compute(dphi, dc, dD)  # graph replay
    e3 = b.compute(dphi, dc, dD)  # eager launches
    assert e1 == e2 == e3
    np.testing.assert_array_equal(a.pairs()["e_pair"], b.pairs()["e_pair"])


def test_host_buffers_match_device(torch, cfg0):
    w, phi, ref = cfg0
    from paper_1911_10630_gb300.exx import Exx
    ex = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, 6, w.tol)
    D = np.empty_like(phi)
    e = ex.compute_host(phi, np.ascontiguousarray(w.centers), D)
    dev = run_gpu(w, phi, torch=torch)
    assert e == dev["E_xx"]
    assert d_maxrel(D, dev["D"]) <= 1e-12
    assert abs(e - ref["E_xx"]) / w.n <= E_GATE_PER_ORBITAL


def test_host_buffers_pinned_and_pageable(torch, cfg0):
    """exx_compute_host copies pinned, device-mapped host buffers with the SMs
    (copy16_kernel) and any other memory with the copy engine: both give the
    same results bit for bit, also from a pinned buffer 8 bytes off the 16-byte
    boundary (which takes the copy engine). D_xx is summed deterministically
    so that the calls can be compared bit for bit."""
    w, phi, _ = cfg0
    from paper_1911_10630_gb300.exx import Exx
    ex = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, 6, w.tol, deterministic=1)
    cen = np.ascontiguousarray(w.centers)
    D0 = np.empty_like(phi)
    e0 = ex.compute_host(phi, cen, D0)
    hphi = torch.from_numpy(phi).pin_memory()
    hD = torch.empty(phi.shape, dtype=torch.float64).pin_memory()
    e1 = ex.compute_host(hphi, torch.from_numpy(cen).pin_memory(), hD)
    assert e1 == e0
    np.testing.assert_array_equal(hD.numpy(), D0)
    flat = torch.empty(phi.size + 1, dtype=torch.float64).pin_memory()
    off = flat[1:].view(phi.shape)
    off.copy_(torch.from_numpy(phi))
    hD2 = torch.empty(phi.size + 1, dtype=torch.float64).pin_memory()[1:].view(phi.shape)
    e2 = ex.compute_host(off, cen, hD2)
    assert e2 == e0
    np.testing.assert_array_equal(hD2.numpy(), D0)
    ex.close()


def test_async_call_matches_and_reports_in_stats(torch, cfg0):
    """exx_compute_async writes E_xx to device memory with no host wait: two calls
    queued back to back on one stream give the synchronous call's E_xx bit for bit
    (fixed-order reduction) and the same D_xx, a kernel the caller queues after
    the call reads the finished E_xx, and the outcome of a call that hits the
    iteration cap is in the statistics rather than in its return value."""
    w, phi, _ = cfg0
    from paper_1911_10630_gb300.exx import Exx, ExxError
    dphi = torch.from_numpy(phi).cuda()
    dcen = torch.from_numpy(np.ascontiguousarray(w.centers)).cuda()
    ex = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, deterministic=1)
    D0 = torch.empty_like(dphi)
    e0 = ex.compute(dphi, dcen, D0)
    s = torch.cuda.Stream()
    E = torch.zeros(2, dtype=torch.float64, device="cuda")
    D1 = torch.empty_like(dphi)
    with torch.cuda.stream(s):
        ex.compute_async(dphi, dcen, D1, E[0:1], stream=s)
        ex.compute_async(dphi, dcen, D1, E[1:2], stream=s)
        twice = E * 2.0  # queued after the calls on the same stream
    s.synchronize()
    assert E[0].item() == e0 and E[1].item() == e0 and twice[1].item() == 2.0 * e0
    assert torch.equal(D1, D0)
    st = ex.stats()
    assert st["n_pair"] == 36 and st["n_nonconv"] == 0 and st["n_dropped"] == 0
    ex.close()
    capped = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, max_iter=5)
    capped.compute_async(dphi, dcen, D1, E[0:1])
    assert capped.stats()["n_nonconv"] == 36
    with pytest.raises(ExxError, match="device"):
        capped.compute_async(dphi, dcen, D1, torch.zeros(1, dtype=torch.float64))  # host memory
    capped.close()


def test_iteration_cap_reports_nonconvergence(torch, cfg0):
    w, phi, _ = cfg0
    out = run_gpu(w, phi, torch=torch, allow_noconv=True, max_iter=5)
    assert out["status"] == -4
    assert out["stats"]["n_nonconv"] == 36
    assert np.all(out["pairs"]["iters"] <= 5)
    assert np.isfinite(out["E_xx"])


@pytest.mark.parametrize("precision,lane_map,preconditioner,cluster", [
    (1, None, 1, 0), (1, None, 1, 2), (1, None, 0, 0), (1, 2, 0, 0), (1, 3, 0, 0), (1, 4, 0, 0), (1, 5, 0, 0),
    (0, None, 0, 0)])
def test_water64_full_size_sampled(torch, precision, lane_map, preconditioner, cluster):
    """The bench workload (water-64 scale, 120^3, 256 orbitals, R_pair = 10 bohr,
    R_PE/R_ME = 24/32, tol 1e-8) in the configuration bench.py times (the FP32
    multigrid PCG in FP64 refinement, one CTA per pair), on the autotuned cluster
    solver and with its z-run and quad thread maps forced, and the multigrid CG
    on 2-CTA clusters; checked on sampled pairs and sampled orbitals the oracle
    computes one by one."""
    w = synth.config1()
    phi = w.orbitals()
    extra = {} if lane_map is None else dict(lane_map=lane_map, autotune=0)
    extra["preconditioner"] = preconditioner
    if cluster:  # the multigrid CG on clusters of this size
        extra.update(solver_kind=2, cluster_size=cluster)
    out = run_gpu(w, phi, torch=torch, precision=precision, **extra)
    if lane_map is not None:
        assert out["stats"]["lane_map"] == lane_map
    ref_pairs = oracle.pair_list(w.centers, w.cell, w.grid, w.r_pair)
    _pairs_equal(out["pairs"], ref_pairs)
    npair = len(ref_pairs[0])
    assert out["stats"]["n_nonconv"] == 0
    rng = np.random.default_rng(1)
    its = out["pairs"]["iters"]
    sample = np.unique(np.concatenate([rng.choice(npair, 20, replace=False), np.argsort(its)[-4:]]))
    sub = tuple(a[sample] for a in ref_pairs)
    orc = oracle.exx(w.cell, w.grid, phi, sub, w.r_pe, w.r_me, w.l_max, tol=1e-13, want_d=False)
    np.testing.assert_allclose(out["pairs"]["e_pair"][sample], orc["E_pair"], rtol=0,
                               atol=E_GATE_PER_ORBITAL / 4)
    # D of two sampled orbitals: every pair touching them, summed by the oracle
    orbs = [int(ref_pairs[0][sample[0]]), int(ref_pairs[1][sample[-1]])]
    mask = np.zeros(w.n, np.int32)
    mask[orbs] = 1
    touch = np.nonzero(mask[ref_pairs[0]] | mask[ref_pairs[1]])[0]
    sub2 = tuple(a[touch] for a in ref_pairs)
    orc2 = oracle.exx(w.cell, w.grid, phi, sub2, w.r_pe, w.r_me, w.l_max, tol=1e-13, want_d=True, dmask=mask)
    for i in orbs:
        den = np.max(np.abs(orc2["D"][i]))
        assert np.max(np.abs(out["D"][i] - orc2["D"][i])) <= D_GATE_MAXREL * den
    # E_xx is the multiplicity-weighted sum of the pair energies
    m = np.where(out["pairs"]["i"] == out["pairs"]["j"], 1.0, 2.0)
    assert abs(out["E_xx"] + np.sum(m * out["pairs"]["e_pair"])) <= 1e-12 * abs(out["E_xx"])


# --------------------------------------------------------------------------
# Per-pair radii, largest pairs first (batched uneven workloads)
# --------------------------------------------------------------------------

def _pairs_radii_equal(gpu_pairs, ref_pairs):
    pi, pj, g, rpe, rme = ref_pairs
    np.testing.assert_array_equal(gpu_pairs["i"], pi)
    np.testing.assert_array_equal(gpu_pairs["j"], pj)
    np.testing.assert_array_equal(gpu_pairs["g"], g)
    np.testing.assert_array_equal(gpu_pairs["radii"][:, 0], rpe)
    np.testing.assert_array_equal(gpu_pairs["radii"][:, 1], rme)


@pytest.mark.parametrize("precision,solver_kind", [(1, 0), (1, 1), (0, 0)])
def test_per_pair_radii_small(torch, precision, solver_kind):
    """Per-pair radii against the oracle: precision 1 runs the cluster solver
    in radius classes (one CTA per ball below R_PE 14, clusters above), or the
    one-CTA solver on request; precision 0 the one-CTA FP64 solver."""
    w = synth.tiny(seed=8, n=6, npts=48, length=9.6, r_pe=16, r_me=22, alpha=(0.5, 2.0), tol=1e-10, min_sep=1.2)
    w.radii_mode = 1
    phi = w.orbitals()
    ref = oracle.exx_workload(w, tol=1e-13, orbitals=phi)
    assert len(set(ref["pairs"][3])) >= 3  # several radii in play
    out = run_gpu(w, phi, torch=torch, precision=precision, solver_kind=solver_kind)
    assert out["stats"]["solver_kind"] == (2 if precision == 1 and solver_kind == 0 else 1)
    _pairs_radii_equal(out["pairs"], ref["pairs"])
    assert out["stats"]["n_nonconv"] == 0
    assert abs(out["E_xx"] - ref["E_xx"]) / w.n <= E_GATE_PER_ORBITAL
    assert d_maxrel(out["D"], ref["D"]) <= D_GATE_MAXREL
    np.testing.assert_allclose(out["pairs"]["e_pair"], ref["E_pair"], rtol=1e-7, atol=1e-12)


@pytest.mark.parametrize("precision", [1, 0])
def test_self_and_nonself_radii(torch, precision):
    """Separate self / non-self proto-subdomains (radii_mode 2): self pairs on
    R_PE/R_ME = 16/20, non-self pairs on 12/16, against the oracle with the
    same per-pair radii."""
    w = synth.config0()
    phi = w.orbitals()
    pi, pj, g = oracle.pair_list(w.centers, w.cell, w.grid, w.r_pair)
    self_ = pi == pj
    rpe = np.where(self_, 16, 12).astype(np.int32)
    rme = np.where(self_, 20, 16).astype(np.int32)
    ref = oracle.exx(w.cell, w.grid, phi, (pi, pj, g, rpe, rme), 16, 20, w.l_max, tol=1e-13, want_d=True)
    out = run_gpu(w, phi, torch=torch, precision=precision, radii_mode=2, r_pe_nonself=12, r_me_nonself=16)
    _pairs_radii_equal(out["pairs"], (pi, pj, g, rpe, rme))
    assert out["stats"]["n_nonconv"] == 0 and out["stats"]["solver_kind"] == 1
    assert abs(out["E_xx"] - ref["E_xx"]) / w.n <= E_GATE_PER_ORBITAL
    assert d_maxrel(out["D"], ref["D"]) <= D_GATE_MAXREL
    np.testing.assert_allclose(out["pairs"]["e_pair"], ref["E_pair"], rtol=1e-7, atol=1e-12)
    # the GPU used the non-self radii: it is far closer to the per-pair-radii
    # oracle than to the fixed-radii one
    fixed = oracle.exx(w.cell, w.grid, phi, (pi, pj, g), 16, 20, w.l_max, tol=1e-13, want_d=False)
    assert abs(out["E_xx"] - fixed["E_xx"]) > 10 * abs(out["E_xx"] - ref["E_xx"])


def test_batched_uneven_full_size_sampled(torch):
    """The batched-uneven workload (150^3, 512 orbitals in 128 clusters,
    alpha ~ U(0.5, 2), per-pair radii 12..32, largest pairs first), checked
    on sampled pairs and one sampled orbital."""
    w = synth.config2()
    phi = w.orbitals()
    out = run_gpu(w, phi, torch=torch, precision=1)
    ref_pairs = oracle.pair_list_radii(w.centers, w.cell, w.grid, w.r_pair, w.alphas, 12, w.r_pe)
    _pairs_radii_equal(out["pairs"], ref_pairs)
    assert out["stats"]["n_nonconv"] == 0
    rpe = ref_pairs[3]
    assert rpe.min() <= 14 and rpe.max() >= 28
    rng = np.random.default_rng(3)
    npair = len(rpe)
    sample = np.unique(np.concatenate([rng.choice(npair, 12, replace=False), [int(np.argmax(rpe)),
                                                                              int(np.argmin(rpe))]]))
    sub = tuple(a[sample] for a in ref_pairs)
    orc = oracle.exx(w.cell, w.grid, phi, sub, w.r_pe, w.r_me, w.l_max, tol=1e-13, want_d=False)
    np.testing.assert_allclose(out["pairs"]["e_pair"][sample], orc["E_pair"], rtol=0,
                               atol=E_GATE_PER_ORBITAL / 4)
    orb = int(ref_pairs[0][sample[0]])
    mask = np.zeros(w.n, np.int32)
    mask[orb] = 1
    touch = np.nonzero(mask[ref_pairs[0]] | mask[ref_pairs[1]])[0]
    sub2 = tuple(a[touch] for a in ref_pairs)
    orc2 = oracle.exx(w.cell, w.grid, phi, sub2, w.r_pe, w.r_me, w.l_max, tol=1e-13, want_d=True, dmask=mask)
    den = np.max(np.abs(orc2["D"][orb]))
    assert np.max(np.abs(out["D"][orb] - orc2["D"][orb])) <= D_GATE_MAXREL * den


# --------------------------------------------------------------------------
# Warm start from the previous call (MD-like sequences)
# --------------------------------------------------------------------------

def test_warm_start_from_previous_step(torch):
    """Two consecutive calls on drifted inputs (centres + N(0, 0.02^2) bohr,
    alpha x (1 + 0.01 xi)): the second starts each kept pair from the first
    call's potential (shifted where its grid centre moved), meets the same
    accuracy gates and needs fewer CG iterations than a cold start."""
    import copy
    from paper_1911_10630_gb300.exx import Exx
    w0 = synth.config0()
    rng = np.random.default_rng(21)
    w1 = copy.deepcopy(w0)
    w1.centers = np.mod(w0.centers + rng.normal(0.0, 0.02, size=w0.centers.shape), w0.cell)
    w1.alphas = w0.alphas * (1.0 + 0.01 * rng.normal(size=w0.n))
    phi0, phi1 = w0.orbitals(), w1.orbitals()
    ex = Exx(w0.cell, w0.grid, w0.r_pair, w0.r_pe, w0.r_me, 6, w0.tol, precision=1, warm_start=1)
    dD = torch.empty(phi0.shape, dtype=torch.float64, device="cuda")
    for w, phi in ((w0, phi0), (w1, phi1)):
        e = ex.compute(torch.from_numpy(phi).cuda(), torch.from_numpy(np.ascontiguousarray(w.centers)).cuda(), dD)
    warm_iters = ex.stats()["iters_total"]
    D = dD.cpu().numpy()
    ref = oracle.exx_workload(w1, tol=1e-13, orbitals=phi1)
    assert abs(e - ref["E_xx"]) / w1.n <= E_GATE_PER_ORBITAL
    assert d_maxrel(D, ref["D"]) <= D_GATE_MAXREL
    cold = run_gpu(w1, phi1, torch=torch, precision=1)
    assert warm_iters < 0.97 * cold["stats"]["iters_total"], (warm_iters, cold["stats"]["iters_total"])
    i0, j0, g0 = oracle.pair_list(w0.centers, w0.cell, w0.grid, w0.r_pair)
    i1, j1, g1 = oracle.pair_list(w1.centers, w1.cell, w1.grid, w1.r_pair)
    before = {(a, b): g for a, b, g in zip(i0.tolist(), j0.tolist(), g0.tolist())}
    moved = [k for k, g in zip(zip(i1.tolist(), j1.tolist()), g1.tolist()) if k in before and before[k] != g]
    assert moved  # some kept pairs' grid centres moved: the shifted start was exercised


# --------------------------------------------------------------------------
# Multigrid-preconditioned CG (preconditioner 1): FP64 on one CTA per pair;
# FP32 inside the FP64 refinement on one CTA per pair (solver_kind 1; 256
# threads by default, 512 or 1024 on request) or on a cluster of C CTAs per
# pair (solver_kind 0 or 2), one or two CTAs per SM
# --------------------------------------------------------------------------
MG_FORMS = [dict(precision=0), dict(precision=1), dict(precision=1, solver_kind=2),
            dict(precision=1, solver_kind=2, cluster_size=2), dict(precision=1, solver_kind=2, cluster_size=4),
            dict(precision=1, solver_kind=2, cluster_size=16),
            dict(precision=1, solver_kind=2, cluster_size=8, ctas_per_sm=1),
            dict(precision=1, threads=512), dict(precision=1, threads=1024)]
MG_IDS = ["fp64", "fp32-cta", "fp32-c8", "fp32-c2", "fp32-c4", "fp32-c16", "fp32-c8-1sm", "fp32-cta512",
          "fp32-cta1024"]


def _mg_form_check(out, form):
    if form.get("solver_kind", 0) != 2:
        assert out["stats"]["solver_kind"] == 1
        assert out["stats"]["threads"] == form.get("threads", 256 if form.get("precision") == 1 else 512)
    else:
        assert out["stats"]["solver_kind"] == 2
        assert out["stats"]["cluster_size"] == form.get("cluster_size", 8)


@pytest.mark.parametrize("form", MG_FORMS, ids=MG_IDS)
def test_multigrid_pcg_meets_the_gates_in_far_fewer_iterations(torch, cfg0, form):
    """Config 0 (R_PE 16 / R_ME 20, tol 1e-10; levels 16, 8, 4, 2): the same
    energies and forces as the oracle under the gates, every pair's E_ij to
    the solve's tolerance, in a small fraction of the plain CG's iterations."""
    w, phi, ref = cfg0
    plain = run_gpu(w, phi, torch=torch, precision=0)
    mg = run_gpu(w, phi, torch=torch, preconditioner=1, **form)
    _mg_form_check(mg, form)
    assert mg["stats"]["n_nonconv"] == 0
    _pairs_equal(mg["pairs"], ref["pairs"])
    assert abs(mg["E_xx"] - ref["E_xx"]) / w.n <= E_GATE_PER_ORBITAL
    assert d_maxrel(mg["D"], ref["D"]) <= D_GATE_MAXREL
    np.testing.assert_allclose(mg["pairs"]["e_pair"], ref["E_pair"], rtol=1e-8, atol=1e-12)
    it_plain, it_mg = plain["stats"]["iters_total"], mg["stats"]["iters_total"]
    assert it_mg < 0.25 * it_plain, (it_mg, it_plain)


@pytest.mark.parametrize("form", MG_FORMS[:4], ids=MG_IDS[:4])
def test_multigrid_pcg_per_pair_radii(torch, form):
    """Per-pair radii (R_PE 12..16): one hierarchy per ball (levels 12, 6, 3 up to
    16, 8, 4, 2) in the same workspace slots, cleared between pairs."""
    w = synth.tiny(seed=8, n=6, npts=48, length=9.6, r_pe=16, r_me=22, alpha=(0.5, 2.0), tol=1e-10, min_sep=1.2)
    w.radii_mode = 1
    phi = w.orbitals()
    ref = oracle.exx_workload(w, tol=1e-13, orbitals=phi)
    assert len(set(ref["pairs"][3])) >= 3
    out = run_gpu(w, phi, torch=torch, preconditioner=1, **form)
    _mg_form_check(out, form)
    _pairs_radii_equal(out["pairs"], ref["pairs"])
    assert out["stats"]["n_nonconv"] == 0
    assert abs(out["E_xx"] - ref["E_xx"]) / w.n <= E_GATE_PER_ORBITAL
    assert d_maxrel(out["D"], ref["D"]) <= D_GATE_MAXREL
    np.testing.assert_allclose(out["pairs"]["e_pair"], ref["E_pair"], rtol=1e-7, atol=1e-12)


@pytest.mark.parametrize("form", MG_FORMS[:4], ids=MG_IDS[:4])
def test_multigrid_pcg_anisotropic_ragged(torch, form):
    """Non-cubic grid and cell (each level's stencil with its own spacings),
    small balls (levels 5, 3), pairs across faces."""
    w = synth.tiny(seed=3, n=6, npts=28, length=6.5, r_pe=5, r_me=9, r_pair=3.0, tol=1e-10)
    w.grid = np.array([28, 30, 26])
    w.cell = np.array([6.5, 7.1, 6.2])
    w.centers = np.mod(w.centers, w.cell)
    w.centers[0] = [0.05, 3.0, 6.1]
    w.centers[1] = [6.3, 3.2, 0.2]
    phi = w.orbitals()
    ref = oracle.exx_workload(w, tol=1e-13, orbitals=phi)
    out = run_gpu(w, phi, torch=torch, preconditioner=1, **form)
    _mg_form_check(out, form)
    _pairs_equal(out["pairs"], ref["pairs"])
    assert abs(out["E_xx"] - ref["E_xx"]) / w.n <= E_GATE_PER_ORBITAL
    assert d_maxrel(out["D"], ref["D"]) <= D_GATE_MAXREL


@pytest.mark.parametrize("form", [MG_FORMS[1], MG_FORMS[2]], ids=[MG_IDS[1], MG_IDS[2]])
def test_multigrid_deterministic_dxx_is_bitwise_reproducible(torch, cfg0, form):
    """With deterministic = 1 the multigrid forms give the same D_xx bit for bit
    from call to call (order-independent integer accumulation, fixed-order sums
    within a pair), and the same D_xx as the FP64-atomic mode within roundoff."""
    w, phi, ref = cfg0
    a = run_gpu(w, phi, torch=torch, preconditioner=1, deterministic=1, **form)
    b = run_gpu(w, phi, torch=torch, preconditioner=1, deterministic=1, **form)
    c = run_gpu(w, phi, torch=torch, preconditioner=1, **form)
    assert a["E_xx"] == b["E_xx"]
    np.testing.assert_array_equal(a["D"], b["D"])
    # each contribution rounds to a multiple of 2^-40 (9.1e-13), and a grid
    # point sums a few dozen of them: far below 1e-9 of max |D| on this case
    assert np.max(np.abs(a["D"] - c["D"])) <= 64 * 2.0 ** -40
    assert d_maxrel(a["D"], c["D"]) <= 1e-9
    assert d_maxrel(a["D"], ref["D"]) <= D_GATE_MAXREL


def test_multigrid_smallest_balls_on_clusters(torch):
    """Self pairs on R_PE/R_ME = 8/12 (levels 8, 4, 2), non-self pairs on 3/7: a
    ball of radius 3 has no coarse level, so the cluster PCG runs those pairs
    with the identity preconditioner, and its 7 planes are fewer than the 8
    CTAs. With every ball of radius 3 there is no hierarchy at all and the
    one-CTA solver takes the call."""
    w = synth.tiny(seed=9, n=5, npts=32, length=8.0, r_pe=8, r_me=12, tol=1e-10)
    phi = w.orbitals()
    pi, pj, g = oracle.pair_list(w.centers, w.cell, w.grid, w.r_pair)
    self_ = pi == pj
    rpe = np.where(self_, 8, 3).astype(np.int32)
    rme = np.where(self_, 12, 7).astype(np.int32)
    ref = oracle.exx(w.cell, w.grid, phi, (pi, pj, g, rpe, rme), 8, 12, w.l_max, tol=1e-13, want_d=True)
    out = run_gpu(w, phi, torch=torch, precision=1, preconditioner=1, solver_kind=2, cluster_size=8,
                  radii_mode=2, r_pe_nonself=3, r_me_nonself=7)
    assert out["stats"]["solver_kind"] == 2 and out["stats"]["n_nonconv"] == 0
    _pairs_radii_equal(out["pairs"], (pi, pj, g, rpe, rme))
    assert abs(out["E_xx"] - ref["E_xx"]) / w.n <= E_GATE_PER_ORBITAL
    assert d_maxrel(out["D"], ref["D"]) <= D_GATE_MAXREL
    np.testing.assert_allclose(out["pairs"]["e_pair"], ref["E_pair"], rtol=1e-7, atol=1e-12)
    w3 = synth.tiny(seed=9, n=4, npts=20, length=5.0, r_pe=3, r_me=7, tol=1e-10)
    phi3 = w3.orbitals()
    ref3 = oracle.exx_workload(w3, tol=1e-13, orbitals=phi3)
    out3 = run_gpu(w3, phi3, torch=torch, precision=1, preconditioner=1)
    assert out3["stats"]["solver_kind"] == 1 and out3["stats"]["n_nonconv"] == 0
    assert abs(out3["E_xx"] - ref3["E_xx"]) / w3.n <= E_GATE_PER_ORBITAL


def test_multigrid_option_errors(torch):
    from paper_1911_10630_gb300.exx import Exx, ExxError
    w = synth.config0()
    with pytest.raises(ExxError, match="precision"):
        Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, precision=0, preconditioner=1, solver_kind=2)
    with pytest.raises(ExxError, match="multigrid"):
        Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, precision=1, preconditioner=1, cluster_size=9)
