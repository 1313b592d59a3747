"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: exact
polynomial results of the stencil (Eq. d2_1), closed-form Gaussian potentials
and energies, exact multipoles (Eq. mepole) against SciPy's spherical
harmonics, a direct Coulomb sum (Eq. me), an FFT solve with the stencil's own
symbol, dense direct solves, brute-force enumeration, and invariants of the
scatter (Eqs. Dxx_mlwf, exx_omega). A plausible mistake in any step of the
oracle (a dropped boundary leg, a wrong weight, sign, index or wrap, a missing
4 pi/(2l+1), a wrong pair multiplicity) fails at least one of them.
"""
import math

import numpy as np
import pytest

from paper_1911_10630_gb300 import synth

W = np.array([-49.0 / 18.0, 3.0 / 2.0, -3.0 / 20.0, 1.0 / 90.0])  # Eq. d2_1, n = 3


def _nint(x):
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


def _minimg(x, L):
    return x - L * np.floor(x / L + 0.5)


# --------------------------------------------------------------------------
# Algorithm 2 and the pair list (brute force)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("r_pe,r_me", [(3, 6), (5, 8), (7, 7), (9, 12)])
def test_proto_subdomain_bruteforce(oracle_mod, r_pe, r_me):
    off, npe = oracle_mod.proto_subdomain(r_pe, r_me)
    g = np.arange(-r_me, r_me + 1)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    s = (X * X + Y * Y + Z * Z).ravel()
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    pe = pts[s <= r_pe * r_pe]
    sh = pts[(s > r_pe * r_pe) & (s <= r_me * r_me)]
    assert npe == len(pe)
    np.testing.assert_array_equal(off, np.concatenate([pe, sh]))


def test_ball_counts_match_known_values(oracle_mod):
    # lattice points with |o|^2 <= R^2 (the sizes the configs run at)
    for r, count in [(12, 7153), (16, 17077), (20, 33401), (24, 57777), (32, 137065)]:
        _, npe = oracle_mod.proto_subdomain(r, r)
        assert npe == count


def _pairs_numpy(centers, cell, grid, r_pair):
    delta = cell / grid
    out = []
    n = len(centers)
    for i in range(n):
        for j in range(i, n):
            d = _minimg(centers[j] - centers[i], cell)
            if d @ d < r_pair * r_pair:
                c = centers[i] + 0.5 * d
                g = np.mod(_nint(c / delta).astype(np.int64), grid)
                out.append((i, j, *g))
    return np.array(out, dtype=np.int64).reshape(-1, 5)


def test_pair_list_bruteforce(oracle_mod):
    rng = np.random.default_rng(7)
    cell = np.array([10.0, 11.0, 9.5])
    grid = np.array([40, 44, 38])
    centers = rng.uniform(0, 1, size=(40, 3)) * cell
    centers[0] = [0.05, 10.95, 4.0]   # straddles the periodic faces
    centers[1] = [9.9, 0.1, 4.2]
    for r_pair in (2.5, 4.0, 1e9):
        pi, pj, g = oracle_mod.pair_list(centers, cell, grid, r_pair)
        ref = _pairs_numpy(centers, cell, grid, r_pair)
        got = np.concatenate([pi[:, None], pj[:, None], g], 1)
        np.testing.assert_array_equal(got, ref)
        assert np.all(pi <= pj)
        assert np.sum(pi == pj) == len(centers)  # every self pair is kept


def test_pair_list_nint_ties_and_strict_cutoff(oracle_mod):
    cell = np.array([8.0, 8.0, 8.0])
    grid = np.array([16, 16, 16])  # delta = 0.5
    # midpoint at x = 1.25 = 2.5 delta -> NINT rounds half away from zero -> 3
    c = np.array([[1.0, 2.0, 3.0], [1.5, 2.0, 3.0], [5.0, 5.0, 5.0]])
    pi, pj, g = oracle_mod.pair_list(c, cell, grid, 0.5)      # |d| = 0.5 is not < 0.5
    assert list(zip(pi, pj)) == [(0, 0), (1, 1), (2, 2)]
    pi, pj, g = oracle_mod.pair_list(c, cell, grid, 0.5000001)
    k = list(zip(pi, pj)).index((0, 1))
    assert list(g[k]) == [3, 4, 6]
    # a pair across the face: midpoint of 7.9 and 0.3 (min image) is 8.1 -> wraps to g = 0
    c2 = np.array([[7.9, 1.0, 1.0], [0.3, 1.0, 1.0]])
    pi, pj, g = oracle_mod.pair_list(c2, cell, grid, 1.0)
    k = list(zip(pi, pj)).index((0, 1))
    assert list(g[k]) == [0, 2, 2]


# --------------------------------------------------------------------------
# Eq. d2_1: the stencil (P1) and its Fourier symbol
# --------------------------------------------------------------------------

def test_stencil_weights_match_golden():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "stencil_weights.txt")
    vals = {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            k, num, den = line.split()
            vals[int(k)] = float(num) / float(den)
    np.testing.assert_array_equal([vals[q] for q in range(4)], W)
    assert W[0] + 2 * W[1:].sum() == 0.0


def test_stencil_exact_on_degree7_polynomials(oracle_mod):
    dims = (14, 15, 16)
    delta = np.array([0.3, 0.25, 0.2])
    x = (np.arange(dims[0]) - 6.3) * delta[0]
    y = (np.arange(dims[1]) - 7.1) * delta[1]
    z = (np.arange(dims[2]) - 7.7) * delta[2]
    X, Y, Z = np.meshgrid(x, y, z, indexing="ij")
    sl = (slice(3, -3),) * 3
    for (a, b, c) in [(7, 0, 0), (0, 7, 0), (0, 0, 7), (2, 3, 4), (7, 7, 7), (6, 1, 5), (0, 0, 0)]:
        f = X ** a * Y ** b * Z ** c
        lap = (a * (a - 1) * X ** max(a - 2, 0) * Y ** b * Z ** c if a >= 2 else 0) \
            + (b * (b - 1) * X ** a * Y ** max(b - 2, 0) * Z ** c if b >= 2 else 0) \
            + (c * (c - 1) * X ** a * Y ** b * Z ** max(c - 2, 0) if c >= 2 else 0)
        lap = np.broadcast_to(lap, f.shape)
        got = oracle_mod.laplacian_box(f, delta)
        scale = np.max(np.abs(f[sl])) / delta.min() ** 2
        assert np.max(np.abs(got[sl] - lap[sl])) <= 1e-11 * scale


def test_stencil_degree8_error_is_72_delta6(oracle_mod):
    # sum_q w_q q^8 / 8! * f^(8) delta^6 with f = x^8: exactly 72 delta^6, everywhere
    dims = (12, 7, 7)
    delta = np.array([0.37, 1.0, 1.0])
    x = (np.arange(dims[0]) - 5.5) * delta[0]
    f = np.broadcast_to((x ** 8)[:, None, None], dims).copy()
    got = oracle_mod.laplacian_box(f, delta)[3:-3, 3, 3]
    exact = 56 * x[3:-3] ** 6
    np.testing.assert_allclose(got - exact, 72 * delta[0] ** 6, rtol=1e-6)


def test_stencil_symbol_is_theta2_minus_theta8_over_560():
    th = np.array([0.05, 0.1, 0.2])
    lam = -(W[0] + 2 * sum(W[q] * np.cos(q * th) for q in (1, 2, 3)))
    np.testing.assert_allclose(lam - th ** 2, -th ** 8 / 560, rtol=2e-2)


# --------------------------------------------------------------------------
# CG (P6 periodic FFT, P7 dense solve on a small ball)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [16, 24])
def test_periodic_cg_matches_fft_with_stencil_symbol(oracle_mod, n):
    rng = np.random.default_rng(n)
    dims = (n, n, n)
    delta = np.array([0.3, 0.3, 0.3])
    rho = rng.normal(size=dims)
    rho -= rho.mean()
    b = 4 * np.pi * rho
    v, it = oracle_mod.cg_periodic(b, delta, tol=1e-13)
    k = [2 * np.pi * np.fft.fftfreq(n) for _ in range(3)]
    lam = 0
    for a in range(3):
        th = k[a]
        sym = -(W[0] + 2 * sum(W[q] * np.cos(q * th) for q in (1, 2, 3))) / delta[a] ** 2
        shape = [1, 1, 1]
        shape[a] = n
        lam = lam + sym.reshape(shape)
    bh = np.fft.fftn(b)
    lam = np.where(lam == 0, 1.0, lam)
    vh = bh / lam
    vh[0, 0, 0] = 0.0
    vref = np.real(np.fft.ifftn(vh))
    assert np.max(np.abs(v - vref)) <= 1e-10 * np.max(np.abs(vref))


def _dense_ball_operator(r_pe, delta):
    g = np.arange(-r_pe, r_pe + 1)
    pts = [(x, y, z) for x in g for y in g for z in g if x * x + y * y + z * z <= r_pe * r_pe]
    idx = {p: k for k, p in enumerate(pts)}
    n = len(pts)
    A = np.zeros((n, n))
    for k, p in enumerate(pts):
        for a in range(3):
            A[k, k] -= W[0] / delta[a] ** 2
            for q in (1, 2, 3):
                for s in (-1, 1):
                    u = list(p)
                    u[a] += s * q
                    t = idx.get(tuple(u))
                    if t is not None:
                        A[k, t] -= W[q] / delta[a] ** 2
    return A


def test_ball_operator_dense_and_cg_vs_cholesky(oracle_mod):
    r_pe, r_me = 5, 8
    delta = np.array([0.2, 0.22, 0.25])
    A = _dense_ball_operator(r_pe, delta)
    n = A.shape[0]
    cols = np.stack([oracle_mod.ball_apply(r_pe, r_me, delta, e) for e in np.eye(n)], 1)
    np.testing.assert_allclose(cols, A, rtol=0, atol=1e-12 * np.abs(A).max())
    np.testing.assert_allclose(A, A.T, atol=0)
    Lc = np.linalg.cholesky(A)  # raises unless SPD
    rng = np.random.default_rng(3)
    b = rng.normal(size=n)
    x_ref = np.linalg.solve(Lc.T, np.linalg.solve(Lc, b))
    x, it = oracle_mod.ball_cg(r_pe, r_me, delta, b, tol=1e-13)
    assert np.max(np.abs(x - x_ref)) <= 1e-10 * np.max(np.abs(x_ref))
    assert 0 < it < n


# --------------------------------------------------------------------------
# Real spherical harmonics and multipoles (P4, P5)
# --------------------------------------------------------------------------

def _scipy_real_ylm(lmax, x, y, z):
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    r = math.sqrt(x * x + y * y + z * z)
    th = math.acos(z / r)
    ph = math.atan2(y, x) % (2 * math.pi)
    out = np.zeros((lmax + 1) ** 2)
    for l in range(lmax + 1):
        for m in range(0, l + 1):
            c = complex(sp.sph_harm_y(l, m, th, ph))
            # SciPy includes the Condon-Shortley phase; the real set has none
            c *= (-1) ** m
            if m == 0:
                out[l * l + l] = c.real
            else:
                out[l * l + l + m] = math.sqrt(2) * c.real
                out[l * l + l - m] = math.sqrt(2) * c.imag
    return out


def test_real_ylm_against_scipy_and_addition_theorem(oracle_mod):
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(11)
    for _ in range(6):
        a = rng.normal(size=3)
        b = rng.normal(size=3)
        ya = oracle_mod.real_ylm(8, *a)
        np.testing.assert_allclose(ya, _scipy_real_ylm(8, *a), atol=1e-13)
        yb = oracle_mod.real_ylm(8, *b)
        cosg = a @ b / np.linalg.norm(a) / np.linalg.norm(b)
        for l in range(9):
            s = ya[l * l:(l + 1) ** 2] @ yb[l * l:(l + 1) ** 2]
            assert abs(s - (2 * l + 1) / (4 * np.pi) * sp.eval_legendre(l, cosg)) < 1e-13


def _gauss_pair_grid(N, L, center, alpha):
    cell = np.full(3, float(L))
    grid = np.full(3, N)
    phi = synth.orbitals(cell, grid, np.asarray([center]), [alpha], np.zeros((1, 3)))
    return cell, grid, phi


def test_multipoles_of_offset_gaussian_are_exact(oracle_mod):
    # rho = phi^2 is a unit Gaussian charge (beta = 2 alpha) at C; about an origin g
    # the moments are exactly |c|^l Y_lm(c^) with c = C - g delta (mean-value property)
    N, L, alpha = 48, 9.6, 1.5
    C = np.array([4.61, 4.93, 5.07])
    cell, grid, phi = _gauss_pair_grid(N, L, C, alpha)
    g = np.array([22, 25, 24])
    res = oracle_mod.pair_solve(cell, grid, phi, 0, 0, g, r_pe=18, r_me=21, lmax=6, tol=1e-8)
    c = C - g * (L / N)
    want = _scipy_real_ylm(6, *c)
    r = np.linalg.norm(c)
    for l in range(7):
        want[l * l:(l + 1) ** 2] *= r ** l
    np.testing.assert_allclose(res["Q"], want, atol=2e-11)


def test_shell_expansion_converges_to_direct_coulomb_sum(oracle_mod):
    # Eq. me vs the direct sum_q rho_q dV / |r - r_q| on the shell, l_max = 0..6
    w = synth.tiny(seed=5, n=2, npts=32, length=8.0, r_pe=9, r_me=13, alpha=(1.2, 1.6), p_sigma=0.4)
    phi = w.orbitals()
    pi, pj, g = oracle_mod.pair_list(w.centers, w.cell, w.grid, math.inf)
    k = int(np.nonzero(pi != pj)[0][0])
    errs = []
    for lmax in range(7):
        res = oracle_mod.pair_solve(w.cell, w.grid, phi, pi[k], pj[k], g[k], w.r_pe, w.r_me, lmax=lmax, tol=1e-6)
        off, npe = res["off"], res["n_pe"]
        rq = off[:npe] * w.delta
        rs = off[npe:] * w.delta
        dv = np.prod(w.delta)
        direct = np.array([np.sum(res["rho"][:npe] * dv / np.linalg.norm(rq - r, axis=1)) for r in rs])
        errs.append(np.max(np.abs(res["v"][npe:] - direct)) / np.max(np.abs(direct)))
    assert errs[-1] < 2e-4
    assert all(errs[l + 1] < errs[l] for l in range(6)), errs


# --------------------------------------------------------------------------
# Closed-form potentials and energies (P2, P3, P12)
# --------------------------------------------------------------------------

def test_gaussian_charge_potential_is_erf_over_r_at_sixth_order(oracle_mod):
    # unit Gaussian charge (beta = 2 alpha) centred on a grid point; v -> erf(sqrt(beta) r)/r
    from math import erf
    alpha = 1.0
    beta = 2 * alpha
    errs = []
    for N, r_pe, r_me in [(32, 12, 15), (64, 24, 30)]:
        L = 8.0
        cell, grid, phi = _gauss_pair_grid(N, L, np.full(3, L / 2), alpha)
        g = np.array([N // 2] * 3)
        res = oracle_mod.pair_solve(cell, grid, phi, 0, 0, g, r_pe, r_me, lmax=6, tol=1e-13)
        off, npe = res["off"], res["n_pe"]
        r = np.linalg.norm(off[:npe] * (L / N), axis=1)
        exact = np.array([erf(math.sqrt(beta) * x) / x if x > 0 else 2 * math.sqrt(beta / math.pi) for x in r])
        errs.append(np.max(np.abs(res["v"][:npe] - exact)))
    assert errs[1] < 1e-5
    assert 30 < errs[0] / errs[1] < 130, errs  # 2^6 = 64


def test_single_s_orbital_energy_closed_form(oracle_mod):
    # E_xx = -(rho|rho) = -2 sqrt(alpha/pi) for phi = (2 alpha/pi)^(3/4) exp(-alpha r^2)
    alpha = 1.0
    errs = []
    for N, r_pe, r_me in [(32, 12, 15), (64, 24, 30)]:
        cell, grid, phi = _gauss_pair_grid(N, 8.0, np.array([4.03, 3.93, 4.11]), alpha)
        pairs = oracle_mod.pair_list(np.array([[4.03, 3.93, 4.11]]), cell, grid, math.inf)
        out = oracle_mod.exx(cell, grid, phi, pairs, r_pe, r_me, 6, tol=1e-13, want_d=False)
        errs.append(abs(out["E_xx"] + 2 * math.sqrt(alpha / math.pi)))
    assert errs[1] < 1e-6
    assert 30 < errs[0] / errs[1] < 130, errs


def _closed_form_exx(centers, alphas, cell):
    # s Gaussians: rho_ij is a Gaussian charge q_ij with exponent beta = a_i + a_j,
    # (rho_ij|rho_ij) = q_ij^2 sqrt(2 beta / pi); ordered sum over ij
    e = 0.0
    n = len(alphas)
    for i in range(n):
        for j in range(n):
            a, b = alphas[i], alphas[j]
            beta = a + b
            mu = a * b / beta
            d = _minimg(centers[j] - centers[i], cell)
            q = (2 * a / np.pi) ** 0.75 * (2 * b / np.pi) ** 0.75 * np.exp(-mu * d @ d) * (np.pi / beta) ** 1.5
            e += q * q * np.sqrt(2 * beta / np.pi)
    return -e


@pytest.mark.slow
def test_multi_orbital_s_type_energy_closed_form(oracle_mod):
    rng = np.random.default_rng(2)
    L = 8.0
    centers = np.array([[1.0, 4.0, 4.0], [2.4, 4.6, 3.7], [7.3, 3.2, 4.5]])  # 0 and 2 meet across x = 0
    alphas = rng.uniform(1.0, 1.4, size=3)
    ref = _closed_form_exx(centers, alphas, np.full(3, L))
    errs = []
    for N, r_pe, r_me in [(32, 12, 15), (64, 24, 30)]:
        cell = np.full(3, L)
        grid = np.full(3, N)
        phi = synth.orbitals(cell, grid, centers, alphas, np.zeros((3, 3)))
        pairs = oracle_mod.pair_list(centers, cell, grid, math.inf)
        out = oracle_mod.exx(cell, grid, phi, pairs, r_pe, r_me, 6, tol=1e-13, want_d=False)
        errs.append(abs(out["E_xx"] - ref))
    assert errs[1] < 2e-6 * abs(ref)
    assert 20 < errs[0] / errs[1] < 130, errs


# --------------------------------------------------------------------------
# Invariants of the pipeline (P8, P9, P10, P11)
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def tiny_case(oracle_mod):
    w = synth.tiny(seed=1, n=3, npts=24, length=6.0, r_pe=6, r_me=9, alpha=(1.2, 2.0))
    phi = w.orbitals()
    out = oracle_mod.exx_workload(w, tol=1e-13, orbitals=phi)
    return w, phi, out


def test_pair_swap_symmetry(oracle_mod, tiny_case):
    w, phi, out = tiny_case
    pi, pj, g = out["pairs"]
    for k in range(len(pi)):
        a = oracle_mod.pair_solve(w.cell, w.grid, phi, pi[k], pj[k], g[k], w.r_pe, w.r_me, tol=1e-13)
        b = oracle_mod.pair_solve(w.cell, w.grid, phi, pj[k], pi[k], g[k], w.r_pe, w.r_me, tol=1e-13)
        assert a["E"] == b["E"]
        np.testing.assert_array_equal(a["v"], b["v"])


def test_scatter_invariant(oracle_mod, tiny_case):
    # sum_i <D^i, phi_i> dV = -E_xx + sum_pairs m_ij sum_{shell} rho v dV
    w, phi, out = tiny_case
    pi, pj, g = out["pairs"]
    dv = np.prod(w.delta)
    lhs = sum(np.sum(out["D"][i] * phi[i]) for i in range(w.n)) * dv
    shell = 0.0
    for k in range(len(pi)):
        r = oracle_mod.pair_solve(w.cell, w.grid, phi, pi[k], pj[k], g[k], w.r_pe, w.r_me, tol=1e-13)
        npe = r["n_pe"]
        shell += (1 if pi[k] == pj[k] else 2) * np.sum(r["rho"][npe:] * r["v"][npe:]) * dv
    rhs = -out["E_xx"] + shell
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_periodic_roll_invariance(oracle_mod, tiny_case):
    w, phi, out = tiny_case
    shift = np.array([5, -7, 11])
    phi2 = np.roll(phi, tuple(shift), axis=(1, 2, 3))
    c2 = np.mod(w.centers + shift * w.delta, w.cell)
    pairs2 = oracle_mod.pair_list(c2, w.cell, w.grid, w.r_pair)
    out2 = oracle_mod.exx(w.cell, w.grid, phi2, pairs2, w.r_pe, w.r_me, 6, tol=1e-13)
    np.testing.assert_array_equal(pairs2[0], out["pairs"][0])
    np.testing.assert_array_equal(pairs2[2], np.mod(out["pairs"][2] + shift, w.grid))
    assert abs(out2["E_xx"] - out["E_xx"]) <= 1e-13 * abs(out["E_xx"])
    D2 = np.roll(out2["D"], tuple(-shift), axis=(1, 2, 3))
    assert np.max(np.abs(D2 - out["D"])) <= 1e-13 * np.max(np.abs(out["D"]))


def test_directional_derivative_matches_minus_4_D(oracle_mod, tiny_case):
    # d/dt E_xx(phi + t eta) at t = 0 equals -4 sum_i <D^i, eta_i> dV up to the
    # asymmetry of the ME boundary map and the shell part of D (small here)
    w, phi, out = tiny_case
    rng = np.random.default_rng(4)
    eta = np.stack([synth.orbital(w.cell, w.grid, w.centers[i] + rng.normal(0, 0.2, 3), 2.5, np.zeros(3))
                    for i in range(w.n)]) * rng.normal(size=(w.n, 1, 1, 1))
    t = 1e-4
    pairs = out["pairs"]
    ep = oracle_mod.exx(w.cell, w.grid, phi + t * eta, pairs, w.r_pe, w.r_me, 6, tol=1e-13, want_d=False)["E_xx"]
    em = oracle_mod.exx(w.cell, w.grid, phi - t * eta, pairs, w.r_pe, w.r_me, 6, tol=1e-13, want_d=False)["E_xx"]
    fd = (ep - em) / (2 * t)
    an = -4 * np.sum(out["D"] * eta) * np.prod(w.delta)
    assert abs(fd - an) <= 2e-3 * abs(an), (fd, an)
    # a factor-2 or sign slip in D is far outside that band
    assert abs(fd - an / 2) > 0.1 * abs(an) and abs(fd + an) > 0.1 * abs(an)


# --------------------------------------------------------------------------
# P13: an independent dense restatement with SciPy's complex harmonics
# --------------------------------------------------------------------------

def _numpy_exx(cell, grid, phi, centers, r_pe, r_me, lmax):
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    delta = cell / grid
    dv = np.prod(delta)
    rng_ = np.arange(-r_me, r_me + 1)
    X, Y, Z = np.meshgrid(rng_, rng_, rng_, indexing="ij")
    o = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    s = np.sum(o * o, 1)
    pe = o[s <= r_pe ** 2]
    sh = o[(s > r_pe ** 2) & (s <= r_me ** 2)]
    pe_idx = {tuple(p): k for k, p in enumerate(pe)}
    sh_idx = {tuple(p): k for k, p in enumerate(sh)}
    A = _dense_ball_operator(r_pe, delta)
    n = len(centers)
    D = np.zeros_like(phi)
    E = 0.0
    for i in range(n):
        for j in range(i, n):
            d = _minimg(centers[j] - centers[i], cell)
            gc = np.mod(_nint((centers[i] + 0.5 * d) / delta).astype(np.int64), grid)
            gpe = np.mod(gc + pe, grid)
            gsh = np.mod(gc + sh, grid)
            rho = phi[i][tuple(gpe.T)] * phi[j][tuple(gpe.T)]
            rp = pe * delta
            rr = np.linalg.norm(rp, axis=1)
            th = np.arccos(np.divide(rp[:, 2], rr, out=np.ones_like(rr), where=rr > 0))
            ph = np.mod(np.arctan2(rp[:, 1], rp[:, 0]), 2 * np.pi)
            rs = sh * delta
            rsn = np.linalg.norm(rs, axis=1)
            ths = np.arccos(rs[:, 2] / rsn)
            phs = np.mod(np.arctan2(rs[:, 1], rs[:, 0]), 2 * np.pi)
            vsh = np.zeros(len(sh), dtype=complex)
            for l in range(lmax + 1):
                for m in range(-l, l + 1):
                    Q = np.sum(np.conj(sp.sph_harm_y(l, m, th, ph)) * rr ** l * rho) * dv
                    vsh += 4 * np.pi * Q / (2 * l + 1) * sp.sph_harm_y(l, m, ths, phs) / rsn ** (l + 1)
            vsh = vsh.real
            b = 4 * np.pi * rho.copy()
            for k, p in enumerate(pe):
                for a in range(3):
                    for q in (1, 2, 3):
                        for sg in (-1, 1):
                            u = p.copy()
                            u[a] += sg * q
                            t = sh_idx.get(tuple(u))
                            if t is not None:
                                b[k] += W[q] * vsh[t] / delta[a] ** 2
            vpe = np.linalg.solve(A, b)
            e = np.sum(rho * vpe) * dv
            E += e if i == j else 2 * e
            np.add.at(D[i], tuple(gpe.T), vpe * phi[j][tuple(gpe.T)])
            np.add.at(D[i], tuple(gsh.T), vsh * phi[j][tuple(gsh.T)])
            if i != j:
                np.add.at(D[j], tuple(gpe.T), vpe * phi[i][tuple(gpe.T)])
                np.add.at(D[j], tuple(gsh.T), vsh * phi[i][tuple(gsh.T)])
    return -E, D


@pytest.mark.slow
def test_bruteforce_dense_restatement(oracle_mod):
    w = synth.tiny(seed=9, n=3, npts=20, length=5.0, r_pe=5, r_me=8, alpha=(1.5, 2.5))
    phi = w.orbitals()
    ref_e, ref_d = _numpy_exx(w.cell, w.grid, phi, w.centers, w.r_pe, w.r_me, 6)
    out = oracle_mod.exx_workload(w, tol=1e-14, orbitals=phi)
    assert abs(out["E_xx"] - ref_e) <= 1e-11 * abs(ref_e)
    assert np.max(np.abs(out["D"] - ref_d)) <= 1e-10 * np.max(np.abs(ref_d))


# --------------------------------------------------------------------------
# Per-pair radii (spread-dependent subdomains)
# --------------------------------------------------------------------------

def test_pair_radius_rule_bounds_the_envelope(oracle_mod):
    # brute force: beyond R_PE grid steps from the pair centre the product of the
    # two Gaussian envelopes is below eps = 1e-14 (unless R_PE was clamped)
    rng = np.random.default_rng(12)
    delta = 0.197
    for _ in range(40):
        ai, aj = rng.uniform(0.5, 2.0, 2)
        d = rng.normal(size=3) * rng.uniform(0.0, 3.0)
        r, rme = oracle_mod.pair_radius(ai, aj, d @ d, delta, 12, 32)
        ci, cj = np.zeros(3), d
        cij = 0.5 * d
        dirs = rng.normal(size=(400, 3))
        dirs /= np.linalg.norm(dirs, axis=1)[:, None]
        pts = cij + dirs * (r * delta * (1.0 + 1e-9))
        env = np.exp(-ai * np.sum((pts - ci) ** 2, 1) - aj * np.sum((pts - cj) ** 2, 1))
        if 12 < r < 32:
            assert env.max() <= 1e-14 * (1 + 1e-9)
            # and one step less would not bound it everywhere (the radius is tight)
            pts_in = cij + dirs * ((r - 1) * delta)
            env_in = np.exp(-ai * np.sum((pts_in - ci) ** 2, 1) - aj * np.sum((pts_in - cj) ** 2, 1))
            cbar = aj / (ai + aj) * d
            toward = cij + (cbar - cij) / max(np.linalg.norm(cbar - cij), 1e-300) * ((r - 1) * delta)
            worst = np.exp(-ai * np.sum((toward - ci) ** 2) - aj * np.sum((toward - cj) ** 2))
            assert max(env_in.max(), worst) > 1e-14 * 0.999 or np.linalg.norm(cbar - cij) < 1e-12
        assert 12 <= r <= 32 and rme == r + max(3, -(-r // 3))
        assert (r, rme) == oracle_mod.pair_radius(aj, ai, d @ d, delta, 12, 32)  # symmetric in i, j


def test_pair_radius_self_pair_closed_form(oracle_mod):
    # d = 0: s_eps = sqrt(ln(1e14) / (2 alpha)), R = ceil(s_eps / delta)
    for alpha in (0.5, 0.8, 1.0, 1.5, 2.0):
        r, _ = oracle_mod.pair_radius(alpha, alpha, 0.0, 0.19733, 12, 32)
        want = min(32, max(12, math.ceil(math.sqrt(math.log(1e14) / (2 * alpha)) / 0.19733)))
        assert r == want
    assert oracle_mod.pair_radius(0.5, 0.5, 0.0, 0.19733, 12, 32)[0] == 29


def test_exx_with_per_pair_radii_matches_fixed_when_radii_agree(oracle_mod):
    # the per-pair form with every pair at the same radii equals the fixed form
    w = synth.tiny(seed=6, n=3, npts=24, length=6.0, r_pe=6, r_me=9)
    phi = w.orbitals()
    pi, pj, g = oracle_mod.pair_list(w.centers, w.cell, w.grid, w.r_pair)
    a = oracle_mod.exx(w.cell, w.grid, phi, (pi, pj, g), 6, 9, tol=1e-13)
    rp = np.full(len(pi), 6, np.int32)
    rm = np.full(len(pi), 9, np.int32)
    b = oracle_mod.exx(w.cell, w.grid, phi, (pi, pj, g, rp, rm), 6, 9, tol=1e-13)
    assert a["E_xx"] == b["E_xx"]
    np.testing.assert_array_equal(a["D"], b["D"])
    # and mixed radii change the per-pair subdomains
    rp2 = np.where(pi == pj, 7, 5).astype(np.int32)
    rm2 = rp2 + 3
    c = oracle_mod.exx(w.cell, w.grid, phi, (pi, pj, g, rp2, rm2), 7, 10, tol=1e-13)
    for k in range(len(pi)):
        e = oracle_mod.pair_solve(w.cell, w.grid, phi, pi[k], pj[k], g[k], int(rp2[k]), int(rm2[k]), tol=1e-13)["E"]
        assert abs(e - c["E_pair"][k]) <= 1e-14 * max(abs(e), 1e-300)
