"""The multigrid preconditioner itself, one V-cycle at a time
(exx_apply_preconditioner), against the properties that make the
preconditioned CG a CG and a fast one: M is symmetric (the V-cycle's pre- and
post-smoothing are the same symmetric Jacobi sweep, restriction is the
transpose of prolongation up to its factor, the coarsest solve is a symmetric
inverse) and positive definite, and one cycle takes any right-hand side most
of the way to the solution of A z = r: the error of z = M r in the A-norm
against z* from a CG run here on an operator built from the paper's stencil
weights (Eq. d2_1). A model of the cycle gives 0.29-0.35 for the cases below;
the PCG's measured 16 iterations to 1e-8 mean about 0.32 per iteration; a
cycle without its coarse correction leaves almost all of a smooth error.
A second context in the FP32 multigrid form gives the same z bit for bit (the
call clears the cubes the FP32 solver leaves floats in) and the same E_xx
after the call as before it (the call leaves the workspace as the solvers
expect)."""
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_1911_10630_gb300 import synth
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu

CASES = [dict(grid=(48, 48, 48), cell=(9.6, 9.6, 9.6)), dict(grid=(48, 50, 46), cell=(9.6, 10.4, 9.0))]


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def _context(torch, case, precision):
    from paper_1911_10630_gb300.exx import Exx
    return Exx(np.array(case["cell"]), np.array(case["grid"]), 4.0, 16, 20, 6, 1e-10, precision=precision,
               preconditioner=1)


def _apply(torch, ex, r):
    dr = torch.from_numpy(np.ascontiguousarray(r)).cuda()
    dz = torch.empty_like(dr)
    ex.apply_preconditioner(dr, dz)
    return dz.cpu().numpy()


def _weights():
    path = os.path.join(os.path.dirname(__file__), "golden", "stencil_weights.txt")
    w = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            q, num, den = (int(t) for t in line.split())
            w[q] = float(Fraction(num, den))
    return [w[q] for q in range(4)]


def _ball_operator(pts, d):
    """-lap of Eq. d2_1 on the ball's points, zero outside (sparse)."""
    w = _weights()
    index = {tuple(p): k for k, p in enumerate(pts)}
    rows, cols, vals = [], [], []
    for k, p in enumerate(pts):
        rows.append(k), cols.append(k), vals.append(-w[0] * sum(1.0 / h ** 2 for h in d))
        for a in range(3):
            for q in (1, 2, 3):
                for s in (-1, 1):
                    o = list(p)
                    o[a] += s * q
                    j = index.get(tuple(o))
                    if j is not None:
                        rows.append(k), cols.append(j), vals.append(-w[q] / d[a] ** 2)
    return sp.csr_matrix((vals, (rows, cols)), shape=(len(pts), len(pts)))


def _solve(A, r, rtol=1e-12):
    x, res = np.zeros_like(r), r.copy()
    p, rr = res.copy(), res @ res
    for _ in range(20000):
        ap = A @ p
        al = rr / (p @ ap)
        x += al * p
        res -= al * ap
        rn = res @ res
        if rn <= rtol ** 2 * (r @ r):
            return x
        p = res + (rn / rr) * p
        rr = rn
    raise AssertionError("reference CG did not converge")


@pytest.mark.parametrize("case", CASES, ids=["cubic", "anisotropic"])
def test_vcycle_is_symmetric_positive_and_reduces_the_error(torch, case):
    ex = _context(torch, case, 0)
    n_pe, _ = ex.ball_size()
    pts = oracle.proto_subdomain(16, 20)[0][:n_pe]
    d = np.array(case["cell"]) / np.array(case["grid"])
    A = _ball_operator(pts, d)
    rng = np.random.default_rng(7)
    r1, r2 = rng.standard_normal(n_pe), rng.standard_normal(n_pe)
    z1, z2 = _apply(torch, ex, r1), _apply(torch, ex, r2)
    assert r1 @ z1 > 0 and r2 @ z2 > 0
    assert abs(r2 @ z1 - r1 @ z2) <= 1e-11 * np.sqrt((r1 @ z1) * (r2 @ z2))
    o = pts * d
    smooth = [np.exp(-(o ** 2).sum(axis=1) / (2 * s ** 2)) for s in (0.8, 1.2)]
    for r, z in [(r1, z1)] + [(rs, _apply(torch, ex, rs)) for rs in smooth]:
        zs = _solve(A, r)
        e = z - zs
        err = np.sqrt(e @ (A @ e) / (zs @ (A @ zs)))
        assert err < 0.45, err
    ex.close()


def test_vcycle_is_the_same_on_an_fp32_context_and_leaves_it_clean(torch):
    case = CASES[0]
    w = synth.tiny(seed=4, n=4, npts=48, length=9.6, r_pe=16, r_me=20, tol=1e-10)
    phi = w.orbitals()
    dphi = torch.from_numpy(phi).cuda()
    dcen = torch.from_numpy(np.ascontiguousarray(w.centers)).cuda()
    dD = torch.empty_like(dphi)
    ref = _context(torch, case, 0)
    ex = _context(torch, case, 1)
    e0 = ex.compute(dphi, dcen, dD)  # the FP32 solver leaves floats in the cubes
    n_pe, _ = ex.ball_size()
    r = np.random.default_rng(11).standard_normal(n_pe)
    np.testing.assert_array_equal(_apply(torch, ex, r), _apply(torch, ref, r))
    e1 = ex.compute(dphi, dcen, dD)
    assert e1 == e0
    ex.close()
    ref.close()


def test_refused_without_a_hierarchy(torch):
    from paper_1911_10630_gb300.exx import Exx, ExxError
    case = CASES[0]
    ex = Exx(np.array(case["cell"]), np.array(case["grid"]), 4.0, 16, 20, 6, 1e-10, precision=0)
    r = torch.zeros(10, dtype=torch.float64, device="cuda")
    with pytest.raises(ExxError, match="hierarchy"):
        ex.apply_preconditioner(r, r)
    ex.close()
