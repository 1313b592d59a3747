"""The multigrid hierarchy's host tables (exx_mg_levels), checked on the CPU
against what defines them: ball radii R_l = ceil(R_{l-1} / 2) down to the
first R_l <= 3, each ball's points counted by brute force, the cube side
2 R_l + 7, and the coarsest level's dense inverse against an operator built
here from the paper's stencil weights (Eq. d2_1, tests/golden) at spacing
2^L delta, zero outside the ball."""
import os
from fractions import Fraction

import numpy as np
import pytest


@pytest.fixture(scope="module")
def exx():
    from paper_1911_10630_gb300 import build, exx as _exx
    build.build(quiet=True)
    _exx.load()
    return _exx


def golden_weights():
    path = os.path.join(os.path.dirname(__file__), "golden", "stencil_weights.txt")
    w = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        q, num, den = (int(t) for t in line.split())
        w[q] = float(Fraction(num, den))
    return [w[q] for q in range(4)]


def ball_points(R):
    """The ball |o|^2 <= R^2 in lexicographic (x, y, z) order."""
    return [(x, y, z) for x in range(-R, R + 1) for y in range(-R, R + 1) for z in range(-R, R + 1)
            if x * x + y * y + z * z <= R * R]


def coarse_radii(r_pe):
    out, R = [], r_pe
    while R > 3:
        R = -(-R // 2)
        out.append(R)
    return out


@pytest.mark.parametrize("r_pe", [4, 5, 7, 12, 16, 24, 29, 32, 64])
def test_levels_follow_the_halving_rule(exx, r_pe):
    m = exx.mg_levels(r_pe, [0.2, 0.2, 0.2])
    want = coarse_radii(r_pe)
    assert list(m["radius"]) == want
    assert list(m["side"]) == [2 * R + 7 for R in want]
    assert list(m["points"]) == [len(ball_points(R)) for R in want]
    assert m["radius"][-1] <= 3 and (len(want) == 1 or m["radius"][-2] > 3)


@pytest.mark.parametrize("r_pe, delta", [(16, (0.25, 0.25, 0.25)), (24, (0.19583, 0.19583, 0.19583)),
                                         (13, (0.2321, 0.2367, 0.2385)), (5, (0.3, 0.2, 0.25))])
def test_coarsest_inverse_matches_a_dense_operator(exx, r_pe, delta):
    m = exx.mg_levels(r_pe, delta, want_minv=True)
    L = len(m["radius"])
    pts = ball_points(int(m["radius"][-1]))
    n = len(pts)
    assert m["minv"].shape == (n, n)
    w = golden_weights()
    h2 = [(d * 2.0 ** L) ** 2 for d in delta]
    index = {p: k for k, p in enumerate(pts)}
    A = np.zeros((n, n))
    for k, p in enumerate(pts):
        A[k, k] = -w[0] * sum(1.0 / h for h in h2)
        for a in range(3):
            for q in (1, 2, 3):
                for s in (-1, 1):
                    o = list(p)
                    o[a] += s * q
                    j = index.get(tuple(o))
                    if j is not None:
                        A[k, j] -= w[q] / h2[a]
    # the operator is symmetric positive definite on the ball, and so is its inverse
    assert np.all(np.linalg.eigvalsh(A) > 0)
    np.testing.assert_allclose(m["minv"], m["minv"].T, rtol=0, atol=1e-12 * np.abs(m["minv"]).max())
    np.testing.assert_allclose(m["minv"] @ A, np.eye(n), rtol=0, atol=1e-10)
    np.testing.assert_allclose(m["minv"], np.linalg.inv(A), rtol=1e-10, atol=1e-14 * np.abs(m["minv"]).max())


def test_bad_arguments_are_rejected(exx):
    from paper_1911_10630_gb300.exx import ExxError
    for r_pe in (3, 0, 128):
        with pytest.raises(ExxError, match="exx_mg_levels"):
            exx.mg_levels(r_pe, [0.2, 0.2, 0.2])
    with pytest.raises(ExxError, match="spacings"):
        exx.mg_levels(16, [0.2, 0.0, 0.2])
    with pytest.raises(ExxError, match="spacings"):
        exx.mg_levels(16, [0.2, float("nan"), 0.2])
