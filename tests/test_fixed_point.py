"""The arithmetic behind the fixed-point FP64 residuals of the cluster kernel
(exx_options.fixed_residual = 0), checked on the host: 180 delta^2 times the
Eq. d2_1 weights are integers, the int64 stencil of round(v 2^E) reproduces the
FP64 stencil of v to within the quantisation bound, and no partial sum leaves
the int64 range when |v| 2^E < 2^50."""
from fractions import Fraction

import numpy as np

W = [Fraction(-49, 18), Fraction(3, 2), Fraction(-3, 20), Fraction(1, 90)]  # Eq. d2_1, n = 3
IW = [-490, 270, -27, 2]


def test_scaled_weights_are_the_integers():
    assert [w * 180 for w in W] == IW
    assert sum(abs(w) for w in IW[1:]) * 6 + 3 * abs(IW[0]) == 3264  # |weights| of the 19-point sum


def _lap_int(f):
    """180 delta^2 lap on the interior of an int64 cube (the kernel's lap_fix)."""
    c = f[3:-3, 3:-3, 3:-3]
    out = 3 * IW[0] * c
    for q in (1, 2, 3):
        s = np.zeros_like(c)
        for ax in range(3):
            sl_p = [slice(3, -3)] * 3
            sl_m = [slice(3, -3)] * 3
            sl_p[ax] = slice(3 + q, f.shape[ax] - 3 + q)
            sl_m[ax] = slice(3 - q, f.shape[ax] - 3 - q)
            s = s + f[tuple(sl_p)] + f[tuple(sl_m)]
        out = out + IW[q] * s
    return out


def _lap64(v, delta):
    c = v[3:-3, 3:-3, 3:-3]
    out = 3 * float(W[0]) * c
    for q in (1, 2, 3):
        for ax in range(3):
            sl_p = [slice(3, -3)] * 3
            sl_m = [slice(3, -3)] * 3
            sl_p[ax] = slice(3 + q, v.shape[ax] - 3 + q)
            sl_m[ax] = slice(3 - q, v.shape[ax] - 3 - q)
            out = out + float(W[q]) * (v[tuple(sl_p)] + v[tuple(sl_m)])
    return out / (delta * delta)


def test_integer_stencil_matches_fp64_within_the_quantisation_bound():
    rng = np.random.default_rng(7)
    delta = 0.19583
    x = np.linspace(-1, 1, 24)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    v = 3.7 * np.exp(-2 * (X ** 2 + Y ** 2 + Z ** 2)) + 1e-3 * rng.standard_normal(X.shape)
    bound = 2 * np.max(np.abs(v))
    _, e = np.frexp(bound)  # bound < 2^e
    E = 50 - int(e)
    vf = np.rint(v * 2.0 ** E).astype(np.int64)
    assert np.max(np.abs(vf)) < 2 ** 50
    li = _lap_int(vf)
    assert np.max(np.abs(li)) < 2 ** 62
    lap_fix = li.astype(np.float64) * (2.0 ** -E / (180 * delta * delta))
    lap_ref = _lap64(v, delta)
    # quantisation: each of the 19 values moves by <= 2^-E / 2, weighted by |w| / delta^2
    q = 3264 / 180 / delta ** 2 * 2.0 ** -(E + 1)
    assert np.max(np.abs(lap_fix - lap_ref)) <= q + 1e-12 * np.max(np.abs(lap_ref))
