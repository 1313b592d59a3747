"""Pins of the U-Net oracle (oracle/unet.py) against definitions it does not
share code with: brute-force loops, SciPy's correlate, adjoint identities and
central finite differences of the loss."""
import numpy as np
import pytest

from oracle import unet


def _brute_conv(x, W, b):
    B, D, H, Wd, ci = x.shape
    co = W.shape[2]
    y = np.zeros((B, D, H, Wd, co))
    for bb in range(B):
        for z in range(D):
            for yy in range(H):
                for xx in range(Wd):
                    acc = b.copy()
                    for t in range(27):
                        dz, dy, dx = t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1
                        z2, y2, x2 = z + dz, yy + dy, xx + dx
                        if 0 <= z2 < D and 0 <= y2 < H and 0 <= x2 < Wd:
                            acc = acc + x[bb, z2, y2, x2, :] @ W[t]
                    y[bb, z, yy, xx] = acc
    return y


def test_conv3_matches_brute_force_loops():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 4, 5, 3))
    W = rng.normal(size=(27, 3, 2))
    b = rng.normal(size=2)
    np.testing.assert_allclose(unet.conv3(x, W, b), _brute_conv(x, W, b), rtol=1e-12, atol=1e-12)


def test_conv3_matches_scipy_correlate():
    nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(1)
    x = rng.normal(size=(1, 6, 5, 7, 2))
    W = rng.normal(size=(27, 2, 3))
    y = unet.conv3(x, W)
    for co in range(3):
        ref = np.zeros((6, 5, 7))
        for ci in range(2):
            k = W[:, ci, co].reshape(3, 3, 3)
            ref += nd.correlate(x[0, ..., ci], k, mode="constant", cval=0.0)
        np.testing.assert_allclose(y[0, ..., co], ref, rtol=1e-12, atol=1e-12)


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 8, 8, 8, 3))
    y = rng.normal(size=(2, 4, 4, 4, 3))
    assert np.isclose(np.sum(unet.pool(x) * y), np.sum(x * unet.pool_backward(y)))
    assert np.isclose(np.sum(unet.upsample(y) * x), np.sum(y * unet.upsample_backward(x)))
    # pooling a constant field is the constant; up-sampling then pooling is the identity
    assert np.allclose(unet.pool(np.full((1, 4, 4, 4, 2), 3.5)), 3.5)
    assert np.allclose(unet.pool(unet.upsample(y)), y)


def test_bf16_rounding_is_nearest_even():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even mantissa wins (1.0)
    assert unet.bf16_round(np.float32(1.0 + 2.0 ** -8)) == 1.0
    assert unet.bf16_round(np.float32(1.0 + 3 * 2.0 ** -8)) == 1.0 + 2.0 ** -6
    assert unet.bf16_round(np.float32(-2.75)) == -2.75


def _sample(S, B, seed):
    rng = np.random.default_rng(seed)
    c = (np.arange(S) - S / 2)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    r2 = x * x + y * y + z * z
    inp = np.zeros((B, S, S, S, 3))
    tgt = np.zeros((B, S, S, S))
    for b in range(B):
        a = rng.uniform(0.05, 0.2)
        sh = rng.normal(0, 1.0, 3)
        rho = np.exp(-a * ((x - sh[0]) ** 2 + (y - sh[1]) ** 2 + (z - sh[2]) ** 2))
        mask = r2 <= (S / 2 - 1) ** 2
        inp[b, ..., 0] = rho * mask
        inp[b, ..., 1] = rng.normal(0, 1, (S, S, S)) * ~mask
        inp[b, ..., 2] = mask
        tgt[b] = rng.normal(0, 1, (S, S, S)) * mask
    return inp, tgt


def test_gradient_matches_central_differences():
    S, B = 8, 1
    inp, tgt = _sample(S, B, 3)
    p = unet.init_params(4).astype(np.float64)
    p += np.random.default_rng(5).normal(0, 0.05, p.size)  # nonzero biases too
    loss, g = unet.loss_and_gradient(p, inp, tgt)
    rng = np.random.default_rng(6)
    sizes = unet.param_sizes()
    offs = np.concatenate([[0], np.cumsum(sizes)])
    idx = [int(rng.integers(offs[l], offs[l + 1])) for l in range(len(sizes)) for _ in range(3)]
    idx += [int(offs[-1] - 1), int(offs[-2])]  # head bias, head weight 0
    eps = 1e-6
    for k in idx:
        pp, pm = p.copy(), p.copy()
        pp[k] += eps
        pm[k] -= eps
        lp, _ = unet.loss_and_gradient(pp, inp, tgt)
        lm, _ = unet.loss_and_gradient(pm, inp, tgt)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-5 * max(abs(fd), abs(g[k])) + 1e-9, (k, fd, g[k])


def test_param_count_matches_layer_table():
    # 27 cin cout + cout per 3x3x3 layer, 16 + 1 for the head
    expect = sum(27 * a * b + b for a, b in zip(unet.CIN[:-1], unet.COUT[:-1])) + 17
    assert unet.param_count() == expect == len(unet.init_params(0))
