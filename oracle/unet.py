"""CPU oracle of the learned warm start's 3D U-Net (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and bench.py's CPU legs may use
anything under ``oracle/``; the product path never imports it.

The network is this library's addition to the method (the paper names better
CG initial guesses as the way to fewer iterations, Sec. III.C Step IV and the
conclusions, without a network). This module restates it from its definition
in plain NumPy FP64: 3x3x3 cross-correlations with zero padding, ReLU, 2x2x2
average pooling, nearest up-sampling, channel concatenation, a 1x1x1 head, the
masked squared-error loss, and the backward pass written out layer by layer
from the chain rule. With ``bf16=True`` it rounds to bfloat16 (nearest even) at
the points where the device stores BF16: tensor-core layer weights, every
activation after the input layer, and every activation gradient.

Layouts follow include/exx_guess.h: samples [B][S][S][S][C] channels last,
parameters one flat FP32 vector, W[27][cin][cout] then bias per layer.
"""
from __future__ import annotations

import numpy as np

CIN = (3, 16, 16, 32, 32, 64, 64, 128, 192, 64, 96, 32, 48, 16, 16)
MASK = 2  # input channels: rho / s, the multipole boundary values, the ball mask
COUT = (16, 16, 32, 32, 64, 64, 128, 128, 64, 64, 32, 32, 16, 16, 1)
HEAD = 14
TAPS = [(dz, dy, dx) for dz in range(3) for dy in range(3) for dx in range(3)]


def param_sizes():
    return [(CIN[l] if l == HEAD else 27 * CIN[l]) * COUT[l] + COUT[l] for l in range(len(CIN))]


def param_count() -> int:
    return int(sum(param_sizes()))


def unpack(params):
    """Flat vector -> list of (W, b); W is [27][cin][cout] (head: [cin][cout])."""
    out, off = [], 0
    for l in range(len(CIN)):
        nw = (CIN[l] if l == HEAD else 27 * CIN[l]) * COUT[l]
        W = np.asarray(params[off:off + nw], np.float64)
        W = W.reshape(CIN[l], COUT[l]) if l == HEAD else W.reshape(27, CIN[l], COUT[l])
        b = np.asarray(params[off + nw:off + nw + COUT[l]], np.float64)
        out.append((W, b))
        off += nw + COUT[l]
    return out


def pack(grads):
    return np.concatenate([np.concatenate([g[0].ravel(), g[1].ravel()]) for g in grads])


def bf16_round(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = (a + 0x7FFF + ((a >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3(x, W, b=None):
    """y[v][co] = sum_tap sum_ci x[v + tap - 1][ci] W[tap][ci][co] (+ b), zero padding."""
    B, D, H, Wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((B, D, H, Wd, W.shape[2]))
    for t, (dz, dy, dx) in enumerate(TAPS):
        y += xp[:, dz:dz + D, dy:dy + H, dx:dx + Wd, :] @ W[t]
    if b is not None:
        y += b
    return y


def conv3_backward(x, W, g):
    """Gradients of sum(g * conv3(x, W, b)) with respect to x, W and b."""
    B, D, H, Wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1), (0, 0)))
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for t, (dz, dy, dx) in enumerate(TAPS):
        sl = (slice(None), slice(dz, dz + D), slice(dy, dy + H), slice(dx, dx + Wd), slice(None))
        dW[t] = np.einsum("bzyxi,bzyxo->io", xp[sl], g)
        dxp[sl] += g @ W[t].T
    return dxp[:, 1:-1, 1:-1, 1:-1, :], dW, g.sum(axis=(0, 1, 2, 3))


def pool(x):
    B, S, _, _, C = x.shape
    return x.reshape(B, S // 2, 2, S // 2, 2, S // 2, 2, C).mean(axis=(2, 4, 6))


def pool_backward(g):
    return np.repeat(np.repeat(np.repeat(g, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def upsample(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def upsample_backward(g):
    B, S, _, _, C = g.shape
    return g.reshape(B, S // 2, 2, S // 2, 2, S // 2, 2, C).sum(axis=(2, 4, 6))


def relu(x):
    return np.maximum(x, 0.0)


def forward(params, inp, bf16=False):
    """inp [B][S][S][S][3] -> (out [B][S][S][S], cache of activations)."""
    P = unpack(params)
    r = bf16_round if bf16 else (lambda a: a)
    Wq = [(P[l][0] if l in (0, HEAD) else r(P[l][0]), P[l][1]) for l in range(len(P))]
    a = {"in": np.asarray(inp, np.float64)}

    def conv(x, l):
        return r(relu(conv3(x, Wq[l][0], Wq[l][1])))

    a["x0a"] = conv(a["in"], 0)
    a["x0"] = conv(a["x0a"], 1)
    a["p0"] = r(pool(a["x0"]))
    a["x1a"] = conv(a["p0"], 2)
    a["x1"] = conv(a["x1a"], 3)
    a["p1"] = r(pool(a["x1"]))
    a["x2a"] = conv(a["p1"], 4)
    a["x2"] = conv(a["x2a"], 5)
    a["p2"] = r(pool(a["x2"]))
    a["x3a"] = conv(a["p2"], 6)
    a["x3"] = conv(a["x3a"], 7)
    a["c2"] = np.concatenate([upsample(a["x3"]), a["x2"]], axis=-1)
    a["y2a"] = conv(a["c2"], 8)
    a["y2"] = conv(a["y2a"], 9)
    a["c1"] = np.concatenate([upsample(a["y2"]), a["x1"]], axis=-1)
    a["y1a"] = conv(a["c1"], 10)
    a["y1"] = conv(a["y1a"], 11)
    a["c0"] = np.concatenate([upsample(a["y1"]), a["x0"]], axis=-1)
    a["y0a"] = conv(a["c0"], 12)
    a["y0"] = conv(a["y0a"], 13)
    hw, hb = Wq[HEAD]
    out = (a["y0"] @ hw)[..., 0] + hb[0]
    return out, (a, Wq)


def loss_and_gradient(params, inp, target, bf16=False):
    """Loss sum(m (out - t)^2) / (B S^3), m = input channel 1 > 0.5, and its
    gradient with respect to the flat parameters."""
    out, (a, Wq) = forward(params, inp, bf16)
    r = bf16_round if bf16 else (lambda x: x)
    n = out.size
    m = (a["in"][..., MASK] > 0.5).astype(np.float64)
    diff = out - np.asarray(target, np.float64)
    loss = float(np.sum(m * diff * diff) / n)
    gout = 2.0 * m * diff / n
    grads = [None] * len(CIN)
    hw, hb = Wq[HEAD]
    grads[HEAD] = (np.einsum("bzyxc,bzyx->c", a["y0"], gout)[:, None], np.array([gout.sum()]))
    g = r(gout[..., None] * hw[:, 0] * (a["y0"] > 0))

    def back(l, x, g, mask_input):
        """g: gradient at layer l's pre-activation; returns the gradient at its input."""
        dx, dW, db = conv3_backward(x, Wq[l][0], g)
        grads[l] = (dW, db)
        if mask_input is not None:
            dx = dx * (mask_input > 0)
        return r(dx)

    g = back(13, a["y0a"], g, a["y0a"])
    g_c0 = back(12, a["c0"], g, None)
    g = r(upsample_backward(g_c0[..., :32]) * (a["y1"] > 0))
    g = back(11, a["y1a"], g, a["y1a"])
    g_c1 = back(10, a["c1"], g, None)
    g = r(upsample_backward(g_c1[..., :64]) * (a["y2"] > 0))
    g = back(9, a["y2a"], g, a["y2a"])
    g_c2 = back(8, a["c2"], g, None)
    g = r(upsample_backward(g_c2[..., :128]) * (a["x3"] > 0))
    g = back(7, a["x3a"], g, a["x3a"])
    g_p2 = back(6, a["p2"], g, None)
    g = r((pool_backward(g_p2) + g_c2[..., 128:]) * (a["x2"] > 0))
    g = back(5, a["x2a"], g, a["x2a"])
    g_p1 = back(4, a["p1"], g, None)
    g = r((pool_backward(g_p1) + g_c1[..., 64:]) * (a["x1"] > 0))
    g = back(3, a["x1a"], g, a["x1a"])
    g_p0 = back(2, a["p0"], g, None)
    g = r((pool_backward(g_p0) + g_c0[..., 32:]) * (a["x0"] > 0))
    g = back(1, a["x0a"], g, a["x0a"])
    dx, dW, db = conv3_backward(a["in"], Wq[0][0], g)
    grads[0] = (dW, db)
    return loss, pack(grads)


def init_params(seed: int, scale: float = 1.0):
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(len(CIN)):
        fan = CIN[l] if l == HEAD else 27 * CIN[l]
        nw = fan * COUT[l]
        bound = scale * np.sqrt(6.0 / fan)
        parts.append(rng.uniform(-bound, bound, nw))
        parts.append(np.zeros(COUT[l]))
    return np.concatenate(parts).astype(np.float32)
