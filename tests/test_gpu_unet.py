"""The learned warm start's U-Net on the GPU against its CPU oracle
(oracle/unet.py): the tcgen05 implicit-GEMM convolution (forward and data
gradient), the whole forward pass, every parameter gradient, and training."""
import numpy as np
import pytest

from oracle import unet as ounet
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def _bf16_tensor(torch, a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).cuda()


@pytest.mark.parametrize("B,D,H,W,cin,cout,mode", [
    (1, 4, 16, 8, 16, 16, 1),      # exactly one tile
    (2, 5, 20, 11, 32, 48, 0),     # ragged in every axis, two input chunks
    (1, 3, 3, 3, 64, 128, 1),      # smaller than one tile
    (1, 6, 17, 9, 192, 64, 1),     # widest input (up-path concat)
    (2, 5, 18, 10, 64, 32, 2),     # data gradient, cout -> cin
    (1, 4, 16, 16, 192, 64, 2),    # data gradient with 192 outputs (two TMEM slices of 192)
    # depth-folded tiles (one MMA of N = 3 x outputs per (dh, dw)): 16 outputs
    # (8 slices per tile) and 32 outputs (4 slices), ragged depth, 1-3 chunks
    (2, 10, 20, 12, 16, 32, 1),
    (1, 9, 16, 8, 48, 16, 0),
    (1, 3, 5, 4, 32, 16, 1),       # depth shorter than a tile
    (2, 6, 18, 9, 16, 32, 2),      # data gradient onto 16 channels
    (1, 5, 17, 9, 32, 48, 2),      # data gradient onto 32 channels
])
def test_conv3_tensor_core_matches_oracle(torch, B, D, H, W, cin, cout, mode):
    from paper_1911_10630_gb300 import exx
    rng = np.random.default_rng(cin * 7 + cout + mode)
    if mode == 2:
        xin = ounet.bf16_round(rng.normal(size=(B, D, H, W, cout)))
        mask = ounet.bf16_round(rng.normal(size=(B, D, H, W, cin)))
    else:
        xin = ounet.bf16_round(rng.normal(size=(B, D, H, W, cin)))
        mask = None
    w = rng.normal(0, 0.2, size=(27, cin, cout)).astype(np.float32)
    bias = rng.normal(0, 0.5, size=cout).astype(np.float32)
    wq = ounet.bf16_round(w)
    if mode == 2:
        g = xin
        xp = np.zeros((B, D, H, W, cin))
        dx, _, _ = ounet.conv3_backward(xp, wq, g)
        ref = dx * (mask > 0)
        ycha = cin
    else:
        ref = ounet.conv3(xin, wq, bias.astype(np.float64))
        if mode == 1:
            ref = np.maximum(ref, 0)
        ycha = cout
    dx_ = _bf16_tensor(torch, xin)
    dw = torch.from_numpy(w).cuda()
    db = torch.from_numpy(bias).cuda()
    dm = _bf16_tensor(torch, mask) if mask is not None else None
    dy = torch.empty((B, D, H, W, ycha), dtype=torch.bfloat16, device="cuda")
    exx.unet_conv3d(dx_, dw, db if mode != 2 else None, dm, dy, B, D, H, W, cin, cout, mode)
    torch.cuda.synchronize()
    y = dy.float().cpu().numpy().astype(np.float64)
    scale = np.max(np.abs(ref))
    err = np.abs(y - ref)
    # FP32 accumulation of BF16 products, one BF16 rounding of the result
    assert np.max(err) <= 8e-3 * scale + 1e-6, (np.max(err), scale)
    assert np.linalg.norm(y - ref) <= 4e-3 * np.linalg.norm(ref)


def _batch(S, B, seed):
    rng = np.random.default_rng(seed)
    c = np.arange(S) - S / 2
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    r2 = x * x + y * y + z * z
    inp = np.zeros((B, S, S, S, 3), np.float32)
    tgt = np.zeros((B, S, S, S), np.float32)
    for b in range(B):
        a = rng.uniform(0.05, 0.2)
        sh = rng.normal(0, 1.5, 3)
        rho = np.exp(-a * ((x - sh[0]) ** 2 + (y - sh[1]) ** 2 + (z - sh[2]) ** 2))
        mask = r2 <= (S / 2) ** 2
        d = np.sqrt((x - sh[0]) ** 2 + (y - sh[1]) ** 2 + (z - sh[2]) ** 2) + 1.0
        inp[b, ..., 0] = rho * mask
        inp[b, ..., 1] = (5.0 / d) * ~mask  # boundary-like values outside the ball
        inp[b, ..., 2] = mask
        tgt[b] = (5.0 / d) * mask
    return inp, tgt


def test_forward_and_gradients_match_oracle(torch):
    from paper_1911_10630_gb300.exx import GuessNet
    S, B = 16, 2
    inp, tgt = _batch(S, B, 11)
    p = ounet.init_params(12)
    p = p + np.random.default_rng(13).normal(0, 0.02, p.size).astype(np.float32)
    net = GuessNet(S, B)
    assert net.n_params == ounet.param_count()
    net.set_params(p)
    assert np.array_equal(net.get_params(), p)
    di = torch.from_numpy(inp).cuda()
    dt = torch.from_numpy(tgt).cuda()
    do = torch.empty((B, S, S, S), dtype=torch.float32, device="cuda")
    net.forward(di, do, B)
    torch.cuda.synchronize()
    out = do.cpu().numpy()
    ref, _ = ounet.forward(p, inp, bf16=True)
    assert np.linalg.norm(out - ref) <= 2e-2 * np.linalg.norm(ref), np.linalg.norm(out - ref) / np.linalg.norm(ref)
    loss, g = net.gradient(di, dt, B)
    rloss, rg = ounet.loss_and_gradient(p, inp, tgt, bf16=True)
    assert abs(loss - rloss) <= 2e-2 * abs(rloss)
    offs = np.concatenate([[0], np.cumsum(ounet.param_sizes())])
    for l in range(len(ounet.CIN)):
        a, b = g[offs[l]:offs[l + 1]], rg[offs[l]:offs[l + 1]]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        # Both sides round to BF16 (8-bit mantissa) at the same points, but an
        # FP32 (device) and an FP64 (oracle) value on either side of a
        # rounding boundary round one BF16 step apart, and such flips pass on
        # through the layers. The bottleneck layers (6, 7: 2^3 voxels per
        # sample at S = 16) sum their weight gradients over 16 voxels only, so
        # the flips do not average out there.
        assert rel <= (8e-2 if l in (6, 7) else 5e-2), (l, rel)
    net.close()


def test_training_reduces_the_loss(torch):
    from paper_1911_10630_gb300.exx import GuessNet
    S, B = 16, 8
    inp, tgt = _batch(S, B, 21)
    net = GuessNet(S, B)
    net.set_params(ounet.init_params(22))
    di = torch.from_numpy(inp).cuda()
    dt = torch.from_numpy(tgt).cuda()
    losses = [net.train_step(di, dt, B, 2e-3) for _ in range(60)]
    assert all(np.isfinite(losses))
    assert losses[-1] < 0.25 * losses[0], (losses[0], losses[-1])
    net.close()
