"""Compact per-orbital storage (exx_compute_boxes): each orbital kept only on a
periodic box of grid points around its support.

Boxes of side 2 (ceil(R_pair / (2 delta)) + R_ME + 1) + 1 around each orbital's
nearest grid point hold every ME ball of every pair of the orbital, so the
results must equal the full-grid ones: E_xx, every E_ij and, in the
deterministic mode (order-independent integer accumulation), D_xx on each box
bit for bit. A box too small for some pairs is reported (n_clipped) and then
equals the full-grid result with those orbitals cut to zero outside their
boxes."""
import math

import numpy as np
import pytest

from paper_1911_10630_gb300 import synth
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def _boxes(phi, w, side):
    """The orbitals cut to boxes of the given side around their nearest grid points."""
    n = phi.shape[0]
    N = np.asarray(w.grid)
    g = np.floor(np.asarray(w.centers) / w.delta + 0.5).astype(np.int64) % N
    org = (g - side // 2) % N
    idx = [(org[:, a, None] + np.arange(side)[None, :]) % N[a] for a in range(3)]
    box = np.empty((n, side, side, side))
    for i in range(n):
        box[i] = phi[i][np.ix_(idx[0][i], idx[1][i], idx[2][i])]
    return box, org.astype(np.int32), idx


@pytest.mark.parametrize("precision,preconditioner", [(1, 0), (0, 0), (1, 1), (0, 1)])
def test_boxes_equal_full_grids(torch, precision, preconditioner):
    from paper_1911_10630_gb300.exx import Exx
    w = synth.tiny(seed=5, n=6, npts=40, length=8.0, r_pe=6, r_me=9, r_pair=3.0, tol=1e-10)
    phi = w.orbitals()
    side = 2 * (math.ceil(w.r_pair / (2 * w.delta[0])) + w.r_me + 1) + 1
    assert side < w.grid[0]
    box, org, idx = _boxes(phi, w, side)
    dcen = torch.from_numpy(np.ascontiguousarray(w.centers)).cuda()
    ex = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, precision=precision, deterministic=1,
             preconditioner=preconditioner)
    dphi = torch.from_numpy(phi).cuda()
    dD = torch.empty_like(dphi)
    e_full = ex.compute(dphi, dcen, dD)
    D_full = dD.cpu().numpy()
    pairs_full = ex.pairs()
    dbox = torch.from_numpy(box).cuda()
    dDb = torch.empty_like(dbox)
    e_box = ex.compute_boxes(dbox, torch.from_numpy(org).cuda(), dcen, dDb)
    st = ex.stats()
    assert st["n_clipped"] == 0 and st["n_pair"] == len(pairs_full["i"]) > w.n
    assert e_box == e_full
    np.testing.assert_array_equal(ex.pairs()["e_pair"], pairs_full["e_pair"])
    Db = dDb.cpu().numpy()
    for i in range(w.n):
        np.testing.assert_array_equal(Db[i], D_full[i][np.ix_(idx[0][i], idx[1][i], idx[2][i])])
        # nothing of D^i lies outside its box
        outside = np.ones(tuple(w.grid), bool)
        outside[np.ix_(idx[0][i], idx[1][i], idx[2][i])] = False
        assert np.all(D_full[i][outside] == 0.0)
    ex.close()


def test_clipped_boxes_are_counted_and_equal_cut_orbitals(torch):
    from paper_1911_10630_gb300.exx import Exx
    w = synth.tiny(seed=5, n=6, npts=40, length=8.0, r_pe=6, r_me=9, r_pair=3.0, tol=1e-10)
    phi = w.orbitals()
    side = 2 * w.r_me + 3  # too small for the pairs whose centre is off the orbital's own
    box, org, idx = _boxes(phi, w, side)
    cut = np.zeros_like(phi)
    for i in range(w.n):
        cut[i][np.ix_(idx[0][i], idx[1][i], idx[2][i])] = box[i]
    dcen = torch.from_numpy(np.ascontiguousarray(w.centers)).cuda()
    ex = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, precision=1, deterministic=1)
    dcut = torch.from_numpy(cut).cuda()
    dD = torch.empty_like(dcut)
    e_cut = ex.compute(dcut, dcen, dD)
    D_cut = dD.cpu().numpy()
    dbox = torch.from_numpy(box).cuda()
    dDb = torch.empty_like(dbox)
    e_box = ex.compute_boxes(dbox, torch.from_numpy(org).cuda(), dcen, dDb)
    assert ex.stats()["n_clipped"] > 0
    assert e_box == e_cut
    Db = dDb.cpu().numpy()
    for i in range(w.n):
        np.testing.assert_array_equal(Db[i], D_cut[i][np.ix_(idx[0][i], idx[1][i], idx[2][i])])
    ex.close()


def test_box_dim_is_validated(torch):
    from paper_1911_10630_gb300.exx import Exx, ExxError
    w = synth.tiny(seed=5, n=4, npts=40, length=8.0, r_pe=6, r_me=9, r_pair=3.0)
    ex = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, precision=1)
    small = torch.zeros((w.n, 2 * w.r_me, 2 * w.r_me, 2 * w.r_me), dtype=torch.float64, device="cuda")
    org = torch.zeros((w.n, 3), dtype=torch.int32, device="cuda")
    cen = torch.from_numpy(np.ascontiguousarray(w.centers)).cuda()
    with pytest.raises(ExxError, match="box_dim"):
        ex.compute_boxes(small, org, cen, torch.empty_like(small))
    ex.close()
