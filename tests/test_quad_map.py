"""Host logic of the cluster solver's quad thread map (exx_quad_map), checked
against an independent enumeration of the PE ball (Algorithm 2 order: x, y, z
lexicographic, |o|^2 <= R_PE^2). Needs only the library, no GPU."""
import numpy as np
import pytest

from paper_1911_10630_gb300 import exx


def _ball(R):
    pts = [(x, y, z) for x in range(-R, R + 1) for y in range(-R, R + 1) for z in range(-R, R + 1)
           if x * x + y * y + z * z <= R * R]
    return np.array(pts, np.int64)


@pytest.mark.parametrize("R,C,NT,Q,bank", [(24, 9, 512, 4, 1), (24, 9, 512, 4, 0), (16, 4, 1024, 2, 1),
                                           (16, 9, 512, 4, 1), (5, 2, 512, 4, 1)])
def test_quad_map_covers_the_ball(R, C, NT, Q, bank):
    pk, kk, info = exx.quad_map(R, C, NT, Q, bank)
    pts = _ball(R)
    syz, sp2, cap = int(info[1]), int(info[2]), int(info[3])
    assert syz % 4 == 0 and syz >= 2 * R + 7 and sp2 == (2 * R + 7) * syz
    ranks = info[4:].reshape(C, 4)  # x0, planes, k0, k1
    # slabs: whole x planes, >= 3 each, contiguous, covering the ball in order
    assert ranks[0, 0] == -R and ranks[0, 2] == 0 and ranks[-1, 3] == len(pts)
    for r in range(C):
        x0, planes, k0, k1 = ranks[r]
        assert planes >= 3 and planes <= cap
        if r + 1 < C:
            assert ranks[r + 1, 0] == x0 + planes and ranks[r + 1, 2] == k1
        assert np.all((pts[k0:k1, 0] >= x0) & (pts[k0:k1, 0] < x0 + planes))
    seen = np.zeros(len(pts), np.int64)
    for r in range(C):
        x0, planes, k0, k1 = ranks[r]
        p = pk[r].reshape(-1).astype(np.int64)
        k = kk[r].reshape(-1).astype(np.int64)
        off, mask, xl = p & 0xFFFFF, (p >> 20) & 15, p >> 24
        assert np.all(off % 4 == 0)
        for i in range(4):
            sel = (mask >> i) & 1 == 1
            ki = k[sel] + i
            assert np.all((ki >= k0) & (ki < k1))
            x, y, z = pts[ki, 0], pts[ki, 1], pts[ki, 2]
            np.testing.assert_array_equal(x - x0, xl[sel])
            np.testing.assert_array_equal((x - x0) * sp2 + (y + R + 3) * syz + (z + R + 3), off[sel] + i)
            np.add.at(seen, ki, 1)
        # idle slots: no valid element, a quad outside the ball in every plane, all
        # 15 stencil legs inside the slab array with its 3 halo planes per side
        idle = mask == 0
        rows, zs = off[idle] // syz, off[idle] % syz
        y = rows - (R + 3)
        for i in range(4):
            assert np.all(y * y + (zs + i - (R + 3)) ** 2 > R * R)
        legs = np.concatenate([[0, -4, 4], [q * syz for q in (-3, -2, -1, 1, 2, 3)],
                               [q * sp2 for q in (-3, -2, -1, 1, 2, 3)]])
        lo, hi = -3 * sp2, (planes + 3) * sp2
        a = off[:, None] + legs[None, :]
        assert np.all(a >= lo) and np.all(a + 3 < hi)
        if bank:
            g = ((off >> 2) & 7).reshape(-1, 8)
            assert all(len(set(row)) == 8 for row in g.tolist())
    assert np.all(seen == 1)


def test_quad_map_rejects_what_does_not_fit():
    with pytest.raises(exx.ExxError):
        exx.quad_map(24, 9, 256, 2, 1)   # 512 slots for ~1,900 quads per CTA
    with pytest.raises(exx.ExxError):
        exx.quad_map(24, 20, 512, 4, 0)  # more CTAs than the cluster limit
