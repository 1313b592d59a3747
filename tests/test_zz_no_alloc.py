"""The allocation-free pair list (exx_pair_list_static) against exx_compute's.

exx_pair_list_static serves callers that cannot allocate device memory:
applications whose device memory all goes through their own pool or a fixed
budget, and latency-bound loops that cannot take cudaMalloc's implicit
synchronisation. Its scratch is a static device array shared by all calls and
kept between them. The test therefore calls it twice in a row, on two
different inputs. Each result must equal, bit for bit, the pair list that
exx_compute built for the same input (the pair list is integer output,
compared exactly).
"""
import ctypes
import math

import numpy as np
import pytest

from paper_1911_10630_gb300 import synth
from tests.gpu_util import require_gpu, run_gpu

pytestmark = pytest.mark.gpu


def _static_pairs(torch, w, cap=None):
    from paper_1911_10630_gb300 import exx
    lib = exx.load()
    n = w.n
    cap = n * (n + 1) // 2 if cap is None else cap
    dcen = torch.from_numpy(np.ascontiguousarray(w.centers)).cuda()
    out = torch.full((max(cap, 1), 5), -1, dtype=torch.int32, device="cuda")
    cell = np.ascontiguousarray(w.cell, np.float64)
    grid = np.ascontiguousarray(w.grid, np.int32)
    count = ctypes.c_int(-1)
    r_pair = float(w.r_pair) if math.isfinite(w.r_pair) else float("inf")
    st = lib.exx_pair_list_static(dcen.data_ptr(), n, cell.ctypes.data_as(exx._d), grid.ctypes.data_as(exx._i),
                                  r_pair, out.data_ptr(), cap, ctypes.byref(count), None)
    torch.cuda.synchronize()
    return st, count.value, out.cpu().numpy(), exx.exx_last_error(None)


def _reference_pairs(torch, w):
    ref = run_gpu(w, torch=torch)["pairs"]
    return np.stack([ref["i"], ref["j"], ref["g"][:, 0], ref["g"][:, 1], ref["g"][:, 2]], 1)


def test_static_pair_list_matches_exx_compute_on_two_calls():
    torch = require_gpu()
    ragged = synth.tiny(seed=3, n=6, npts=28, length=6.5, r_pe=5, r_me=9, r_pair=3.0)
    ragged.grid = np.array([28, 30, 26])
    ragged.cell = np.array([6.5, 7.1, 6.2])
    ragged.centers = np.mod(ragged.centers, ragged.cell)
    ragged.centers[0] = [0.05, 3.0, 6.1]
    ragged.centers[1] = [6.3, 3.2, 0.2]
    for w in (synth.config0(), ragged):  # two calls in a row on the shared scratch
        ref = _reference_pairs(torch, w)
        st, count, got, err = _static_pairs(torch, w)
        assert st == 0, err
        assert count == len(ref)
        np.testing.assert_array_equal(got[:count], ref)


def test_static_pair_list_rejects_sizes_beyond_its_scratch():
    torch = require_gpu()
    w = synth.config0()
    w.centers = np.tile(w.centers, (2049, 1))[:16385]  # one more orbital than the static array holds
    st, count, _, err = _static_pairs(torch, w, cap=1)
    assert st == -1 and "16384" in err
    # a capacity smaller than the pair count reports the count and writes only cap records
    w2 = synth.config0()
    st, count, got, err = _static_pairs(torch, w2, cap=10)
    assert st == -1 and count == 36 and "cap" in err
    ref = _reference_pairs(torch, w2)
    np.testing.assert_array_equal(got[:10], ref[:10])
