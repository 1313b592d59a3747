"""The ball tables the kernels index (exx_ball_tables), checked on the CPU:
the proto-subdomain of Algorithm 2 point for point against the oracle's
brute-force construction, the packed offsets and cube indices against their
definitions, and the FP64 shell layer against the reach of the stencil of
Eq. d2_1, by brute force: every shell point that the stencil reads from a PE
point must have its far-field potential evaluated in FP64."""
import numpy as np
import pytest

import oracle

RADII = [(1, 4), (3, 6), (5, 9), (6, 9), (12, 15), (13, 17), (16, 20), (24, 32), (29, 32), (32, 35)]


@pytest.fixture(scope="module")
def exx():
    from paper_1911_10630_gb300 import build, exx as _exx
    build.build(quiet=True)
    _exx.load()
    return _exx


def unpack(off):
    off = off.astype(np.int64)
    return np.stack([(off & 0xff) - 128, ((off >> 8) & 0xff) - 128, ((off >> 16) & 0xff) - 128], axis=1)


@pytest.mark.parametrize("r_pe, r_me", RADII)
def test_tables_equal_the_oracle_subdomain(exx, r_pe, r_me):
    t = exx.ball_tables(r_pe, r_me)
    ref, n_pe = oracle.proto_subdomain(r_pe, r_me)
    assert t["n_pe"] == n_pe and t["n_me"] == len(ref)
    np.testing.assert_array_equal(unpack(t["off"]), ref)
    S = 2 * r_me + 1
    o = ref.astype(np.int64) + r_me
    np.testing.assert_array_equal(t["cube"], (o[:, 0] * S + o[:, 1]) * S + o[:, 2])


@pytest.mark.parametrize("r_pe, r_me", RADII)
def test_every_shell_point_the_stencil_reads_is_fp64(exx, r_pe, r_me):
    t = exx.ball_tables(r_pe, r_me)
    o = unpack(t["off"])
    n_pe = t["n_pe"]
    assert not t["near"][:n_pe].any()
    shell = o[n_pe:]
    needed = np.zeros(len(shell), bool)
    for a in range(3):
        for q in (1, 2, 3):
            for s in (-1, 1):
                p = shell.copy()
                p[:, a] += s * q
                needed |= (p * p).sum(axis=1) <= r_pe * r_pe
    near = t["near"][n_pe:].astype(bool)
    assert needed.any()
    missing = shell[needed & ~near]
    assert len(missing) == 0, missing[:5]


def test_bad_arguments_are_rejected(exx):
    from paper_1911_10630_gb300.exx import ExxError
    for r_pe, r_me in ((0, 4), (6, 6), (8, 5), (10, 65)):
        with pytest.raises(ExxError, match="exx_ball_tables"):
            exx.ball_tables(r_pe, r_me)
