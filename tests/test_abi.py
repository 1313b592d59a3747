"""The C-ABI library builds, loads and exports every symbol include/exx.h
declares; argument validation happens on the host before any CUDA call."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "exx.h")
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def lib():
    from paper_1911_10630_gb300 import build, exx
    build.build(quiet=True)
    return exx.load()


def declared_functions():
    text = "\n".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(exx_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("exx_init", "exx_compute", "exx_compute_async", "exx_compute_host", "exx_get_stats", "exx_last_error",
                     "exx_destroy", "exx_default_options"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1911_10630_gb300 import exx
    names = declared_functions()
    bound = {n for n, _, _ in exx.SIGNATURES}
    for n in names:
        assert hasattr(lib, n), n
        assert n in bound, f"binding lacks {n}"


def test_default_options(lib):
    o = lib.exx_default_options()
    assert o.precision == 0 and o.batched == 1 and o.max_iter == 20000
    assert o.inner_max_iter == 4000 and o.inner_tol == 0.0  # library choice: 1e-4 multigrid, else 1e-5


def _init(lib, cell=(9.0, 9.0, 9.0), grid=(48, 48, 48), r_pair=math.inf, r_pe=16, r_me=20, lmax=6, tol=1e-10,
          opt=None):
    from paper_1911_10630_gb300 import exx
    ctx = ctypes.c_void_p()
    c = np.asarray(cell, np.float64)
    g = np.asarray(grid, np.int32)
    st = lib.exx_init(ctypes.byref(ctx), c.ctypes.data_as(exx._d), g.ctypes.data_as(exx._i), r_pair, r_pe, r_me,
                      lmax, tol, ctypes.byref(opt) if opt is not None else None)
    return st, ctx


@pytest.mark.parametrize("kw,frag", [
    (dict(r_me=18), "r_pe + 3"),
    (dict(grid=(48, 48, 40)), "2 r_me + 1"),
    (dict(lmax=7), "l_max"),
    (dict(tol=0.0), "tol"),
    (dict(tol=1.5), "tol"),
    (dict(r_pair=-1.0), "r_pair"),
    (dict(cell=(9.0, -1.0, 9.0)), "cell"),
    (dict(r_pe=0, r_me=3), "r_pe"),
    (dict(r_pe=61, r_me=64, grid=(200, 200, 200)), "r_me"),
])
def test_init_rejects_invalid_arguments_before_cuda(lib, kw, frag):
    st, ctx = _init(lib, **kw)
    assert st == -1
    assert not ctx.value
    assert frag in lib.exx_last_error(None).decode()


def test_init_rejects_bad_options(lib):
    o = lib.exx_default_options()
    o.precision = 3
    st, ctx = _init(lib, opt=o)
    assert st == -1 and "precision" in lib.exx_last_error(None).decode()
    o = lib.exx_default_options()
    o.threads = 300
    st, ctx = _init(lib, opt=o)
    assert st == -1 and "threads" in lib.exx_last_error(None).decode()
    # separate self / non-self radii: the non-self ball must fit inside the self one
    for pe, me in ((0, 16), (17, 20), (12, 14), (12, 21)):
        o = lib.exx_default_options()
        o.radii_mode = 2
        o.r_pe_nonself, o.r_me_nonself = pe, me
        st, ctx = _init(lib, opt=o)
        assert st == -1 and "r_pe_nonself" in lib.exx_last_error(None).decode(), (pe, me)
    o = lib.exx_default_options()
    o.radii_mode = 2
    o.r_pe_nonself, o.r_me_nonself = 12, 16
    o.solver_kind = 2
    st, ctx = _init(lib, opt=o)
    assert st == -1 and "solver_kind 1" in lib.exx_last_error(None).decode()
    o = lib.exx_default_options()
    assert o.fixed_residual == 0
    o.fixed_residual = 3
    st, ctx = _init(lib, opt=o)
    assert st == -1 and "fixed_residual" in lib.exx_last_error(None).decode()
    o = lib.exx_default_options()
    o.warm_start = 4
    st, ctx = _init(lib, opt=o)
    assert st == -1 and "warm_start" in lib.exx_last_error(None).decode()
    o = lib.exx_default_options()
    assert o.deterministic == 0
    o.deterministic = 2
    st, ctx = _init(lib, opt=o)
    assert st == -1 and "deterministic" in lib.exx_last_error(None).decode()
    o = lib.exx_default_options()
    assert o.preconditioner == 0 and o.inject_wait_timeout == 0
    o.preconditioner = 2
    st, ctx = _init(lib, opt=o)
    assert st == -1 and "preconditioner" in lib.exx_last_error(None).decode()
    o = lib.exx_default_options()
    o.preconditioner = 1
    o.precision = 0
    o.solver_kind = 2  # the multigrid CG on clusters is FP32 inside FP64 refinement
    st, ctx = _init(lib, opt=o)
    assert st == -1 and "precision" in lib.exx_last_error(None).decode()
    o = lib.exx_default_options()
    o.preconditioner = 1
    o.precision = 1
    o.cluster_size = 9  # cluster sizes of the multigrid CG: 2, 4, 8, 16
    st, ctx = _init(lib, opt=o)
    assert st == -1 and "multigrid" in lib.exx_last_error(None).decode()
    o = lib.exx_default_options()
    o.preconditioner = 1
    o.precision = 1
    o.warm_start = 1
    st, ctx = _init(lib, opt=o)
    assert st == -1 and "multigrid" in lib.exx_last_error(None).decode()
    o = lib.exx_default_options()
    o.inject_wait_timeout = -1
    st, ctx = _init(lib, opt=o)
    assert st == -1 and "inject_wait_timeout" in lib.exx_last_error(None).decode()


def test_null_and_destroy_are_safe(lib):
    from paper_1911_10630_gb300 import exx
    e = ctypes.c_double()
    assert lib.exx_compute(None, None, None, 1, None, ctypes.byref(e), None, None) == -1
    lib.exx_destroy(None)
    s = exx.exx_stats()
    assert lib.exx_get_stats(None, ctypes.byref(s)) == -1


def test_init_without_a_gpu_reports_cuda_error(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, ctx = _init(lib)
    assert st == -3
    assert lib.exx_last_error(None).decode()


def test_binding_fails_loudly_without_the_library(tmp_path):
    import importlib
    from paper_1911_10630_gb300 import exx
    m = importlib.reload(exx)  # a fresh binding with no library loaded yet
    with pytest.raises(OSError):
        m.load(str(tmp_path / "missing.so"))


def test_guess_param_count_matches_the_oracle_network(lib):
    from oracle import unet
    assert lib.exx_guess_param_count() == unet.param_count()


def test_guess_create_rejects_bad_sizes(lib):
    import ctypes
    h = ctypes.c_void_p()
    assert lib.exx_guess_create(ctypes.byref(h), 12, 4) == -1
    assert "multiple of 8" in lib.exx_last_error(None).decode()
    assert lib.exx_guess_create(ctypes.byref(h), 16, 0) == -1
    assert not h.value


C_CALLER = r"""
#include <stdio.h>
#include <stdlib.h>
#include "exx.h"
#include "exx_guess.h"

int main(void) {
    int n_pe = 0, n_me = 0, levels = 0, radius[8], points[8], side[8];
    const double delta[3] = {0.2, 0.2, 0.2};
    int *off = (int *)malloc(sizeof(int) * 40000);
    if (!off) return 2;
    if (exx_ball_tables(16, 20, off, NULL, NULL, 40000, &n_pe, &n_me) != EXX_OK) return 3;
    if (exx_mg_levels(24, delta, radius, points, side, 8, &levels, NULL, 0) != EXX_OK) return 4;
    printf("%d %d %d", n_pe, n_me, levels);
    for (int l = 0; l < levels; ++l) printf(" %d", radius[l]);
    printf("\n");
    free(off);
    return exx_mg_levels(3, delta, radius, points, side, 8, &levels, NULL, 0) == EXX_EINVAL ? 0 : 5;
}
"""


def test_a_c_program_compiles_links_and_calls_the_boundary(tmp_path, lib):
    """The headers are plain C (C99, warnings as errors); a C program links the
    library and calls host-only entry points without any GPU: the ball counts
    of R 16 / 20 (17,077 and 33,401 points) and the levels of an R_PE 24
    hierarchy (12, 6, 3)."""
    import shutil
    import subprocess
    from paper_1911_10630_gb300 import exx
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "caller.c"
    src.write_text(C_CALLER)
    exe = tmp_path / "caller"
    libdir = os.path.dirname(exx.LIB_PATH)
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-L", libdir, "-lexx_gb300", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
    assert out.stdout.split() == ["17077", "33401", "3", "12", "6", "3"]
