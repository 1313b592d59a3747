"""The radius sweeps on a small case: relative errors in E_xx fall as R_pair
and the self / non-self R_PE grow and gamma_xx falls as R_ME grows (the
trends of the paper's accuracy study). Unlike orthonormal MLWFs, the
synthetic clusters of overlapping Gaussians give the non-self pairs a large
share of E_xx (their densities carry monopoles), so no share is asserted."""
import numpy as np
import pytest

from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def _decreasing(vals):
    v = np.asarray(vals)
    floor = 1e-12  # below the solver tolerance the trend is noise
    return all(b <= a * 1.05 or b < floor for a, b in zip(v[:-1], v[1:]))


def test_radius_sweeps_converge(torch):
    from paper_1911_10630_gb300 import radius_sweep
    res = radius_sweep.sweep(n_orbitals=16, r_ref=28, shell=8, tol=1e-11, pe_radii=(10, 14, 18, 22),
                             default_self=(20, 32), default_nonself=(16, 24), me_self=(24, 28, 32, 36),
                             me_nonself=(19, 24, 28, 32, 36), log=lambda m: None)
    assert 0.0 < res["self_share"] < 1.0
    assert _decreasing([r["rel_err"] for r in res["r_pair"]])
    assert _decreasing([r["rel_err"] for r in res["r_pe_self"]])
    assert _decreasing([r["rel_err"] for r in res["r_pe_nonself"]])
    assert _decreasing([g["gamma_xx"] for g in res["gamma_r_me_self"]])
    assert _decreasing([g["gamma_xx"] for g in res["gamma_r_me_nonself"]])
    assert res["gamma_r_me_self"][-1]["gamma_xx"] < 1e-9  # the reference point itself
    assert res["r_pe_self"][0]["rel_err"] > res["r_pe_self"][-1]["rel_err"]
