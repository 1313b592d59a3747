"""The MD-like sequence at full size (1024 orbitals, 190^3, about 43k pairs per
step): two steps with the previous-step warm start, and four with the
polynomial extrapolation (the last step from 3 v1 - 3 v2 + v3), the last step
checked on sampled pairs and one sampled orbital's D_xx against the oracle
(which gets the very device input arrays, copied back)."""
import numpy as np
import pytest

import oracle
from tests.gpu_util import D_GATE_MAXREL, E_GATE_PER_ORBITAL, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


@pytest.mark.parametrize("warm,steps", [(1, 2), (3, 4)])
def test_md_sequence_warm_start_full_size(torch, warm, steps):
    from paper_1911_10630_gb300 import md_sequence
    checked = {}

    def check(step, w, phi, D, ex):
        if step != steps - 1:
            return
        pairs = ex.pairs()
        n = len(pairs["i"])
        rng = np.random.default_rng(5)
        sample = np.sort(rng.choice(n, 6, replace=False))
        o = int(pairs["i"][sample[0]])  # this orbital's D: every pair touching it
        touch = np.nonzero((pairs["i"] == o) | (pairs["j"] == o))[0]
        orbs = sorted(set(pairs["i"][sample].tolist()) | set(pairs["j"][sample].tolist()) |
                      set(pairs["i"][touch].tolist()) | set(pairs["j"][touch].tolist()))
        loc = {g: k for k, g in enumerate(orbs)}
        sub_phi = np.stack([phi[g].cpu().numpy() for g in orbs])

        def remap(a):
            return np.array([loc[int(x)] for x in a], np.int32)

        ref = oracle.exx(w.cell, w.grid, sub_phi, (remap(pairs["i"][sample]), remap(pairs["j"][sample]),
                                                   pairs["g"][sample]), w.r_pe, w.r_me, w.l_max, tol=1e-13,
                         want_d=False)
        np.testing.assert_allclose(pairs["e_pair"][sample], ref["E_pair"], rtol=0, atol=E_GATE_PER_ORBITAL / 4)
        mask = np.zeros(len(orbs), np.int32)
        mask[loc[o]] = 1
        ref2 = oracle.exx(w.cell, w.grid, sub_phi, (remap(pairs["i"][touch]), remap(pairs["j"][touch]),
                                                    pairs["g"][touch]), w.r_pe, w.r_me, w.l_max, tol=1e-13,
                          want_d=True, dmask=mask)
        dref = ref2["D"][loc[o]]
        dgot = D[o].cpu().numpy()
        checked["d_err"] = float(np.max(np.abs(dgot - dref)) / np.max(np.abs(dref)))

    recs = md_sequence.run(steps=steps, warm=warm, on_step=check)
    assert recs[0]["n_pair"] > 40000 and all(r["n_nonconv"] == 0 for r in recs)
    assert checked["d_err"] <= D_GATE_MAXREL
    if warm == 1:
        # the warm second step needs fewer iterations per pair than the cold first
        per0 = recs[0]["iters_total"] / recs[0]["n_pair"]
        per1 = recs[1]["iters_total"] / recs[1]["n_pair"]
        assert per1 < 0.99 * per0, (per0, per1)
