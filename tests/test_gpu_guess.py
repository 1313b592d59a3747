"""The learned warm start end to end: training samples exported by the
solver agree with the oracle's pair solution, and a network trained on the
GPU (the library's own forward/backward/Adam kernels) starts the CG closer to
the solution: same accuracy gates, fewer iterations."""
import numpy as np
import pytest

import oracle
from paper_1911_10630_gb300 import synth
from tests.gpu_util import D_GATE_MAXREL, E_GATE_PER_ORBITAL, d_maxrel, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def test_exported_samples_match_the_oracle_pair_solution(torch):
    from paper_1911_10630_gb300.exx import Exx
    w = synth.config0()
    phi = w.orbitals()
    ex = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, precision=1, warm_start=1)
    dphi = torch.from_numpy(phi).cuda()
    dD = torch.empty_like(dphi)
    ex.compute(dphi, torch.from_numpy(np.ascontiguousarray(w.centers)).cuda(), dD)
    S = 40  # larger than the ME ball but for its +20 poles
    inp = torch.empty((36, S, S, S, 3), dtype=torch.float32, device="cuda")
    tgt = torch.empty((36, S, S, S), dtype=torch.float32, device="cuda")
    n = ex.export_samples(dphi, S, inp, tgt, 36)
    assert n == 36
    inp, tgt = inp.cpu().numpy(), tgt.cpu().numpy()
    pairs = ex.pairs()
    d2 = float(np.cbrt(np.prod(w.delta ** 2)))
    for k in (0, 5, 17, 35):
        i, j, g = int(pairs["i"][k]), int(pairs["j"][k]), pairs["g"][k]
        ref = oracle.pair_solve(w.cell, w.grid, phi, i, j, g, w.r_pe, w.r_me)
        off, npe = ref["off"][:ref["n_pe"]], ref["n_pe"]
        idx = tuple((off + S // 2).T)
        rho = ref["rho"][:npe]
        s = np.max(np.abs(rho))
        # density channel, mask channel, target = v / (s delta^2) on the ball
        np.testing.assert_allclose(inp[k][idx][:, 0], rho / s, rtol=1e-6, atol=1e-7)
        assert np.all(inp[k][idx][:, 2] == 1.0)
        assert inp[k][..., 2].sum() == npe
        assert np.all(inp[k][idx][:, 1] == 0.0)
        v = ref["v"][:npe]
        np.testing.assert_allclose(tgt[k][idx] * s * d2, v, rtol=0, atol=2e-6 * np.max(np.abs(v)))
        # boundary channel on the shell points in the cube: the oracle's
        # multipole expansion (Eq. me, FP64) against the FP32 channel
        sh = ref["off"][npe:]
        inside = np.all(sh + S // 2 < S, axis=1)
        sidx = tuple((sh[inside] + S // 2).T)
        vsh = ref["v"][npe:][inside]
        np.testing.assert_allclose(inp[k][sidx][:, 1] * s * d2, vsh, rtol=0, atol=1e-4 * np.max(np.abs(vsh)))
        outside = np.ones((S, S, S), bool)
        outside[idx] = False
        assert np.all(inp[k][outside][:, 0] == 0.0) and np.all(inp[k][outside][:, 2] == 0.0)
        assert np.all(tgt[k][outside] == 0.0)
    ex.close()


def test_learned_warm_start_meets_the_gates_with_fewer_iterations(torch):
    """Training is bitwise reproducible (fixed-order gradient reductions, seeded
    initialisation and batch order, solver samples from one fixed launch
    shape), so the gain is one number per GPU model and build: 5.9 % fewer CG
    iterations over these three held-out workloads with 7,200 training samples
    on GB300 (12.8 % over 40 workloads with 18,000 samples), asserted at 3 % to
    leave room for the rounding differences of another build."""
    from paper_1911_10630_gb300 import guess_train
    from paper_1911_10630_gb300.exx import Exx, guess_model_blob
    inp, tgt = guess_train.solve_and_export(range(1000, 1200), torch=torch)
    net, hist = guess_train.train(inp, tgt, epochs=8, batch=32, lr=1e-3)
    assert hist[-1] < 0.01 * hist[0]
    blob = guess_model_blob(guess_train.CUBE, net.get_params())
    net.close()
    del inp, tgt
    iters = {0: 0, 2: 0}
    for seed in (7, 8, 9):  # not among the training workloads
        w = synth.config0(seed)
        phi = w.orbitals()
        dphi = torch.from_numpy(phi).cuda()
        dcen = torch.from_numpy(np.ascontiguousarray(w.centers)).cuda()
        dD = torch.empty_like(dphi)
        for warm in (0, 2):
            ex = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, precision=1, warm_start=warm,
                     autotune=0)
            if warm == 2:
                ex.load_guess_model(blob)
            e = ex.compute(dphi, dcen, dD)
            st = ex.stats()
            iters[warm] += st["iters_total"]
            if warm == 2:
                assert st["guess_ms"] > 0.0
                ref = oracle.exx_workload(w, tol=1e-13, orbitals=phi)
                assert abs(e - ref["E_xx"]) / w.n <= E_GATE_PER_ORBITAL
                assert d_maxrel(dD.cpu().numpy(), ref["D"]) <= D_GATE_MAXREL
            ex.close()
    print("CG iterations from zero", iters[0], "from the learned guess", iters[2])
    assert iters[2] < 0.97 * iters[0], iters


def test_warm_start_2_without_a_model_is_rejected(torch):
    from paper_1911_10630_gb300.exx import Exx, ExxError
    w = synth.config0()
    ex = Exx(w.cell, w.grid, w.r_pair, w.r_pe, w.r_me, w.l_max, w.tol, precision=1, warm_start=2)
    dphi = torch.from_numpy(w.orbitals()).cuda()
    with pytest.raises(ExxError, match="exx_load_guess_model"):
        ex.compute(dphi, torch.from_numpy(np.ascontiguousarray(w.centers)).cuda(), torch.empty_like(dphi))
    with pytest.raises(ExxError, match="magic"):
        ex.load_guess_model(b"\0" * 64)
    ex.close()
