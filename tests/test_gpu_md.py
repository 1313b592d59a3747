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


# --------------------------------------------------------------------------
# The MD-like protocol: zero / previous-step / learned warm starts over the
# sequence, E_xx drift of every step against the oracle on a fixed subset of
# pairs, p50 / p99 step time. The full protocol (20 steps, a 24-orbital
# subset, a network trained on 6,000 water-64-form samples) runs with
# EXX_MD_STEPS=20 EXX_MD_SUBSET=24 EXX_MD_TRAIN=full and writes its summary to
# EXX_MD_OUT; by default it runs 3 steps on a 12-orbital subset with a briefly
# trained network (the learned arm's path under the gates, not its payoff).
# --------------------------------------------------------------------------

def _subset_pairs(w, n_orb):
    """The listed pairs among the n_orb orbitals nearest (minimum image) to
    orbital 0: (global orbital indices, [(i, j)])."""
    d = w.centers - w.centers[0]
    d -= w.cell * np.floor(d / w.cell + 0.5)
    orbs = np.sort(np.argsort(np.sum(d * d, axis=1))[:n_orb])
    pi, pj, _ = oracle.pair_list(w.centers[orbs], w.cell, w.grid, w.r_pair)
    return orbs, [(int(orbs[a]), int(orbs[b])) for a, b in zip(pi, pj)]


def _oracle_subset(cell, grid, sub_phi, centers, r_pair, r_pe, r_me, l_max, orbs, subset):
    """E_ij of the subset pairs by the oracle (run in a spawned worker)."""
    pi, pj, g = oracle.pair_list(centers, cell, grid, r_pair)
    have = {(int(orbs[a]), int(orbs[b])): k for k, (a, b) in enumerate(zip(pi, pj))}
    ref = oracle.exx(cell, grid, sub_phi, (pi, pj, g), r_pe, r_me, l_max, tol=1e-13, want_d=False)
    return np.array([ref["E_pair"][have[p]] if p in have else np.nan for p in subset])


def _learned_model(torch, full):
    from paper_1911_10630_gb300 import guess_train, synth
    from paper_1911_10630_gb300.exx import guess_model_blob
    nw, per, epochs = (15, 400, 8) if full else (2, 64, 2)
    inp, tgt = guess_train.solve_and_export(range(2000, 2000 + nw), S=guess_train.CUBE_R24, torch=torch,
                                            workload=synth.config1, per_workload=per)
    net, hist = guess_train.train(inp, tgt, S=guess_train.CUBE_R24, epochs=epochs, batch=32, lr=1e-3)
    blob = guess_model_blob(guess_train.CUBE_R24, net.get_params())
    net.close()
    del inp, tgt
    torch.cuda.empty_cache()
    return blob, hist


def test_md_protocol_three_warm_starts(torch):
    import concurrent.futures
    import json
    import multiprocessing
    import os

    from paper_1911_10630_gb300 import md_sequence, synth
    steps = int(os.environ.get("EXX_MD_STEPS", "3"))
    n_orb = int(os.environ.get("EXX_MD_SUBSET", "12"))
    full = os.environ.get("EXX_MD_TRAIN", "small") == "full"
    w0 = synth.config4(0, 0)
    orbs, subset = _subset_pairs(w0, n_orb)
    assert len(subset) >= n_orb
    blob, hist = _learned_model(torch, full)
    refs = [None] * steps
    pool = concurrent.futures.ProcessPoolExecutor(1, mp_context=multiprocessing.get_context("spawn"))
    futs = {}

    def submit(step, w, phi, D, ex):  # the oracle of each step, beside the GPU's later steps
        sub_phi = np.stack([phi[int(g)].cpu().numpy() for g in orbs])
        futs[step] = pool.submit(_oracle_subset, w.cell, w.grid, sub_phi, w.centers[orbs], w.r_pair, w.r_pe,
                                 w.r_me, w.l_max, orbs, subset)

    arms = {}
    try:
        arms["zero"] = md_sequence.run(steps=steps, warm=0, subset=subset, on_step=submit)
        arms["previous"] = md_sequence.run(steps=steps, warm=1, subset=subset)
        arms["learned"] = md_sequence.run(steps=steps, warm=2, model_blob=blob, subset=subset)
        for s in range(steps):
            refs[s] = futs[s].result()
    finally:
        pool.shutdown()
    m = np.array([1.0 if i == j else 2.0 for i, j in subset])
    summary = {"steps": steps, "subset_orbitals": int(n_orb), "subset_pairs": len(subset),
               "training_loss": [hist[0], hist[-1]], "arms": {}}
    for name, recs in arms.items():
        assert all(r["n_nonconv"] == 0 for r in recs), name
        drift = []
        for s, r in enumerate(recs):
            e = np.array(r["e_sub"])
            ok = np.isfinite(e) & np.isfinite(refs[s])
            assert ok.sum() >= 0.9 * len(subset)
            # every pair and the subset's E_xx per orbital within the gate of
            # |dE_xx| / N_o (a pair's error is part of its orbitals' share)
            assert np.max(np.abs(e[ok] - refs[s][ok])) <= E_GATE_PER_ORBITAL, (name, s)
            de = abs(float(np.sum(m[ok] * (e[ok] - refs[s][ok])))) / n_orb
            assert de <= E_GATE_PER_ORBITAL, (name, s, de)
            drift.append(de)
        p50, p99 = md_sequence.step_time_percentiles(recs)
        summary["arms"][name] = {
            "p50_ms": p50, "p99_ms": p99,
            "pair_solves_per_s": float(np.sum([r["n_pair"] for r in recs]) / (np.sum([r["total_ms"] for r in recs]) / 1e3)),
            "iters_per_pair": [r["iters_total"] / r["n_pair"] for r in recs],
            "guess_ms": [r["guess_ms"] for r in recs], "total_ms": [r["total_ms"] for r in recs],
            "dE_subset_per_orbital": drift, "n_pair": [r["n_pair"] for r in recs]}
    if os.environ.get("EXX_MD_OUT"):
        with open(os.environ["EXX_MD_OUT"], "w") as f:
            json.dump(summary, f, indent=1)
    # the previous step's potential starts every later step closer than zero
    z = summary["arms"]["zero"]["iters_per_pair"]
    p = summary["arms"]["previous"]["iters_per_pair"]
    assert all(p[s] < 0.99 * z[s] for s in range(1, steps))
