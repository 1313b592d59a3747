"""Convergence of E_xx and D_xx with the pair cutoff and the subdomain radii.

Reproduces, on the synthetic water-64-form workload, the structure of the
paper's accuracy study (Sec. IV: E_xx against R_pair, the self R_PE and the
non-self R_PE with every other parameter at its largest value; the force
metric gamma_xx of Eqs. gammaxx_i / gammaxx against the self and non-self
R_ME with the PE radii at their defaults). Radii are in grid points.

E_xx sweeps need few solves: a run's per-pair energies split into the self
and the non-self sums, and each sum depends only on its own radius, so
E_xx(R_pe_self, R_pe_nonself) = E_self(R_pe_self) + E_nonself(R_pe_nonself);
the R_pair sweep re-sums the reference run's pairs closer than R_pair.

    python -m paper_1911_10630_gb300.radius_sweep --orbitals 64
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import synth
from .exx import Exx


def _minimg_dist(ci, cj, cell):
    d = cj - ci
    d -= cell * np.floor(d / cell + 0.5)
    return np.sqrt(np.sum(d * d, axis=-1))


def _run(w, phi, cen, D, r_pair, r_pe, r_me, tol, **opts):
    ex = Exx(w.cell, w.grid, r_pair, r_pe, r_me, w.l_max, tol, precision=1, **opts)
    e = ex.compute(phi, cen, D)
    pairs = ex.pairs()
    st = ex.stats()
    ex.close()
    m = np.where(pairs["i"] == pairs["j"], 1.0, 2.0)
    self_ = pairs["i"] == pairs["j"]
    return dict(E=e, pairs=pairs, e_self=-float(np.sum((m * pairs["e_pair"])[self_])),
                e_nonself=-float(np.sum((m * pairs["e_pair"])[~self_])), nonconv=st["n_nonconv"])


def gamma_xx(D, Dref):
    """Eqs. gammaxx_i, gammaxx: mean over orbitals of the relative L1 error."""
    num = (D - Dref).abs().sum(dim=(1, 2, 3))
    den = Dref.abs().sum(dim=(1, 2, 3))
    return float((num / den).mean())


def sweep(n_orbitals=64, r_ref=40, shell=12, tol=1e-11, pe_radii=(12, 16, 20, 24, 28, 32),
          default_self=(31, 51), default_nonself=(26, 36), me_self=(36, 40, 44, 48, 52),
          me_nonself=(29, 32, 36, 40, 44, 48), log=print):
    """Runs the sweeps; radii in grid points. The defaults mirror the paper's
    R_PE 6.0 / 5.0 bohr and R_ME 10.0 / 7.0 bohr (self / non-self) on the
    0.196-bohr grid, with the reference radii r_ref / r_ref + shell."""
    import torch
    w = synth.config1()
    w.centers, w.alphas, w.pvecs = w.centers[:n_orbitals], w.alphas[:n_orbitals], w.pvecs[:n_orbitals]
    phi = synth.orbitals_torch(w)
    cen = torch.from_numpy(np.ascontiguousarray(w.centers)).cuda()
    D = torch.empty_like(phi)
    half = 0.5 * float(np.min(w.cell)) - 1e-6
    out = {"workload": f"{w.name} (first {n_orbitals} orbitals)", "delta_bohr": float(w.delta[0]),
           "r_ref": r_ref, "shell": shell, "tol": tol}
    # reference: every pair within L/2, all radii at r_ref
    ref = _run(w, phi, cen, D, half, r_ref, r_ref + shell, tol)
    e_ref = ref["E"]
    out["E_ref"] = e_ref
    out["self_share"] = ref["e_self"] / e_ref
    log(f"reference E_xx {e_ref:.10f}  self share {ref['e_self'] / e_ref:.3f}  pairs {len(ref['pairs']['i'])}")
    # R_pair: re-sum the reference pairs closer than R_pair
    p = ref["pairs"]
    dist = _minimg_dist(w.centers[p["i"]], w.centers[p["j"]], w.cell)
    m = np.where(p["i"] == p["j"], 1.0, 2.0)
    rows = []
    for rp in (2.0, 3.0, 4.0, 5.0, 6.0, 8.0, 10.0):
        e = -float(np.sum((m * p["e_pair"])[dist < rp]))
        rows.append({"r_pair_bohr": rp, "rel_err": abs(e - e_ref) / abs(e_ref)})
    out["r_pair"] = rows
    # self and non-self R_PE
    runs = {}
    for r in pe_radii:
        runs[r] = _run(w, phi, cen, D, half, r, r + shell, tol)
        log(f"R_PE {r}: E_self {runs[r]['e_self']:.10f} E_nonself {runs[r]['e_nonself']:.10f}")
    out["r_pe_self"] = [{"r_pe": r, "r_pe_bohr": r * float(w.delta[0]),
                         "rel_err": abs(runs[r]["e_self"] + ref["e_nonself"] - e_ref) / abs(e_ref)} for r in pe_radii]
    out["r_pe_nonself"] = [{"r_pe": r, "r_pe_bohr": r * float(w.delta[0]),
                            "rel_err": abs(ref["e_self"] + runs[r]["e_nonself"] - e_ref) / abs(e_ref)}
                           for r in pe_radii]
    # gamma_xx against R_ME with the PE radii at their defaults (self and
    # non-self proto-subdomains, R_pair 8 bohr). The self sweep keeps the
    # non-self R_ME at its default and compares with self R_ME = r_ref + shell;
    # the non-self sweep keeps the self R_ME at r_ref + shell and compares with
    # non-self R_ME = r_ref + shell (the non-self ball never exceeds the self one).
    rs, ms = default_self
    rn, mn = default_nonself
    rme_max = r_ref + shell
    Dref = torch.empty_like(phi)
    _run(w, phi, cen, Dref, 8.0, rs, rme_max, tol, radii_mode=2, r_pe_nonself=rn, r_me_nonself=mn)
    gs = []
    for me in me_self:
        _run(w, phi, cen, D, 8.0, rs, me, tol, radii_mode=2, r_pe_nonself=rn, r_me_nonself=mn)
        gs.append({"r_me_self": me, "r_me_self_bohr": me * float(w.delta[0]), "gamma_xx": gamma_xx(D, Dref)})
    out["gamma_r_me_self"] = gs
    _run(w, phi, cen, Dref, 8.0, rs, rme_max, tol, radii_mode=2, r_pe_nonself=rn, r_me_nonself=rme_max)
    gn = []
    for me in me_nonself:
        _run(w, phi, cen, D, 8.0, rs, rme_max, tol, radii_mode=2, r_pe_nonself=rn, r_me_nonself=me)
        gn.append({"r_me_nonself": me, "r_me_nonself_bohr": me * float(w.delta[0]), "gamma_xx": gamma_xx(D, Dref)})
    out["gamma_r_me_nonself"] = gn
    # the paper-like defaults in this grid: R_pair 8 bohr, R_PE 31/26, R_ME 51/36
    dflt = _run(w, phi, cen, D, 8.0, rs, ms, tol, radii_mode=2, r_pe_nonself=rn, r_me_nonself=mn)
    out["defaults"] = {"r_pair_bohr": 8.0, "r_pe_self": rs, "r_me_self": ms, "r_pe_nonself": rn, "r_me_nonself": mn,
                       "rel_err_E": abs(dflt["E"] - e_ref) / abs(e_ref),
                       "gamma_xx_vs_max_r_me": gamma_xx(D, Dref)}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--orbitals", type=int, default=64)
    ap.add_argument("--r-ref", type=int, default=40)
    args = ap.parse_args()
    res = sweep(args.orbitals, args.r_ref)
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
