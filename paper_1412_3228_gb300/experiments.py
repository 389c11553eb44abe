"""Drivers for the paper's numerical experiment (section 3, Fig. 1) on the hot path.

* `axial_stress_sweep` - spatial convergence study: the average axial stress <sigma_11> of the
  centred-disk cell under a uniaxial mean strain, for every (filter rule, filter radius, grid
  size), computed as ONE batched filter build and ONE batched solve (every cell of every rule and
  radius in the same launch sequence).
* `n_within` - N_1%: the smallest resolution from which every larger resolution of the study
  stays within a relative tolerance (1 %) of the converged value.
* `n1pct_vs_radius` - N_1% as a function of the filter radius, per rule (Fig. 1-B and D).
* `iteration_sweep` - section 5, Fig. 3: iterations at convergence against the elastic contrast
  (reference medium at the optimal choice) and against the scale alpha of the reference medium
  (fixed contrast), per filter radius, each as ONE batched solve.
* `extrapolation_study` - section 6, Fig. 4: the truncated Fourier series of c~_11 on a finer grid,
  per filter radius, with its overshoot beyond the phase range and its L2 gap to a point-sampled
  exact microstructure supplied by the caller.

Grid sizes factor into 2, 3, 5, 7, 11 and 13.  The frequency set J of section 2 is defined for odd N;
even N (the paper's sweep includes them) take the library's Nyquist convention (zero strain at
wave vectors with a Nyquist component).  The converged value is the unfiltered stress at a large resolution `n_ref` (the
filters' pixel-sized smoothing vanishes as the grid is refined, so every rule converges to it).

    python -m paper_1412_3228_gb300.experiments --contrast 1000 --sizes 9,15,21,25,27,35,45,63,75,81,105,125
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
from typing import Dict, Iterable, List, Optional, Sequence

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

import hom_inputs as H  # noqa: E402

RULES = {"none": H.RULE_NONE, "voigt": H.RULE_VOIGT, "reuss": H.RULE_REUSS, "2-layers": H.RULE_TWO_LAYER}


def n_within(sizes: Sequence[int], values: Sequence[float], reference: float, rel: float = 0.01) -> Optional[int]:
    """Smallest n of `sizes` such that |v(n') - reference| <= rel |reference| for every n' >= n in
    the study (None if even the largest size misses the band)."""
    order = np.argsort(np.asarray(sizes))
    s = np.asarray(sizes)[order]
    v = np.asarray(values, dtype=np.float64)[order]
    ok = np.abs(v - reference) <= rel * abs(reference)
    if not ok[-1]:
        return None
    i = len(s) - 1
    while i > 0 and ok[i - 1]:
        i -= 1
    return int(s[i])


def axial_stress_sweep(sizes: Iterable[int], contrast: float, rules: Iterable[str] = ("none", "voigt", "2-layers"),
                       radii: Iterable[float] = (0.55, 1.0), vf: float = 0.2, subgrid: int = 16,
                       precision: Optional[int] = None, criterion: Optional[int] = None, tol: float = 1e-4,
                       max_iter: int = 100000, n_ref: Optional[int] = None, device=None) -> Dict:
    """<sigma_11> of the centred disk (volume fraction vf) under E = (1, 0, 0) for every rule x radius
    x size, in one batched filter build and solve.  Returns a dict with the records, the converged
    reference (unfiltered value at n_ref, if given) and the solver status of every cell."""
    import paper_1412_3228_gb300 as hom
    precision = hom.HOM_FP64 if precision is None else precision
    criterion = hom.HOM_CRIT_E if criterion is None else criterion
    sizes = [int(n) for n in sizes]
    for n in sizes + ([n_ref] if n_ref else []):
        if not _factors_supported(n):
            raise ValueError("grid size %d must factor into 2, 3, 5, 7, 11, 13" % n)
    phases = H.two_phases(contrast)
    cells, keys = [], []
    for rule in rules:
        radius_list = [1.0] if rule == "none" else list(radii)
        for r in radius_list:
            for n in sizes:
                cells.append(H.centred_disk_cell(n, vf=vf, rule=RULES[rule], radius_px=r, subgrid=subgrid))
                keys.append((rule, r, n))
    if n_ref:
        cells.append(H.centred_disk_cell(n_ref, vf=vf, rule=H.RULE_NONE, subgrid=subgrid))
        keys.append(("reference", 0.0, n_ref))
    c0 = [H.mean_lame(phases)] * len(cells)
    mat = hom.hom_filter_build(cells, phases, device=device)
    res = hom.hom_solve(mat, np.array([[1.0, 0.0, 0.0]]), c0, precision=precision, criterion=criterion, tol=tol,
                        max_iter=max_iter, fields=False)
    records = []
    ref = None
    for i, (rule, r, n) in enumerate(keys):
        s11 = float(res["mean_sigma"][i, 0, 0])
        if rule == "reference":
            ref = s11
            continue
        records.append(dict(rule=rule, radius_px=r, n=n, sigma11=s11, iterations=int(res["iterations"][i, 0]),
                            status=int(res["status"][i, 0])))
    return dict(contrast=contrast, vf=vf, subgrid=subgrid, tol=tol, reference=ref, n_ref=n_ref, records=records)


def n1pct_vs_radius(study: Dict, rel: float = 0.01, reference: Optional[float] = None) -> List[Dict]:
    """N_1% of every (rule, radius) curve of `axial_stress_sweep` (Fig. 1-B and D)."""
    ref = study["reference"] if reference is None else reference
    if ref is None:
        raise ValueError("no converged reference: pass n_ref to axial_stress_sweep or a reference value")
    curves: Dict = {}
    for rec in study["records"]:
        curves.setdefault((rec["rule"], rec["radius_px"]), []).append((rec["n"], rec["sigma11"]))
    out = []
    for (rule, r), pts in sorted(curves.items()):
        pts.sort()
        out.append(dict(rule=rule, radius_px=r, n_1pct=n_within([p[0] for p in pts], [p[1] for p in pts], ref, rel)))
    return out


def iteration_sweep(n: int = 65, contrasts: Sequence[float] = (1e-3, 1e-2, 0.1, 10.0, 100.0, 1e3),
                    alphas: Sequence[float] = (0.9, 1.0, 1.25, 1.5, 2.0, 3.0), alpha_contrast: float = 1e3,
                    radii: Sequence[float] = (0.55, 1.0, 1.5), rule: str = "2-layers", radius: float = math.pi / 15,
                    subgrid: int = 16, tol: float = 1e-4, max_iter: int = 20000, diverge_window: int = 50,
                    precision: Optional[int] = None, criterion: Optional[int] = None, device=None) -> Dict:
    """Iterations of the basic scheme at convergence (section 5, Fig. 3) on the centred disk.

    A radius of 0 stands for the unfiltered cell.  Part A: one cell per (radius, contrast) with the
    reference medium at the optimal choice
    (lam0, mu0) = mid-range of the phase constants.  Part B: one cell per (radius, alpha) at contrast
    `alpha_contrast` with the reference medium alpha * (lam0, mu0).  Each part is one filter build and
    one solve over all its cells (every cell carries its own phase pair and reference medium).  A
    record's status is 0 when the equilibrium error fell below `tol`, 1 at max_iter, 2 on
    divergence (non-finite error, or `diverge_window` successive increases)."""
    import paper_1412_3228_gb300 as hom
    precision = hom.HOM_FP64 if precision is None else precision
    criterion = hom.HOM_CRIT_E if criterion is None else criterion
    if not _factors_supported(n):
        raise ValueError("grid size %d must factor into 2, 3, 5, 7, 11, 13" % n)

    def run(keys):
        cells, phases, c0 = [], [], []
        for r, contrast, alpha in keys:
            cell = H.centred_disk_cell(n, rule=RULES[rule] if r else H.RULE_NONE, radius_px=r if r else 1.0,
                                       subgrid=subgrid, radius=radius)
            cells.append(H.remap_phases(cell, len(phases)))
            pair = H.two_phases(contrast)
            phases.extend(pair)
            lam0, mu0 = H.mean_lame(pair)
            c0.append((alpha * lam0, alpha * mu0))
        mat = hom.hom_filter_build(cells, phases, device=device)
        res = hom.hom_solve(mat, np.array([[1.0, 0.0, 0.0]]), c0, precision=precision, criterion=criterion,
                            tol=tol, max_iter=max_iter, diverge_window=diverge_window, fields=False)
        return [dict(radius_px=r, contrast=contrast, alpha=alpha, iterations=int(res["iterations"][i, 0]),
                     status=int(res["status"][i, 0]), err=float(res["err"][i, 0]))
                for i, (r, contrast, alpha) in enumerate(keys)]

    part_a = run([(r, float(c), 1.0) for r in radii for c in contrasts])
    part_b = run([(r, float(alpha_contrast), float(a)) for r in radii for a in alphas])
    return dict(n=n, rule=rule, tol=tol, vs_contrast=part_a, vs_alpha=part_b)


def extrapolation_study(n: int = 65, m: int = 325, radii: Sequence[float] = (0.0, 0.3, 0.55, 1.0, 1.5),
                        rule: str = "voigt", contrast: float = 1e-3, radius: float = math.pi / 15, subgrid: int = 16,
                        exact: Optional[np.ndarray] = None, device=None) -> Dict:
    """Fourier extrapolation of c~_11 (section 6, Fig. 4) for each filter radius (0 = no filter), all
    cells in one filter build.  Returns the fine-grid fields and, per radius, the overshoot of the
    extrapolation beyond the phase range (relative to the range) and, if `exact` (the m^2 exact
    property, e.g. point-sampled phases) is given, the relative L2 gap to it."""
    import paper_1412_3228_gb300 as hom
    phases = H.two_phases(contrast)
    vals = [lam + 2.0 * mu for lam, mu in phases]            # c_11 of each isotropic phase
    span = max(vals) - min(vals)
    cells = [H.centred_disk_cell(n, rule=RULES[rule] if r else H.RULE_NONE, radius_px=r if r else 1.0,
                                 subgrid=subgrid, radius=radius) for r in radii]
    mat = hom.hom_filter_build(cells, phases, device=device)
    records, fields = [], []
    for i, r in enumerate(radii):
        f = hom.hom_fourier_extrapolate(mat, i, m, 0)
        fields.append(f)
        fmax, fmin = float(f.max()), float(f.min())
        rec = dict(radius_px=float(r), overshoot=max(fmax - max(vals), min(vals) - fmin) / span)
        if exact is not None:
            d = f.cpu().numpy() - exact
            rec["l2_gap"] = float(np.sqrt(np.mean(d * d)) / span)
        records.append(rec)
    return dict(n=n, m=m, rule=rule, contrast=contrast, records=records, fields=fields)


def _factors_supported(n: int) -> bool:
    for p in (2, 3, 5, 7, 11, 13):
        while n % p == 0:
            n //= p
    return n == 1


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--contrast", type=float, default=1000.0)
    ap.add_argument("--sizes", default="9,15,21,25,27,35,45,63,75,81,105,125")
    ap.add_argument("--rules", default="none,voigt,2-layers")
    ap.add_argument("--radii", default="0.3,0.55,0.75,1.0,1.25,1.5")
    ap.add_argument("--n-ref", type=int, default=405)
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--fp32", action="store_true", help="FP32 fields (criterion e_n) instead of FP64")
    ap.add_argument("--study", choices=("resolution", "iterations"), default="resolution",
                    help="resolution: section 3, Fig. 1; iterations: section 5, Fig. 3")
    args = ap.parse_args(argv)
    import torch
    import paper_1412_3228_gb300 as hom
    from paper_1412_3228_gb300 import _build_lib
    _build_lib.build()
    torch.cuda.set_device(0)
    if args.study == "iterations":
        print(json.dumps(iteration_sweep(n=65, tol=args.tol, radii=[float(x) for x in args.radii.split(",")])))
        return
    study = axial_stress_sweep([int(x) for x in args.sizes.split(",")], args.contrast, args.rules.split(","),
                               [float(x) for x in args.radii.split(",")], tol=args.tol, n_ref=args.n_ref,
                               precision=hom.HOM_FP32 if args.fp32 else hom.HOM_FP64,
                               criterion=hom.HOM_CRIT_EN if args.fp32 else hom.HOM_CRIT_E)
    study["n_1pct"] = n1pct_vs_radius(study)
    print(json.dumps(study))


if __name__ == "__main__":
    main()
