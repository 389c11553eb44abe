"""Drivers for the paper's numerical experiment (section 3, Fig. 1) on the hot path.

* `axial_stress_sweep` - spatial convergence study: the average axial stress <sigma_11> of the
  centred-disk cell under a uniaxial mean strain, for every (filter rule, filter radius, grid
  size), computed as ONE batched filter build and ONE batched solve (every cell of every rule and
  radius in the same launch sequence).
* `n_within` - N_1%: the smallest resolution from which every larger resolution of the study
  stays within a relative tolerance (1 %) of the converged value.
* `n1pct_vs_radius` - N_1% as a function of the filter radius, per rule (Fig. 1-B and D).

Grid sizes must be odd (the frequency set J of section 1 is defined for odd N) and factor into
3, 5 and 7.  The converged value is the unfiltered stress at a large resolution `n_ref` (the
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
        if n % 2 == 0 or not _factors_357(n):
            raise ValueError("grid size %d must be odd with factors 3, 5, 7" % n)
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


def _factors_357(n: int) -> bool:
    for p in (3, 5, 7):
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
    args = ap.parse_args(argv)
    import torch
    import paper_1412_3228_gb300 as hom
    from paper_1412_3228_gb300 import _build_lib
    _build_lib.build()
    torch.cuda.set_device(0)
    study = axial_stress_sweep([int(x) for x in args.sizes.split(",")], args.contrast, args.rules.split(","),
                               [float(x) for x in args.radii.split(",")], tol=args.tol, n_ref=args.n_ref,
                               precision=hom.HOM_FP32 if args.fp32 else hom.HOM_FP64,
                               criterion=hom.HOM_CRIT_EN if args.fp32 else hom.HOM_CRIT_E)
    study["n_1pct"] = n1pct_vs_radius(study)
    print(json.dumps(study))


if __name__ == "__main__":
    main()
