"""Writes the stored expected values of the full-size parity tests, computed by the FP64 oracle:

* tests/golden/sweep2d_ceff.json -- C_eff of the 2D resolution sweep (centred disk of volume
  fraction 0.2; n in {45, 135, 405, 1215}; contrasts 10 and 0.1; no filter, Voigt, Reuss, 2-layer
  with radius 1 pixel and a 16x16 subgrid; c0 = mean Lamé constants; 3 unit Mandel loads) to an
  equilibrium error e < 1e-10 (section 2 criterion);
* tests/golden/spheres3d_ceff.json (--case 3d) -- C_eff of the 81^3 and 135^3 random-sphere cells
  (seed 1000 + n, radii U[0.05, 0.1], volume fraction 0.3, surface gap 1/243 of the cell, contrasts
  10 and 0.1, 2-layer filter of radius 1 pixel on an 8x8x8 subgrid, 6 unit Mandel loads) to e < 1e-9.

Only the oracle is called.  Usage: python tests/golden/make_golden.py [--case 2d|3d] [--sizes ..] [--jobs 8]
(--case 3d --sizes 135 adds the 135^3 cells and keeps the entries already stored.)
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import hom_inputs as H  # noqa: E402
import oracle as O  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sweep2d_ceff.json")
OUT3D = os.path.join(os.path.dirname(os.path.abspath(__file__)), "spheres3d_ceff.json")
TOL = 1e-10
TOL3D = 1e-9


def one(args):
    n, contrast, rule = args
    t = time.time()
    phases = H.two_phases(contrast)
    cell = H.centred_disk_cell(n, vf=0.2, rule=rule, radius_px=1.0, subgrid=16)
    fb = O.filter_build(cell, phases)
    lam0, mu0 = O.default_reference(phases)
    r = O.solve(fb["ctilde"], 2, n, lam0, mu0, np.eye(3), tol=TOL, max_iter=5000, criterion=O.CRIT_E)
    C = O.effective_stiffness(r["mean_sigma"], np.eye(3))
    return dict(n=n, contrast=contrast, rule=H.RULE_NAMES[rule], ceff=C.tolist(),
                iterations=[int(i) for i in r["iterations"]], status=r["status"], tol=TOL,
                seconds=time.time() - t)


def sphere_cell(n):
    return H.rsa_spheres_cell(n, seed=1000 + n, vf=0.3, rmin=0.05, rmax=0.1, rule=H.RULE_TWO_LAYER,
                              radius_px=1.0, subgrid=8, gap_voxels=n / 243.0)


def filter3d(args):
    """Oracle filter build of one sphere cell, written to a scratch .npy for the solves."""
    n, contrast, path = args
    t = time.time()
    fb = O.filter_build(sphere_cell(n), H.two_phases(contrast))
    np.save(path, fb["ctilde"])
    return n, contrast, time.time() - t


def one3d(args):
    n, contrast, load, path = args
    t = time.time()
    phases = H.two_phases(contrast)
    ctilde = np.load(path)
    lam0, mu0 = O.default_reference(phases)
    E = np.eye(6)[load:load + 1]
    r = O.solve(ctilde, 3, n, lam0, mu0, E, tol=TOL3D, max_iter=5000, criterion=O.CRIT_E)
    return dict(n=n, contrast=contrast, load=load, mean_sigma=r["mean_sigma"][0].tolist(),
                iterations=int(r["iterations"][0]), status=r["status"][0], seconds=time.time() - t)


def main3d(sizes, jobs):
    import tempfile
    tmp = tempfile.mkdtemp(prefix="hom_golden3d_")
    contrasts = (10.0, 0.1)
    paths = {(n, c): os.path.join(tmp, "ctilde_%d_%g.npy" % (n, c)) for n in sizes for c in contrasts}
    with mp.get_context("spawn").Pool(jobs) as pool:
        for n, c, sec in pool.imap_unordered(filter3d, [(n, c, paths[(n, c)]) for n in sizes for c in contrasts]):
            print("filter 3d", n, c, "%.0fs" % sec, flush=True)
        res = {}
        tasks = [(n, c, l, paths[(n, c)]) for n in sizes for c in contrasts for l in range(6)]
        for r in pool.imap_unordered(one3d, tasks):
            res[(r["n"], r["contrast"], r["load"])] = r
            print("done 3d", r["n"], r["contrast"], r["load"], r["iterations"], "%.0fs" % r["seconds"], flush=True)
    for p in paths.values():
        os.remove(p)
    os.rmdir(tmp)
    old = []
    if os.path.exists(OUT3D):
        old = [e for e in json.load(open(OUT3D))["cells"] if e["n"] not in sizes]
    cells = list(old)
    for n in sizes:
        for c in contrasts:
            S = np.array([res[(n, c, l)]["mean_sigma"] for l in range(6)])
            cells.append(dict(n=n, contrast=c, seed=1000 + n, ceff=O.effective_stiffness(S, np.eye(6)).tolist(),
                              iterations=[res[(n, c, l)]["iterations"] for l in range(6)], tol=TOL3D))
    cells.sort(key=lambda e: (e["n"], -e["contrast"]))
    json.dump({"description": "C_eff of random-sphere cells (make_golden.py --case 3d)", "cells": cells},
              open(OUT3D, "w"), indent=1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="2d", choices=["2d", "3d"])
    ap.add_argument("--sizes", default=None, help="2d: 45,135,405,1215 (default); 3d: 81 (default)")
    ap.add_argument("--jobs", type=int, default=os.cpu_count())
    a = ap.parse_args()
    if a.case == "3d":
        main3d([int(s) for s in (a.sizes or "81").split(",")], a.jobs)
        return
    sizes = [int(s) for s in (a.sizes or "45,135,405,1215").split(",")]
    tasks = [(n, c, r) for n in sizes for c in (10.0, 0.1)
             for r in (H.RULE_NONE, H.RULE_VOIGT, H.RULE_REUSS, H.RULE_TWO_LAYER)]
    tasks.sort(key=lambda t: -t[0])
    old = {}
    if os.path.exists(OUT):
        for e in json.load(open(OUT))["cells"]:
            old[(e["n"], e["contrast"], e["rule"])] = e
    todo = [t for t in tasks if (t[0], t[1], H.RULE_NAMES[t[2]]) not in old]
    with mp.get_context("spawn").Pool(a.jobs) as pool:
        for res in pool.imap_unordered(one, todo):
            old[(res["n"], res["contrast"], res["rule"])] = res
            cells = sorted(old.values(), key=lambda e: (e["n"], -e["contrast"], e["rule"]))
            json.dump({"description": __doc__.strip().splitlines()[0], "tol": TOL, "cells": cells},
                      open(OUT, "w"), indent=1)
            print("done", res["n"], res["contrast"], res["rule"], "%.0fs" % res["seconds"], flush=True)


if __name__ == "__main__":
    main()
