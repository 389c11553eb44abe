"""Writes tests/golden/sweep2d_ceff.json: C_eff of the 2D resolution sweep (centred disk of
volume fraction 0.2; n in {45, 135, 405, 1215}; contrasts 10 and 0.1; no filter, Voigt, Reuss,
2-layer with radius 1 pixel and a 16x16 subgrid; c0 = mean Lamé constants; 3 unit Mandel loads)
computed by the FP64 oracle to an equilibrium error e < 1e-10 (section 2 criterion).

Only the oracle is called.  Usage: python tests/golden/make_golden.py [--sizes 45,135] [--jobs 8]
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
TOL = 1e-10


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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", default="45,135,405,1215")
    ap.add_argument("--jobs", type=int, default=os.cpu_count())
    a = ap.parse_args()
    sizes = [int(s) for s in a.sizes.split(",")]
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
