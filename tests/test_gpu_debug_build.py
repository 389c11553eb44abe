"""GPU test of the bounds-checked build (-DHOM_DEBUG): every solver kernel checks its global
indices and task descriptors and poisons its dynamic shared memory with NaN before use.  The same
solves (specialised and generic passes, FP32 and FP64, 2D and 3D, odd and even grids, the
Eyre-Milton scheme, a warm start, conjugate gradients, the adjoint) run in a child process on the
debug library and here on the release library: the debug build must report no failed check
(HOM_ERR_BOUNDS) and no NaN, and give the release build's iteration counts and mean stresses."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

hom = pytest.importorskip("paper_1412_3228_gb300")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = r'''
import json, sys
import numpy as np, torch
import paper_1412_3228_gb300 as hom
import hom_inputs as H

def run():
    out = {}
    ph = H.two_phases(10.0)
    c0 = H.mean_lame(ph)
    def solve(name, cells, dim, **kw):
        mat = hom.hom_filter_build(cells, ph)
        nc = 3 if dim == 2 else 6
        kw.setdefault("c0", [c0] * len(cells))
        c = kw.pop("c0")
        r = hom.hom_solve(mat, np.eye(nc), c, criterion=hom.HOM_CRIT_EN, max_iter=400, **kw)
        f = r["eps"].double()
        out[name] = dict(it=r["iterations"].tolist(), ms=r["mean_sigma"].tolist(),
                         fsum=float(f.abs().sum()), fnan=bool(torch.isnan(f).any()))
        return mat, r
    disk = lambda n, rule=H.RULE_TWO_LAYER: H.centred_disk_cell(n, rule=rule)
    sph = lambda n: H.rsa_spheres_cell(n, seed=n, vf=0.12, rmin=0.12, rmax=0.16, subgrid=4, gap_voxels=0.5)
    solve("fast2d_fp32", [disk(45), disk(75, H.RULE_VOIGT)], 2, precision=hom.HOM_FP32, tol=1e-5)
    solve("fast3d_fp32", [sph(27)], 3, precision=hom.HOM_FP32, tol=1e-5)
    solve("generic2d_fp64", [disk(27), disk(16, H.RULE_REUSS)], 2, precision=hom.HOM_FP64, tol=1e-9)
    solve("generic3d_fp32", [sph(15)], 3, precision=hom.HOM_FP32, tol=1e-5, passes=hom.HOM_PASSES_GENERIC)
    solve("generic3d_fp64_even", [sph(10)], 3, precision=hom.HOM_FP64, tol=1e-9)
    solve("em_fp64", [disk(21)], 2, precision=hom.HOM_FP64, tol=1e-9, scheme=hom.HOM_SCHEME_EYRE_MILTON,
          c0=[H.geometric_lame(ph, 2)])
    solve("em_fp32_fast2d", [disk(45), disk(135, H.RULE_VOIGT)], 2, precision=hom.HOM_FP32, tol=1e-6,
          scheme=hom.HOM_SCHEME_EYRE_MILTON, c0=[H.geometric_lame(ph, 2)] * 2)
    solve("em_fp32_fast3d", [sph(27)], 3, precision=hom.HOM_FP32, tol=1e-6, scheme=hom.HOM_SCHEME_EYRE_MILTON,
          c0=[H.geometric_lame(ph, 3)])
    rng = np.random.default_rng(3)
    eps0 = torch.tensor(rng.standard_normal(3 * 3 * 21 * 21), dtype=torch.float64, device="cuda")
    solve("warm_fp64", [disk(21)], 2, precision=hom.HOM_FP64, tol=1e-9, eps0=eps0)
    mat = hom.hom_filter_build([disk(27)], ph)
    rc = hom.hom_solve_cg(mat, np.eye(3), precision=hom.HOM_FP64, tol=1e-9, max_iter=400)
    out["cg_fp64"] = dict(it=rc["iterations"].tolist(), ms=rc["mean_sigma"].tolist(), fsum=0.0, fnan=False)
    fwd = hom.hom_solve(mat, np.eye(3), [c0], precision=hom.HOM_FP64, criterion=hom.HOM_CRIT_E, tol=1e-10,
                        max_iter=2000)
    b = hom.hom_solve_backward(mat, fwd, [c0], dL_dC=np.eye(3)[None], precision=hom.HOM_FP64)
    out["backward"] = dict(it=[0], ms=np.asarray(b["dphase"]).tolist(), fsum=0.0, fnan=False)
    return out

if __name__ == "__main__":
    if sys.argv[1] == "debug":
        hom.use_debug_library()
        assert hom.lib().hom_build_flags() == 1
    torch.cuda.set_device(0)
    print(json.dumps(run()))
'''


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_3228_gb300 import _build_lib
    _build_lib.build()
    _build_lib.build(debug=True)


def _run(kind):
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CASES, kind], capture_output=True, text=True, cwd=ROOT, env=env,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_build_checks_pass_and_match_release():
    dbg = _run("debug")
    rel = _run("release")
    assert dbg.keys() == rel.keys()
    for k in rel:
        assert not dbg[k]["fnan"], k
        assert dbg[k]["it"] == rel[k]["it"], (k, dbg[k]["it"], rel[k]["it"])
        a, b = np.asarray(dbg[k]["ms"]), np.asarray(rel[k]["ms"])
        assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max(), k
        assert abs(dbg[k]["fsum"] - rel[k]["fsum"]) <= 1e-6 * max(rel[k]["fsum"], 1.0), k
