"""Full-size GPU parity of the 3D workloads (random-sphere cells of 135^3 and 243^3, 2-layer
filter, all 6 loads in one launch, in the launch configuration bench.py times).

* The specialised FP32 3D passes (compile-time plans for 135 = 15 x 9 and 243 = 3 x 9 x 9) against
  the generic passes on the same inputs, element by element after a fixed number of iterations:
  two independent FFT implementations of eqs. 1-2 must agree to FP32 rounding.
* C_eff of the 135^3 cells against the FP64 oracle's values stored in tests/golden (written by
  tests/golden/make_golden.py, which calls only the oracle).
* The filtered stiffness of sampled 135^3 voxels against the oracle's definitions, voxel by voxel."""
import json
import os

import numpy as np
import pytest
import torch

import hom_inputs as H
import oracle as O

pytestmark = pytest.mark.gpu

hom = pytest.importorskip("paper_1412_3228_gb300")
from gpu_helpers import dense_ctilde, unpack  # noqa: E402
from test_gpu_fullsize import _oracle_voxel_ctilde  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_3228_gb300 import _build_lib
    _build_lib.build()
    torch.cuda.set_device(0)


def _sphere_cell(n):
    return H.rsa_spheres_cell(n, seed=1000 + n, vf=0.3, rmin=0.05, rmax=0.1, rule=H.RULE_TWO_LAYER, radius_px=1.0,
                              subgrid=8, gap_voxels=n / 243.0)


def _dev_rel(a, b):
    """(L2, max) error of a against b, relative to b's RMS and largest magnitude (on the device)."""
    d = (a.double() - b.double())
    bb = b.double()
    return (float(d.pow(2).mean().sqrt() / bb.pow(2).mean().sqrt()), float(d.abs().max() / bb.abs().max()))


@pytest.mark.parametrize("n", [135, 243])
def test_specialised_and_generic_3d_agree_fixed_steps(n):
    """Five iterations from eps = E on both pass families (tol < 0: no early stop), contrast 10.
    The two FP32 transforms round differently, so the fields agree to FP32 accuracy, not bit for
    bit; the mean stresses (FP64 sums of FP32 products) agree to 1e-6."""
    cell = _sphere_cell(n)
    phases = H.two_phases(10.0)
    c0 = [H.mean_lame(phases)]
    E = np.eye(6)
    mat = hom.hom_filter_build([cell], phases)
    kw = dict(precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, tol=-1.0, max_iter=5)
    fast = hom.hom_solve(mat, E, c0, passes=hom.HOM_PASSES_AUTO, **kw)
    np.testing.assert_array_equal(fast["iterations"], 5)
    ef, sf, msf = fast["eps"], fast["sigma"], fast["mean_sigma"]
    del fast
    gen = hom.hom_solve(mat, E, c0, passes=hom.HOM_PASSES_GENERIC, **kw)
    np.testing.assert_array_equal(gen["iterations"], 5)
    assert float(np.abs(msf - gen["mean_sigma"]).max() / np.abs(gen["mean_sigma"]).max()) < 1e-6
    for got, want in ((ef, gen["eps"]), (sf, gen["sigma"])):
        l2, mx = _dev_rel(got, want)
        assert l2 < 2e-6 and mx < 2e-5, (l2, mx)


def _golden(n):
    p = os.path.join(GOLDEN, "spheres3d_ceff.json")
    gold = {}
    if os.path.exists(p):
        gold = {e["contrast"]: np.array(e["ceff"]) for e in json.load(open(p))["cells"] if e["n"] == n}
    if len(gold) < 2:
        pytest.skip("golden C_eff of the %d^3 cells not generated" % n)
    return gold


@pytest.mark.parametrize("precision,crit,tol,bar", [(1, 0, 1e-10, 1e-8), (0, 1, 1e-6, 1e-5)], ids=["fp64", "fp32"])
def test_spheres_135_ceff_matches_oracle(precision, crit, tol, bar):
    """135^3 random-sphere cells at contrasts 10 and 0.1, 6 loads each, in one call: FP64 (generic
    passes) within 1e-8 of the oracle's C_eff (converged to e < 1e-9), FP32 (specialised passes)
    within 1e-5."""
    gold = _golden(135)
    base = _sphere_cell(135)
    phases, cells = [], []
    for contrast in (10.0, 0.1):
        cells.append(H.remap_phases(base, len(phases)))
        phases.extend(H.two_phases(contrast))
    c0 = [H.mean_lame(phases[0:2]), H.mean_lame(phases[2:4])]
    mat = hom.hom_filter_build(cells, phases)
    r = hom.hom_solve(mat, np.eye(6), c0, precision=precision, criterion=crit, tol=tol, max_iter=3000, fields=False)
    assert (r["status"] == 0).all()
    C = hom.hom_effective_stiffness(np.eye(6), r["mean_sigma"], 3)
    for i, contrast in enumerate((10.0, 0.1)):
        g = gold[contrast]
        assert float(np.abs(C[i] - g).max() / np.abs(g).max()) < bar


def test_spheres_135_filter_sampled_voxels():
    cell = _sphere_cell(135)
    phases = H.two_phases(10.0)
    mat = hom.hom_filter_build([cell], phases)
    got, mixed = dense_ctilde(mat, 0)
    rng = np.random.default_rng(135)
    n = 135
    pick = np.concatenate([rng.choice(np.nonzero(mixed)[0], 25, replace=False), rng.integers(0, n ** 3, 25)])
    for v in pick:
        a = (v % n, (v // n) % n, v // (n * n))
        C, is_mixed = _oracle_voxel_ctilde(cell, phases, a)
        assert bool(mixed[v]) == is_mixed, v
        np.testing.assert_allclose(unpack(got[v], 6), C, rtol=0, atol=1e-12 * np.abs(C).max())
