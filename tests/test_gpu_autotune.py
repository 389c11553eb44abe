"""The FFT-plan autotuner (hom_solve_opts.tune): the first FP32 solve of a batch shape times the
candidate plans on that batch and keeps the fastest; every later solve of the shape runs it.  The
choice changes FP32 rounding only: results stay within the FP32 bar of the untuned solve, and
repeated solves of the shape give identical results."""
import numpy as np
import pytest
import torch

import hom_inputs as H

pytestmark = pytest.mark.gpu

hom = pytest.importorskip("paper_1412_3228_gb300")


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_3228_gb300 import _build_lib
    _build_lib.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("sizes", [(45, 135, 135), (45, 33, 75)], ids=["specialised-sizes", "with-generic-only-size"])
def test_autotuned_solve(sizes):
    phases, cells = [], []
    for i, n in enumerate(sizes):
        cells.append(H.remap_phases(H.centred_disk_cell(n, rule=(H.RULE_VOIGT, H.RULE_TWO_LAYER, H.RULE_REUSS)[i]),
                                    len(phases)))
        phases.extend(H.two_phases((10.0, 0.1, 5.0)[i]))
    c0 = [H.mean_lame(phases[2 * i:2 * i + 2]) for i in range(len(cells))]
    mat = hom.hom_filter_build(cells, phases)
    kw = dict(precision=hom.HOM_FP32, criterion=hom.HOM_CRIT_EN, tol=1e-6, max_iter=3000)
    ref = hom.hom_solve(mat, np.eye(3), c0, **kw)
    a = hom.hom_solve(mat, np.eye(3), c0, tune=True, **kw)
    b = hom.hom_solve(mat, np.eye(3), c0, tune=True, **kw)
    report = hom.hom_autotune_report()
    key = " ".join("%dx%d" % (n, sizes.count(n)) for n in sorted(set(sizes)))
    line = [ln for ln in report.splitlines() if ln.split(":")[0].endswith(key)]
    assert len(line) == 1, report
    assert line[0].count(" ms") == 4 and "->" in line[0]
    assert (a["status"] == 0).all()
    Ca = hom.hom_effective_stiffness(np.eye(3), a["mean_sigma"], 2)
    Cr = hom.hom_effective_stiffness(np.eye(3), ref["mean_sigma"], 2)
    assert float(np.abs(Ca - Cr).max() / np.abs(Cr).max()) < 1e-5
    np.testing.assert_array_equal(a["mean_sigma"], b["mean_sigma"])
    assert torch.equal(a["eps"].cpu(), b["eps"].cpu())
