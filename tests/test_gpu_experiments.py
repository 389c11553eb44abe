"""GPU test of the resolution-study driver (section 3, Fig. 1): with a compliant inclusion
(contrast 1e-3) the Voigt filter of radius 0.55 pixel reaches the 1 % band of the converged axial
stress at a much smaller resolution than the unfiltered cell (the paper reports factors of 2.6 to
7.2 for its disk; this cell's disk has volume fraction 0.2)."""
import pytest
import torch

pytestmark = pytest.mark.gpu

hom = pytest.importorskip("paper_1412_3228_gb300")
from paper_1412_3228_gb300 import experiments as X  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_3228_gb300 import _build_lib
    _build_lib.build()
    torch.cuda.set_device(0)


def test_voigt_filter_divides_the_required_resolution_for_a_compliant_inclusion():
    study = X.axial_stress_sweep([9, 15, 21, 25, 27, 35, 45, 63, 75, 81, 105, 125], 1e-3, ("none", "voigt"),
                                 (0.55, 1.0), tol=1e-4, n_ref=405)
    assert all(r["status"] == 0 for r in study["records"])
    n1 = {(r["rule"], r["radius_px"]): r["n_1pct"] for r in X.n1pct_vs_radius(study)}
    assert n1[("voigt", 0.55)] is not None and n1[("none", 1.0)] is not None
    assert 2 * n1[("voigt", 0.55)] <= n1[("none", 1.0)]
    # the larger radius needs more resolution than the near-optimal 0.55 (section 3)
    assert n1[("voigt", 1.0)] >= n1[("voigt", 0.55)]


def test_iteration_counts_against_contrast_and_reference_medium():
    """Section 5, Fig. 3 (65^2): filtering neither helps nor hurts the basic scheme's iteration count
    (the curves of radii 0.55, 1.0 and 1.5 and of the unfiltered cell stay within a factor 1.5 of each
    other while the count itself spans orders of magnitude, so they coincide on a log axis); the count grows
    with the contrast on both sides of 1; below the optimal reference medium (alpha < 1) the scheme
    does not converge; far above it the count grows with alpha (here 1.5 -> 3; the paper states no
    monotonicity right above the optimum, where the count measured at 1.25 is below the one at 1)."""
    radii = (0.0, 0.55, 1.0, 1.5)
    sweep = X.iteration_sweep(n=65, contrasts=(1e-3, 0.1, 10.0, 1e3), alphas=(0.9, 1.0, 1.5, 3.0), radii=radii)
    a = {(r["radius_px"], r["contrast"]): r for r in sweep["vs_contrast"]}
    assert all(r["status"] == 0 for r in sweep["vs_contrast"]), sweep["vs_contrast"]
    for c in (1e-3, 0.1, 10.0, 1e3):
        its = [a[(r, c)]["iterations"] for r in radii]
        assert max(its) <= 1.5 * min(its), (c, its)    # within 0.18 decade on a log axis
    for r in radii:
        assert a[(r, 1e3)]["iterations"] > 2 * a[(r, 10.0)]["iterations"]
        assert a[(r, 1e-3)]["iterations"] > 2 * a[(r, 0.1)]["iterations"]
    b = {(r["radius_px"], r["alpha"]): r for r in sweep["vs_alpha"]}
    for r in radii:
        assert b[(r, 0.9)]["status"] != 0, b[(r, 0.9)]
        assert all(b[(r, al)]["status"] == 0 for al in (1.0, 1.5, 3.0))
        assert b[(r, 1.5)]["iterations"] < b[(r, 3.0)]["iterations"]
    for al in (1.0, 1.5, 3.0):
        its = [b[(r, al)]["iterations"] for r in radii]
        assert max(its) <= 1.5 * min(its), (al, its)
