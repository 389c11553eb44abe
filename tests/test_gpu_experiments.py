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
