"""The generic mixed-radix FFT (radices 2 ... 49, primes 11 and 13) run on the host: every supported
length from 3 to 2187 (odd and even), DIF and DIT, forward and inverse, several thread schedules, against a
long-double DFT at sampled bins.  Needs nvcc (compiles tests/fft_host_check.cu as host code); no GPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("fft") / "fft_host_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"), "-o", exe,
                    os.path.join(HERE, "fft_host_check.cu")], check=True, capture_output=True)
    return exe


@pytest.mark.parametrize("max_radix", [15, 27, 45])
@pytest.mark.parametrize("lo,hi", [(3, 255), (257, 1023), (1025, 2187)])
def test_generic_fft_every_length(checker, lo, hi, max_radix):
    """max_radix as the kernels use it: FP64 plans up to radix 15, FP32 up to 27 (default) or 45."""
    out = subprocess.run([checker, str(lo), str(hi), str(max_radix)], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout[-2000:]
    assert out.stdout.strip().endswith("ok")
