"""Host-only checks of the kernels' per-site arithmetic (no GPU): the header with
the densities, forces and energy differences compiles for the host too, and a small
nvcc-built program checks that the cancellation-free energy differences used by the
arrest test equal e(a) - e(a - delta) of the kernels' own density functions
evaluated in higher precision."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "device_math_check.cu")
EXE = os.path.join(ROOT, "_build", "device_math_check")


@pytest.fixture(scope="module")
def results():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    os.makedirs(os.path.dirname(EXE), exist_ok=True)
    subprocess.run([nvcc, "-O2", "-std=c++17", "-diag-suppress", "20208", "-x", "cu", SRC, "-o", EXE], check=True,
                   capture_output=True)
    out = subprocess.run([EXE], check=True, capture_output=True, text=True).stdout
    return {k: float(v) for k, v in (line.split() for line in out.strip().splitlines())}


def test_energy_difference_is_exact_algebra_in_fp64(results):
    # a wrong term would leave O(1) relative errors; exact algebra leaves rounding only
    for name, err in results.items():
        if "_f64_" in name:
            assert err < 1e-7, (name, err)


def test_energy_difference_error_scales_with_the_difference_in_fp32(results):
    # relative to the difference itself, even for delta = 1e-6 where a direct FP32
    # difference of the two energies would carry ~6e-8 |e| / |de| ~ 1e-1 relative error
    for name, err in results.items():
        if "_f32_" in name:
            assert err < 1e-2, (name, err)
