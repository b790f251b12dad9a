"""The compact float sin/cos that the FP32-mixed KPP flux inlines at every
quadrature point (Cody-Waite reduction by pi/2 and fitted polynomials)
must stay within 1.2e-7 of float64 sin and cos, on a dense sweep of
[-200, 200], on the KPP range and on the wide-argument fallback (host build of
the same device function with nvcc; no GPU needed)."""
import json
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_kpp_sincos_accuracy(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "kpp_sincos_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-o", exe, os.path.join(HERE, "native", "kpp_sincos_check.cu")],
                   check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True, check=True)
    out = json.loads(r.stdout)
    assert out["points"] > 1000000
    assert out["max_abs_err"] <= 1.2e-7, out
    assert out["max_abs_err_kpp_range"] <= 1.2e-7, out
    assert out["max_abs_err_wide"] <= 1.2e-7, out
