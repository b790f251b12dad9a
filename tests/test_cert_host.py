"""The float32 certificate that lets the FP32-mixed Euler limiter skip the
float64 Appendix-A formula where the factor is certainly 1 must never
certify a node whose float64 factor differs from 1 (host build of the same
device code with nvcc; no GPU needed)."""
import json
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_certificate_never_wrong(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "cert_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-o", exe, os.path.join(HERE, "native", "cert_check.cu")],
                   check=True, capture_output=True)
    r = subprocess.run([exe, "1000000"], capture_output=True, text=True)
    out = json.loads(r.stdout)
    assert r.returncode == 0 and out["wrong"] == 0, (out, r.stderr)
    # not trivially false: most random contributions are certified, and
    # near-ties are mostly left to float64
    assert out["certified"] > 0.3 * out["trials"], out
    assert out["near"] > 0.1 * out["trials"], out
