"""The integer helpers of the uniform-grid location (csrc/dlm_device.cuh),
compiled for the host and checked without a GPU: the first-cell xi from the
bits of d against the FP64 arithmetic of the definition (2 t - 1, one
rounding), the exact double built from an integer and an exponent, and the
multiply-shift division of element indices against integer division.  The
GPU location tests compare the kernels with the oracle bit for bit; this pins
the three helpers on inputs the random points rarely reach (rounding ties,
subnormals, every exponent)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_location_bit_helpers(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = tmp_path / "locate_bits_check"
    src = os.path.join(ROOT, "tests", "host", "locate_bits_check.cu")
    inc = [os.path.join(ROOT, "paper_2601_08266_gb300", "csrc"), os.path.join(ROOT, "include")]
    subprocess.run([nvcc, "-std=c++17", "-O2", "-diag-suppress", "1444", "-x", "cu",
                    *[f"-I{p}" for p in inc], src, "-o", str(exe)], check=True,
                   capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout
