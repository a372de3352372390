"""The register FFT of the CUDA path (csrc/fft_reg.cuh) against a direct DFT, on the host.

fft_reg.cuh is host/device code, so nvcc builds a host program that checks every supported
length (2..32, prime-factor and Cooley-Tukey paths, float and double, both directions)
against an O(N^2) DFT in long double.  No GPU is needed.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_register_fft_matches_direct_dft(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "fftchk")
    src = os.path.join(HERE, "native", "fft_reg_check.cu")
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O2", "-x", "cu", src, "-o", exe],
                   check=True, capture_output=True, text=True)
    res = subprocess.run([exe], capture_output=True, text=True)
    assert res.returncode == 0, res.stdout
    assert res.stdout.count(" ok") == 18
