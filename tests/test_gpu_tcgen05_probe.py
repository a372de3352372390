"""Measured prototype of the tensor-core DFT on the fifth-generation tensor cores (tcgen05).

tests/native/tc5_dft_probe.cu transforms tiles of 128 pencils of 24 complex values (the unit
of work of the Y and X stages of the 24^3 kernel, Sec. II C) two ways: as one split-TF32 GEMM
per tile with tcgen05.mma (operands in shared memory, accumulator in Tensor Memory, three
products hi*hi + hi*lo + lo*hi) and with the register FFT of csrc/fft_reg.cuh.  Both are
checked against an FP64 DFT of sampled pencils (relative error below 1e-5); the printed times
per tile feed the comparison recorded in the design notes.
"""
import json
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_tcgen05_dft_prototype_matches_fp64_and_is_timed(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "tc5probe")
    src = os.path.join(HERE, "native", "tc5_dft_probe.cu")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "--expt-relaxed-constexpr",
                    src, "-o", exe], check=True, capture_output=True, text=True)
    res = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(res.stdout)
    lines = {d["mode"]: d for d in (json.loads(s) for s in res.stdout.strip().splitlines() if s.startswith("{"))}
    assert res.returncode == 0, res.stdout
    g, c = lines["global"], lines["on_chip"]
    assert g["status"] == 0 and c["status"] == 0
    # one transform against the FP64 DFT
    assert g["err_tc"] < 1e-5 and g["err_reg"] < 1e-5
    # 256 unitary transforms on chip bring the tile back ((F / sqrt 24)^4 = 1), within the
    # round-off of 256 transforms
    assert c["reps"] % 4 == 0 and c["back_tc"] < 1e-6 * c["reps"] and c["back_reg"] < 1e-6 * c["reps"]
