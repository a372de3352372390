"""Host audit of the fused kernels' index arithmetic (no GPU; in place of a device-side bounds
checker, which this pool does not run).

tests/native/index_audit.cu includes the kernel headers and, for every supported grid side and
every pencil layout the launchers can choose, checks on the host that each shared-memory,
stage-buffer, pencil-blocked and Tensor Memory index the kernels form stays inside its buffer,
that each transform stage addresses every grid cell exactly once (also in the bank-spread X
order, which must be a permutation with distinct banks per half-warp group), that the
pencil-blocked layout the kernels read is the one the relayout kernel writes, and that the
barriers the kernels leave out (x-slab named barriers at 24^3, warp-local planes at 8^3 and
16^3) separate only data the same threads wrote.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_kernel_indices_stay_in_bounds_and_cover_the_grid(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "index_audit")
    src = os.path.join(HERE, "native", "index_audit.cu")
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O1", "-diag-suppress", "177,1886", "-x", "cu",
                    src, "-o", exe], check=True, capture_output=True, text=True)
    res = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    print(res.stdout)
    assert res.returncode == 0, res.stdout
    assert res.stdout.strip().endswith("index audit ok")
    # every side was audited, and the 24^3 one-pencil layout's slab groups were checked
    for n in (4, 6, 8, 10, 12, 16, 18, 20, 24):
        assert f"n={n} stages:" in res.stdout
    assert "n=24 PPT=1 TS=576: 6 slab groups of 96 threads are closed under Z <-> Y" in res.stdout
