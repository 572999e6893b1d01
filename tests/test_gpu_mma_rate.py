"""Issue rate of the tcgen05 MMA shapes the kernels use (tests/gpu_mma_rate.cu, built with nvcc for
sm_103a): cycles per 128 x N x 16 bf16 MMA for N = 64, 128, 256.  N = 64 reads its operands from
shared memory at the full shared-memory rate and runs at two thirds of the bf16 rate, so the
exact-slice kernel issues one MMA per run of up to four slice levels whose 64-column TMEM accumulators
are adjacent (N up to 256); the split-bf16 kernel uses N = 256.  The measured figures are printed; the
test checks that every launch completed (no timeout, no CUDA error) and that the per-clock rate does
not fall as N grows."""
import os
import re
import shutil
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_mma_rate_by_width():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "mma_rate")
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-o", exe,
                        os.path.join(HERE, "gpu_mma_rate.cu")], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, timeout=120).stdout
    print(out)
    rates = {}
    for m in re.finditer(r"N=(\d+): (.+?) timeout=(\d)\s+([\d.]+) cycles per MMA.*?([\d.]+) flop/clk/SM", out):
        n, err, to, cyc, rate = int(m.group(1)), m.group(2), int(m.group(3)), float(m.group(4)), float(m.group(5))
        assert err == "no error" and to == 0
        rates[n] = rate
    assert set(rates) == {64, 128, 256}
    assert rates[64] <= rates[128] * 1.05 and rates[128] <= rates[256] * 1.05
