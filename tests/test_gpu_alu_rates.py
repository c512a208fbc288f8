"""The GPU's arithmetic-unit rates (tests/native/alu_rates.cu): the FP64 FMA
rate is the peak the bench reports the FP64-bound orthogonalisation passes
against, so it is measured here and must stay close to the figure the bench
uses.  Prints the measured JSON (pytest -s)."""
import json
import os
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_alu_rates():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "alu_rates")
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-o", exe,
                        os.path.join(HERE, "native", "alu_rates.cu")], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    r = json.loads(out)
    print(out)
    # FP32 and FP64 pipes as this design assumes them: FP64 about 1/70 of FP32
    assert r["fp32_fma_per_s"] > 30 * r["fp64_fma_per_s"]
    assert 0.8 < r["fp64_fma_per_s"] / bench.FP64_FMA_PER_S < 1.25
