"""The FP64 pipe's measured throughput on the GPU (tests/fp64_pipe_probe.cu).

Two facts the FP64 kernels' design and roofline rest on:
* a warp instruction costs the pipe the same whatever number of its lanes is
  active, so lanes left idle by a schedule are lost throughput (the batched
  kernel's packing is measured by its lane fill);
* the sustained FMA rate, against which the pair kernel's FP64 instruction
  count sets its speed of light.
Run with -s to see the figures.
"""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    pytest.skip("nvcc not found")


def test_fp64_pipe_cost_is_per_warp_instruction(tmp_path):
    exe = tmp_path / "fp64_pipe_probe"
    subprocess.run([_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                    os.path.join(HERE, "fp64_pipe_probe.cu"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    rates = {}
    for ln in out.splitlines():
        f = ln.split()
        if f[0] == "k":
            rates[int(f[1])] = (float(f[5]), float(f[7]))
    print(out)
    full = rates[32][0]
    # the same warp-instruction rate for 32, 16, 8 and 1 active lanes
    for k, (winst, _) in rates.items():
        assert abs(winst / full - 1.0) < 0.05, (k, winst, full)
    # a full warp: the sustained FMA rate (two flops each), in TFLOP/s
    print("FP64 FMA peak %.3f TFLOP/s" % (2.0 * rates[32][1] / 1e12))
    assert rates[32][1] > 0
