"""csrc/fp64_emu.cuh on the GPU (tests/fp64_emu_probe.cu): the integer-pipe
multiply (also with its first operand negated), add and fused multiply-add
that the FP64 pair kernels use in place
of part of their FP64 instructions, compared bit for bit with the GPU's own
FP64 instructions (__dmul_rn, __dadd_rn, __fma_rn) on 10 million cases of
each operand kind of tests/fp64_emu_cases.h (every class of double, typical
magnitudes, exact results and ties, boundary values, cancellation, results
next to the rounding's halfway point).  The same routines are checked on the
host against the host's IEEE arithmetic (tests/test_fp64_emu_host.py); this
test shows that the device build, with its fallback calls to the hardware
instructions, gives the GPU's results."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
MIN_FAST = {0: 0.7, 1: 1.0, 2: 1.0, 3: 0.25, 4: 0.7, 5: 0.7, 6: 1.0}


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    pytest.skip("nvcc not found")


def test_device_emulation_bit_exact_against_fp64_instructions(tmp_path):
    exe = tmp_path / "fp64_emu_probe"
    subprocess.run([_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                    os.path.join(HERE, "fp64_emu_probe.cu"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    print(out)
    lines = [ln.split() for ln in out.splitlines() if ln.startswith("op ")]
    assert len(lines) == 26
    for f in lines:
        op, kind, cases, mism, fast = int(f[1]), int(f[3]), int(f[5]), int(f[7]), int(f[9])
        assert mism == 0, f"op {op} kind {kind}: {mism} mismatches, first operands {f[10:13]}"
        assert fast >= MIN_FAST[kind] * cases, f"op {op} kind {kind}: fast path {fast} of {cases}"
