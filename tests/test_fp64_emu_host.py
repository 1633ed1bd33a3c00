"""csrc/fp64_emu.cuh on the host: the integer-pipe IEEE binary64 multiply
(also with its first operand negated), add and fused multiply-add that the
FP64 pair kernels use in place of part of their FP64 instructions, compared
bit for bit with the host's own IEEE 754 arithmetic (x * y, -x * y, x + y and
std::fma, each correctly rounded to nearest-even by the standard's
definition).

The operand kinds (tests/fp64_emu_host.cpp) cover every class of double
(random bit patterns: zeros, subnormals, infinities, NaN), typical
magnitudes, significands with trailing zeros (exact results and exact
ties), boundary values (the least and largest normals, powers of two next to
the exponent limits), near-cancellations, and results next to the halfway
point of the rounding with and without bits further down.  The test also
checks that the fast path (the integer arithmetic) took most cases, so a
routine that sent everything to the hardware instruction would fail.

Each planted mistake tried while writing these (the sticky bit of the
multiply's low word dropped, the sum's sticky bit dropped, the FMA alignment's
sticky bit dropped, ties rounded away from even) fails at least one case."""
import ctypes
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
N = 400_000


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = tmp_path_factory.mktemp("fp64emu") / "libfp64emu.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                    os.path.join(HERE, "fp64_emu_host.cpp"), "-o", str(out)], check=True)
    L = ctypes.CDLL(str(out))
    L.emu_check.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_long, ctypes.c_uint64,
                            ctypes.POINTER(ctypes.c_uint64)]
    L.emu_check.restype = ctypes.c_int
    return L


OPS = {"mul": 0, "add": 1, "fma": 2, "mul_neg": 3}
KINDS = {"any_bits": 0, "typical": 1, "trailing_zeros": 2, "boundary": 3, "mixed": 4,
         "cancellation": 5, "near_ties": 6}
# the least share of cases the integer path must take, per kind (random bit
# patterns: exponents over the whole range, so products and sums leave the
# normal range often; boundary values: zeros, subnormals, inf and NaN)
MIN_FAST = {0: 0.7, 1: 1.0, 2: 1.0, 3: 0.25, 4: 0.7, 5: 0.7, 6: 1.0}


@pytest.mark.parametrize("kind", list(KINDS), ids=list(KINDS))
@pytest.mark.parametrize("op", list(OPS), ids=list(OPS))
def test_bit_exact_against_host_ieee(lib, op, kind):
    o, k = OPS[op], KINDS[kind]
    if o in (0, 3) and k == 5:
        pytest.skip("cancellation is a property of sums")
    out = (ctypes.c_uint64 * 5)()
    assert lib.emu_check(o, k, N, 0x5EED + 17 * k + o, out) == 0
    mism, fast = out[0], out[1]
    assert mism == 0, (f"{op}/{kind}: {mism} mismatches; first operands "
                       f"{out[2]:016x} {out[3]:016x} {out[4]:016x}")
    assert fast >= MIN_FAST[k] * N, f"{op}/{kind}: fast path took {fast} of {N}"
