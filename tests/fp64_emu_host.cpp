// Host build of csrc/fp64_emu.cuh for tests/test_fp64_emu_host.py: the
// integer-pipe multiply, add and fused multiply-add against the host's own
// IEEE 754 binary64 arithmetic (x * y, x + y, std::fma), bit for bit.
#include "../paper_1402_3325_gb300/csrc/fp64_emu.cuh"
#include "fp64_emu_cases.h"

#include <cmath>
#include <cstdint>

using namespace sakura;
using namespace emucases;

// n cases of op (0: a * b, 1: a + b, 2: fma(a, b, c), 3: (-a) * b) of the
// given kind (fp64_emu_cases.h).  out[0]: mismatches, out[1]: cases the fast
// path took, out[2..4]: the bits of the first mismatch's operands.  Returns 0.
extern "C" int emu_check(int op, int kind, long n, uint64_t seed, uint64_t *out)
{
    uint64_t s = seed;
    out[0] = out[1] = out[2] = out[3] = out[4] = 0;
    for (long i = 0; i < n; ++i) {
        double a, b, c;
        make_case(s, op, kind, a, b, c);
        double want, got, fast;
        bool took;
        if (op == 0) {
            want = a * b;
            got = emu::mul(a, b);
            took = emu::mul_fast(a, b, fast);
        } else if (op == 3) {
            want = -a * b;
            got = emu::mul_neg(a, b);
            took = emu::mul_fast<true>(a, b, fast);
        } else if (op == 1) {
            want = a + b;
            got = emu::add(a, b);
            took = emu::add_fast(a, b, fast);
        } else {
            want = std::fma(a, b, c);
            got = emu::fma(a, b, c);
            took = emu::fma_fast(a, b, c, fast);
        }
        if (took) ++out[1];
        if (!same(want, got) || (took && !same(want, fast))) {
            if (out[0] == 0) {
                out[2] = bits(a);
                out[3] = bits(b);
                out[4] = bits(c);
            }
            ++out[0];
        }
    }
    return 0;
}
