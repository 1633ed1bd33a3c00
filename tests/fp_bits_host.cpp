// Host build of csrc/fp_bits.cuh for tests/test_fp_bits_host.py.
#include "../paper_1402_3325_gb300/csrc/fp_bits.cuh"

extern "C" {
void scale2_many(const double *x, long n, int k, double *out)
{
    for (long i = 0; i < n; ++i) out[i] = sakura::scale2(x[i], k);
}
void f2d_many(const float *f, long n, double *out)
{
    for (long i = 0; i < n; ++i) out[i] = sakura::f2d(f[i]);
}
}
