// Host build of the library's double-word primitives (csrc/df64.cuh) for the
// CPU test of their error bounds (tests/test_df64_host.py).  Built with
// g++ -O2 -ffp-contract=off so that plain float operations round once.
#include "../paper_1402_3325_gb300/csrc/df64.cuh"
#include "../paper_1402_3325_gb300/csrc/kepler_df64.cuh"

using sakura::dw;

#if defined(SAKURA_DW_COUNT)
namespace sakura {
long long sakura_dw_flops = 0, sakura_dw_mufu = 0;
}
using sakura::sakura_dw_flops;
using sakura::sakura_dw_mufu;
#endif

extern "C" {

// op: 0 add, 1 sub, 2 add_f, 3 mul, 4 mul_f, 5 sqr, 6 rcp, 7 rsqrt,
// 8 add without cancellation
void dw_batch(int op, long n, const float *xh, const float *xl, const float *yh,
              const float *yl, float *zh, float *zl)
{
    for (long k = 0; k < n; ++k) {
        const dw x{xh[k], xl[k]}, y{yh[k], yl[k]};
        dw z{0.0f, 0.0f};
        switch (op) {
            case 0: z = sakura::dw_add(x, y); break;
            case 1: z = sakura::dw_sub(x, y); break;
            case 2: z = sakura::dw_add_f(x, yh[k]); break;
            case 3: z = sakura::dw_mul(x, y); break;
            case 4: z = sakura::dw_mul_f(x, yh[k]); break;
            case 5: z = sakura::dw_sqr(x); break;
            case 6: z = sakura::dw_rcp(x); break;
            case 7: z = sakura::dw_rsqrt(x); break;
            case 8: z = sakura::dw_add_nc(x, y); break;
        }
        zh[k] = z.h;
        zl[k] = z.l;
    }
}

static sakura::dw to_dw(double d)
{
    const float h = (float)d;
    return {h, (float)(d - (double)h)};
}

// The double-word pair map for n pairs of relative states (after the
// one-subscript drift): rv[k] = (rx, ry, rz, vx, vy, vz) as doubles, taken
// through the exact three-float differences of (rv, 0).  Writes the
// increments over m and the admitted flag (1: double-word, 0: FP64 class).
void dw_pair_batch(long n, const double *rv, const double *m, double tau, double pre,
                   double post, int guess, double *out, int *admitted, int *evals)
{
    for (long k = 0; k < n; ++k) {
        dw rr[3], vv[3];
        for (int q = 0; q < 3; ++q) {
            float a0, a1, a2, b0, b1, b2;
            sakura::tf_split(rv[6 * k + q], a0, a1, a2);
            sakura::tf_split(0.0, b0, b1, b2);
            rr[q] = sakura::tf_diff(a0, a1, a2, b0, b1, b2);
            sakura::tf_split(rv[6 * k + 3 + q], a0, a1, a2);
            vv[q] = sakura::tf_diff(a0, a1, a2, b0, b1, b2);
        }
        const dw mm = to_dw(m[k]);
        const sakura::K32 o = sakura::dw_phase1(rr, vv, mm, (float)(pre * tau), (float)tau, guess);
        admitted[k] = 0;
        evals[k] = 0;
        for (int q = 0; q < 6; ++q) out[6 * k + q] = 0.0;
        if (!o.ok) continue;
        dw d[6];
        const bool big = std::fabs(o.x) > 0x1p-8f;
        int ev = 0;
        if (!sakura::dw_phase2(rr, vv, mm, to_dw(pre * tau), to_dw(tau), to_dw(post * tau), o.s,
                               big, d, ev))
            continue;
        admitted[k] = 1;
        evals[k] = ev;
        for (int q = 0; q < 6; ++q) out[6 * k + q] = (double)d[q].h + (double)d[q].l;
    }
}

#if defined(SAKURA_DW_COUNT)
// Floating-point work of the pair kernel for each pair (ri, rj, vi, vj as
// doubles after the drift): the six exact differences, the FP32 phase, the
// double-word phase and the two weighted double-word accumulations.
// Returns the flops (FMA = 2) and approximations summed over the admitted
// pairs and their count.
void dw_count_pairs(long n, const double *xi, const double *xj, const double *mi,
                    const double *mj, double tau, double pre, double post, int guess,
                    double *flops, double *mufu, long *admitted)
{
    *flops = 0.0;
    *mufu = 0.0;
    *admitted = 0;
    for (long k = 0; k < n; ++k) {
        sakura_dw_flops = 0;
        sakura_dw_mufu = 0;
        dw rr[3], vv[3];
        for (int q = 0; q < 6; ++q) {
            float a0, a1, a2, b0, b1, b2;
            sakura::tf_split(xi[6 * k + q], a0, a1, a2);
            sakura::tf_split(xj[6 * k + q], b0, b1, b2);
            (q < 3 ? rr[q] : vv[q - 3]) = sakura::tf_diff(a0, a1, a2, b0, b1, b2);
        }
        const dw ma = to_dw(mi[k]), mb = to_dw(mj[k]);
        const dw m = sakura::dw_add(ma, mb);
        const sakura::K32 o = sakura::dw_phase1(rr, vv, m, (float)(pre * tau), (float)tau, guess);
        if (!o.ok) continue;
        dw d[6];
        int ev = 0;
        if (!sakura::dw_phase2(rr, vv, m, to_dw(pre * tau), to_dw(tau), to_dw(post * tau), o.s,
                               std::fabs(o.x) > 0x1p-8f, d, ev))
            continue;
        dw racc[6] = {}, cacc[6] = {};
        for (int q = 0; q < 6; ++q) {
            sakura::dw_acc(racc[q], sakura::dw_mul(mb, d[q]));
            sakura::dw_acc(cacc[q], sakura::dw_mul(sakura::dw_neg(ma), d[q]));
        }
        *flops += (double)sakura_dw_flops;
        *mufu += (double)sakura_dw_mufu;
        ++*admitted;
    }
}
#endif

// exact difference of doubles through their three-float form
void tf_diff_batch(long n, const double *a, const double *b, float *zh, float *zl)
{
    for (long k = 0; k < n; ++k) {
        float a0, a1, a2, b0, b1, b2;
        sakura::tf_split(a[k], a0, a1, a2);
        sakura::tf_split(b[k], b0, b1, b2);
        const dw z = sakura::tf_diff(a0, a1, a2, b0, b1, b2);
        zh[k] = z.h;
        zl[k] = z.l;
    }
}

}
