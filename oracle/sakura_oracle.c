/*
 * sakura_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.
 *
 * A plain, slow, deliberately obvious FP64 CPU statement of the Sakura
 * Keplerian-splitting integrator (Goncalves Ferrari, Boekholt & Portegies
 * Zwart 2014, "A Keplerian-based Hamiltonian splitting for gravitational
 * N-body simulations").  It exists to check the CUDA library: only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header or constant with the CUDA path.
 *
 * Build (see oracle/build.py): gcc -O2 -ffp-contract=off -fno-fast-math
 * -fopenmp -shared -fPIC.  Contraction is off so that x86 and Arm hosts
 * produce bit-identical results.
 *
 * Data layout follows the paper's listing: m[n], r[n][3], v[n][3] (array of
 * structures), G = 1, no softening (Sec. 3: the method admits none).
 *
 * Readings of points the paper leaves open (each is also listed in the
 * design notes):
 *   - Kepler solver: universal variable s with Stumpff functions, Laguerre
 *     iteration of order n = 5 (Conway 1986, the method the paper's
 *     implementation section names), safeguarded by a bracket on the strictly
 *     increasing Kepler function F(s); bisection if 50 steps do not converge.
 *   - Convergence: |ds| <= 4 eps |s|, or |F| <= 4 eps max(|t|, r0 |s|).
 *   - Initial guess: s0 = t / r0 after reducing t modulo the period P for
 *     bound orbits with |t| > P.
 *   - Stumpff functions: power series for |x| < 0.1, closed trigonometric or
 *     hyperbolic forms otherwise.
 *   - order = 1 is phi(tau) of Eq. 24 read right-to-left: W(tau) with pair map
 *     Eq. 19a (Kepler tau, then backward drift tau), then the drift
 *     e^{tau H_T}.  order = -1 is the adjoint phi^dagger: drift tau, then W(tau)
 *     with pair map Eq. 19b (backward drift tau, then Kepler tau).
 *   - Energy sums use Neumaier compensated summation.
 *   - Orders 4, 6, 8 (the paper only says that higher orders come from
 *     compositions, Sec. 2.2): Yoshida's triple jump of the second-order map.
 *
 * Parity status: every exported function here is pinned by tests/ against
 * closed forms, high-precision (mpmath) classical Kepler solutions, an
 * independently written leapfrog (the Eq. 28 limit), invariants, and a
 * high-order reference integrator.  Per-step values for N >= 3 beyond those
 * structural pins have no independent source: "parity unpinned" there.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>

#define ORC_OK 0
#define ORC_E_ARG -2
#define ORC_E_MASS -3
#define ORC_E_COINCIDENT -4
#define ORC_E_NONFINITE -5
#define ORC_E_KEPLER -6

#define ORC_PAIR_KEPLER 0 /* Eq. 18: exact two-body flow                */
#define ORC_PAIR_DKD 1    /* Eq. 28: drift-kick-drift two-body leapfrog */

static const double ORC_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------ */
/* Stumpff functions c_k(x) = sum_{n>=0} (-x)^n / (k+2n)!, k = 0..3.    */
/* ------------------------------------------------------------------ */
static void stumpff_series(double x, double c[4])
{
    for (int k = 0; k < 4; ++k) {
        /* first term 1/k! */
        double term = 1.0;
        for (int q = 2; q <= k; ++q) term /= (double)q;
        double sum = 0.0;
        for (int n = 0; n < 30; ++n) {
            sum += term;
            if (fabs(term) <= 1e-20 * fabs(sum)) break;
            double a = (double)(k + 2 * n + 1), b = (double)(k + 2 * n + 2);
            term *= -x / (a * b);
        }
        c[k] = sum;
    }
}

static void stumpff_closed(double x, double c[4])
{
    if (x > 0.0) {
        double z = sqrt(x);
        c[0] = cos(z);
        c[1] = sin(z) / z;
        c[2] = (1.0 - cos(z)) / x;
        c[3] = (z - sin(z)) / (x * z);
    } else {
        double z = sqrt(-x);
        c[0] = cosh(z);
        c[1] = sinh(z) / z;
        c[2] = (cosh(z) - 1.0) / (-x);
        c[3] = (sinh(z) - z) / (-x * z);
    }
}

void oracle_stumpff(double x, double c[4])
{
    if (fabs(x) < 0.1)
        stumpff_series(x, c);
    else
        stumpff_closed(x, c);
}

/* ------------------------------------------------------------------ */
/* Universal-variable Kepler flow over time t (Eq. 18).                 */
/*   r(s) = r0 + eta0 G1 + zeta0 G2,  t(s) = r0 s + eta0 G2 + zeta0 G3  */
/*   G_k(s) = s^k c_k(beta s^2), beta = 2m/r0 - v0^2, eta0 = r0.v0,      */
/*   zeta0 = m - beta r0.                                                */
/* ------------------------------------------------------------------ */
typedef struct {
    double r0, eta0, zeta0, beta, t;
} kep_t;

static void kep_eval(const kep_t *k, double s, double G[4], double *F, double *Fp,
                     double *Fpp)
{
    double c[4];
    oracle_stumpff(k->beta * s * s, c);
    G[0] = c[0];
    G[1] = s * c[1];
    G[2] = s * s * c[2];
    G[3] = s * s * s * c[3];
    *F = k->r0 * s + k->eta0 * G[2] + k->zeta0 * G[3] - k->t;
    *Fp = k->r0 + k->eta0 * G[1] + k->zeta0 * G[2];
    *Fpp = k->eta0 * G[0] + k->zeta0 * G[1];
}

typedef struct {
    int max_iter;     /* Laguerre steps before bisection (default 50) */
    int use_bisection; /* 1: fall back to bisection, 0: report failure */
    double tol_eps;   /* tolerance in units of DBL_EPSILON (default 4) */
} oracle_kepler_opts;

static const oracle_kepler_opts ORC_KEPLER_DEFAULT = {50, 1, 4.0};

/* Solve F(s) = 0.  Returns the converged s; *iters = Laguerre steps taken
   (plus bisection halvings, if any); *ok = 0 when neither converged. */
static double kep_solve(const kep_t *k, const oracle_kepler_opts *o, int *iters, int *ok)
{
    const double eps = DBL_EPSILON;
    double s = k->t / k->r0; /* standard initial guess */
    double G[4], F, Fp, Fpp;
    double lo, hi;
    int n_it = 0;

    /* Bracket the unique root: F(0) = -t and F'(s) = r(s) > 0.  F grows
       without bound away from 0 on the side of the root, so where its
       evaluation overflows (inf, or inf - inf on a strongly hyperbolic orbit
       whose guess lies far beyond the root) s is past the root: a
       non-finite F counts as "past the root" in every test below. */
    if (k->t > 0.0) {
        lo = 0.0;
        hi = s;
        for (int d = 0; d < 400; ++d) {
            kep_eval(k, hi, G, &F, &Fp, &Fpp);
            if (!(F < 0.0)) break;
            lo = hi;
            hi *= 2.0;
        }
    } else {
        hi = 0.0;
        lo = s;
        for (int d = 0; d < 400; ++d) {
            kep_eval(k, lo, G, &F, &Fp, &Fpp);
            if (!(F > 0.0)) break;
            hi = lo;
            lo *= 2.0;
        }
    }

    const double nl = 5.0; /* Laguerre order (Conway 1986) */
    for (int it = 0; it < o->max_iter; ++it) {
        kep_eval(k, s, G, &F, &Fp, &Fpp);
        ++n_it;
        if (!isfinite(F) || !isfinite(Fp) || !isfinite(Fpp)) {
            /* overflow: s lies past the root; bisect towards it */
            if (s > 0.0)
                hi = s;
            else
                lo = s;
            s = 0.5 * (lo + hi);
            continue;
        }
        if (F == 0.0) {
            *iters = n_it;
            *ok = 1;
            return s;
        }
        double scale = fmax(fabs(k->t), k->r0 * fabs(s));
        if (fabs(F) <= o->tol_eps * eps * scale) {
            *iters = n_it;
            *ok = 1;
            return s;
        }
        if (F < 0.0)
            lo = s;
        else
            hi = s;
        double disc = (nl - 1.0) * (nl - 1.0) * Fp * Fp - nl * (nl - 1.0) * F * Fpp;
        double den = Fp + copysign(sqrt(fabs(disc)), Fp);
        if (!isfinite(disc) || !isfinite(den) || den == 0.0) {
            /* F' = r(s) so large that its square overflows: s lies far past
               the root (at the root r is the pair's separation), and the
               Laguerre step would round to zero; bisect instead */
            s = 0.5 * (lo + hi);
            continue;
        }
        double ds = nl * F / den;
        double snew = s - ds;
        if (fabs(ds) <= o->tol_eps * eps * fabs(snew)) {
            *iters = n_it;
            *ok = 1;
            return snew;
        }
        if (!(snew > lo && snew < hi)) snew = 0.5 * (lo + hi);
        s = snew;
    }
    if (!o->use_bisection) {
        *iters = n_it;
        *ok = 0;
        return s;
    }
    /* Bisection on the bracket down to about two ulp. */
    for (int b = 0; b < 2000; ++b) {
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        if (hi - lo <= 2.0 * eps * fmax(fabs(lo), fabs(hi))) break;
        kep_eval(k, mid, G, &F, &Fp, &Fpp);
        ++n_it;
        if (!isfinite(F)) {
            if (mid > 0.0)
                hi = mid;
            else
                lo = mid;
        } else if (F < 0.0)
            lo = mid;
        else if (F > 0.0)
            hi = mid;
        else {
            lo = hi = mid;
            break;
        }
    }
    *iters = n_it;
    *ok = 1;
    return 0.5 * (lo + hi);
}

/* Advance the relative two-body state (r0v, v0v) with total mass m over time
   tau along the exact Kepler flow (Eq. 18).  Returns ORC_OK or an error. */
int oracle_kepler_ex(double tau, double m, const double r0v[3], const double v0v[3],
                     double r1v[3], double v1v[3], int *iters,
                     const oracle_kepler_opts *opts)
{
    const oracle_kepler_opts *o = opts ? opts : &ORC_KEPLER_DEFAULT;
    int dummy = 0;
    if (!iters) iters = &dummy;
    *iters = 0;
    double r0 = sqrt(r0v[0] * r0v[0] + r0v[1] * r0v[1] + r0v[2] * r0v[2]);
    if (!(r0 > 0.0)) return ORC_E_COINCIDENT;
    if (!(m > 0.0)) return ORC_E_MASS;
    double eta0 = r0v[0] * v0v[0] + r0v[1] * v0v[1] + r0v[2] * v0v[2];
    double v2 = v0v[0] * v0v[0] + v0v[1] * v0v[1] + v0v[2] * v0v[2];
    kep_t k;
    k.r0 = r0;
    k.eta0 = eta0;
    k.beta = 2.0 * m / r0 - v2;
    k.zeta0 = m - k.beta * r0;
    k.t = tau;
    if (k.beta > 0.0) {
        double P = 2.0 * ORC_PI * m / (k.beta * sqrt(k.beta));
        if (fabs(k.t) > P) k.t = fmod(k.t, P);
    }
    if (k.t == 0.0) {
        for (int q = 0; q < 3; ++q) {
            r1v[q] = r0v[q];
            v1v[q] = v0v[q];
        }
        return ORC_OK;
    }
    int ok = 0;
    double s = kep_solve(&k, o, iters, &ok);
    if (!ok) return ORC_E_KEPLER;
    double G[4], F, Fp, Fpp;
    kep_eval(&k, s, G, &F, &Fp, &Fpp);
    double r = Fp;
    /* Lagrange coefficients */
    double f = 1.0 - m * G[2] / r0;
    double g = k.t - m * G[3];
    double fd = -m * G[1] / (r0 * r);
    double gd = 1.0 - m * G[2] / r;
    for (int q = 0; q < 3; ++q) {
        r1v[q] = f * r0v[q] + g * v0v[q];
        v1v[q] = fd * r0v[q] + gd * v0v[q];
    }
    for (int q = 0; q < 3; ++q)
        if (!isfinite(r1v[q]) || !isfinite(v1v[q])) return ORC_E_NONFINITE;
    return ORC_OK;
}

int oracle_kepler(double tau, double m, const double r0v[3], const double v0v[3],
                  double r1v[3], double v1v[3], int *iters)
{
    return oracle_kepler_ex(tau, m, r0v, v0v, r1v, v1v, iters, NULL);
}

/* Same, with explicit iteration controls (used by the failure-path tests). */
int oracle_kepler_opt(double tau, double m, const double r0v[3], const double v0v[3],
                      double r1v[3], double v1v[3], int *iters, int max_iter,
                      int use_bisection, double tol_eps)
{
    oracle_kepler_opts o = {max_iter, use_bisection, tol_eps};
    return oracle_kepler_ex(tau, m, r0v, v0v, r1v, v1v, iters, &o);
}

/* Two-body drift-kick-drift leapfrog over tau: the substitute solver of the
   Eq. 28 limit.  Relative acceleration a = -m r / |r|^3. */
static int pair_dkd(double tau, double m, const double r0v[3], const double v0v[3],
                    double r1v[3], double v1v[3])
{
    double rh[3];
    for (int q = 0; q < 3; ++q) rh[q] = r0v[q] + 0.5 * tau * v0v[q];
    double d2 = rh[0] * rh[0] + rh[1] * rh[1] + rh[2] * rh[2];
    if (!(d2 > 0.0)) return ORC_E_COINCIDENT;
    double d = sqrt(d2);
    double inv3 = 1.0 / (d2 * d);
    for (int q = 0; q < 3; ++q) v1v[q] = v0v[q] - tau * m * rh[q] * inv3;
    for (int q = 0; q < 3; ++q) r1v[q] = rh[q] + 0.5 * tau * v1v[q];
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* The drift operator e^{tau H_T} (Eq. 12): r_i += tau v_i.            */
/* ------------------------------------------------------------------ */
static void evolve_HT(double tau, int64_t n, double *r, const double *v)
{
    for (int64_t i = 0; i < n; ++i)
        for (int q = 0; q < 3; ++q) r[3 * i + q] += v[3 * i + q] * tau;
}

/* ------------------------------------------------------------------ */
/* The W operator e^{tau H_W} (Eq. 14, increments by Eq. 23) with one  */
/* of three per-pair maps:                                             */
/*   pair_map = 2 : Eq. 26, back-drift tau/2, Kepler tau, back-drift   */
/*   pair_map = 1 : Eq. 19a, Kepler tau then back-drift tau            */
/*   pair_map = -1: Eq. 19b, back-drift tau then Kepler tau            */
/* Loops run i ascending outside, j ascending inside, as in the paper's */
/* listing; per-i sums are sequential, so the OpenMP split over i gives */
/* the same bits as a serial run.                                       */
/* ------------------------------------------------------------------ */
typedef struct {
    int64_t pairs;      /* ordered pairs solved */
    int64_t iters;      /* total Kepler iterations */
    int64_t max_iters;  /* largest iteration count of any pair */
} oracle_stats;

static int evolve_HW(double tau, int64_t n, const double *m, double *r, double *v,
                     int pair_map, int pair_solver, int nthreads, oracle_stats *st)
{
    double *dmr = (double *)calloc((size_t)(3 * n), sizeof(double));
    double *dmv = (double *)calloc((size_t)(3 * n), sizeof(double));
    if (!dmr || !dmv) {
        free(dmr);
        free(dmv);
        return ORC_E_ARG;
    }
    int status = ORC_OK;
    int64_t tot_it = 0, max_it = 0;
    double pre = 0.0, post = 0.0; /* backward-drift fractions before / after */
    if (pair_map == 2) {
        pre = 0.5;
        post = 0.5;
    } else if (pair_map == 1) {
        pre = 0.0;
        post = 1.0;
    } else {
        pre = 1.0;
        post = 0.0;
    }
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(+ : tot_it) \
    reduction(max : max_it)
#endif
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            if (i == j) continue;
            double mij = m[i] + m[j];
            double mu = m[i] * m[j] / mij;
            double rr0[3], vv0[3], r0[3], v0[3], r1[3], v1[3], rr1[3];
            for (int q = 0; q < 3; ++q) {
                rr0[q] = r[3 * i + q] - r[3 * j + q];
                vv0[q] = v[3 * i + q] - v[3 * j + q];
            }
            for (int q = 0; q < 3; ++q) {
                r0[q] = rr0[q] - vv0[q] * tau * pre;
                v0[q] = vv0[q];
            }
            int it = 0, rc;
            if (pair_solver == ORC_PAIR_DKD)
                rc = pair_dkd(tau, mij, r0, v0, r1, v1);
            else
                rc = oracle_kepler(tau, mij, r0, v0, r1, v1, &it);
            if (rc != ORC_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
                status = rc;
            }
            tot_it += it;
            if (it > max_it) max_it = it;
            for (int q = 0; q < 3; ++q) rr1[q] = r1[q] - v1[q] * tau * post;
            for (int q = 0; q < 3; ++q) {
                dmr[3 * i + q] += mu * (rr1[q] - rr0[q]);
                dmv[3 * i + q] += mu * (v1[q] - vv0[q]);
            }
        }
    }
    /* Eqs. 27b-c */
    for (int64_t i = 0; i < n; ++i)
        for (int q = 0; q < 3; ++q) {
            r[3 * i + q] += dmr[3 * i + q] / m[i];
            v[3 * i + q] += dmv[3 * i + q] / m[i];
        }
    free(dmr);
    free(dmv);
    if (st) {
        st->pairs += n * (n - 1);
        st->iters += tot_it;
        if (max_it > st->max_iters) st->max_iters = max_it;
    }
    return status;
}

int oracle_step(int64_t n, const double *m, double *r, double *v, double tau, int order,
                int pair_solver, int nthreads, oracle_stats *st);

/* Orders 4, 6 and 8: the paper (Sec. 2.2, after Eqs. 19a-b) builds higher
 * orders by composing the symmetric second-order map, as in symplectic
 * integrators (Yoshida 1990).  Yoshida's triple jump raises a symmetric map
 * S of order 2k - 2 to order 2k:
 *     S_2k(tau) = S(x1 tau) S(x0 tau) S(x1 tau),
 *     x1 = 1 / (2 - 2^(1/(2k-1))),  x0 = -2^(1/(2k-1)) / (2 - 2^(1/(2k-1))),
 * the three maps applied left to right in time (the outer two are equal, so
 * the reading of the operator order does not matter). */
static int step_triple_jump(int64_t n, const double *m, double *r, double *v, double tau,
                            int order, int pair_solver, int nthreads, oracle_stats *st)
{
    const double c = pow(2.0, 1.0 / (double)(order - 1));
    const double x1 = 1.0 / (2.0 - c);
    const double x0 = -c / (2.0 - c);
    int rc = oracle_step(n, m, r, v, x1 * tau, order - 2, pair_solver, nthreads, st);
    if (rc == ORC_OK) rc = oracle_step(n, m, r, v, x0 * tau, order - 2, pair_solver, nthreads, st);
    if (rc == ORC_OK) rc = oracle_step(n, m, r, v, x1 * tau, order - 2, pair_solver, nthreads, st);
    return rc;
}

/* One step of the integrator on m[n], r[n][3], v[n][3] in place.
 *   order =  2: Psi(tau) = D(tau/2) W(tau) D(tau/2), pair map Eq. 26 (Eq. 25,
 *               Eqs. 27a-d, the paper's listing).
 *   order =  1: phi(tau) = W(tau; Eq. 19a) followed by D(tau).
 *   order = -1: phi^dagger(tau) = D(tau) followed by W(tau; Eq. 19b).
 *   order =  4, 6, 8: the triple-jump composition of the order below
 *               (3, 9 or 27 second-order steps, step_triple_jump).
 * pair_solver selects the two-body map inside W: ORC_PAIR_KEPLER (Eq. 18) or
 * ORC_PAIR_DKD (the Eq. 28 substitute).  nthreads: OpenMP threads for the i
 * loop (results do not depend on it).  stats may be NULL. */
int oracle_step(int64_t n, const double *m, double *r, double *v, double tau, int order,
                int pair_solver, int nthreads, oracle_stats *st)
{
    if (n < 1 || !m || !r || !v) return ORC_E_ARG;
    if (order == 4 || order == 6 || order == 8)
        return step_triple_jump(n, m, r, v, tau, order, pair_solver, nthreads, st);
    if (!(order == 2 || order == 1 || order == -1)) return ORC_E_ARG;
    for (int64_t i = 0; i < n; ++i)
        if (!(m[i] > 0.0)) return ORC_E_MASS;
    for (int64_t i = 0; i < 3 * n; ++i)
        if (!isfinite(r[i]) || !isfinite(v[i])) return ORC_E_NONFINITE;
    int rc = ORC_OK;
    if (order == 2) {
        evolve_HT(0.5 * tau, n, r, v);                                     /* 27a */
        rc = evolve_HW(tau, n, m, r, v, 2, pair_solver, nthreads, st);      /* 27b-c */
        evolve_HT(0.5 * tau, n, r, v);                                     /* 27d */
    } else if (order == 1) {
        rc = evolve_HW(tau, n, m, r, v, 1, pair_solver, nthreads, st);
        evolve_HT(tau, n, r, v);
    } else {
        evolve_HT(tau, n, r, v);
        rc = evolve_HW(tau, n, m, r, v, -1, pair_solver, nthreads, st);
    }
    if (rc != ORC_OK) return rc;
    for (int64_t i = 0; i < 3 * n; ++i)
        if (!isfinite(r[i]) || !isfinite(v[i])) return ORC_E_NONFINITE;
    return ORC_OK;
}

/* The step of oracle_step (order 2, 1 or -1, Kepler pair solver) evaluated
   only for the k particles listed in idx[]: writes their post-step positions
   and velocities to r_out[k][3], v_out[k][3].  Each sampled row sums over all
   j != i in ascending order exactly as the full step does, so the values are
   the ones oracle_step would produce for those particles.  The input state is
   not modified. */
int oracle_step_sample(int64_t n, const double *m, const double *r, const double *v,
                       double tau, int order, const int64_t *idx, int64_t k, double *r_out,
                       double *v_out, int nthreads)
{
    if (n < 1 || !m || !r || !v || !idx || k < 0) return ORC_E_ARG;
    if (!(order == 2 || order == 1 || order == -1)) return ORC_E_ARG;
    double drift = order == 2 ? 0.5 * tau : (order == 1 ? 0.0 : tau);
    double pre = order == 2 ? 0.5 : (order == 1 ? 0.0 : 1.0);
    double post = order == 2 ? 0.5 : (order == 1 ? 1.0 : 0.0);
    double *rd = (double *)malloc(sizeof(double) * (size_t)(3 * n));
    if (!rd) return ORC_E_ARG;
    /* the first drift, as evolve_HT computes it */
    for (int64_t i = 0; i < n; ++i)
        for (int q = 0; q < 3; ++q) rd[3 * i + q] = r[3 * i + q] + v[3 * i + q] * drift;
    int status = ORC_OK;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic) num_threads(nthreads)
#endif
    for (int64_t s = 0; s < k; ++s) {
        int64_t i = idx[s];
        double dmr[3] = {0, 0, 0}, dmv[3] = {0, 0, 0};
        for (int64_t j = 0; j < n; ++j) {
            if (i == j) continue;
            double mij = m[i] + m[j];
            double mu = m[i] * m[j] / mij;
            double rr0[3], vv0[3], r0[3], v0[3], r1[3], v1[3], rr1[3];
            for (int q = 0; q < 3; ++q) {
                rr0[q] = rd[3 * i + q] - rd[3 * j + q];
                vv0[q] = v[3 * i + q] - v[3 * j + q];
            }
            for (int q = 0; q < 3; ++q) {
                r0[q] = rr0[q] - vv0[q] * tau * pre;
                v0[q] = vv0[q];
            }
            int it = 0;
            int rc = oracle_kepler(tau, mij, r0, v0, r1, v1, &it);
            if (rc != ORC_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
                status = rc;
            }
            for (int q = 0; q < 3; ++q) rr1[q] = r1[q] - v1[q] * tau * post;
            for (int q = 0; q < 3; ++q) {
                dmr[q] += mu * (rr1[q] - rr0[q]);
                dmv[q] += mu * (v1[q] - vv0[q]);
            }
        }
        for (int q = 0; q < 3; ++q) {
            double x = rd[3 * i + q] + dmr[q] / m[i];
            double u = v[3 * i + q] + dmv[q] / m[i];
            if (order == 2)
                x += u * (0.5 * tau);
            else if (order == 1)
                x += u * tau;
            r_out[3 * s + q] = x;
            v_out[3 * s + q] = u;
        }
    }
    free(rd);
    return status;
}

/* ------------------------------------------------------------------ */
/* Energy (Eqs. 1-3): E = sum_i m_i v_i^2 / 2 - sum_{i<j} m_i m_j / r_ij */
/* Neumaier-compensated sums; T and U are also returned.               */
/* ------------------------------------------------------------------ */
typedef struct {
    double s, c;
} nsum_t;

static void nsum_add(nsum_t *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x))
        a->c += (a->s - t) + x;
    else
        a->c += (x - t) + a->s;
    a->s = t;
}

int oracle_energy(int64_t n, const double *m, const double *r, const double *v,
                  double *E, double *T, double *U)
{
    if (n < 1 || !m || !r || !v) return ORC_E_ARG;
    nsum_t kin = {0.0, 0.0}, pot = {0.0, 0.0};
    for (int64_t i = 0; i < n; ++i) {
        double v2 = v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2];
        nsum_add(&kin, 0.5 * m[i] * v2);
    }
    int status = ORC_OK;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            double dx = r[3 * i] - r[3 * j], dy = r[3 * i + 1] - r[3 * j + 1],
                   dz = r[3 * i + 2] - r[3 * j + 2];
            double d = sqrt(dx * dx + dy * dy + dz * dz);
            if (!(d > 0.0)) status = ORC_E_COINCIDENT;
            nsum_add(&pot, -m[i] * m[j] / d);
        }
    double Tk = kin.s + kin.c, Up = pot.s + pot.c;
    nsum_t tot = {0.0, 0.0};
    nsum_add(&tot, kin.s);
    nsum_add(&tot, pot.s);
    nsum_add(&tot, kin.c);
    nsum_add(&tot, pot.c);
    if (T) *T = Tk;
    if (U) *U = Up;
    if (E) *E = tot.s + tot.c;
    return status;
}

/* ------------------------------------------------------------------ */
/* Precision class of each ordered pair for the mixed-precision form.  */
/* The rule is stated on the pair's Kepler input (r0, v0) of Eq. 26,   */
/* the relative state after the first drift (Eq. 27a) and the backward */
/* drift over pre * tau (Eq. 17), with m = m_i + m_j:                  */
/*   r = |r0|,  E = v0^2 / 2 - m / r,  h^2 = |r0 x v0|^2,              */
/*   e^2 = 1 + 2 E h^2 / m^2           (all in double precision)        */
/*   rule 0: single iff r > r_min and e < e_max                         */
/*   rule 1: single iff r > r_min and (e < e_max or e > e_hyp)          */
/* order selects (drift, pre): 2 -> (tau/2, 1/2), 1 -> (0, 0),          */
/* -1 -> (tau, 1).  Writes one byte per ordered pair (row i, column j;  */
/* diagonal 0) when cls != NULL, and the pair's r^2 and e^2 when r2 and */
/* e2 are not NULL (n x n doubles each, diagonal 0); returns the number */
/* of single-precision pairs.                                           */
/* ------------------------------------------------------------------ */
int64_t oracle_pair_classes(int64_t n, const double *m, const double *r, const double *v,
                            double tau, int order, int rule, double r_min, double e_max,
                            double e_hyp, uint8_t *cls, double *r2out, double *e2out)
{
    double drift = order == 2 ? 0.5 * tau : (order == 1 ? 0.0 : tau);
    double pre = order == 2 ? 0.5 : (order == 1 ? 0.0 : 1.0);
    double *rd = (double *)malloc(sizeof(double) * (size_t)(3 * n));
    if (!rd) return -1;
    for (int64_t i = 0; i < n; ++i)
        for (int q = 0; q < 3; ++q) rd[3 * i + q] = r[3 * i + q] + v[3 * i + q] * drift;
    int64_t count = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            uint8_t c = 0;
            double rsq = 0.0, esq = 0.0;
            if (i != j) {
                double x0[3], u0[3];
                for (int q = 0; q < 3; ++q) {
                    u0[q] = v[3 * i + q] - v[3 * j + q];
                    x0[q] = (rd[3 * i + q] - rd[3 * j + q]) - u0[q] * tau * pre;
                }
                double mm = m[i] + m[j];
                rsq = x0[0] * x0[0] + x0[1] * x0[1] + x0[2] * x0[2];
                double v2 = u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2];
                double hx = x0[1] * u0[2] - x0[2] * u0[1];
                double hy = x0[2] * u0[0] - x0[0] * u0[2];
                double hz = x0[0] * u0[1] - x0[1] * u0[0];
                double h2 = hx * hx + hy * hy + hz * hz;
                double E = 0.5 * v2 - mm / sqrt(rsq);
                esq = 1.0 + 2.0 * E * h2 / (mm * mm);
                int far = sqrt(rsq) > r_min;
                int lowe = sqrt(esq > 0.0 ? esq : 0.0) < e_max;
                int hyp = (rule == 1) && (sqrt(esq > 0.0 ? esq : 0.0) > e_hyp);
                c = (uint8_t)(far && (lowe || hyp));
            }
            if (cls) cls[i * n + j] = c;
            if (r2out) r2out[i * n + j] = rsq;
            if (e2out) e2out[i * n + j] = esq;
            count += c;
        }
    free(rd);
    return count;
}

/* A version string so that loaders can check they found this file. */
const char *oracle_version(void) { return "sakura-oracle-1"; }
