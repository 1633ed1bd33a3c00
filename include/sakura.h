/*
 * sakura.h -- C ABI of the GB300 (sm_103a) implementation of the Sakura
 * Keplerian-splitting N-body step (Goncalves Ferrari, Boekholt & Portegies
 * Zwart 2014).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - G = 1, no softening (the method admits none, Sec. 3).
 *  - A system of n particles is a device structure-of-arrays state
 *    double[6][n] (rows x, y, z, vx, vy, vz, row-major, contiguous) and a
 *    device double[n] of masses.  The caller owns both; the library never
 *    frees or retains caller memory beyond a call.
 *  - Device calls are asynchronous and ordered on the library stream
 *    (sakura_config.stream, or the one given to sakura_set_stream).  Calls
 *    that return host values (sakura_energy, sakura_get_stats, sakura_check,
 *    sakura_evolve_host) synchronise that stream.
 *  - Every function returns SAKURA_OK (0) or a negative SAKURA_E_* code.
 *    Faults found on the device (coincident pair, non-finite state, failed
 *    Kepler solve, non-positive mass) set bits in a device status word; they
 *    are reported by the next synchronising call, or by the call itself when
 *    SAKURA_FLAG_SYNC_CHECK is set.  No kernel traps or waits without bound.
 *  - The library keeps one process-wide context (one device); it is not
 *    thread-safe.  Scratch buffers are owned by the library and grow on
 *    demand (cudaMalloc) outside the timed kernels.
 */
#ifndef SAKURA_H
#define SAKURA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------- */
#define SAKURA_OK 0
#define SAKURA_E_NOINIT -1     /* sakura_init has not been called          */
#define SAKURA_E_ARG -2        /* bad size, order, pointer or option        */
#define SAKURA_E_MASS -3       /* a mass is <= 0 (mu_ij / m_i undefined)    */
#define SAKURA_E_COINCIDENT -4 /* a pair has r0 = 0: the Kepler flow is undefined */
#define SAKURA_E_NONFINITE -5  /* NaN or Inf in the state                   */
#define SAKURA_E_KEPLER -6     /* Laguerre iteration and bisection both failed */
#define SAKURA_E_CUDA -7       /* a CUDA runtime call failed                */
#define SAKURA_E_TIMEOUT -8    /* a bounded device wait ran out             */
#define SAKURA_E_NOMEM -9      /* device allocation failed                  */

/* ---- options --------------------------------------------------------- */
#define SAKURA_PREC_FP64 0  /* every pair solved in FP64                      */
#define SAKURA_PREC_MIXED 1 /* distant, low-eccentricity pairs solved in FP32 */
#define SAKURA_PREC_DF64 2  /* every pair solved to FP64 accuracy in double-word
                               ("double-float") arithmetic on the FP32 pipe:
                               an FP32 Laguerre phase, one double-word
                               correction and the increments in double-word
                               form; pairs outside single-precision range,
                               bound orbits whose step exceeds 0.9 of the
                               period and unconverged pairs are solved in
                               FP64.  Symmetric pair mode only (else as
                               FP64); the initial guess is the second-order
                               one (SAKURA_GUESS_LEARNED included).  Results
                               match the FP64 form to about 2^-46 relative
                               per pair.                                       */

#define SAKURA_MIXED_RULE_LITERAL 0 /* FP32 iff r > r_min and e < e_max           */
#define SAKURA_MIXED_RULE_HYP 1     /* FP32 iff r > r_min and (e < e_max or e > e_hyp) */

#define SAKURA_PAIRS_ORDERED 0   /* solve every ordered pair (i, j), i != j         */
#define SAKURA_PAIRS_SYMMETRIC 1 /* solve every unordered pair once and apply it to
                                    both particles (Newton's third law)            */

#define SAKURA_GUESS_STANDARD 0 /* s0 = t / r0                               */
#define SAKURA_GUESS_LEARNED 1  /* s0 from the loaded MLP (sakura_load_mlp)   */
#define SAKURA_GUESS_TAYLOR 2   /* s0 = (t/r0)(1 - eta0 t / (2 r0^2)): second order in t */
#define SAKURA_GUESS_FP32 3     /* s0 = the root of a single-precision Laguerre solve of
                                   the same pair (from a float copy of the drifted
                                   state, second-order start); the FP64 iteration and
                                   its convergence test follow as for every guess.
                                   Symmetric FP64 step only; elsewhere, and for a pair
                                   whose float solve fails, the second-order guess */

#define SAKURA_FLAG_SYNC_CHECK 1u /* synchronise and report faults on every call */
#define SAKURA_FLAG_STATS 2u      /* collect iteration statistics (small cost)   */
#define SAKURA_FLAG_TIMING 4u     /* time every pair-kernel launch with CUDA events */
#define SAKURA_FLAG_NO_AUTOTUNE 8u /* batched path: skip the block-shape autotuner  */
#define SAKURA_FLAG_NO_SMALL 16u   /* n <= 20: use the multi-kernel step instead of  */
                                   /* the single-block kernel (for comparisons)      */
#define SAKURA_FLAG_TILES 32u      /* symmetric FP64 and mixed steps: always the
                                      systolic tile kernel (per-warp tile segments,
                                      partials per segment: up to 12 n^2 bytes of
                                      scratch), the FP64 default below 4096
                                      bodies (the mixed form's under the literal
                                      rule too; the double-word form's up to about
                                      13400)                                       */
#define SAKURA_FLAG_GROUPS 64u     /* symmetric FP64 and mixed steps: always the
                                      row-group kernel (blocks of warps sweep column
                                      blocks together, column sums reduced per
                                      block: about n^2 / 2.7 bytes), the default
                                      beyond, and the mixed form's under
                                      SAKURA_MIXED_RULE_HYP                        */

#define SAKURA_BATCH_MAX_N 64     /* largest system of sakura_step_batched       */

typedef struct sakura_config {
    int device;           /* CUDA device ordinal                                  */
    void *stream;         /* cudaStream_t for all work; NULL = legacy default    */
    int precision;        /* SAKURA_PREC_*                                        */
    int mixed_rule;       /* SAKURA_MIXED_RULE_*                                  */
    double mixed_r_min;   /* default 0.1                                          */
    double mixed_e_max;   /* default 0.9                                          */
    double mixed_e_hyp;   /* default 10                                           */
    int guess;            /* SAKURA_GUESS_*                                       */
    double kepler_tol;    /* convergence |ds| <= kepler_tol * eps * |s|; default 4 */
    int kepler_max_iter;  /* Laguerre steps before bisection; default 50          */
    int kepler_bisection; /* 1 (default): bisection fallback; 0: report E_KEPLER  */
    unsigned int flags;   /* SAKURA_FLAG_*                                        */
    int block_warps;      /* pair kernel: warps per block (4, 8, 16), 0 = 4       */
    int grid_blocks;      /* pair kernel: blocks of the persistent grid, 0 = one
                             wave of resident blocks                             */
    int pair_mode;        /* SAKURA_PAIRS_* for the FP64 step (default symmetric;
                             ordered when the tile partials would pass 16 GB)   */
} sakura_config;

typedef struct sakura_stats {
    int64_t steps;        /* second-order (or first-order) maps applied since the
                             last reset: one per order-2/1/-1 step, 3 / 9 / 27
                             per step of order 4 / 6 / 8                         */
    int64_t pairs;        /* ordered pairs advanced (per map applied)            */
    int64_t iters;        /* Laguerre/Newton iterations summed over pairs         */
    int64_t max_iters;    /* largest iteration count of any pair                  */
    int64_t warp_slots;   /* sum over warp batches of 32 x (max lane iterations)  */
    int64_t fp32_pairs;   /* pairs solved on the FP32 pipe: in single precision
                             (mixed form) or in double-word arithmetic (df64)  */
    int64_t fallbacks;    /* pairs that needed bisection or a restart             */
    int64_t solves;       /* Kepler solves performed (pairs / 2 + diagonal-tile
                             pairs in the symmetric mode)                        */
    int64_t timed_launches; /* pair-kernel launches timed (SAKURA_FLAG_TIMING)    */
    double pair_kernel_ms;  /* their summed device time, from CUDA events on the
                               library stream                                    */
    int64_t carries;      /* FP64 solves finished by a Laguerre step below 2^-20 of
                             the scale with G1..G3 and r carried to the root by
                             their Taylor series (symmetric FP64 step)          */
    int64_t group_launches; /* pair-kernel launches in the row-group layout (the
                               others: systolic tiles, ordered pairs, the
                               single-block or batched kernels)                 */
} sakura_stats;

/* Fill *cfg with the defaults listed above. */
void sakura_default_config(sakura_config *cfg);

/* Create the process-wide context on cfg->device (NULL: defaults).
 * Allocates the status word and statistics counters.  Calling it again
 * replaces the configuration and keeps scratch buffers. */
int sakura_init(const sakura_config *cfg);

/* Release every library-owned device buffer and the context. */
int sakura_finalize(void);

/* Change the stream used by later calls (cudaStream_t as void*). */
int sakura_set_stream(void *stream);

/* One step of the integrator on a device state, in place (Sec. 2.2).
 *   order =  2: Psi(tau) = e^{tau/2 H_T} e^{tau H_W} e^{tau/2 H_T} (Eq. 25)
 *               with the pair map of Eq. 26, i.e. Eqs. 27a-d.
 *   order =  1: phi(tau) of Eq. 24 read right to left: W(tau) with the pair
 *               map of Eq. 19a (Kepler, then backward drift), then drift tau.
 *   order = -1: phi^dagger(tau): drift tau, then W(tau) with the pair map of
 *               Eq. 19b (backward drift, then Kepler).
 *   order = 4, 6, 8: Yoshida's triple jump of the order below, down to
 *               order-2 maps: S_2k(tau) = S_2k-2(x1 tau) S_2k-2(x0 tau)
 *               S_2k-2(x1 tau), x1 = 1/(2 - 2^(1/(2k-1))), x0 = 1 - 2 x1
 *               (the composition route to higher orders of Sec. 2.2); 3, 9
 *               or 27 order-2 maps per step.  The order-2 map is
 *               time-symmetric only up to O(tau^4) for N > 2, so the
 *               composed steps converge at third order there (exactly for
 *               N = 2).
 * Every ordered pair (i, j), i != j, is advanced by the universal-variable
 * Kepler flow (Eq. 18) and its increments are summed mass-weighted into
 * particle i (Eq. 23).  With cfg.pair_mode = SAKURA_PAIRS_SYMMETRIC (the
 * default) each unordered pair is solved once, its two ordered increments
 * being exact negatives.  The symmetric FP64 step runs on systolic tiles,
 * whose partial sums take up to 8 x 6 x 8 ceil(n/32) n bytes of library
 * scratch (12 MB at n = 1024), below 4096 bodies, and in row-group phases
 * from there, whose partials take about n^2 / 2.7 bytes (0.1 GB at 16384);
 * the mixed form uses row groups under SAKURA_MIXED_RULE_HYP, and under the
 * literal rule the FP64 kernel of its size with an inline class test
 * (SAKURA_FLAG_TILES / SAKURA_FLAG_GROUPS force either kernel).  Where the symmetric scratch
 * would pass 16 GB the ordered kernel is used.  Systems of 2 <= n <= 20 in the
 * FP64 form with symmetric pairs and a non-learned guess run in one launch
 * of a single-block kernel that keeps the system in shared memory and packs
 * the pairs densely over its lanes (no scratch; SAKURA_FLAG_NO_SMALL turns
 * it off).
 *   state:  device double[6][n], updated in place.
 *   masses: device double[n], all > 0.
 *   n >= 1; dt any finite value (negative integrates backwards).
 * Errors: E_NOINIT, E_ARG (n < 1, order not in {2,1,-1,4,6,8}, NULL
 * pointer, non-finite dt); device faults as described above.
 * Stream capture: once a call with the same n, order and configuration has
 * sized the library scratch, a call enqueues kernels on the library stream
 * only (no allocation, no synchronisation unless SAKURA_FLAG_SYNC_CHECK or
 * SAKURA_FLAG_TIMING is set), so runs of steps can be captured into a CUDA
 * graph and replayed. */
int sakura_step(double *state, const double *masses, int64_t n, double dt, int order);

/* nsteps consecutive steps of sakura_step on a device state, in place,
 * asynchronous.  Systems that sakura_step runs in the single-block kernel
 * take all nsteps steps in one launch (the state stays in shared memory
 * between steps); other systems take nsteps sakura_step calls.  nsteps >= 0
 * (0: nothing).  Arguments, errors and stream capture as for sakura_step. */
int sakura_evolve(double *state, const double *masses, int64_t n, double dt, int order,
                  int nsteps);

/* nsteps consecutive steps on HOST buffers: copies state and masses to
 * library-owned device memory, runs the steps, copies the state back and
 * synchronises.  state: host double[6][n]; masses: host double[n].  order
 * as for sakura_step.  Errors as for sakura_step; the call returns (and
 * clears) every device fault pending on the library stream.
 * Page-locked buffers mapped into the device's address space (cudaHostAlloc,
 * cudaMallocHost, or cudaHostRegister, under the unified addressing of
 * 64-bit Linux), with nsteps >= 1: no copy-engine transfers.  The first
 * sub-step's drift kernel reads state and masses in place and the last
 * sub-step's apply kernel writes state in place; sub-steps in between run in
 * library memory.  Both buffers are checked at their first and last byte,
 * and each must be one allocation of at least the stated size.  Pageable
 * buffers are staged through library memory with cudaMemcpyAsync.  Systems
 * of the single-block kernel (see sakura_step) take all nsteps steps in one
 * launch, which reads and writes the mapped buffers directly. */
int sakura_evolve_host(double *state, const double *masses, int64_t n, double dt,
                       int order, int nsteps);

/* Total energy E = sum_i m_i v_i^2 / 2 - sum_{i<j} m_i m_j / r_ij
 * (Eqs. 1-3), accumulated in double-double.  state, masses: device, as
 * above.  *E_out: host double.  Synchronises.  E_COINCIDENT if some r_ij = 0. */
int sakura_energy(const double *state, const double *masses, int64_t n, double *E_out);

/* Many independent systems in one persistent launch (the paper's method
 * applied to each system separately).  The systems are packed end to end:
 * system k owns particles offsets[k] .. offsets[k+1]-1 of state (device
 * double[6][total], total = offsets[nsys]) and masses (device double[total]).
 *   offsets: device int64[nsys+1]; host_offsets: the same values on the host
 *   (used to build the work schedule, rebuilt when they change);
 *   dt: device double[nsys], one step size per system.
 * Runs nsteps steps of the given order (2, 1, -1, 4, 6, 8) on every system, state
 * updated in place.  Each unordered pair of a system is solved once per
 * step.  A block runs all steps of its systems (up to 64 particles in all)
 * with the state in shared memory; their pairs are packed densely over its
 * warps' lanes and each particle's increments are summed over its own
 * system in a fixed order (results independent of the packing and of the
 * block shape); the launch is a CUDA
 * graph (counter reset + kernel), built once per (buffers, schedule, nsteps,
 * order, block shape) and replayed.  The first call with a new schedule
 * times the candidate block shapes (1, 2, 4, 8 warps) on a scratch copy and
 * keeps the fastest unless SAKURA_FLAG_NO_AUTOTUNE is set or
 * cfg.block_warps / cfg.grid_blocks fix it.
 * Systems need 1 <= N <= SAKURA_BATCH_MAX_N particles (else SAKURA_E_ARG). */
int sakura_step_batched(double *state, const double *masses, const int64_t *offsets,
                        const int64_t *host_offsets, int nsys, const double *dt, int order,
                        int nsteps);

/* The block shape the batched autotuner chose (warps per block, blocks) and
 * the time in ms it measured for 1, 2, 4 and 8 warps per block.
 * SAKURA_E_ARG if no batched call has been tuned yet. */
int sakura_batched_tuning(int *warps, int *blocks, double times_ms[4]);

/* The work schedule sakura_step_batched builds for these systems, on the
 * host (no device work, no sakura_init needed): tasks of at most 64
 * particles in all, each run by one block with its pairs packed densely over
 * the block's lanes, listed longest first.
 *   host_offsets: int64[nsys+1] as for sakura_step_batched;
 *   task_begin: caller's int[nsys+1], receives ntasks+1 offsets into task_sys;
 *   task_sys: caller's int[nsys], receives the systems of task t at
 *   task_sys[task_begin[t] .. task_begin[t+1]-1], every system exactly once;
 *   ntasks: receives the number of tasks.
 * Errors: E_ARG (null pointer, nsys < 1, host_offsets[0] != 0, a system of
 * N < 1 or N > SAKURA_BATCH_MAX_N). */
int sakura_batched_schedule(const int64_t *host_offsets, int nsys, int *task_begin,
                            int *task_sys, int *ntasks);

/* The precision class that the mixed form (SAKURA_PREC_MIXED) gives every
 * ordered pair of the step of this order (2, 1 or -1) that starts from
 * state, under the configured rule and thresholds (cfg.mixed_rule,
 * mixed_r_min, mixed_e_max, mixed_e_hyp).  The rule is stated on the pair's
 * Kepler input (r0, v0) of Eq. 26 (after the first drift of Eq. 27a and the
 * backward drift of Eq. 17), with m = m_i + m_j: single precision iff
 * r = |r0| > r_min and e < e_max (or e > e_hyp under
 * SAKURA_MIXED_RULE_HYP), e^2 = 1 + 2 (v0^2/2 - m/r) |r0 x v0|^2 / m^2.
 * The library decides it in single precision, as the mixed pair kernels do
 * (the same device code), so pairs within rounding of a threshold may be
 * classed either way.  A pair of class 1 whose single-precision solve fails
 * is still solved in FP64 by the step.
 *   state, masses: device arrays as for sakura_step; n <= 2^20.
 *   classes: device uint8[n][n]; classes[i * n + j] = 1 for the pair (i, j)
 *   in single precision, 0 in FP64; the diagonal is 0.
 * Uses the library scratch; synchronises and returns device faults.
 * Errors: E_NOINIT, E_ARG (null pointer, n < 1 or n > 2^20, order not in
 * {2, 1, -1}, non-finite dt). */
int sakura_pair_classes(const double *state, const double *masses, int64_t n, double dt,
                        int order, unsigned char *classes);

/* ---- learned initial guess ------------------------------------------
 * The paper leaves the Kepler solver's starting value open (Sec. 2.3 only
 * names a universal-variable solver).  With cfg.guess = SAKURA_GUESS_LEARNED
 * the second-order guess s_T2 is refined by a 6-64-64-1 tanh perceptron:
 *   s0 = s_T2 exp(w g(x)), w = q/(1+q), q = tau'^2 (1 + eta'^2 + |beta'|),
 * tau' = |t| sqrt(m/r0^3), eta' = sign(t) eta0/sqrt(m r0), beta' = beta r0/m,
 * x = (log tau', asinh eta', asinh beta', tanh(eta' tau'), tanh(beta' tau'^2),
 * w) normalised, g clamped to [-4, 4]; a warp of 32 pairs that all have
 * w <= 1e-4 keeps s_T2 without evaluating the network.  The convergence test, the bracket and
 * the bisection fallback are unchanged, so results do not depend on the
 * network.  Inference runs inside the pair kernels with BF16 mma.sync (FP32
 * accumulation), weights in shared memory.  Training runs on the GPU with the
 * kernels below (FP32). */

/* Load the network: weights is a host float32 array laid out as
 * W1[64][6], b1[64], W2[64][64], b2[64], W3[64], b3[1], then the input
 * normalisation mean[6], scale[6] and the output scale, shift (2 floats):
 * 6*64+64+64*64+64+64+1+6+6+2 = 4687 floats.  bytes must equal 4687*4; all
 * values finite and the six input scales > 0 (else SAKURA_E_ARG).
 * Synchronises.  Steps with SAKURA_GUESS_LEARNED before a load return
 * SAKURA_E_ARG. */
int sakura_load_mlp(const void *weights, size_t bytes);

/* Training data from the method itself: for the ordered pairs
 * pair_ids[k] = i * n + j (device int64[count]) of the step of order `order`
 * that starts from state (device double[6][n]) with masses (device double[n]),
 * runs each pair's FP64 Kepler solve (Eq. 18, standard guess) and writes the
 * features (device float[count][6]) and the target g = log(s / s_T2) / w
 * (device float[count]); iters (device int[count] or NULL) receives the
 * evaluations the standard guess needed.  Synchronises; device faults are
 * returned. */
int sakura_sample_pairs(const double *state, const double *masses, int64_t n, double dt,
                        int order, const int64_t *pair_ids, int64_t count, float *features,
                        float *targets, int *iters);

/* Mean squared error of the network with FP32 parameters params (device
 * float[4673], layout as the first 4673 floats of the load blob) on a batch
 * of raw features (device float[batch][6]) normalised by norm (device
 * float[12]: mean[6], scale[6]) against targets (device float[batch]); writes
 * the gradient (device float[4673]) and the loss (device float[1]).
 * Synchronises. */
int sakura_mlp_grad(const float *params, const float *norm, const float *features,
                    const float *targets, int64_t batch, float *grad, float *loss);

/* Adam training (lr, beta1 = 0.9, beta2 = 0.999) of params (device
 * float[4673], updated in place) for `epochs` passes over nsamples samples in
 * consecutive minibatches of `batch` (shuffle the data beforehand).  losses:
 * device float[epochs * (nsamples / batch)] receiving each minibatch loss, or
 * NULL.  Synchronises. */
int sakura_mlp_train(float *params, const float *norm, const float *features,
                     const float *targets, int64_t nsamples, int64_t batch, int epochs, float lr,
                     float *losses);

/* The loaded network's output g (after output scaling and clamping) for raw
 * features (device float[count][6]) into out (device float[count]), with the
 * same BF16 warp inference the pair kernels use.  Synchronises. */
int sakura_mlp_eval(const float *features, int64_t count, float *out);

/* Copy the accumulated statistics (SAKURA_FLAG_STATS) and reset them if
 * reset != 0.  Synchronises. */
int sakura_get_stats(sakura_stats *out, int reset);

/* Synchronise the library stream and return the first pending device fault
 * (and clear it), or SAKURA_OK. */
int sakura_check(void);

/* An FP64 step for callers that cannot allocate device memory: programs
 * whose GPU memory is owned by another allocator (a framework's caching
 * allocator that has reserved the device would make cudaMalloc fail) and
 * latency-critical loops that must not call cudaMalloc/cudaFree.  The paper
 * has no counterpart; this is an interface convenience.  It needs no
 * sakura_init, reads no sakura_config and allocates nothing.  It always runs
 * the ordered-pair FP64 kernels (SAKURA_PAIRS_ORDERED: every ordered pair
 * solved) with the standard initial guess t/r0 and the default Kepler
 * controls (tolerance 4 eps, 50 Laguerre steps, bisection fallback), so its
 * results equal sakura_step's in that configuration to summation order.
 * Its scratch (drifted state and row sums, 20 x SAKURA_NOALLOC_MAX_N
 * doubles = 10 MiB) and its fault status word are file-scope device arrays
 * that every GPU loading the library holds until the process exits.
 *   state, masses: device arrays as for sakura_step; n <= SAKURA_NOALLOC_MAX_N
 *   (larger n returns SAKURA_E_ARG); order 2, 1 or -1; stream: cudaStream_t
 *   or NULL.
 * Runs on the calling thread's current device and synchronises the stream
 * before returning the first device fault of this call (or SAKURA_OK).
 * The first call on a device looks up the arrays' device addresses; make it
 * before any stream capture.  Host threads may make first calls
 * concurrently (the look-up runs once per device).  All calls share the
 * arrays and keep the last call's contents; calls that overlap on the GPU
 * (other streams, other threads) race on them. */
#define SAKURA_NOALLOC_MAX_N 65536
int sakura_step_noalloc(double *state, const double *masses, int64_t n, double dt, int order,
                        void *stream);

/* Static description of a return code. */
const char *sakura_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* SAKURA_H */
