// grp_layout.cuh -- the row-group layout of the symmetric kernels: which
// tile-steps each block of a persistent grid takes and where it writes its
// partial sums.  Plain integer arithmetic, built for the device and the host
// (the host builds the layout; tests check it against an enumeration).
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define GRP_HD __host__ __device__ __forceinline__
#else
#define GRP_HD inline
#endif

namespace sakura {

// Row-group phases of the symmetric (Newton's third law) FP64 and mixed
// kernels (step_grp.cu, step_mixed.cu).  The n particles form nb blocks of
// 32; a group is G consecutive row blocks (G = 8 for the mixed kernel, 4 for
// the FP64 one; the last group has R_g = nb - g G < G of them when G does not
// divide nb).  Group g meets the column blocks J = g G .. nb - 1 in
// L_g = nb - g G phases; phase t (J = g G + t) holds the tiles (g G + r, J)
// with r <= t, r < R_g, one per warp, each solved in 32 systolic steps.
//
// Work is split in steps.  The units (g, t, k), step k of phase t of group
// g, are ordered group by group, phase by phase.  A step of phase t costs
// c(g, t) = wA + wB min(t + 1, R_g): wA for the step's time and wB for each
// of its tiles.  The blocks on an SM share its FP64 pipe warp by warp, so a
// block whose phase has idle warps advances faster than one whose warps are
// all busy, but not in proportion to its tiles: measured on GB300, a step of
// the phases at a group's start (1 to 3 tiles of 4, two on average) took
// 0.64 of a full step with two blocks per SM (the double-word kernel keeps
// (wA, wB) = (2, 1)).  The FP64 kernel, now four blocks per SM with part of
// its multiplies on the integer pipes, measured fastest with steps counted
// alike, (1, 0): 20.43 ms per step at 16384 bodies, against 20.45 with
// (8, 1), 20.56 with (5, 1), 20.73 with (3, 1), 20.85 with (2, 1) and 21.16
// with (1, 1).  The mixed kernel, whose blocks' times vary with their
// pairs' classes more than with this, takes (1, 0) as well.  x(g, t, k), the cost of the
// units before (g, t, k), is grp_phase_x(g, t) + k c(g, t); C = x at the
// end.  The units are dealt in chunks of S consecutive steps of one phase
// (S = 1: single steps, for the FP64 kernel; S = 32: whole phases, for the
// mixed kernel): block b of a persistent grid of B blocks takes the chunks
// starting at an x with floor(x B / C) = b (grp_owner), a contiguous range
// that starts at grp_block_start(b), C / B to within one chunk's cost
// whatever the group and phase boundaries.  B <= C / (32 max c) keeps every
// range about a phase long or longer.  A block works its range in windows of
// up to a few phases of one group, with one block barrier and one reduction
// of the warps' column sums per window.  Partials:
//   colpart[g][6][n]  the column sums of phase (g, J) for the particles of
//                     column block J, from the block that holds its step 0;
//   colx[b][6][32]    the column sums of the phase in which block b starts,
//                     when b starts after its step 0 (a phase split between
//                     blocks; the apply kernel finds these from grp_owner);
//   rowpart[h][6][n]  the row sums of the particles of group g from the h-th
//                     block holding units of g, h = b - grp_owner(x(g, 0, 0))
//                     < Hmax.
// With rev set the layout numbers the particles from the end of the array
// (layout index i is particle n - 1 - i, grp_particle); the partials are
// indexed by layout index.  A particle's pairs with the particles after it
// are row pairs, all solved by the blocks holding its group, and its pairs
// with those before it column pairs, one phase in each earlier group; so the
// first particles of the layout carry most of their pairs in a few blocks.
// N-body initial conditions conventionally put a central massive body, whose
// pairs cost the most (closer orbits: more series terms and seed
// iterations), first in the array: taken last, its pairs are spread over
// every group's blocks.
constexpr int kGrpWindow = 4;
constexpr int kMixedGrpWarps = 8;  // G of the mixed kernel (2 blocks of 8 warps per SM)
constexpr int kFp64GrpWarps = 4;   // G of the FP64 kernel (blocks of 4 warps, 2 to 4 per SM)

struct GrpLayout {
    int64_t nb;  // blocks of 32 particles
    int64_t C;   // cost of all units
    int S;       // steps per chunk: 1 or 32
    int wA, wB;  // a step costs wA + wB x (tiles of its phase)
    int rev;     // layout index i is particle n - 1 - i
    int ng;      // groups
    int G;       // row blocks per group (warps per block)
    int Hmax;    // most row pieces of a group for the grid it was made for
};

// the layout of the FP64 kernel and of the mixed kernel
struct GrpShape {
    int G, S, wA, wB;
    bool rev;
};
constexpr GrpShape kFp64GrpShape{kFp64GrpWarps, 1, 1, 0, true};
constexpr GrpShape kMixedGrpShape{kMixedGrpWarps, 32, 1, 0, false};
// the double-word form (step_df64.cu): one block of 12 warps per SM, whose
// window barrier keeps the SM's warps together (in three blocks of 4 warps
// the warp scheduler's preference let one block end up to 1.4 ms before
// another on the same SM, the last then running alone at a low issue rate
// in this FP32-issue-bound kernel); whole phases (its loop stays free of
// range tests), a step costing 2 + its tiles, particles reversed
constexpr int kDf64GrpWarps = 12;
constexpr GrpShape kDf64GrpShape{kDf64GrpWarps, 32, 2, 1, true};

// row blocks of group g (0 past the last group)
GRP_HD int64_t grp_rows(const GrpLayout &L, int64_t g)
{
    const int64_t r = L.nb - g * L.G;
    return r < 0 ? 0 : (r < L.G ? r : L.G);
}

// phases of groups 0 .. g - 1 (group g' has nb - g' G of them)
GRP_HD int64_t grp_phases_before(const GrpLayout &L, int64_t g)
{
    return g * L.nb - L.G * (g * (g - 1) / 2);
}

// tiles of phases 0 .. t - 1 of a group of R row blocks
GRP_HD int64_t grp_ramp(int64_t t, int64_t R)
{
    return t <= R ? t * (t + 1) / 2 : R * (R + 1) / 2 + (t - R) * R;
}

// tiles of groups 0 .. g - 1: a full group g' has G nb - G^2 g' - G (G - 1)/2
// of them, a last group of R < G row blocks R (R + 1) / 2
GRP_HD int64_t grp_tiles_before(const GrpLayout &L, int64_t g)
{
    const int64_t G = L.G, full = L.nb / G, gf = g < full ? g : full;
    int64_t c = gf * (G * L.nb - G * (G - 1) / 2) - G * G * (gf * (gf - 1) / 2);
    if (g > full) {
        const int64_t R = L.nb - full * G;
        c += R * (R + 1) / 2;
    }
    return c;
}

// cost of one step of phase t of group g
GRP_HD int64_t grp_step_cost(const GrpLayout &L, int64_t g, int64_t t)
{
    const int64_t R = grp_rows(L, g), c = t + 1 < R ? t + 1 : R;
    return L.wA + L.wB * c;
}

// cost of the units before phase t of group g (t = 0: before the group)
GRP_HD int64_t grp_phase_x(const GrpLayout &L, int64_t g, int64_t t)
{
    return 32 * (L.wA * (grp_phases_before(L, g) + t) +
                 L.wB * (grp_tiles_before(L, g) + grp_ramp(t, grp_rows(L, g))));
}

// cost before the last chunk of phase t of group g
GRP_HD int64_t grp_phase_last_x(const GrpLayout &L, int64_t g, int64_t t)
{
    return grp_phase_x(L, g, t) + (32 - L.S) * grp_step_cost(L, g, t);
}

// the particle of layout index i (0 <= i < n)
GRP_HD int64_t grp_particle(const GrpLayout &L, int64_t n, int64_t i) { return L.rev ? n - 1 - i : i; }

// the block whose range holds the chunk with cost x before it
GRP_HD int64_t grp_owner(int64_t x, int64_t B, const GrpLayout &L) { return x * B / L.C; }

struct GrpPos {
    int64_t g, t;  // group, phase within the group
    int k;         // step within the phase
};

// the first unit of block b's range (for b = B: (ng, 0, 0), the end): the
// first chunk whose x is at least ceil(b C / B)
GRP_HD GrpPos grp_block_start(const GrpLayout &L, int64_t b, int64_t B)
{
    const int64_t X = (b * L.C + B - 1) / B;
    if (X >= L.C) return GrpPos{L.ng, 0, 0};
    int64_t lo = 0, hi = L.ng - 1;  // the last group with x(g, 0, 0) <= X
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if (grp_phase_x(L, mid, 0) <= X)
            lo = mid;
        else
            hi = mid - 1;
    }
    const int64_t g = lo, Lg = L.nb - g * L.G, R = grp_rows(L, g);
    // the last phase with x(g, t, 0) <= X: past the first R phases x grows
    // by 32 (wA + wB R) per phase
    const int64_t xr = grp_phase_x(L, g, R < Lg ? R : Lg);
    int64_t t;
    if (R < Lg && X >= xr) {
        t = R + (X - xr) / (32 * (L.wA + L.wB * R));
        if (t > Lg - 1) t = Lg - 1;
    } else {
        t = 0;
        while (t + 1 < Lg && grp_phase_x(L, g, t + 1) <= X) ++t;
    }
    const int64_t c = grp_step_cost(L, g, t);
    int64_t k = (X - grp_phase_x(L, g, t) + c - 1) / c;  // the first step with x >= X
    k = (k + L.S - 1) / L.S * L.S;                        // ... that starts a chunk
    if (k < 32) return GrpPos{g, t, (int)k};
    if (t + 1 < Lg) return GrpPos{g, t + 1, 0};
    return GrpPos{g + 1, 0, 0};
}

// the layout for n particles of the given shape; clamps blocks to
// [1, C / (32 max c)] (each block's range about a phase long or longer)
inline GrpLayout make_grp_layout(int64_t n, const GrpShape &shape, int64_t &blocks)
{
    GrpLayout L;
    L.nb = (n + 31) / 32;
    L.G = shape.G;
    L.S = shape.S;
    L.wA = shape.wA;
    L.wB = shape.wB;
    L.rev = shape.rev ? 1 : 0;
    L.ng = (int)((L.nb + L.G - 1) / L.G);
    L.C = grp_phase_x(L, L.ng, 0);
    const int64_t cap = L.C / (32 * (L.wA + L.wB * L.G));
    blocks = blocks < cap ? blocks : cap;
    if (blocks < 1) blocks = 1;
    L.Hmax = 1;
    for (int64_t g = 0; g < L.ng; ++g) {
        const int64_t x1 = grp_phase_last_x(L, g, L.nb - g * L.G - 1);  // its last chunk
        const int64_t h = grp_owner(x1, blocks, L) - grp_owner(grp_phase_x(L, g, 0), blocks, L) + 1;
        if (h > L.Hmax) L.Hmax = (int)h;
    }
    return L;
}

}  // namespace sakura
