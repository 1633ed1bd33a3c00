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
// Work is split in phase-steps.  The units (g, t, k), step k of phase t of
// group g, are numbered group by group, phase by phase:
// u = 32 (grp_before(g) + t) + k, U = 32 grp_before(ng) in all.  Every unit
// takes the same time whatever number of the block's warps hold a tile in
// its phase: the two blocks on an SM share its FP64 pipe warp by warp, so a
// block's warps advance one step in the same time whether or not its other
// warps are idle (a split by tiles instead gave the blocks holding many
// group starts, whose first phases have idle warps, the longest times).
// The units are dealt in chunks of S consecutive units (S = 1: single steps,
// for the FP64 kernel; S = 32: whole phases, for the mixed kernel, whose
// blocks' times vary with their pairs' classes more than with a phase's
// length, so that splitting phases would only add work): block b of a
// persistent grid of B blocks takes the units u with floor(floor(u / S) B /
// (U / S)) = b (grp_owner), a contiguous range starting at
// grp_block_start(b), U / B units to within one chunk, whatever the group
// and phase boundaries.  B <= U / 32 (the phase count) keeps at least one
// phase per block.  A block works its range in windows of up to a
// few phases of one group, with one block barrier and one reduction of the
// warps' column sums per window.  Partials:
//   colpart[g][6][n]  the column sums of phase (g, J) for the particles of
//                     column block J, from the block that holds its step 0;
//   colx[b][6][32]    the column sums of the phase in which block b starts,
//                     when b starts after its step 0 (a phase split between
//                     blocks; the apply kernel finds these from grp_owner);
//   rowpart[h][6][n]  the row sums of the particles of group g from the h-th
//                     block holding units of g, h = b - grp_owner(32
//                     grp_before(g)) < Hmax.
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
constexpr int kFp64GrpWarps = 4;   // G of the FP64 kernel (2 blocks of 4 warps per SM)
constexpr int kMixedGrpChunk = 32;  // S of the mixed kernel: whole phases
constexpr int kFp64GrpChunk = 1;    // S of the FP64 kernel: single steps

struct GrpLayout {
    int64_t nb;  // blocks of 32 particles
    int64_t U;   // phase-steps of all groups (32 per phase)
    int S;       // units per chunk: 1 or 32
    int rev;     // layout index i is particle n - 1 - i
    int ng;      // groups
    int G;       // row blocks per group (warps per block)
    int Hmax;    // most row pieces of a group for the grid it was made for
};

// row blocks of group g
GRP_HD int64_t grp_rows(const GrpLayout &L, int64_t g)
{
    const int64_t r = L.nb - g * L.G;
    return r < L.G ? r : L.G;
}

// phases of groups 0 .. g - 1 (group g' has nb - g' G of them)
GRP_HD int64_t grp_before(const GrpLayout &L, int64_t g)
{
    return g * L.nb - L.G * (g * (g - 1) / 2);
}

// the particle of layout index i (0 <= i < n)
GRP_HD int64_t grp_particle(const GrpLayout &L, int64_t n, int64_t i) { return L.rev ? n - 1 - i : i; }

// the block whose range holds unit u
GRP_HD int64_t grp_owner(int64_t u, int64_t B, const GrpLayout &L)
{
    return (u / L.S) * B / (L.U / L.S);
}

struct GrpPos {
    int64_t g, t;  // group, phase within the group
    int k;         // step within the phase
};

// the first unit of block b's range (for b = B: (ng, 0, 0), the end)
GRP_HD GrpPos grp_block_start(const GrpLayout &L, int64_t b, int64_t B)
{
    const int64_t nc = L.U / L.S;
    const int64_t u = (b * nc + B - 1) / B * L.S;  // the first chunk c with c B >= b nc
    if (u >= L.U) return GrpPos{L.ng, 0, 0};
    const int64_t p = u >> 5;
    int64_t lo = 0, hi = L.ng - 1;  // the last group starting at or before phase p
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if (grp_before(L, mid) <= p)
            lo = mid;
        else
            hi = mid - 1;
    }
    return GrpPos{lo, p - grp_before(L, lo), (int)(u & 31)};
}

// the layout for n particles with G row blocks per group, chunks of S units
// and the particles in reverse order if rev; clamps blocks to [1, phases]
inline GrpLayout make_grp_layout(int64_t n, int G, int S, bool rev, int64_t &blocks)
{
    GrpLayout L;
    L.nb = (n + 31) / 32;
    L.G = G;
    L.S = S;
    L.rev = rev ? 1 : 0;
    L.ng = (int)((L.nb + G - 1) / G);
    L.U = 32 * grp_before(L, L.ng);
    const int64_t cap = L.U / 32;
    blocks = blocks < cap ? blocks : cap;
    if (blocks < 1) blocks = 1;
    L.Hmax = 1;
    for (int64_t g = 0; g < L.ng; ++g) {
        const int64_t u0 = 32 * grp_before(L, g), u1 = 32 * grp_before(L, g + 1) - 1;
        const int64_t h = grp_owner(u1, blocks, L) - grp_owner(u0, blocks, L) + 1;
        if (h > L.Hmax) L.Hmax = (int)h;
    }
    return L;
}

}  // namespace sakura
