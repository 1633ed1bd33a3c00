// Host build of csrc/grp_layout.cuh for tests/test_grp_layout_host.py: the
// closed forms and the block ranges against a plain enumeration of the units.
#include "../paper_1402_3325_gb300/csrc/grp_layout.cuh"

#include <vector>

using namespace sakura;

// Checks the layout of n particles with G row blocks per group, chunks of S
// steps, step cost wA + wB x tiles, particles in reverse order if rev, on a
// grid of `blocks` blocks (clamped as the library clamps it).  out[0..6]:
// blocks used, total cost C, Hmax, the least and the most cost of a block,
// the number of blocks that start inside a phase, the largest chunk cost.
// Returns 0, or the number of the first check that failed.
extern "C" int grp_layout_check(long n, int G, int S, int wA, int wB, int rev, long blocks,
                                long *out)
{
    int64_t B = blocks;
    const GrpShape shape{G, S, wA, wB, rev != 0};
    const GrpLayout L = make_grp_layout(n, shape, B);
    if (L.nb != (n + 31) / 32 || L.ng != (L.nb + G - 1) / G) return 1;
    // layout index to particle: a permutation, the identity or the reversal
    std::vector<char> seen(n, 0);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t p = grp_particle(L, n, i);
        if (p < 0 || p >= n || seen[p] || p != (rev ? n - 1 - i : i)) return 2;
        seen[p] = 1;
    }
    // enumerate the chunks in order: the cost before each, its owner
    std::vector<int64_t> first(B, -1), cost(B, 0);
    std::vector<GrpPos> cp;
    int64_t x = 0, prev_owner = 0, phases = 0, tiles = 0, cmaxchunk = 0;
    int hmax = 0;
    for (int64_t g = 0; g < L.ng; ++g) {
        const int64_t R = L.nb - g * G < G ? L.nb - g * G : G;
        if (grp_rows(L, g) != R) return 3;
        if (grp_phases_before(L, g) != phases || grp_tiles_before(L, g) != tiles) return 4;
        int64_t gfirst = -1, glast = -1;
        for (int64_t t = 0; t < L.nb - g * G; ++t, ++phases) {
            int64_t c = 0;  // tiles of the phase: rows r <= t
            for (int64_t r = 0; r < R; ++r) c += (r <= t) ? 1 : 0;
            tiles += c;
            const int64_t w = wA + wB * c;  // cost of one step
            if (grp_step_cost(L, g, t) != w || grp_phase_x(L, g, t) != x) return 5;
            int64_t pf = -1, pl = -1;
            for (int k = 0; k < 32; k += S) {
                const int64_t b = grp_owner(x, B, L);
                if (b < prev_owner || b >= B) return 6;  // owners ascend and stay in range
                if (first[b] < 0) {
                    if (b > 0 && first[b - 1] < 0) return 7;  // no empty block
                    first[b] = (int64_t)cp.size();
                }
                prev_owner = b;
                if (gfirst < 0) gfirst = b;
                glast = b;
                if (pf < 0) pf = b;
                pl = b;
                cost[b] += S * w;
                cmaxchunk = S * w > cmaxchunk ? S * w : cmaxchunk;
                cp.push_back(GrpPos{g, t, k});
                x += S * w;
            }
            // the owners of a phase's chunks are those the apply kernel
            // derives from its first and last chunk
            if (pf != grp_owner(grp_phase_x(L, g, t), B, L) ||
                pl != grp_owner(grp_phase_last_x(L, g, t), B, L))
                return 8;
        }
        if (glast - gfirst + 1 > hmax) hmax = (int)(glast - gfirst + 1);
    }
    if (x != L.C || grp_phase_x(L, L.ng, 0) != x) return 9;
    if (B < 1 || (B > 1 && B > x / (32 * (wA + wB * G)))) return 10;
    if (L.Hmax != hmax) return 11;
    if (first[B - 1] < 0) return 12;
    long starts_inside = 0;
    for (int64_t b = 0; b <= B; ++b) {
        const GrpPos p = grp_block_start(L, b, B);
        if (b == B) {
            if (p.g != L.ng || p.t != 0 || p.k != 0) return 13;
            continue;
        }
        const GrpPos &q = cp[first[b]];
        if (p.g != q.g || p.t != q.t || p.k != q.k) return 14;
        if (p.k > 0) ++starts_inside;
    }
    int64_t lo = cost[0], hi = cost[0];
    for (int64_t b = 1; b < B; ++b) {
        lo = cost[b] < lo ? cost[b] : lo;
        hi = cost[b] > hi ? cost[b] : hi;
    }
    out[0] = (long)B;
    out[1] = (long)L.C;
    out[2] = L.Hmax;
    out[3] = (long)lo;
    out[4] = (long)hi;
    out[5] = starts_inside;
    out[6] = (long)cmaxchunk;
    return 0;
}
