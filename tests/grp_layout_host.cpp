// Host build of csrc/grp_layout.cuh for tests/test_grp_layout_host.py: the
// closed forms and the block ranges against a plain enumeration of the units.
#include "../paper_1402_3325_gb300/csrc/grp_layout.cuh"

#include <vector>

using namespace sakura;

// Checks the layout of n particles, G row blocks per group, chunks of S
// units, particles in reverse order if rev, on a grid of `blocks` blocks
// (clamped as the library clamps it).  out[0..5]: blocks used,
// total units U, Hmax, the least and the most units of a block, the number
// of blocks that start inside a phase.  Returns 0, or the number of the
// first check that failed.
extern "C" int grp_layout_check(long n, int G, int S, int rev, long blocks, long *out)
{
    int64_t B = blocks;
    const GrpLayout L = make_grp_layout(n, G, S, rev != 0, B);
    if (L.nb != (n + 31) / 32 || L.ng != (L.nb + G - 1) / G) return 1;
    // layout index to particle: a permutation, the identity or the reversal
    std::vector<char> seen(n, 0);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t p = grp_particle(L, n, i);
        if (p < 0 || p >= n || seen[p] || p != (rev ? n - 1 - i : i)) return 14;
        seen[p] = 1;
    }
    // enumerate the units in order: their owners and each block's first
    std::vector<int64_t> first(B, -1), units(B, 0);
    std::vector<GrpPos> up;
    int64_t u = 0, prev_owner = 0, phases = 0;
    int hmax = 0;
    for (int64_t g = 0; g < L.ng; ++g) {
        const int64_t R = L.nb - g * G < G ? L.nb - g * G : G;
        if (grp_rows(L, g) != R) return 2;
        if (grp_before(L, g) != phases) return 3;
        int64_t gfirst = -1, glast = -1;
        for (int64_t t = 0; t < L.nb - g * G; ++t, ++phases) {
            int64_t pf = -1, pl = -1;
            for (int k = 0; k < 32; ++k, ++u) {
                const int64_t b = grp_owner(u, B, L);
                if (b != grp_owner(u - u % S, B, L)) return 13;  // chunks are not split
                if (b < prev_owner || b >= B) return 4;  // owners ascend and stay in range
                if (first[b] < 0) {
                    if (b > 0 && first[b - 1] < 0) return 5;  // no empty block
                    first[b] = (int64_t)up.size();
                }
                prev_owner = b;
                if (gfirst < 0) gfirst = b;
                glast = b;
                if (pf < 0) pf = b;
                pl = b;
                ++units[b];
                up.push_back(GrpPos{g, t, k});
            }
            // the owners of a phase's units are those the apply kernel
            // derives from its first and last unit
            const int64_t u0 = 32 * (grp_before(L, g) + t);
            if (pf != grp_owner(u0, B, L) || pl != grp_owner(u0 + 31, B, L)) return 6;
        }
        if (glast - gfirst + 1 > hmax) hmax = (int)(glast - gfirst + 1);
    }
    if (u != L.U || phases * 32 != L.U) return 7;
    if (B < 1 || (B > 1 && B > phases)) return 8;  // at least one phase per block
    if (L.Hmax != hmax) return 9;
    if (first[B - 1] < 0) return 10;
    long starts_inside = 0;
    for (int64_t b = 0; b <= B; ++b) {
        const GrpPos p = grp_block_start(L, b, B);
        if (b == B) {
            if (p.g != L.ng || p.t != 0 || p.k != 0) return 11;
            continue;
        }
        const GrpPos &q = up[first[b]];
        if (p.g != q.g || p.t != q.t || p.k != q.k) return 12;
        if (p.k > 0) ++starts_inside;
    }
    int64_t cmin = units[0], cmax = units[0];
    for (int64_t b = 1; b < B; ++b) {
        cmin = units[b] < cmin ? units[b] : cmin;
        cmax = units[b] > cmax ? units[b] : cmax;
    }
    out[0] = (long)B;
    out[1] = (long)L.U;
    out[2] = L.Hmax;
    out[3] = (long)cmin;
    out[4] = (long)cmax;
    out[5] = starts_inside;
    return 0;
}
