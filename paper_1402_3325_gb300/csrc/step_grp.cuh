// step_grp.cuh -- the row-group kernels (step_grp.cu: FP64; step_mixed.cu:
// mixed form) and their apply kernel: launchers and the partial-sum
// buffers.  Only their sources and the host code include it, so that the
// row-group layout (grp_layout.cuh) is no part of the other kernels' sources.
#pragma once

#include "grp_layout.cuh"
#include "step_common.cuh"

namespace sakura {

// the partial sums of a row-group step: row [Hmax][6][n], col [ng][6][n],
// colx [blocks][6][32] (grp_layout.cuh)
struct GrpParts {
    double *row, *col, *colx;
};
// a.X32 (the float copy, as ma.X32) set: FP64-class pairs seeded by a
// single-precision solve
void launch_pair_step_grp_mixed(const StepArgs &a, const MixedArgs &ma, const GrpLayout &L,
                                const GrpParts &parts, int blocks, bool stats, cudaStream_t s);
int pair_step_grp_mixed_blocks_per_sm(bool stats, bool seed);
// Eqs. 27b-d for the row-group layout; fuse: also the next sub-step's drift
// (next_drift), writing its drifted copy to X (and X32, if not null) as the
// prep kernel would, so that a run of steps needs no prep kernel after its
// first
void launch_apply_grp(double *state, double *X, float *X32, const GrpParts &parts, int64_t n,
                      const GrpLayout &L, int64_t blocks, double post_drift, bool fuse,
                      double next_drift, unsigned *status, cudaStream_t s);
// the symmetric FP64 pair kernel in row-group phases (a.mlp: learned guess;
// a.X32: single-precision seed; a.mixed: the mixed form's inline class test,
// a.mixed == 2 with the seed, as in launch_pair_step_sym)
void launch_pair_step_grp(const StepArgs &a, const GrpLayout &L, const GrpParts &parts,
                          int blocks, bool stats, cudaStream_t s);
int pair_step_grp_blocks_per_sm(bool stats, bool learned, bool seed, bool mixed = false);
// the double-word form in row-group phases (step_df64.cu): X3 from
// launch_prep_df64, partial sums in FP64 for launch_apply_grp
void launch_pair_step_grp_df64(const StepArgs &a, const DwArgs &da, const GrpLayout &L,
                               const GrpParts &parts, int blocks, bool stats, cudaStream_t s);
int pair_step_grp_df64_blocks_per_sm(bool stats);

}  // namespace sakura
