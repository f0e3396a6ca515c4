// pair.cuh -- tile configurations and parameters of the FP32 pair-moment
// kernel (kernels_pair.cu); shared with the host planner and the autotuner.
#pragma once

#include <stdint.h>

#include "common.cuh"

namespace lg {

// Tile configurations of the FP32 pair-moment kernel.  A warp owns wi x wj
// ordered pairs (i, j) and its 32 lanes split the samples; wgi x wgj warps
// form the CTA tile (wi wgi) x (wj wgj); `stages` chunk buffers of PAIR_S
// samples sit in shared memory, filled by TMA (thread 0 issues the copies).
// The register caps set how many CTAs share an SM in each form.  The
// autotuner picks a configuration and a split schedule per range of p.
struct PairCfg {
    int wi, wj, wgi, wgj, stages;
    int reg_fast, reg_acc;   // register cap per thread (fast / accurate form)
    int groups;              // groups of 4 samples per lane and iteration (1 or 2)
    int fold;                // chunks between compensated folds of the FP32 partial sums
    int packed;              // fast form: two samples per paired-FP32 instruction
    int sub;                 // 0: one chunk per ring stage (pair_block); >= 1: the streamlined
                             // block (pair_block_v2) with `sub` chunks per stage
    int absadd;              // streamlined paired form: 1 sums |u| as f32x2 pairs
    int hmajor;              // streamlined paired form: 1 loads every row first and runs the
                             // sample steps outermost (all WI x WJ pairs per step)
    constexpr int ti() const { return wi * wgi; }
    constexpr int tj() const { return wj * wgj; }
    constexpr int warps() const { return wgi * wgj; }
    constexpr int threads() const { return 32 * wgi * wgj; }
};
constexpr PairCfg PAIR_CFGS[] = {
    {4, 4, 2, 4, 4, 248, 128, 1, 4},   // 0: 256 threads, 8 x 16 tile
    {4, 4, 1, 4, 3, 168, 128, 1, 4},   // 1: 128 threads, 4 x 16 tile
    {4, 2, 2, 4, 4, 128, 96, 1, 4},    // 2: 256 threads, 8 x 8 tile
    {2, 4, 2, 4, 4, 128, 96, 1, 4},    // 3: 256 threads, 4 x 16 tile
    {4, 4, 2, 2, 4, 168, 128, 1, 4},   // 4: 128 threads, 8 x 8 tile
    {4, 4, 1, 4, 3, 168, 168, 2, 4},   // 5: as 1, 8 samples per lane and iteration
    {4, 2, 1, 4, 3, 128, 96, 2, 4},    // 6: 128 threads, 4 x 8 tile, 8 samples per lane
    {4, 2, 2, 4, 4, 128, 96, 2, 4},    // 7: as 2, 8 samples per lane
    {2, 4, 2, 4, 4, 128, 96, 2, 4},    // 8: as 3, 8 samples per lane
    {4, 2, 1, 4, 3, 128, 96, 2, 8},    // 9: as 6, folds every 8 chunks
    {4, 2, 1, 4, 3, 128, 96, 2, 8, 1}, // 10: as 9, paired FP32 (f32x2) arithmetic
    {4, 4, 1, 4, 3, 168, 168, 2, 8, 1},// 11: as 5, paired, folds every 8 chunks
    {4, 2, 2, 4, 4, 128, 96, 2, 8, 1}, // 12: as 7, paired, folds every 8 chunks
    {2, 2, 1, 4, 3, 80, 80, 2, 8, 1},  // 13: 128 threads, 2 x 8 tile, paired, 6 CTAs per SM
    {2, 2, 2, 4, 4, 80, 80, 2, 8, 1},  // 14: 256 threads, 4 x 8 tile, paired, 3 CTAs per SM
    {4, 2, 1, 4, 3, 96, 96, 2, 8, 1},  // 15: as 10 with 96 registers, 5 CTAs per SM
    // streamlined block: row-by-row loads, float2 S2 sums kept across chunks,
    // incremental ring bookkeeping, `sub` chunks per ring stage
    {4, 2, 1, 4, 2, 128, 128, 2, 8, 1, 2},   // 16: 4 x 8 tile, 2 stages of 2 chunks, 4 CTAs per SM
    {2, 2, 1, 4, 2, 80, 80, 2, 8, 1, 2},     // 17: 2 x 8 tile, 2 stages of 2 chunks, 5 CTAs per SM
    {4, 2, 2, 4, 2, 128, 128, 2, 8, 1, 2},   // 18: 8 x 8 tile, 256 threads, 2 CTAs per SM
    {2, 2, 2, 4, 2, 80, 80, 2, 8, 1, 2},     // 19: 4 x 8 tile, 256 threads, 3 CTAs per SM
    {4, 2, 1, 4, 3, 96, 96, 2, 8, 1, 1},     // 20: as 15, streamlined
    {2, 2, 1, 4, 3, 80, 80, 2, 8, 1, 1},     // 21: as 13, streamlined, 6 CTAs per SM
    {2, 2, 2, 4, 3, 80, 80, 2, 8, 1, 2},     // 22: as 19 with 3 stages
    {2, 2, 2, 4, 2, 80, 80, 2, 8, 1, 4},     // 23: as 19 with stages of 4 chunks, 2 CTAs per SM
    {2, 2, 2, 4, 3, 80, 80, 2, 16, 1, 2},    // 24: as 22, folds every 16 chunks
    {4, 2, 1, 4, 2, 128, 128, 2, 16, 1, 2},  // 25: as 16, folds every 16 chunks
    {2, 2, 2, 4, 3, 80, 80, 2, 16, 1, 2, 1}, // 26: as 24, |u| sums as f32x2 pairs
    {4, 2, 1, 4, 2, 128, 128, 2, 16, 1, 2, 1}, // 27: as 25, |u| sums as f32x2 pairs
    {2, 4, 2, 2, 3, 128, 128, 2, 16, 1, 2, 1}, // 28: 2 x 4 pairs per warp, 4 x 8 tile, 3 CTAs per SM
    {4, 2, 2, 4, 2, 128, 128, 2, 16, 1, 2, 1}, // 29: as 27 with 8 warps (8 x 8 tile), 2 CTAs per SM
    {4, 2, 1, 4, 3, 128, 128, 2, 16, 1, 2, 1}, // 30: as 27 with 3 stages, 3 CTAs per SM
    {4, 2, 1, 4, 2, 128, 128, 2, 16, 1, 2, 1, 1}, // 31: as 27, sample steps outermost
    {2, 2, 2, 4, 3, 80, 80, 2, 16, 1, 2, 1, 1},   // 32: as 26, sample steps outermost
};
constexpr int PAIR_NCFG = (int)(sizeof(PAIR_CFGS) / sizeof(PAIR_CFGS[0]));
constexpr int PAIR_S = 256;                  // samples per TMA chunk
static_assert(SHARD_BLOCK % 16 == 0, "tile sides (at most 16) divide the shard block");

// Scale folded into the fast-form residual: u~ = KSC * u makes
// 2^(-u~^2) = exp(-u^2/2).
constexpr double KSC = 0.84932180028801904272;   // sqrt(log2(e) / 2)

enum PairMode { PAIR_ACCURATE = 0, PAIR_FAST = 1 };

struct PairParams {
    const double *C;      // FP64 covariance of the residual data, [d][ldc]
    int64_t ldc;
    const int32_t *U;     // position -> original variable, p entries
    int p, n;
    int tiles_i, tiles_j;
    int nchunks;          // ceil(n / PAIR_S)
    int cps;              // chunks per sample split
    int nsplit;
    float2 *mom;          // out [nsplit][p][p][2] moment sums of entry (i, j), each as a
                          // double-float (hi, lo)
    uint32_t *status;
    int row0;             // first row of this instance in the z tensor
    const double *isd;    // [p] 1 / sqrt(C_ii) by position
    int shard_rank, shard_n;   // shard_n > 1: only tiles this rank owns (shard_owner)
    float *ra;            // out [p][p] 1 / sqrt(1 - rho_ij^2) (FP32, as the score kernel's
                          // error model takes it), written by the first sample split
};

}  // namespace lg
