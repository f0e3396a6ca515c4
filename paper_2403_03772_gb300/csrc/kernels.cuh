// kernels.cuh -- launch interface between the host orchestration and kernels.
#pragma once

#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "df.cuh"
#include "pair.cuh"

namespace lg {

// High-precision pair moments (kernels_refine.cu): tier 1 double-float from
// the split standardised residuals, tier 2 FP64 from the residual data.
constexpr int HP_THREADS = 256;

struct HpParams {
    const double *R;      // tier 2: FP64 residual data [d][ldr] by original index
    int64_t ldr;
    const float *zhi;     // tier 1: standardised residuals z = zhi + zlo, [p][ldz]
    const float *zlo;     //   by position (same rows as the FP32 pair kernel)
    int64_t ldz;
    const double *isd;    // tier 1: [p] 1 / sqrt(C_ii) by position
    const double *C;
    int64_t ldc;
    const int32_t *U;
    int p, n;
    int mode;             // 0: all pairs + variables; 1: re-score of candidate rows
    int with_vars;        // mode 1: also the variable moments
    const DevState *state;
    double *mom;          // mode 0: [nsplit][p][p][2]; mode 1: [nsplit][d][p][4] by candidate slot
    double *hz;           // [nsplit][p][2] variable moment sums
    uint32_t *status;
    const float *I32;     // mode 1: [p][p] lower bound of I(i, j) from the FP32 scores,
                          // or null; entries with I32 >= 0 contribute 0 and are skipped
    int nsplit;           // sample ranges per work item (partial sums per range)
    int sps;              // samples per range
    int64_t mom_sstride;  // elements between the ranges' moment records
    int64_t woff;         // warp that takes this instance's first unit: the
                          // instances of one launch start where the previous
                          // one's expected units end, so all warps share the work
};

// Per-entry bound on |I_fp32(i, j) - I(i, j)| (FP32-scored steps).  Each of
// the four entropies of I is h(m1, m2) = -K1 (m1 - GAMMA)^2 - K2 m2^2, so a
// moment error (dm1, dm2) moves it by at most
//     2 K1 |m1 - GAMMA| dm1 + 2 K2 |m2| dm2 + K1 dm1^2 + K2 dm2^2.
// Residual moments: dm1 <= d1 + da a, dm2 <= d2 + da a with
// a = 1 / sqrt(1 - rho^2) (the FP32 residual a z_i - b z_j loses absolute
// accuracy in proportion to a); variable moments: dv1, dv2.
struct ErrModel {
    double d1, d2, da;    // residual-moment error terms of the pair kernel
    double dv1, dv2;      // variable-moment error terms (regress kernel)
};

struct ScoreParams {
    const double *mom;    // [nsplit][p][p][2] FP64 sums (steps scored in high precision)
    const float2 *mom2;   // or [nsplit][p][p][2] double-float sums from the FP32 pair kernel
    int nsplit, p, n;
    const double *hz;     // [nsplit_hz][p][2]
    int nsplit_hz;
    double a1, b1, a2;    // entry moments: m1 = a1 S1/n + b1, m2 = a2 S2/n
    double ha1, hb1, ha2; // variable moments, same form
    double epsI;          // fixed bound on |I - I_exact| unless use_model (0 when exact)
    int use_model;        // 1: per-entry bounds from `model` (FP32-scored steps)
    ErrModel model;
    const double *C;      // model: covariance by original index, and
    int64_t ldc;          //   1 / sqrt(C_ii) by position, for rho_ij
    const double *isd;
    const int32_t *U;
    double *M;            // out [p]
    double *E;            // out [p] error bound of M
    double *hist;         // optional [d][d] score history (row already offset)
    double *Iout;         // optional [p][p] I(i, j) by position (step-measure calls)
    float *I32;           // optional [p][p] lower bound of I(i, j) (rounded down), read by
                          // the re-score passes: entries with I32 >= 0 are skipped
    double *epsOut;       // optional [p][p] the entry bounds (step-measure calls)
    int shard_rank, shard_n;   // shard_n > 1 (FP32-scored steps): only owned entries count
    const float *ra;      // FP32-scored steps: [p][p] 1 / sqrt(1 - rho^2) from the pair kernel
    float4 *hvar;         // FP32-scored steps: [p] h(z_j) as (hi, lo) and its bound (k_hvar_b)
};

// Bound on the change of h(m1, m2) for moment errors (e1, e2), in FP32 (a
// bound needs no more precision; the 1 % factor covers its own rounding).
__device__ __forceinline__ float h_err(float m1, float m2, float e1, float e2)
{
    return 1.01f * (2.0f * (float)K1 * fabsf(m1 - (float)GAMMA) * e1 +
                    2.0f * (float)K2 * fabsf(m2) * e2 + (float)K1 * e1 * e1 +
                    (float)K2 * e2 * e2);
}

// h(z_j) of the variable at position j and its error term (0 without model).
__device__ __forceinline__ void score_var(const ScoreParams &P, int j, double invn, double &h,
                                         float &w)
{
    double S1 = 0.0, S2 = 0.0;
    for (int s = 0; s < P.nsplit_hz; ++s) {
        S1 += P.hz[((size_t)s * P.p + j) * 2 + 0];
        S2 += P.hz[((size_t)s * P.p + j) * 2 + 1];
    }
    const double m1 = P.ha1 * S1 * invn + P.hb1, m2 = P.ha2 * S2 * invn;
    h = neg_entropy_part(m1, m2);
    w = P.use_model ? h_err((float)m1, (float)m2, (float)P.model.dv1, (float)P.model.dv2) : 0.0f;
}

// h = -K1 (m1 - GAMMA)^2 - K2 m2^2 in double-float (the FP32-scored steps:
// their moment sums arrive as double-floats, so no FP64 arithmetic is needed
// per entry; GB300 runs FP64 at 1/75 of the FP32 rate).
constexpr float K1_HI = (float)K1, K1_LO = (float)(K1 - (double)(float)K1);
constexpr float K2_HI = (float)K2, K2_LO = (float)(K2 - (double)(float)K2);
constexpr float GAMMA_HI = (float)GAMMA, GAMMA_LO = (float)(GAMMA - (double)(float)GAMMA);

__device__ __forceinline__ dfl df_neg_entropy(dfl m1, dfl m2)
{
    const dfl a = df_add(m1, dfl{-GAMMA_HI, -GAMMA_LO});
    const dfl t1 = df_mul(df_mul(a, a), dfl{K1_HI, K1_LO});
    const dfl t2 = df_mul(df_mul(m2, m2), dfl{K2_HI, K2_LO});
    return df_neg(df_add(t1, t2));
}

// I(i, j) of an FP32-scored step in double-float from the double-float pair
// moment sums; c1, b1, c2 scale the sums to moments (m1 = c1 S1 + b1,
// m2 = c2 S2); hd holds h(z_j) as double-floats.  Also returns the FP32
// moments of both residuals for the error model.
__device__ __forceinline__ dfl score_entry_df(const ScoreParams &P, int i, int j, const dfl *hd,
                                              dfl c1, dfl b1, dfl c2, float (&mf)[4])
{
    const size_t plane = (size_t)P.p * P.p * 2;
    dfl a1{0.0f, 0.0f}, a2{0.0f, 0.0f}, e1{0.0f, 0.0f}, e2{0.0f, 0.0f};
    const float2 *pij = P.mom2 + ((size_t)i * P.p + j) * 2;
    const float2 *pji = P.mom2 + ((size_t)j * P.p + i) * 2;
    for (int s = 0; s < P.nsplit; ++s) {
        const float2 x1 = pij[s * plane], x2 = pij[s * plane + 1];
        const float2 y1 = pji[s * plane], y2 = pji[s * plane + 1];
        a1 = df_add(a1, dfl{x1.x, x1.y});
        a2 = df_add(a2, dfl{x2.x, x2.y});
        e1 = df_add(e1, dfl{y1.x, y1.y});
        e2 = df_add(e2, dfl{y2.x, y2.y});
    }
    const dfl mi1 = df_add(df_mul(a1, c1), b1), mi2 = df_mul(a2, c2);
    const dfl mj1 = df_add(df_mul(e1, c1), b1), mj2 = df_mul(e2, c2);
    mf[0] = mi1.hi;
    mf[1] = mi2.hi;
    mf[2] = mj1.hi;
    mf[3] = mj2.hi;
    const dfl hij = df_neg_entropy(mi1, mi2), hji = df_neg_entropy(mj1, mj2);
    return df_add(df_add(hd[j], hij), df_neg(df_add(hd[i], hji)));
}

// I(i, j) (Algorithm 1) of positions i != j from the pair moments and the
// variable entropies hsh, and its error bound eps: the fixed epsI, or the
// moment-error model (ErrModel) with a = 1 / sqrt(1 - rho_ij^2).  Every
// kernel that needs an entry's FP32 value or bound calls this, so they agree
// bit for bit.
__device__ __forceinline__ void score_entry(const ScoreParams &P, int i, int j, const double *hsh,
                                           const float *wsh, double invn, double &I, double &eps)
{
    const size_t plane = (size_t)P.p * P.p * 2;
    double a1 = 0.0, a2 = 0.0, b1 = 0.0, b2 = 0.0;
    const double *pij = P.mom + ((size_t)i * P.p + j) * 2;
    const double *pji = P.mom + ((size_t)j * P.p + i) * 2;
    for (int s = 0; s < P.nsplit; ++s) {
        a1 += pij[s * plane];
        a2 += pij[s * plane + 1];
        b1 += pji[s * plane];
        b2 += pji[s * plane + 1];
    }
    const double mi1 = P.a1 * a1 * invn + P.b1, mi2 = P.a2 * a2 * invn;
    const double mj1 = P.a1 * b1 * invn + P.b1, mj2 = P.a2 * b2 * invn;
    const double hij = neg_entropy_part(mi1, mi2);
    const double hji = neg_entropy_part(mj1, mj2);
    I = (hsh[j] + hij) - (hsh[i] + hji);
    eps = P.epsI;
    if (P.use_model) {
        const int oi = P.U[i], oj = P.U[j];
        const double rho = P.C[(int64_t)min(oi, oj) * P.ldc + max(oi, oj)] * P.isd[i] * P.isd[j];
        const float ra = rsqrtf(fmaxf((float)fma(-rho, rho, 1.0), 1e-12f)) * 1.01f;
        const float e1 = (float)P.model.d1 + (float)P.model.da * ra;
        const float e2 = (float)P.model.d2 + (float)P.model.da * ra;
        eps = (double)(h_err((float)mi1, (float)mi2, e1, e2) + h_err((float)mj1, (float)mj2, e1, e2) +
                       wsh[i] + wsh[j]);
    }
}

struct SelectParams {
    const double *M, *E;
    const int32_t *U;
    int p;
    DevState *state;
    int32_t *scratch;     // [p] candidate list workspace
    int tier;             // tier of the first re-score (1 double-float, 2 FP64)
    const int8_t *prior;  // [ldp][ldp] ancestry knowledge by original index, or null:
    int64_t ldp;          //   prior[i ldp + j] = 1 x_j is an ancestor of x_i, 0 is not, -1 unknown
    uint8_t *allow;       // [p] workspace: positions that may be chosen at this step
};

struct RefineSelectParams {
    const double *mom;    // [nsplit][d][p][4] by candidate slot
    const double *hz;     // [nsplit][p][2]
    int p, n;
    int nsplit;           // partial records per value, summed in range order
    int64_t mom_sstride;
    const int32_t *U;
    DevState *state;
    double *hist;         // optional row of the score history
    int tier;             // 1: double-float passes, 2: FP64 pass
    double epsI;          // tier 1: bound on the error of each re-scored I(i, j)
    int last;             // tier 1: the last double-float pass of the step
};

struct RegressParams {
    double *R;            // FP64 residual data [d][ldr], updated in place
    int64_t ldr;
    float *z;             // FP32 standardised residuals [d][ldz], compacted by position
    int64_t ldz;
    const double *C;
    int64_t ldc;
    const int32_t *U;     // current positions
    int32_t *Unext;       // next positions (compacted)
    int p, n;
    int sps;              // samples per split
    DevState *state;
    int32_t *order;       // order[t] = chosen variable
    int t;
    double *hzpart;       // out [nsplit][p'][2] variable moment sums of z
    const double *ref_var;
    double *lcoef;        // optional [d][d]: lcoef[i*d + m] = regression coefficient (L of LDL^T)
    int64_t ldl;
    uint32_t *status;
    double *isd_out;      // [p'] 1 / sqrt(variance) of the next step's positions
};

// Low parts of the standardised columns (k_zlo_b): z = zhi + zlo.
struct ZloParams {
    const double *R;      // FP64 residual data [d][ldr] by original index
    int64_t ldr;
    const float *zhi;     // [p][ldz] by position
    float *zlo;           // out [p][ldz]
    int64_t ldz;
    const double *isd;    // [p] 1 / sqrt(C_ii) by position
    const int32_t *U;
    int p, n;
    const DevState *state;
    int always;           // 1: every pair scored in double-float at this step
};

struct GramParams {
    const double *R;
    int64_t ldr;
    int n, d, ksplit;
    double *Cpart;        // [ksplit][d][d]
    double *C;            // [d][ldc]
    int64_t ldc;
    double *ref_var;      // diag(C) of the original data
};

struct IotaParams {
    int32_t *U;
    int d;
    DevState *state;
};

struct DowndateParams {
    double *C;
    int64_t ldc;
    const int32_t *U;
    int p;
    const DevState *state;
};

struct FinishParams {
    const int32_t *U;
    int32_t *order;
    int d;
    double *hist_row;
};

// ---- launchers (return the launch error) ----
// Batched launchers take a device array of per-instance parameters.
cudaError_t launch_gate_wait(const uint32_t *flag, uint64_t limit_ns, uint32_t *status,
                             cudaStream_t s);
cudaError_t launch_pack(const void *X, int is_f64, int layout, int64_t ld, int n, int d,
                        double *R, int64_t ldr, uint32_t *status, cudaStream_t s);
cudaError_t launch_center(double *R, int64_t ldr, int n, int d, cudaStream_t s);
cudaError_t launch_gram_f64(const double *R, int64_t ldr, int n, int d, double *Cpart,
                            int ksplit, double *C, int64_t ldc, double *ref_var,
                            cudaStream_t s);
cudaError_t launch_gram_b(const GramParams *P, int count, int maxd, int maxksplit, cudaStream_t s);
int gram_ksplit(int n, int d, int num_sms);
cudaError_t launch_iota_b(const IotaParams *P, int count, int maxd, cudaStream_t s);
// Flattened batched launches: prefix[k] = first block of instance k (count + 1
// entries); the *_blocks functions give an instance's block count.
int regress_blocks(int cols, int n, int sps);
cudaError_t launch_regress_b(const RegressParams *P, const int *prefix, int count, bool init,
                             int total_blocks, cudaStream_t s);
int downdate_blocks(int p);
cudaError_t launch_downdate_b(const DowndateParams *P, const int *prefix, int count,
                              int total_blocks, cudaStream_t s);
cudaError_t launch_finish_b(const FinishParams *P, int count, cudaStream_t s);

cudaError_t pair_kernel_setup();
size_t pair_smem_bytes(int cfg);
// CTAs of configuration cfg resident per SM in the given form (occupancy API).
int pair_ctas_per_sm(int mode, int cfg);
cudaError_t launch_pair_b(int mode, int cfg, const CUtensorMap *tmI, const CUtensorMap *tmJ,
                          const PairParams *P, const int *prefix, int count, int total_ctas,
                          cudaStream_t s);

// Sample splits of one pair-kernel launch: with `tiles` CTA tiles in total
// and a target of `target` CTAs, the samples of an instance with nchunks
// chunks are cut into nsplit ranges of cps chunks.
inline void pair_split(int64_t tiles, int64_t target, int nchunks, int *cps, int *nsplit)
{
    const int ns_pair = tiles > 0 ? (int)std::max<int64_t>(1, (target + tiles - 1) / tiles) : 1;
    const int ns = std::max(1, std::min(ns_pair, nchunks));
    *cps = (nchunks + ns - 1) / ns;
    *nsplit = (nchunks + *cps - 1) / *cps;
}
cudaError_t launch_pairs_hp_b(int tier, const HpParams *P, int count, int blocks, cudaStream_t s);
cudaError_t df_tables_setup();
int score_blocks(int p);
cudaError_t launch_score_b(const ScoreParams *P, const int *prefix, int count, int total_blocks,
                           int maxp, cudaStream_t s);
cudaError_t launch_select_b(const SelectParams *P, int count, cudaStream_t s);
cudaError_t launch_set_rescore_cond(const DevState *st, const unsigned long long *cond,
                                    cudaStream_t s);
cudaError_t launch_refine_select_b(const RefineSelectParams *P, int count, int maxp,
                                   cudaStream_t s);

cudaError_t launch_pack_gather(const float *X, int64_t ld, const int32_t *rows, int n, int d,
                               double *R, int64_t ldr, uint32_t *status, cudaStream_t s);

// Adjacency / VAR helpers
cudaError_t launch_ldl_step(double *C, int64_t ldc, const int32_t *pivots, int t, int d,
                            double *L, int64_t ldl, cudaStream_t s);
cudaError_t launch_unit_lower_inverse(const double *L, int64_t ldl, const int32_t *perm, int d,
                                      double *W, int64_t ldw, cudaStream_t s);

cudaError_t launch_regress_cols(double *R, int64_t ldr, const double *L, int64_t ldl, int t, int q,
                                int n, int nsplit, cudaStream_t s);
cudaError_t launch_var_coefficients(const double *L, int64_t ldl, int nz, int d, double *M,
                                    cudaStream_t s);
cudaError_t launch_var_transform(const double *B0, const double *M, int lags, int d, double *Bt,
                                 cudaStream_t s);
cudaError_t launch_iota_plain(int32_t *v, int q, cudaStream_t s);
cudaError_t launch_fill_nan(double *p, size_t count, cudaStream_t s);
cudaError_t launch_zlo_b(const ZloParams *P, int count, int blocks, cudaStream_t s);
cudaError_t launch_fill_test_z(float *z, int64_t ldz, int rows, int n, cudaStream_t s);

// Tensor-core covariance (kernels_gram_tc.cu): slice planes S [6][d_pad][ldk]
// BF16 described by tmS (box 64 x 128, 128-byte swizzle), expo
// [periods][d_pad] per 128-sample period, part [ksplit][d][d] FP64.
cudaError_t gram_tc_setup();
int gram_tc_dpad(int d);
int64_t gram_tc_ldk(int n);
int64_t gram_tc_expo_count(int n, int d);   // [drain periods][d_pad] exponents
int gram_tc_ksplit(int n, int d, int num_sms);
cudaError_t launch_gram_tc(const CUtensorMap *tmS, const double *R, int64_t ldr, int n, int d,
                           __nv_bfloat16 *S, int *expo, double *part, int ksplit, double *C,
                           int64_t ldc, double *ref_var, uint32_t *status, cudaStream_t s);

// Graph read-outs (kernels_effects.cu)
cudaError_t launch_total_effects_prep(const double *B, const int32_t *order, int d, int32_t *pos,
                                      double *L, uint32_t *status, cudaStream_t s);
cudaError_t launch_identity_minus(const double *W, int d, double *T, cudaStream_t s);
cudaError_t launch_var_window(const double *B0, const double *Bt, int d, int lags,
                              const int32_t *order0, double *A, int32_t *order, cudaStream_t s);
cudaError_t launch_influence(const double *T, int d, double *exert, double *receive,
                             int32_t *rank_exert, int32_t *rank_receive, cudaStream_t s);
void prune_workspace(int d, int num_sms, int *blocks, size_t *dbl, size_t *ints);
cudaError_t launch_prune(const double *C, const double *Bols, const int32_t *order, int d, int n,
                         double gamma, int L, double eps, int blocks, double *Cp, double *ws,
                         int *iws, double *B, uint32_t *status, cudaStream_t s);
cudaError_t launch_edge_stats(const double *const *Bs, int count, int d, double threshold,
                              double *prob, double *mean, uint32_t *status, cudaStream_t s);

cudaError_t launch_peak_probe(int which, int blocks, int iters, unsigned long long *cycles,
                              unsigned long long *ns, float *sink, cudaStream_t s);

}  // namespace lg
