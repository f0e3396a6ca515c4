// kernels_pair.cu -- the entropy-moment kernels of the causal-ordering step.
//
// Algorithm 1 (AcceleratedLiNGAM, arXiv 2403.03772) needs, for every ordered
// pair (i, j) of the p remaining variables, the entropy approximation of the
// standardised least-squares residual r_i^j of x_i on x_j.  With z the
// standardised columns and rho = C_ij / sqrt(C_ii C_jj) from the FP64
// covariance, that residual standardised by its own deviation sqrt(1 - rho^2)
// is u = (z_i - rho z_j) / sqrt(1 - rho^2) = a z_i - b z_j, one FMA per
// sample.  The kernels accumulate, per ordered pair,
//     S1 = sum_s log cosh(u_s)   (in a form that depends on the variant)
//     S2 = sum_s u_s exp(-u_s^2 / 2)
// over the n samples; k_score combines them into I(i, j) and M(i).
#include <cuda.h>
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace lg {

// ------------------------------------------------------------------------
// FP32 pair-moment kernel (TMA-staged, warp-tiled)
// ------------------------------------------------------------------------
//
// CTA tile: TI positions i x TJ positions j.  Thread 0 streams chunks of S
// samples of the TI + TJ standardised columns into shared memory with 2-D
// bulk tensor copies (one box for the i rows, one for the j rows) into a
// STAGES-deep ring guarded by full/empty mbarriers.  Each warp owns WI x WJ
// ordered pairs; lane l handles the four consecutive samples 128 it + 4 l ..
// + 3 of a chunk (conflict-free 16-byte loads), so all 32 lanes of a warp
// share the pair coefficients and the moments are reduced across lanes once,
// after the last chunk.
//
// Variants:
//   PAIR_ACCURATE: per sample  log cosh u + ln2 = |u| + log1pf(expf(-2|u|)),
//                  u exp(-u^2/2) with expf; plain FP32 running sums.
//   PAIR_FAST:     the residual is pre-scaled, u~ = k u with k^2 = log2(e)/2,
//                  so exp(-u^2/2) = ex2(-u~^2) and exp(-2|u|) = ex2(c2 |u~|);
//                  S1 accumulates log2(2 cosh u) = |u~| log2(e)/k +
//                  lg2(1 + ex2(c2 |u~|)) with the MUFU ex2/lg2 units, S2
//                  accumulates u~ exp(-u^2/2).  Per-chunk partial sums are
//                  folded into (hi, lo) pairs with TwoSum (compensated).

// Per-sample terms of the accurate form: log cosh u + ln 2 and u exp(-u^2/2).
__device__ __forceinline__ void accurate_terms(float u, float &t1, float &t2)
{
    const float au = fabsf(u);
    t1 = au + log1pf(expf(-2.0f * au));
    t2 = u * expf(-0.5f * u * u);
}

// Constants of the fast form: c2 = -2 log2(e) / k, c3 = log2(e) / k.
constexpr float FAST_C2 = (float)(-2.0 * LOG2E_D / KSC);
constexpr float FAST_C3 = (float)(LOG2E_D / KSC);

// One chunk of S samples for the WI x WJ pairs of a warp.  An iteration
// covers G x 128 samples: lane l takes the G groups of four consecutive
// samples g 128 + 4 l .. + 3 (one 16-byte shared load per column and group,
// conflict-free).  Fast form: sum_s log2(2 cosh u_s) = log2(e)/k sum |u~_s| +
// sum_s log2(1 + y_s); the second sum is taken as log2 of the product of
// the 4 G factors (1 + y_s) in (1, 2^(4G)], one MUFU lg2 per 4 G samples (the
// logarithm of a product is the sum of the logarithms).
//
// Paired form (PK, full chunks of the fast form): samples 2h and 2h + 1 of a
// lane travel together through the f32x2 multiply / FMA instructions of
// sm_100-class GPUs (one issue slot for two FP32 results); each lane keeps two
// interleaved partial sums of u exp(-u^2/2) and two product chains, joined
// once per pair and iteration.  The MUFU ex2/lg2 work is unchanged.
template <int MODE, bool TAIL, int WI, int WJ, int S, int G, bool PK>
__device__ __forceinline__ void pair_chunk(const float *__restrict__ rows,
                                           const float *__restrict__ cols,
                                           const float (&ca)[WI][WJ], const float (&cb)[WI][WJ],
                                           float (&a1)[WI][WJ], float (&a2)[WI][WJ], int lane,
                                           int valid)
{
    constexpr int V = 4 * G;   // samples per lane and iteration
#pragma unroll 1
    for (int it = 0; it < S / (128 * G); ++it) {
        const int s0 = it * 128 * G + lane * 4;
        float zi[WI][V], zj[WJ][V];
#pragma unroll
        for (int g = 0; g < G; ++g) {
#pragma unroll
            for (int r = 0; r < WI; ++r) {
                const float4 t = *reinterpret_cast<const float4 *>(rows + r * S + s0 + g * 128);
                zi[r][4 * g] = t.x;
                zi[r][4 * g + 1] = t.y;
                zi[r][4 * g + 2] = t.z;
                zi[r][4 * g + 3] = t.w;
            }
#pragma unroll
            for (int c = 0; c < WJ; ++c) {
                const float4 t = *reinterpret_cast<const float4 *>(cols + c * S + s0 + g * 128);
                zj[c][4 * g] = t.x;
                zj[c][4 * g + 1] = t.y;
                zj[c][4 * g + 2] = t.z;
                zj[c][4 * g + 3] = t.w;
            }
        }
        bool ok[V];
#pragma unroll
        for (int v = 0; v < V; ++v) ok[v] = !TAIL || (s0 + (v / 4) * 128 + (v % 4)) < valid;
#pragma unroll
        for (int r = 0; r < WI; ++r) {
#pragma unroll
            for (int c = 0; c < WJ; ++c) {
                if (MODE == PAIR_FAST && PK && !TAIL) {
                    const float2 A = make_float2(ca[r][c], ca[r][c]);
                    const float2 NB = make_float2(-cb[r][c], -cb[r][c]);
                    const float2 C2 = make_float2(FAST_C2, FAST_C2);
                    float2 acc = make_float2(a2[r][c], 0.0f), pr = make_float2(1.0f, 1.0f);
                    float asum = 0.0f;
#pragma unroll
                    for (int h = 0; h < V / 2; ++h) {
                        const float2 zi2 = make_float2(zi[r][2 * h], zi[r][2 * h + 1]);
                        const float2 zj2 = make_float2(zj[c][2 * h], zj[c][2 * h + 1]);
                        const float2 u = __ffma2_rn(A, zi2, __fmul2_rn(NB, zj2));
                        const float2 sq = __fmul2_rn(u, u);
                        const float2 e = make_float2(ex2_approx(-sq.x), ex2_approx(-sq.y));
                        acc = __ffma2_rn(u, e, acc);
                        const float2 q = __fmul2_rn(u, C2);   // C2 < 0: exp(-2|u|) = ex2(-|q|)
                        const float2 y = make_float2(ex2_approx(-fabsf(q.x)),
                                                     ex2_approx(-fabsf(q.y)));
                        pr = h == 0 ? make_float2(1.0f + y.x, 1.0f + y.y) : __ffma2_rn(y, pr, pr);
                        asum = h == 0 ? fabsf(u.x) + fabsf(u.y)
                                      : asum + fabsf(u.x) + fabsf(u.y);
                    }
                    a2[r][c] = acc.x + acc.y;
                    a1[r][c] += fmaf(asum, FAST_C3, lg2_approx(pr.x * pr.y));
                } else if (MODE == PAIR_FAST) {
                    float yv[V], au[V];
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const float u = fmaf(ca[r][c], zi[r][v], -(cb[r][c] * zj[c][v]));
                        const float e = ex2_approx(-(u * u));        // exp(-u^2/2)
                        float g = u * e;
                        float a = fabsf(u);
                        float y = ex2_approx(a * FAST_C2);           // exp(-2|u|)
                        if (TAIL && !ok[v]) {
                            g = 0.0f;
                            a = 0.0f;
                            y = 0.0f;
                        }
                        a2[r][c] += g;
                        yv[v] = y;
                        au[v] = a;
                    }
                    // prod (1 + y_v) by q <- q + y q: one add and V - 1 FMAs
                    float prod = 1.0f + yv[V - 1];
#pragma unroll
                    for (int v = V - 2; v >= 0; --v) prod = fmaf(yv[v], prod, prod);
                    float asum = au[0];
#pragma unroll
                    for (int v = 1; v < V; ++v) asum += au[v];
                    a1[r][c] += fmaf(asum, FAST_C3, lg2_approx(prod));
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const float u = fmaf(ca[r][c], zi[r][v], -(cb[r][c] * zj[c][v]));
                        float t1, t2;
                        accurate_terms(u, t1, t2);
                        if (TAIL && !ok[v]) {
                            t1 = 0.0f;
                            t2 = 0.0f;
                        }
                        a1[r][c] += t1;
                        a2[r][c] += t2;
                    }
                }
            }
        }
    }
}

template <int MODE, int CFG>
__device__ __forceinline__ void pair_block(const CUtensorMap *tmI, const CUtensorMap *tmJ,
                                           const PairParams &P, const int ti, const int tj,
                                           const int split)
{
    constexpr PairCfg G = PAIR_CFGS[CFG];
    constexpr int WI = G.wi, WJ = G.wj, WGJ = G.wgj;
    constexpr int NCW = G.warps();
    constexpr int TI = G.ti(), TJ = G.tj(), S = PAIR_S, STAGES = G.stages;
    constexpr uint32_t STAGE_FLOATS = (TI + TJ) * S;
    constexpr uint32_t STAGE_BYTES = STAGE_FLOATS * 4;
    constexpr bool COMP = true;   // compensated (hi, lo) folds in both forms
    constexpr bool PK = G.packed != 0;

    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + STAGES;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 512);
    float *buf = reinterpret_cast<float *>(smem + 1024);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = split * P.cps;
    const int c1 = min(c0 + P.cps, P.nchunks);
    const int nck = c1 - c0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        // a wait that expired earlier in this run ends every later CTA at once
        *abort_flag = (*(volatile uint32_t *)P.status & ST_TIMEOUT) ? 1 : 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (nck <= 0 || *abort_flag) return;

    // Thread 0 issues the bulk tensor copies: chunks 0 .. STAGES-2 up front,
    // then chunk k + STAGES - 1 at iteration k, into the stage that chunk
    // k - 1 used (free once every warp has finished chunk k - 1).  No warp is
    // set aside for this: register allocation rounds a CTA up to a multiple
    // of four warps, so 8 warps keep the full register budget.
    int issued = 0;
    auto issue = [&](int k) -> bool {
        const int st = k % STAGES;
        if (k >= STAGES && !mbar_wait_bounded(&empty[st], ((k / STAGES) - 1) & 1)) return false;
        float *dst = buf + st * STAGE_FLOATS;
        const int x = (c0 + k) * S;
        mbar_arrive_expect_tx(&full[st], STAGE_BYTES);
        tma_load_2d(dst, tmI, x, P.row0 + ti * TI, &full[st]);
        tma_load_2d(dst + TI * S, tmJ, x, P.row0 + tj * TJ, &full[st]);
        issued = k + 1;
        return true;
    };
    if (threadIdx.x == 0) {
        prefetch_tensormap(tmI);
        prefetch_tensormap(tmJ);
        for (int k = 0; k < min(STAGES - 1, nck); ++k) (void)issue(k);
    }

    // ---------------- every warp computes -----------------------------------
    const int wi = warp / WGJ, wj = warp % WGJ;
    const int ri0 = wi * WI, cj0 = wj * WJ;
    const int pi0 = ti * TI + ri0, pj0 = tj * TJ + cj0;

    float ca[WI][WJ], cb[WI][WJ];
    {
        // rho and 1 - rho^2 in FP64 (cancellation near |rho| = 1), the
        // reciprocal square root in FP32 from that exact-to-rounding value
        float a = 0.0f, b = 0.0f;
        if (lane < WI * WJ) {
            const int pi = pi0 + lane / WJ, pj = pj0 + lane % WJ;
            if (pi < P.p && pj < P.p && pi != pj) {
                const int oi = P.U[pi], oj = P.U[pj];
                const int lo = min(oi, oj), hi = max(oi, oj);
                const double rho = P.C[(int64_t)lo * P.ldc + hi] * P.isd[pi] * P.isd[pj];
                const double s2 = fma(-rho, rho, 1.0);
                // the score kernel's error model reads this entry's factor
                if (P.ra && split == 0)
                    P.ra[(size_t)pi * P.p + pj] = rsqrtf(fmaxf((float)s2, 1e-12f));
                if (s2 > 1e-12) {
                    a = rsqrtf((float)s2);
                    b = (float)rho * a;
                } else {
                    set_status(P.status, ST_DEGENERATE);
                    a = 1.0f;
                }
                if (MODE == PAIR_FAST) {
                    a *= (float)KSC;
                    b *= (float)KSC;
                }
            }
        }
        const float fa = a, fb = b;
#pragma unroll
        for (int e = 0; e < WI * WJ; ++e) {
            ca[e / WJ][e % WJ] = __shfl_sync(0xffffffffu, fa, e);
            cb[e / WJ][e % WJ] = __shfl_sync(0xffffffffu, fb, e);
        }
    }

    float s1[WI][WJ], s2[WI][WJ], e1[WI][WJ], e2[WI][WJ];
#pragma unroll
    for (int r = 0; r < WI; ++r)
#pragma unroll
        for (int c = 0; c < WJ; ++c) s1[r][c] = s2[r][c] = e1[r][c] = e2[r][c] = 0.0f;
    float a1[WI][WJ], a2[WI][WJ];    // chunk partial sums (compensated form)
#pragma unroll
    for (int r = 0; r < WI; ++r)
#pragma unroll
        for (int c = 0; c < WJ; ++c) a1[r][c] = a2[r][c] = 0.0f;
    constexpr int FOLD = G.fold;

    for (int k = 0; k < nck; ++k) {
        if (threadIdx.x == 0 && k + STAGES - 1 < nck && !*abort_flag) {
            if (!issue(k + STAGES - 1)) {
                set_status(P.status, ST_TIMEOUT);
                *abort_flag = 1;
            }
        }
        const int st = k % STAGES;
        const uint32_t par = (k / STAGES) & 1;
        if (!mbar_wait_bounded(&full[st], par)) {
            set_status(P.status, ST_TIMEOUT);
            *abort_flag = 1;
            break;
        }
        const float *rows = buf + st * STAGE_FLOATS + ri0 * S;
        const float *cols = buf + st * STAGE_FLOATS + TI * S + cj0 * S;
        const int valid = min(S, P.n - (c0 + k) * S);
        if (COMP) {
            if (valid == S)
                pair_chunk<MODE, false, WI, WJ, S, G.groups, PK>(rows, cols, ca, cb, a1, a2, lane,
                                                                 valid);
            else
                pair_chunk<MODE, true, WI, WJ, S, G.groups, PK>(rows, cols, ca, cb, a1, a2, lane,
                                                                valid);
            // fold the partial sums of FOLD chunks into (hi, lo) pairs
            if ((k % FOLD) == FOLD - 1 || k == nck - 1) {
#pragma unroll
                for (int r = 0; r < WI; ++r)
#pragma unroll
                    for (int c = 0; c < WJ; ++c) {
                        float t, err;
                        two_sum(s1[r][c], a1[r][c], t, err);
                        s1[r][c] = t;
                        e1[r][c] += err;
                        two_sum(s2[r][c], a2[r][c], t, err);
                        s2[r][c] = t;
                        e2[r][c] += err;
                        a1[r][c] = a2[r][c] = 0.0f;
                    }
            }
        } else {
            if (valid == S)
                pair_chunk<MODE, false, WI, WJ, S, G.groups, PK>(rows, cols, ca, cb, s1, s2, lane,
                                                                 valid);
            else
                pair_chunk<MODE, true, WI, WJ, S, G.groups, PK>(rows, cols, ca, cb, s1, s2, lane,
                                                                valid);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
        if (*abort_flag) break;
    }

    // never leave with a copy in flight: thread 0 waits (bounded) for the
    // last phase issued on every stage (already consumed ones return at once)
    if (threadIdx.x == 0)
        for (int k = max(0, issued - STAGES); k < issued; ++k)
            (void)mbar_wait_bounded(&full[k % STAGES], (k / STAGES) & 1);

    // ---------------- cross-lane reduction (fixed xor tree) ------------------
    float2 *mom = P.mom + (size_t)split * P.p * P.p * 2;
#pragma unroll
    for (int r = 0; r < WI; ++r) {
#pragma unroll
        for (int c = 0; c < WJ; ++c) {
            float h1 = s1[r][c], l1 = e1[r][c], h2 = s2[r][c], l2 = e2[r][c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float oh1 = __shfl_xor_sync(0xffffffffu, h1, o);
                const float ol1 = __shfl_xor_sync(0xffffffffu, l1, o);
                const float oh2 = __shfl_xor_sync(0xffffffffu, h2, o);
                const float ol2 = __shfl_xor_sync(0xffffffffu, l2, o);
                if (COMP) {
                    float t, err;
                    two_sum(h1, oh1, t, err);
                    h1 = t;
                    l1 = (l1 + ol1) + err;
                    two_sum(h2, oh2, t, err);
                    h2 = t;
                    l2 = (l2 + ol2) + err;
                } else {
                    h1 += oh1;
                    h2 += oh2;
                }
            }
            const int pi = pi0 + r, pj = pj0 + c;
            if (lane == r * WJ + c && pi < P.p && pj < P.p && pi != pj) {
                // normalised (hi, lo) pairs for the double-float score
                float2 *o = mom + ((size_t)pi * P.p + pj) * 2;
                float t, err;
                two_sum(h1, l1, t, err);
                o[0] = make_float2(t, err);
                two_sum(h2, l2, t, err);
                o[1] = make_float2(t, err);
            }
        }
    }
}

// ------------------------------------------------------------------------
// Streamlined block (tile configurations with sub >= 1)
// ------------------------------------------------------------------------
//
// The same per-pair arithmetic as pair_block, with less bookkeeping per
// residual-sample: a ring stage holds `sub` consecutive chunks (fewer barrier
// waits and arrivals per sample), stage and parity advance incrementally, the
// fold test uses a power-of-two chunk count, each lane loads the WJ column
// samples once per chunk and the WI row samples one row at a time (fewer live
// registers), the paired-FP32 u exp(-u^2/2) sums stay float2 across the
// chunks of a fold period, and the product of the 1 + y factors starts from
// (1, 1) so every sample pair takes one f32x2 FMA.

// One full chunk of the paired fast form for the WI x WJ pairs of a warp
// (groups of four samples g 128 + 4 l .. + 3, g = 0, 1, as in pair_chunk).
// The product of the 1 + y factors and the |u| sum run on in pr / asum across
// the chunks of a ring stage (FIRST starts them); the caller takes one lg2 of
// the product of up to 8 SUB factors (at most 2^16) when the stage ends.
template <int WI, int WJ, int S, bool FIRST, bool ABS2>
__device__ __forceinline__ void pair_chunk_pk(const float *__restrict__ rows,
                                              const float *__restrict__ cols,
                                              const float2 (&A)[WI][WJ],
                                              const float2 (&NB)[WI][WJ], float2 (&pr)[WI][WJ],
                                              float (&asum)[WI][WJ], float2 (&acc)[WI][WJ],
                                              int lane)
{
    static_assert(S == 256, "one iteration of 8 samples per lane covers a chunk");
    const int s0 = lane * 4;
    float zj[WJ][8];
#pragma unroll
    for (int c = 0; c < WJ; ++c) {
        const float4 t0 = *reinterpret_cast<const float4 *>(cols + c * S + s0);
        const float4 t1 = *reinterpret_cast<const float4 *>(cols + c * S + s0 + 128);
        zj[c][0] = t0.x; zj[c][1] = t0.y; zj[c][2] = t0.z; zj[c][3] = t0.w;
        zj[c][4] = t1.x; zj[c][5] = t1.y; zj[c][6] = t1.z; zj[c][7] = t1.w;
    }
    const float2 C2 = make_float2(FAST_C2, FAST_C2);
    const float2 ONE = make_float2(1.0f, 1.0f);
#pragma unroll
    for (int r = 0; r < WI; ++r) {
        float zi[8];
        {
            const float4 t0 = *reinterpret_cast<const float4 *>(rows + r * S + s0);
            const float4 t1 = *reinterpret_cast<const float4 *>(rows + r * S + s0 + 128);
            zi[0] = t0.x; zi[1] = t0.y; zi[2] = t0.z; zi[3] = t0.w;
            zi[4] = t1.x; zi[5] = t1.y; zi[6] = t1.z; zi[7] = t1.w;
        }
#pragma unroll
        for (int c = 0; c < WJ; ++c) {
            float2 pc = FIRST ? ONE : pr[r][c];
            float as = asum[r][c];
            float2 as2 = make_float2(FIRST ? 0.0f : as, 0.0f);
            float2 ac = acc[r][c];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float2 zi2 = make_float2(zi[2 * h], zi[2 * h + 1]);
                const float2 zj2 = make_float2(zj[c][2 * h], zj[c][2 * h + 1]);
                const float2 u = __ffma2_rn(A[r][c], zi2, __fmul2_rn(NB[r][c], zj2));
                const float2 sq = __fmul2_rn(u, u);
                const float2 e = make_float2(ex2_approx(-sq.x), ex2_approx(-sq.y));
                ac = __ffma2_rn(u, e, ac);
                const float2 q = __fmul2_rn(u, C2);   // C2 < 0: exp(-2|u|) = ex2(-|q|)
                const float2 y = make_float2(ex2_approx(-fabsf(q.x)), ex2_approx(-fabsf(q.y)));
                pc = __ffma2_rn(y, pc, pc);
                if (ABS2)
                    as2 = __fadd2_rn(as2, make_float2(fabsf(u.x), fabsf(u.y)));
                else
                    as = (FIRST && h == 0) ? fabsf(u.x) + fabsf(u.y) : as + fabsf(u.x) + fabsf(u.y);
            }
            acc[r][c] = ac;
            pr[r][c] = pc;
            asum[r][c] = ABS2 ? as2.x + as2.y : as;
        }
    }
}

// The same chunk with every row loaded first and the sample steps outermost:
// each step h runs all WI x WJ pairs, so WI WJ independent chains lie between
// a MUFU result and its use.
template <int WI, int WJ, int S, bool FIRST, bool ABS2>
__device__ __forceinline__ void pair_chunk_pk_h(const float *__restrict__ rows,
                                                const float *__restrict__ cols,
                                                const float2 (&A)[WI][WJ],
                                                const float2 (&NB)[WI][WJ], float2 (&pr)[WI][WJ],
                                                float (&asum)[WI][WJ], float2 (&acc)[WI][WJ],
                                                int lane)
{
    static_assert(S == 256, "one iteration of 8 samples per lane covers a chunk");
    const int s0 = lane * 4;
    float zi[WI][8], zj[WJ][8];
#pragma unroll
    for (int r = 0; r < WI; ++r) {
        const float4 t0 = *reinterpret_cast<const float4 *>(rows + r * S + s0);
        const float4 t1 = *reinterpret_cast<const float4 *>(rows + r * S + s0 + 128);
        zi[r][0] = t0.x; zi[r][1] = t0.y; zi[r][2] = t0.z; zi[r][3] = t0.w;
        zi[r][4] = t1.x; zi[r][5] = t1.y; zi[r][6] = t1.z; zi[r][7] = t1.w;
    }
#pragma unroll
    for (int c = 0; c < WJ; ++c) {
        const float4 t0 = *reinterpret_cast<const float4 *>(cols + c * S + s0);
        const float4 t1 = *reinterpret_cast<const float4 *>(cols + c * S + s0 + 128);
        zj[c][0] = t0.x; zj[c][1] = t0.y; zj[c][2] = t0.z; zj[c][3] = t0.w;
        zj[c][4] = t1.x; zj[c][5] = t1.y; zj[c][6] = t1.z; zj[c][7] = t1.w;
    }
    const float2 C2 = make_float2(FAST_C2, FAST_C2);
    const float2 ONE = make_float2(1.0f, 1.0f);
    float2 as2[WI][WJ];
#pragma unroll
    for (int r = 0; r < WI; ++r)
#pragma unroll
        for (int c = 0; c < WJ; ++c) {
            if (FIRST) pr[r][c] = ONE;
            as2[r][c] = make_float2(FIRST ? 0.0f : asum[r][c], 0.0f);
        }
#pragma unroll
    for (int h = 0; h < 4; ++h) {
#pragma unroll
        for (int r = 0; r < WI; ++r) {
#pragma unroll
            for (int c = 0; c < WJ; ++c) {
                const float2 zi2 = make_float2(zi[r][2 * h], zi[r][2 * h + 1]);
                const float2 zj2 = make_float2(zj[c][2 * h], zj[c][2 * h + 1]);
                const float2 u = __ffma2_rn(A[r][c], zi2, __fmul2_rn(NB[r][c], zj2));
                const float2 sq = __fmul2_rn(u, u);
                const float2 e = make_float2(ex2_approx(-sq.x), ex2_approx(-sq.y));
                acc[r][c] = __ffma2_rn(u, e, acc[r][c]);
                const float2 q = __fmul2_rn(u, C2);
                const float2 y = make_float2(ex2_approx(-fabsf(q.x)), ex2_approx(-fabsf(q.y)));
                pr[r][c] = __ffma2_rn(y, pr[r][c], pr[r][c]);
                if (ABS2) {
                    as2[r][c] = __fadd2_rn(as2[r][c], make_float2(fabsf(u.x), fabsf(u.y)));
                } else {
                    as2[r][c].x = as2[r][c].x + fabsf(u.x) + fabsf(u.y);
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < WI; ++r)
#pragma unroll
        for (int c = 0; c < WJ; ++c) asum[r][c] = ABS2 ? as2[r][c].x + as2[r][c].y : as2[r][c].x;
}

template <int MODE, int CFG>
__device__ __forceinline__ void pair_block_v2(const CUtensorMap *tmI, const CUtensorMap *tmJ,
                                              const PairParams &P, const int ti, const int tj,
                                              const int split)
{
    constexpr PairCfg G = PAIR_CFGS[CFG];
    constexpr int WI = G.wi, WJ = G.wj, WGJ = G.wgj;
    constexpr int NCW = G.warps();
    constexpr int TI = G.ti(), TJ = G.tj(), S = PAIR_S, STAGES = G.stages, SUB = G.sub;
    constexpr uint32_t CHUNK_FLOATS = (TI + TJ) * S;
    constexpr uint32_t STAGE_FLOATS = CHUNK_FLOATS * SUB;
    constexpr bool PK = MODE == PAIR_FAST && G.packed != 0;
    constexpr int FOLD = G.fold;
    static_assert(SUB >= 1 && (FOLD & (FOLD - 1)) == 0 && FOLD % SUB == 0,
                  "streamlined block: power-of-two folds, a multiple of the stage");
    static_assert(!PK || G.groups == 2, "the paired chunk takes 8 samples per lane");

    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + STAGES;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + 512);
    float *buf = reinterpret_cast<float *>(smem + 1024);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = split * P.cps;
    const int c1 = min(c0 + P.cps, P.nchunks);
    const int nck = c1 - c0;
    const int nst = (nck + SUB - 1) / SUB;   // ring stages of this sample range

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NCW);
        }
        *abort_flag = (*(volatile uint32_t *)P.status & ST_TIMEOUT) ? 1 : 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (nck <= 0 || *abort_flag) return;

    // Thread 0 fills stage k with the chunks k SUB .. k SUB + SUB - 1 of the
    // range that exist (the last stage may hold fewer), once every warp has
    // released what that ring slot held before.
    int issued = 0;
    auto issue = [&](int k) -> bool {
        const int st = k % STAGES;
        if (k >= STAGES && !mbar_wait_bounded(&empty[st], ((k / STAGES) - 1) & 1)) return false;
        float *dst = buf + st * STAGE_FLOATS;
        const int nb = min(SUB, nck - k * SUB);
        mbar_arrive_expect_tx(&full[st], (uint32_t)nb * CHUNK_FLOATS * 4u);
        for (int b = 0; b < nb; ++b) {
            const int x = (c0 + k * SUB + b) * S;
            tma_load_2d(dst + b * CHUNK_FLOATS, tmI, x, P.row0 + ti * TI, &full[st]);
            tma_load_2d(dst + b * CHUNK_FLOATS + TI * S, tmJ, x, P.row0 + tj * TJ, &full[st]);
        }
        issued = k + 1;
        return true;
    };
    if (threadIdx.x == 0) {
        prefetch_tensormap(tmI);
        prefetch_tensormap(tmJ);
        for (int k = 0; k < min(STAGES - 1, nst); ++k) (void)issue(k);
    }

    const int wi = warp / WGJ, wj = warp % WGJ;
    const int ri0 = wi * WI, cj0 = wj * WJ;
    const int pi0 = ti * TI + ri0, pj0 = tj * TJ + cj0;

    float ca[WI][WJ], cb[WI][WJ];
    {
        // rho and 1 - rho^2 in FP64, the reciprocal square root in FP32
        float a = 0.0f, b = 0.0f;
        if (lane < WI * WJ) {
            const int pi = pi0 + lane / WJ, pj = pj0 + lane % WJ;
            if (pi < P.p && pj < P.p && pi != pj) {
                const int oi = P.U[pi], oj = P.U[pj];
                const int lo = min(oi, oj), hi = max(oi, oj);
                const double rho = P.C[(int64_t)lo * P.ldc + hi] * P.isd[pi] * P.isd[pj];
                const double s2 = fma(-rho, rho, 1.0);
                // the score kernel's error model reads this entry's factor
                if (P.ra && split == 0)
                    P.ra[(size_t)pi * P.p + pj] = rsqrtf(fmaxf((float)s2, 1e-12f));
                if (s2 > 1e-12) {
                    a = rsqrtf((float)s2);
                    b = (float)rho * a;
                } else {
                    set_status(P.status, ST_DEGENERATE);
                    a = 1.0f;
                }
                if (MODE == PAIR_FAST) {
                    a *= (float)KSC;
                    b *= (float)KSC;
                }
            }
        }
#pragma unroll
        for (int e = 0; e < WI * WJ; ++e) {
            ca[e / WJ][e % WJ] = __shfl_sync(0xffffffffu, a, e);
            cb[e / WJ][e % WJ] = __shfl_sync(0xffffffffu, b, e);
        }
    }
    float2 A[WI][WJ], NB[WI][WJ];
#pragma unroll
    for (int r = 0; r < WI; ++r)
#pragma unroll
        for (int c = 0; c < WJ; ++c) {
            A[r][c] = make_float2(ca[r][c], ca[r][c]);
            NB[r][c] = make_float2(-cb[r][c], -cb[r][c]);
        }

    // (hi, lo) folded sums, and the FP32 sums of the current fold period
    // (S2 as two interleaved float2 halves in the paired form)
    float s1[WI][WJ], s2[WI][WJ], e1[WI][WJ], e2[WI][WJ], a1[WI][WJ], asum[WI][WJ];
    float2 acc[WI][WJ], pr[WI][WJ];
#pragma unroll
    for (int r = 0; r < WI; ++r)
#pragma unroll
        for (int c = 0; c < WJ; ++c) {
            s1[r][c] = s2[r][c] = e1[r][c] = e2[r][c] = asum[r][c] = 0.0f;
            acc[r][c] = pr[r][c] = make_float2(0.0f, 0.0f);
        }

    // Stages whose SUB chunks all exist take the straight-line path, the
    // instance's last chunk included when it is short: its samples past n
    // read as zeros (the z rows are zero-padded, the TMA fills past the
    // tensor with zeros), so each gives u = 0, adds 0 to the u exp(-u^2/2)
    // sum and exactly 1 to the log2(2 cosh u) sum (a factor 1 + 1 in the
    // product, |u| = 0).  Each lane starts its log2 sums at minus its count
    // of such slots.  A last stage with fewer than SUB chunks takes the
    // general path (masked tail).
    const int nfs = PK ? nck / SUB : 0;
    int ninv = 0;
    if (PK && nck % SUB == 0 && (int64_t)c1 * S > P.n) {
        const int64_t base = (int64_t)(c1 - 1) * S + lane * 4;
#pragma unroll
        for (int g = 0; g < 2; ++g)
#pragma unroll
            for (int v = 0; v < 4; ++v) ninv += base + g * 128 + v >= P.n;
    }
#pragma unroll
    for (int r = 0; r < WI; ++r)
#pragma unroll
        for (int c = 0; c < WJ; ++c) a1[r][c] = -(float)ninv;
    int st = 0;
    uint32_t ph = 0;
    for (int k = 0; k < nst; ++k) {
        if (threadIdx.x == 0 && k + STAGES - 1 < nst && !*abort_flag) {
            if (!issue(k + STAGES - 1)) {
                set_status(P.status, ST_TIMEOUT);
                *abort_flag = 1;
            }
        }
        if (!mbar_wait_bounded(&full[st], ph)) {
            set_status(P.status, ST_TIMEOUT);
            *abort_flag = 1;
            break;
        }
        const float *sb = buf + st * STAGE_FLOATS;
        // a chunk after the first of a stage exists only if the first was
        // full (a short chunk is the last of the instance)
        bool pending = false;
        if (PK && k < nfs) {
            // every chunk of the stage is full: no per-chunk checks
            if constexpr (G.hmajor != 0)
                pair_chunk_pk_h<WI, WJ, S, true, G.absadd != 0>(sb + ri0 * S, sb + TI * S + cj0 * S,
                                                                A, NB, pr, asum, acc, lane);
            else
                pair_chunk_pk<WI, WJ, S, true, G.absadd != 0>(sb + ri0 * S, sb + TI * S + cj0 * S,
                                                              A, NB, pr, asum, acc, lane);
#pragma unroll
            for (int b = 1; b < SUB; ++b) {
                const float *rb = sb + b * CHUNK_FLOATS + ri0 * S;
                const float *cb2 = sb + b * CHUNK_FLOATS + TI * S + cj0 * S;
                if constexpr (G.hmajor != 0)
                    pair_chunk_pk_h<WI, WJ, S, false, G.absadd != 0>(rb, cb2, A, NB, pr, asum, acc,
                                                                     lane);
                else
                    pair_chunk_pk<WI, WJ, S, false, G.absadd != 0>(rb, cb2, A, NB, pr, asum, acc,
                                                                   lane);
            }
            pending = true;
        } else
#pragma unroll
        for (int b = 0; b < SUB; ++b) {
            const int ch = k * SUB + b;
            if (ch >= nck) break;
            const float *rows = sb + b * CHUNK_FLOATS + ri0 * S;
            const float *cols = sb + b * CHUNK_FLOATS + TI * S + cj0 * S;
            const int valid = min(S, P.n - (c0 + ch) * S);
            if (PK && valid == S) {
                if (b == 0)
                    pair_chunk_pk<WI, WJ, S, true, G.absadd != 0>(rows, cols, A, NB, pr, asum, acc,
                                                                  lane);
                else
                    pair_chunk_pk<WI, WJ, S, false, G.absadd != 0>(rows, cols, A, NB, pr, asum, acc,
                                                                   lane);
                pending = true;
            } else {
                float tca[WI][WJ], tcb[WI][WJ], t2[WI][WJ];
#pragma unroll
                for (int r = 0; r < WI; ++r)
#pragma unroll
                    for (int c = 0; c < WJ; ++c) {
                        tca[r][c] = A[r][c].x;
                        tcb[r][c] = -NB[r][c].x;
                        t2[r][c] = 0.0f;
                    }
                if (valid == S)
                    pair_chunk<MODE, false, WI, WJ, S, G.groups, false>(rows, cols, tca, tcb, a1,
                                                                        t2, lane, valid);
                else
                    pair_chunk<MODE, true, WI, WJ, S, G.groups, false>(rows, cols, tca, tcb, a1,
                                                                       t2, lane, valid);
#pragma unroll
                for (int r = 0; r < WI; ++r)
#pragma unroll
                    for (int c = 0; c < WJ; ++c) acc[r][c].x += t2[r][c];
            }
        }
        if (PK && pending) {
            // sum log2(2 cosh u) over the stage's full chunks: C3 sum |u~| +
            // lg2 of the product of their 1 + y factors
#pragma unroll
            for (int r = 0; r < WI; ++r)
#pragma unroll
                for (int c = 0; c < WJ; ++c)
                    a1[r][c] += fmaf(asum[r][c], FAST_C3, lg2_approx(pr[r][c].x * pr[r][c].y));
        }
        // fold the period's FP32 sums into (hi, lo) pairs every FOLD chunks
        // (FOLD is a multiple of SUB) and after the last stage
        if ((((k + 1) * SUB) & (FOLD - 1)) == 0 || k == nst - 1) {
#pragma unroll
            for (int r = 0; r < WI; ++r)
#pragma unroll
                for (int c = 0; c < WJ; ++c) {
                    float t, err;
                    two_sum(s1[r][c], a1[r][c], t, err);
                    s1[r][c] = t;
                    e1[r][c] += err;
                    two_sum(s2[r][c], acc[r][c].x + acc[r][c].y, t, err);
                    s2[r][c] = t;
                    e2[r][c] += err;
                    a1[r][c] = 0.0f;
                    acc[r][c] = make_float2(0.0f, 0.0f);
                }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
        if (++st == STAGES) {
            st = 0;
            ph ^= 1u;
        }
        if (*abort_flag) break;
    }

    // never leave with a copy in flight (bounded waits on the last phases)
    if (threadIdx.x == 0)
        for (int k = max(0, issued - STAGES); k < issued; ++k)
            (void)mbar_wait_bounded(&full[k % STAGES], (k / STAGES) & 1);

    // Cross-lane reduction through shared memory, one moment at a time: each
    // lane stores its (hi, lo) sums, then lane L adds the sums of 32 / LPC
    // source lanes for one pair (compensated, fixed order) and LPC lanes
    // join by xor shuffles.  The ring is free once every warp has passed the
    // barrier below (thread 0 has waited for the last copies).
    __syncthreads();
    constexpr int NP = WI * WJ;
    constexpr int LPC = 32 / NP;   // lanes per pair
    constexpr int SRC = 32 / LPC;  // source lanes summed by each lane
    static_assert(32 % NP == 0, "pairs per warp divide the warp");
    float *red = buf + warp * (NP * 2 * 33);   // [NP][hi, lo][33], padded rows
    float2 *mom = P.mom + (size_t)split * P.p * P.p * 2;
    const int e = lane / LPC, part = lane % LPC;
    const int pi = pi0 + e / WJ, pj = pj0 + e % WJ;
#pragma unroll
    for (int m = 0; m < 2; ++m) {
#pragma unroll
        for (int r = 0; r < WI; ++r)
#pragma unroll
            for (int c = 0; c < WJ; ++c) {
                const int q = r * WJ + c;
                red[(q * 2 + 0) * 33 + lane] = m == 0 ? s1[r][c] : s2[r][c];
                red[(q * 2 + 1) * 33 + lane] = m == 0 ? e1[r][c] : e2[r][c];
            }
        __syncwarp();
        float h = 0.0f, l = 0.0f;
#pragma unroll
        for (int k2 = 0; k2 < SRC; ++k2) {
            const int src = part * SRC + k2;
            float t, err;
            two_sum(h, red[(e * 2 + 0) * 33 + src], t, err);
            h = t;
            l = (l + red[(e * 2 + 1) * 33 + src]) + err;
        }
#pragma unroll
        for (int o = LPC / 2; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, h, o);
            const float ol = __shfl_xor_sync(0xffffffffu, l, o);
            float t, err;
            two_sum(h, oh, t, err);
            h = t;
            l = (l + ol) + err;
        }
        if (part == 0 && pi < P.p && pj < P.p && pi != pj) {
            float t, err;
            two_sum(h, l, t, err);
            mom[((size_t)pi * P.p + pj) * 2 + m] = make_float2(t, err);
        }
        __syncwarp();
    }
}

// One launch covers the tiles of every instance in the batch: prefix[k] is the
// first CTA of instance k (tiles_i * tiles_j * nsplit CTAs each).
template <int MODE, int CFG>
__device__ __forceinline__ void pair_dispatch(const CUtensorMap *tmI, const CUtensorMap *tmJ,
                                              const PairParams *__restrict__ Ps,
                                              const int *__restrict__ prefix, int count)
{
    const int b = blockIdx.x;
    const int lo = find_instance(prefix, count, b);
    const PairParams P = Ps[lo];
    const int local = b - prefix[lo];
    const int tiles = P.tiles_i * P.tiles_j;
    const int split = local / tiles, tile = local % tiles;
    if (P.shard_n > 1 &&
        shard_owner((tile / P.tiles_j) * PAIR_CFGS[CFG].ti(), (tile % P.tiles_j) * PAIR_CFGS[CFG].tj(),
                    P.p, P.shard_n) != P.shard_rank)
        return;   // another rank's tile
    if constexpr (PAIR_CFGS[CFG].sub > 0)
        pair_block_v2<MODE, CFG>(tmI, tmJ, P, tile / P.tiles_j, tile % P.tiles_j, split);
    else
        pair_block<MODE, CFG>(tmI, tmJ, P, tile / P.tiles_j, tile % P.tiles_j, split);
}

// One kernel per form and tile configuration; the register cap of each
// fixes how many CTAs share an SM (see PAIR_CFGS).
template <int CFG>
__global__ void __maxnreg__(PAIR_CFGS[CFG].reg_fast)
    k_pair_fast_b(const __grid_constant__ CUtensorMap tmI, const __grid_constant__ CUtensorMap tmJ,
                  const PairParams *__restrict__ Ps, const int *__restrict__ prefix, int count)
{
    pair_dispatch<PAIR_FAST, CFG>(&tmI, &tmJ, Ps, prefix, count);
}

template <int CFG>
__global__ void __maxnreg__(PAIR_CFGS[CFG].reg_acc)
    k_pair_accurate_b(const __grid_constant__ CUtensorMap tmI,
                      const __grid_constant__ CUtensorMap tmJ, const PairParams *__restrict__ Ps,
                      const int *__restrict__ prefix, int count)
{
    pair_dispatch<PAIR_ACCURATE, CFG>(&tmI, &tmJ, Ps, prefix, count);
}

using PairKernel = void (*)(const CUtensorMap, const CUtensorMap, const PairParams *, const int *,
                            int);

template <int... C>
struct PairTable {
    static constexpr PairKernel fast[sizeof...(C)] = {k_pair_fast_b<C>...};
    static constexpr PairKernel acc[sizeof...(C)] = {k_pair_accurate_b<C>...};
};
using PairKernels = PairTable<0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19,
                              20, 21, 22, 23, 24, 25, 26, 27, 28, 29, 30, 31, 32>;
static_assert(PAIR_NCFG == 33, "PairKernels lists every configuration");

static PairKernel pair_kernel(int mode, int cfg)
{
    return mode == PAIR_FAST ? PairKernels::fast[cfg] : PairKernels::acc[cfg];
}

size_t pair_smem_bytes(int cfg)
{
    const PairCfg &G = PAIR_CFGS[cfg];
    return 1024 + (size_t)G.stages * (G.sub > 0 ? G.sub : 1) * (G.ti() + G.tj()) * PAIR_S * 4;
}

static int g_pair_occ[2][PAIR_NCFG];

cudaError_t pair_kernel_setup()
{
    for (int mode = 0; mode < 2; ++mode)
        for (int c = 0; c < PAIR_NCFG; ++c) {
            const void *fn = reinterpret_cast<const void *>(pair_kernel(mode, c));
            cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)pair_smem_bytes(c));
            if (e != cudaSuccess) return e;
            int occ = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, PAIR_CFGS[c].threads(),
                                                              pair_smem_bytes(c));
            if (e != cudaSuccess) return e;
            g_pair_occ[mode][c] = std::max(1, occ);
        }
    return cudaSuccess;
}

int pair_ctas_per_sm(int mode, int cfg) { return g_pair_occ[mode == PAIR_FAST][cfg]; }

cudaError_t launch_pair_b(int mode, int cfg, const CUtensorMap *tmI, const CUtensorMap *tmJ,
                          const PairParams *P, const int *prefix, int count, int total_ctas,
                          cudaStream_t s)
{
    if (total_ctas <= 0 || count <= 0) return cudaSuccess;
    if (cfg < 0 || cfg >= PAIR_NCFG) return cudaErrorInvalidValue;
    pair_kernel(mode, cfg)<<<total_ctas, PAIR_CFGS[cfg].threads(), pair_smem_bytes(cfg), s>>>(
        *tmI, *tmJ, P, prefix, count);
    return cudaGetLastError();
}

}  // namespace lg
