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

// One chunk of S samples for the WI x WJ pairs of a warp: lane l takes the
// four consecutive samples 128 it + 4 l .. + 3 (one 16-byte shared load per
// column).  Fast form: sum_s log2(2 cosh u_s) = log2(e)/k sum |u~_s| +
// sum_s log2(1 + y_s); the second sum is taken as log2 of the product of
// the four (1 + y_s) in (1, 16], one MUFU lg2 per four samples instead of
// four (the logarithm of a product is the sum of the logarithms).
template <int MODE, bool TAIL, int WI, int WJ, int S>
__device__ __forceinline__ void pair_chunk(const float *__restrict__ rows,
                                           const float *__restrict__ cols,
                                           const float (&ca)[WI][WJ], const float (&cb)[WI][WJ],
                                           float (&a1)[WI][WJ], float (&a2)[WI][WJ], int lane,
                                           int valid)
{
#pragma unroll 1
    for (int it = 0; it < S / 128; ++it) {
        const int s = it * 128 + lane * 4;
        float4 zi[WI], zj[WJ];
#pragma unroll
        for (int r = 0; r < WI; ++r) zi[r] = *reinterpret_cast<const float4 *>(rows + r * S + s);
#pragma unroll
        for (int c = 0; c < WJ; ++c) zj[c] = *reinterpret_cast<const float4 *>(cols + c * S + s);
        bool ok[4] = {true, true, true, true};
        if (TAIL) {
#pragma unroll
            for (int v = 0; v < 4; ++v) ok[v] = (s + v) < valid;
        }
#pragma unroll
        for (int r = 0; r < WI; ++r) {
            const float zr[4] = {zi[r].x, zi[r].y, zi[r].z, zi[r].w};
#pragma unroll
            for (int c = 0; c < WJ; ++c) {
                const float zc[4] = {zj[c].x, zj[c].y, zj[c].z, zj[c].w};
                if (MODE == PAIR_FAST) {
                    float q[4], au[4];
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const float u = fmaf(ca[r][c], zr[v], -(cb[r][c] * zc[v]));
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
                        q[v] = 1.0f + y;
                        au[v] = a;
                    }
                    const float prod = (q[0] * q[1]) * (q[2] * q[3]);
                    const float asum = (au[0] + au[1]) + (au[2] + au[3]);
                    a1[r][c] += fmaf(asum, FAST_C3, lg2_approx(prod));
                } else {
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const float u = fmaf(ca[r][c], zr[v], -(cb[r][c] * zc[v]));
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

template <int MODE>
__device__ __forceinline__ void pair_block(const CUtensorMap *tmI, const CUtensorMap *tmJ,
                                           const PairParams &P, const int ti, const int tj,
                                           const int split)
{
    constexpr int WI = PAIR_WI, WJ = PAIR_WJ, WGJ = PAIR_WGJ;
    constexpr int NCW = PAIR_WGI * PAIR_WGJ;
    constexpr int TI = PAIR_TI, TJ = PAIR_TJ, S = PAIR_S, STAGES = PAIR_STAGES;
    constexpr uint32_t STAGE_FLOATS = (TI + TJ) * S;
    constexpr uint32_t STAGE_BYTES = STAGE_FLOATS * 4;
    constexpr bool COMP = (MODE == PAIR_FAST);

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
    constexpr int FOLD = 4;

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
                pair_chunk<MODE, false, WI, WJ, S>(rows, cols, ca, cb, a1, a2, lane, valid);
            else
                pair_chunk<MODE, true, WI, WJ, S>(rows, cols, ca, cb, a1, a2, lane, valid);
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
                pair_chunk<MODE, false, WI, WJ, S>(rows, cols, ca, cb, s1, s2, lane, valid);
            else
                pair_chunk<MODE, true, WI, WJ, S>(rows, cols, ca, cb, s1, s2, lane, valid);
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
    double *mom = P.mom + (size_t)split * P.p * P.p * 2;
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
                double *o = mom + ((size_t)pi * P.p + pj) * 2;
                o[0] = (double)h1 + (double)l1;
                o[1] = (double)h2 + (double)l2;
            }
        }
    }
}

// One launch covers the tiles of every instance in the batch: prefix[k] is the
// first CTA of instance k (tiles_i * tiles_j * nsplit CTAs each).
template <int MODE>
__device__ __forceinline__ void pair_dispatch(const CUtensorMap *tmI, const CUtensorMap *tmJ,
                                              const PairParams *__restrict__ Ps,
                                              const int *__restrict__ prefix, int count)
{
    int lo = 0, hi = count - 1;
    const int b = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const PairParams P = Ps[lo];
    const int local = b - prefix[lo];
    const int tiles = P.tiles_i * P.tiles_j;
    const int split = local / tiles, tile = local % tiles;
    pair_block<MODE>(tmI, tmJ, P, tile / P.tiles_j, tile % P.tiles_j, split);
}

// Register budgets (256 threads per CTA): the compensated fast form keeps
// three FP32 words per accumulator and runs one CTA per SM with up to 248
// registers; the accurate form runs two CTAs per SM with up to 120.
__global__ void __maxnreg__(248)
    k_pair_fast_b(const __grid_constant__ CUtensorMap tmI, const __grid_constant__ CUtensorMap tmJ,
                  const PairParams *__restrict__ Ps, const int *__restrict__ prefix, int count)
{
    pair_dispatch<PAIR_FAST>(&tmI, &tmJ, Ps, prefix, count);
}

__global__ void __maxnreg__(120)
    k_pair_accurate_b(const __grid_constant__ CUtensorMap tmI,
                      const __grid_constant__ CUtensorMap tmJ, const PairParams *__restrict__ Ps,
                      const int *__restrict__ prefix, int count)
{
    pair_dispatch<PAIR_ACCURATE>(&tmI, &tmJ, Ps, prefix, count);
}

static size_t pair_smem_bytes()
{
    return 1024 + (size_t)PAIR_STAGES * (PAIR_TI + PAIR_TJ) * PAIR_S * 4;
}

cudaError_t pair_kernel_setup()
{
    cudaError_t e = cudaFuncSetAttribute(k_pair_accurate_b,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pair_smem_bytes());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_pair_fast_b, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)pair_smem_bytes());
}

cudaError_t launch_pair_b(int mode, const CUtensorMap *tmI, const CUtensorMap *tmJ,
                          const PairParams *P, const int *prefix, int count, int total_ctas,
                          cudaStream_t s)
{
    if (total_ctas <= 0 || count <= 0) return cudaSuccess;
    if (mode == PAIR_FAST)
        k_pair_fast_b<<<total_ctas, PAIR_THREADS, pair_smem_bytes(), s>>>(*tmI, *tmJ, P, prefix,
                                                                         count);
    else
        k_pair_accurate_b<<<total_ctas, PAIR_THREADS, pair_smem_bytes(), s>>>(*tmI, *tmJ, P,
                                                                             prefix, count);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// FP64 pair moments (whole step in FP64 mode, or re-scoring of candidates)
// ------------------------------------------------------------------------
//
// One warp per work item, lanes stride the samples, FP64 throughout with the
// CUDA double exp/log1p.  An item is either an unordered pair {a, b} (both
// residual directions) or a single variable (moments of z itself).
__device__ __forceinline__ void f64_terms(double u, double &t1, double &t2)
{
    const double au = fabs(u);
    t1 = au + log1p(exp(-2.0 * au));      // log cosh u + ln 2
    t2 = u * exp(-0.5 * u * u);
}

__device__ __forceinline__ void pairs_f64_body(const F64Params &P)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    int cbeg = 0;
    int64_t npair_items;
    bool with_vars = true;
    if (P.mode == 1) {
        if (P.state->resolved) return;
        cbeg = P.state->pass_begin;
        const int cend = P.state->pass_end;
        if (cend <= cbeg) return;
        npair_items = (int64_t)(cend - cbeg) * P.p;
        with_vars = (P.pass == 1);
    } else {
        npair_items = (int64_t)P.p * (P.p - 1) / 2;
    }
    const int64_t nitems = npair_items + (with_vars ? P.p : 0);

    for (int64_t q = gw; q < nitems; q += nw) {
        if (q >= npair_items) {
            const int a = (int)(q - npair_items);
            const int oa = P.U[a];
            const double inv = 1.0 / sqrt(P.C[(int64_t)oa * P.ldc + oa]);
            const double *ra = P.R + (int64_t)oa * P.ldr;
            double s1 = 0.0, s2 = 0.0;
            for (int s = lane; s < P.n; s += 32) {
                double t1, t2;
                f64_terms(ra[s] * inv, t1, t2);
                s1 += t1;
                s2 += t2;
            }
            s1 = warp_sum_xor(s1);
            s2 = warp_sum_xor(s2);
            if (lane == 0) {
                P.hz[(size_t)a * 2 + 0] = s1;
                P.hz[(size_t)a * 2 + 1] = s2;
            }
            continue;
        }
        int a, b, cidx = 0;
        if (P.mode == 1) {
            cidx = cbeg + (int)(q / P.p);
            a = P.state->cand[cidx];
            b = (int)(q % P.p);
            // I32(a, b) >= epsI proves I(a, b) >= 0: min(0, I)^2 = 0 exactly,
            // so the entry needs no FP64 moments (marked by a negative sum)
            if (a == b || (P.I32 && P.I32[(size_t)a * P.p + b] >= P.epsI)) {
                if (lane == 0) {
                    double *o = P.mom + ((size_t)cidx * P.p + b) * 4;
                    o[0] = -1.0;
                    o[1] = o[2] = o[3] = 0.0;
                }
                continue;
            }
        } else {
            // unordered pair index q -> (a, b), a < b
            const double pp = (double)P.p;
            int64_t aa = (int64_t)floor(((2.0 * pp - 1.0) -
                                         sqrt((2.0 * pp - 1.0) * (2.0 * pp - 1.0) - 8.0 * (double)q)) /
                                        2.0);
            auto first = [&](int64_t x) { return x * (2 * (int64_t)P.p - x - 1) / 2; };
            if (aa < 0) aa = 0;
            while (aa > 0 && first(aa) > q) --aa;
            while (first(aa + 1) <= q) ++aa;
            a = (int)aa;
            b = (int)(a + 1 + (q - first(aa)));
        }
        const int oa = P.U[a], ob = P.U[b];
        const int lo = min(oa, ob), hi = max(oa, ob);
        const double caa = P.C[(int64_t)oa * P.ldc + oa], cbb = P.C[(int64_t)ob * P.ldc + ob];
        const double rho = P.C[(int64_t)lo * P.ldc + hi] / (sqrt(caa) * sqrt(cbb));
        double s2v = 1.0 - rho * rho;
        if (!(s2v > 1e-12)) {
            if (lane == 0) set_status(P.status, ST_DEGENERATE);
            s2v = 1.0;
        }
        const double isd = 1.0 / sqrt(s2v);
        const double ia = 1.0 / sqrt(caa), ib = 1.0 / sqrt(cbb);
        const double *ra = P.R + (int64_t)oa * P.ldr, *rb = P.R + (int64_t)ob * P.ldr;
        double ab1 = 0.0, ab2 = 0.0, ba1 = 0.0, ba2 = 0.0;
        for (int s = lane; s < P.n; s += 32) {
            const double za = ra[s] * ia, zb = rb[s] * ib;
            double t1, t2;
            f64_terms((za - rho * zb) * isd, t1, t2);    // residual of a given b
            ab1 += t1;
            ab2 += t2;
            f64_terms((zb - rho * za) * isd, t1, t2);    // residual of b given a
            ba1 += t1;
            ba2 += t2;
        }
        ab1 = warp_sum_xor(ab1);
        ab2 = warp_sum_xor(ab2);
        ba1 = warp_sum_xor(ba1);
        ba2 = warp_sum_xor(ba2);
        if (lane == 0) {
            if (P.mode == 1) {
                double *o = P.mom + ((size_t)cidx * P.p + b) * 4;
                o[0] = ab1;
                o[1] = ab2;
                o[2] = ba1;
                o[3] = ba2;
            } else {
                double *o = P.mom + ((size_t)a * P.p + b) * 2;
                o[0] = ab1;
                o[1] = ab2;
                o = P.mom + ((size_t)b * P.p + a) * 2;
                o[0] = ba1;
                o[1] = ba2;
            }
        }
    }
}

// blockIdx.y selects the instance; the x blocks stride its work items.
__global__ void __launch_bounds__(256) k_pairs_f64_b(const F64Params *__restrict__ Ps)
{
    const F64Params P = Ps[blockIdx.y];
    pairs_f64_body(P);
}

cudaError_t launch_pairs_f64_b(const F64Params *P, int count, int blocks_per_inst, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    k_pairs_f64_b<<<dim3(blocks_per_inst, count), 256, 0, s>>>(P);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// Score: I(i, j) and M(i) (Algorithm 1, deterministic FP64 combine)
// ------------------------------------------------------------------------
//
// I(i, j) = (h(z_j) + h(r_i^j)) - (h(z_i) + h(r_j^i)) with h = H - H(nu);
// M(i) = -sum_{j != i} min(0, I(i, j))^2, summed by each lane over j in
// ascending order and across lanes by a fixed xor tree.  E(i) bounds |M(i) -
// M_exact(i)| given |I - I_exact| <= epsI.
__global__ void __launch_bounds__(256) k_score_b(const ScoreParams *__restrict__ Ps)
{
    extern __shared__ double hsh[];   // h(z_j), j < p
    const ScoreParams P = Ps[blockIdx.y];
    if ((int)blockIdx.x * (int)(blockDim.x >> 5) >= P.p) return;
    const double invn = 1.0 / (double)P.n;
    for (int j = threadIdx.x; j < P.p; j += blockDim.x) {
        double S1 = 0.0, S2 = 0.0;
        for (int s = 0; s < P.nsplit_hz; ++s) {
            S1 += P.hz[((size_t)s * P.p + j) * 2 + 0];
            S2 += P.hz[((size_t)s * P.p + j) * 2 + 1];
        }
        hsh[j] = neg_entropy_part(P.ha1 * S1 * invn + P.hb1, P.ha2 * S2 * invn);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= P.p) return;
    const size_t plane = (size_t)P.p * P.p * 2;
    const double hi = hsh[i];
    double acc = 0.0, err = 0.0;
    const double eps = P.epsI;
    for (int j = lane; j < P.p; j += 32) {
        if (j == i) continue;
        double a1 = 0.0, a2 = 0.0, b1 = 0.0, b2 = 0.0;
        const double *pij = P.mom + ((size_t)i * P.p + j) * 2;
        const double *pji = P.mom + ((size_t)j * P.p + i) * 2;
        for (int s = 0; s < P.nsplit; ++s) {
            a1 += pij[s * plane];
            a2 += pij[s * plane + 1];
            b1 += pji[s * plane];
            b2 += pji[s * plane + 1];
        }
        const double hij = neg_entropy_part(P.a1 * a1 * invn + P.b1, P.a2 * a2 * invn);
        const double hji = neg_entropy_part(P.a1 * b1 * invn + P.b1, P.a2 * b2 * invn);
        const double I = (hsh[j] + hij) - (hi + hji);
        const double v = fmin(0.0, I);
        acc += v * v;
        if (I < eps) err += 2.0 * fabs(v) * eps + eps * eps;
        if (P.Iout) P.Iout[(size_t)i * P.p + j] = I;
        if (P.I32) P.I32[(size_t)i * P.p + j] = (float)I;
    }
    acc = warp_sum_xor(acc);
    err = warp_sum_xor(err);
    if (lane == 0) {
        P.M[i] = -acc;
        P.E[i] = err;
        if (P.hist) P.hist[P.U[i]] = -acc;
    }
}

cudaError_t launch_score_b(const ScoreParams *P, int count, int maxp, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    const int rows_per_block = 8;
    dim3 grid((maxp + rows_per_block - 1) / rows_per_block, count);
    k_score_b<<<grid, 256, sizeof(double) * maxp, s>>>(P);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// Select: argmax of M (ties to the smallest original index) and the set of
// candidates whose score intervals [M - E, M + E] reach the leader's.
// ------------------------------------------------------------------------
__device__ __forceinline__ bool better(double m, int u, double bm, int bu)
{
    return (m > bm) || (m == bm && u < bu);
}

__global__ void __launch_bounds__(1024) k_select_b(const SelectParams *__restrict__ Ps)
{
    const SelectParams P = Ps[blockIdx.x];
    __shared__ double sm[32];
    __shared__ int su[32], sp[32];
    __shared__ int s_top, s_cnt;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    double bm = -INFINITY;
    int bu = 0x7fffffff, bp = -1;
    for (int q = tid; q < P.p; q += blockDim.x) {
        const double m = P.M[q];
        const int u = P.U[q];
        if (bp < 0 || better(m, u, bm, bu)) {
            bm = m;
            bu = u;
            bp = q;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double om = __shfl_xor_sync(0xffffffffu, bm, o);
        const int ou = __shfl_xor_sync(0xffffffffu, bu, o);
        const int op = __shfl_xor_sync(0xffffffffu, bp, o);
        if (op >= 0 && (bp < 0 || better(om, ou, bm, bu))) {
            bm = om;
            bu = ou;
            bp = op;
        }
    }
    if (lane == 0) {
        sm[w] = bm;
        su[w] = bu;
        sp[w] = bp;
    }
    if (tid == 0) s_cnt = 0;
    __syncthreads();
    if (tid == 0) {
        int best = -1;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k)
            if (sp[k] >= 0 && (best < 0 || better(sm[k], su[k], sm[best], su[best]))) best = k;
        s_top = sp[best];
    }
    __syncthreads();
    const int top = s_top;
    const double thr = P.M[top] - P.E[top];
    // unordered compaction of the candidates (their order is fixed below)
    for (int q = tid; q < P.p; q += blockDim.x)
        if (P.M[q] + P.E[q] >= thr) P.scratch[atomicAdd(&s_cnt, 1)] = q;
    __syncthreads();
    const int cnt = s_cnt;
    DevState *st = P.state;
    if (cnt <= 1) {
        if (tid == 0) {
            st->m_pos = top;
            st->ncand = 1;
            st->resolved = 1;
            st->pass_begin = st->pass_end = 0;
        }
        return;
    }
    // rank by upper bound M + E descending, ties to the smaller original index;
    // keep the first MAXC
    for (int k = tid; k < cnt; k += blockDim.x) {
        const int q = P.scratch[k];
        const double ub = P.M[q] + P.E[q];
        const int u = P.U[q];
        int rank = 0;
        for (int k2 = 0; k2 < cnt; ++k2) {
            const int q2 = P.scratch[k2];
            const double ub2 = P.M[q2] + P.E[q2];
            rank += (ub2 > ub) || (ub2 == ub && P.U[q2] < u);
        }
        if (rank < MAXC) {
            st->cand[rank] = q;
            st->ub[rank] = ub;
        }
    }
    if (tid == 0) {
        const int nc = min(cnt, MAXC);
        st->m_pos = top;
        st->ncand = nc;
        st->resolved = 0;
        st->pass_begin = 0;
        st->pass_end = min(2, nc);
        st->refined_steps += 1;
        if (cnt > st->cand_max) st->cand_max = cnt;
        if (cnt > MAXC) st->cand_overflow += 1;
    }
}

cudaError_t launch_select_b(const SelectParams *P, int count, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    k_select_b<<<count, 1024, 0, s>>>(P);
    return cudaGetLastError();
}

// FP64 re-score of a pass of candidates.  Pass 1 scores the two candidates
// with the highest upper bounds; if the better of them beats every remaining
// upper bound the step is decided, otherwise pass 2 scores the rest and the
// argmax is taken over all FP64 scores (ties to the smallest original index).
__global__ void __launch_bounds__(256) k_refine_select_b(const RefineSelectParams *__restrict__ Ps)
{
    extern __shared__ double h64[];
    const RefineSelectParams P = Ps[blockIdx.x];
    DevState *st = P.state;
    if (st->resolved) return;
    const int cb = st->pass_begin, ce = st->pass_end, nc = st->ncand;
    const double invn = 1.0 / (double)P.n;
    for (int j = threadIdx.x; j < P.p; j += blockDim.x)
        h64[j] = neg_entropy_part(P.hz[(size_t)j * 2] * invn - LN2_D, P.hz[(size_t)j * 2 + 1] * invn);
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = cb + w; c < ce; c += nw) {
        const int pc = st->cand[c];
        double acc = 0.0;
        for (int j = lane; j < P.p; j += 32) {
            if (j == pc) continue;
            const double *o = P.mom + ((size_t)c * P.p + j) * 4;
            if (o[0] < 0.0) continue;
            const double hcj = neg_entropy_part(o[0] * invn - LN2_D, o[1] * invn);
            const double hjc = neg_entropy_part(o[2] * invn - LN2_D, o[3] * invn);
            const double I = (h64[j] + hcj) - (h64[pc] + hjc);
            const double v = fmin(0.0, I);
            acc += v * v;
        }
        acc = warp_sum_xor(acc);
        if (lane == 0) st->m64[c] = -acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int best = 0;
        for (int c = 1; c < ce; ++c)
            if (better(st->m64[c], P.U[st->cand[c]], st->m64[best], P.U[st->cand[best]])) best = c;
        st->fp64_candidates += ce - cb;
        if (P.hist)
            for (int c = cb; c < ce; ++c) P.hist[P.U[st->cand[c]]] = st->m64[c];
        if (ce < nc && !(st->m64[best] > st->ub[ce])) {
            st->pass_begin = ce;       // undecided: score the rest in pass 2
            st->pass_end = nc;
            return;
        }
        double mx = 0.0, gap = INFINITY;
        for (int c = 0; c < ce; ++c) mx = fmax(mx, fabs(st->m64[c]));
        for (int c = 0; c < ce; ++c)
            if (c != best) gap = fmin(gap, st->m64[best] - st->m64[c]);
        if (gap <= 1e-9 * mx) st->genuine_ties += 1;
        st->m_pos = st->cand[best];
        st->resolved = 1;
    }
}

cudaError_t launch_refine_select_b(const RefineSelectParams *P, int count, int maxp, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    k_refine_select_b<<<count, 256, sizeof(double) * maxp, s>>>(P);
    return cudaGetLastError();
}

}  // namespace lg
