// kernels_refine.cu -- high-precision re-scoring of near-tied candidates.
//
// The FP32 pair-moment kernel gives every I(i, j) of Algorithm 1 with a known
// error bound; at steps where the top scores M(i) lie within that bound of
// each other the argmax is decided by re-scoring the candidates:
//
//   tier 1  double-float ("df"): every quantity carried as an unevaluated sum
//           hi + lo of two FP32 numbers (about 48 significant bits), with
//           table-driven exp and log written for it, so the work runs on the
//           FP32 pipe.  Each I(i, j) carries a bound epsI2 on its error.
//   tier 2  FP64 with the CUDA double-precision exp/log1p, for the candidates
//           whose df score intervals still overlap.  GB300 runs FP64 at about
//           1/75 of its FP32 rate, so this tier only sees genuine near-ties.
//
// The same kernels also score whole steps (mode 0: every pair) in df or FP64.
// Work item = one unordered pair {a, b} (both residual directions) or one
// variable (moments of z itself), cut into sample ranges; a warp owns one
// (item, range) unit and its lanes stride the samples, and the sums run over
// fixed xor trees (deterministic results).

#include <math.h>

#include "df.cuh"
#include "kernels.cuh"

namespace lg {

// ln2/128 split as L1 + L2 + L3: L1 = 709 * 2^-17 has 10 significant bits, so
// N * L1 is exact for |N| < 2^14; L2 and L3 are the next FP32 pieces
// (remainder below 5e-21).
constexpr float EXP_L1 = 0x1.628p-8f;
constexpr float EXP_L2 = 0x1.90bfbep-18f;
constexpr float EXP_L3 = 0x1.1cf79ap-43f;
constexpr float EXP_INV_L = 0x1.715476p+7f;   // 128 / ln2
constexpr int EXP_TAB = 128;                  // 2^(j/128), j < 128
constexpr int LOG_TAB = 257;                  // c_k = 1 + k/256, k <= 256

__device__ float2 g_exp_tab[EXP_TAB];         // hi, lo of 2^(j/128)
__device__ float4 g_log_tab[LOG_TAB];         // hi, lo of 1/c_k; hi, lo of log c_k

// exp(x) for x <= 0 by the table-driven method of P. T. P. Tang (ACM TOMS
// 15(2), 1989), in double-float: x = (128 m + j) ln2/128 + r with
// |r| <= ln2/256, exp(x) = 2^m 2^(j/128) exp(r), exp(r) by its Taylor series
// to r^5 (the r^6 term is below 6e-19).  Returns 0 for x < -87 (exp(x) below
// the smallest normal FP32 number).
__device__ __forceinline__ dfl df_exp_nonpos(dfl x, const float2 *tab)
{
    if (!(x.hi > -87.0f)) return {0.0f, 0.0f};
    const float N = rintf(__fmul_rn(x.hi, EXP_INV_L));      // -16066 <= N <= 0
    const int Ni = __float2int_rn(N);
    const int j = Ni & (EXP_TAB - 1), m = Ni >> 7;          // Ni = 128 m + j
    const float t0 = __fmaf_rn(-N, EXP_L1, x.hi);           // exact (Sterbenz)
    const dfl pq = df_two_prod(N, EXP_L2);
    const dfl s = df_two_sum(t0, -pq.hi);
    const float low = __fadd_rn(__fsub_rn(s.lo, pq.lo), __fsub_rn(x.lo, __fmul_rn(N, EXP_L3)));
    const dfl r = df_two_sum(s.hi, low);
    dfl r2 = df_two_prod(r.hi, r.hi);
    r2.lo = __fmaf_rn(__fmul_rn(2.0f, r.hi), r.lo, r2.lo);
    const float rh = r.hi;
    const float q = rh * rh * rh * (1.0f / 6.0f + rh * (1.0f / 24.0f + rh * (1.0f / 120.0f)));
    const dfl a = df_fast_two_sum(1.0f, r.hi);
    const dfl b = df_fast_two_sum(a.hi, __fmul_rn(0.5f, r2.hi));
    const float lo = __fadd_rn(__fadd_rn(a.lo, b.lo),
                               __fadd_rn(r.lo, __fmaf_rn(0.5f, r2.lo, q)));
    const dfl e = df_fast_two_sum(b.hi, lo);
    const float2 T = tab[j];
    const dfl v = df_mul(e, dfl{T.x, T.y});
    const float sc = __int_as_float((m + 127) << 23);       // 2^m, m >= -126
    return {__fmul_rn(v.hi, sc), __fmul_rn(v.lo, sc)};
}

// log(1 + v) for 0 <= v <= 1 by table-driven reduction (P. T. P. Tang, ACM
// TOMS 16(4), 1990): 1 + v = c_k (1 + d) with c_k = 1 + k/256, |d| <= 1/512,
// log(1 + v) = log c_k + log(1 + d), the latter by its Taylor series to d^5
// (the d^6 term is below 1e-17).
__device__ __forceinline__ dfl df_log1p_unit(dfl v, const float4 *tab)
{
    const dfl w = df_fast_two_sum(1.0f, v.hi);
    const float wlo = __fadd_rn(w.lo, v.lo);
    const int k = min(max(__float2int_rn(__fmul_rn(__fsub_rn(w.hi, 1.0f), 256.0f)), 0),
                      LOG_TAB - 1);
    const float4 T = tab[k];
    const float dh = __fsub_rn(w.hi, __fmaf_rn((float)k, 0x1p-8f, 1.0f));   // exact
    const float p = __fmul_rn(dh, T.x);
    float e = __fmaf_rn(dh, T.x, -p);
    e = __fmaf_rn(dh, T.y, e);
    e = __fmaf_rn(wlo, T.x, e);
    const dfl d = df_two_sum(p, e);
    dfl d2 = df_two_prod(d.hi, d.hi);
    d2.lo = __fmaf_rn(__fmul_rn(2.0f, d.hi), d.lo, d2.lo);
    const float dd = d.hi;
    const float q = dd * dd * dd * (1.0f / 3.0f + dd * (-0.25f + dd * 0.2f));
    const dfl s1 = df_two_sum(T.z, d.hi);
    const dfl s2 = df_two_sum(s1.hi, __fmul_rn(-0.5f, d2.hi));
    const float lo = __fadd_rn(__fadd_rn(s1.lo, s2.lo),
                               __fadd_rn(T.w, __fadd_rn(d.lo, __fmaf_rn(-0.5f, d2.lo, q))));
    return df_fast_two_sum(s2.hi, lo);
}

// The two moment terms of one residual value u:
//   t1 = log cosh u + ln 2 = |u| + log(1 + exp(-2|u|)),   t2 = u exp(-u^2/2).
__device__ __forceinline__ void df_terms(dfl u, dfl &t1, dfl &t2, const float2 *et,
                                         const float4 *lt)
{
    const dfl a = u.hi < 0.0f ? dfl{-u.hi, -u.lo} : u;
    const dfl v = df_exp_nonpos(dfl{-2.0f * a.hi, -2.0f * a.lo}, et);
    t1 = df_add(a, df_log1p_unit(v, lt));
    dfl u2 = df_two_prod(u.hi, u.hi);
    u2.lo = __fmaf_rn(__fmul_rn(2.0f, u.hi), u.lo, u2.lo);
    t2 = df_mul(u, df_exp_nonpos(dfl{-0.5f * u2.hi, -0.5f * u2.lo}, et));
}

// alpha * za - beta * zb in double-float.
__device__ __forceinline__ dfl df_resid(dfl al, dfl be, dfl za, dfl zb)
{
    const float p1 = __fmul_rn(al.hi, za.hi);
    float e1 = __fmaf_rn(al.hi, za.hi, -p1);
    e1 = __fmaf_rn(al.hi, za.lo, e1);
    e1 = __fmaf_rn(al.lo, za.hi, e1);
    const float p2 = __fmul_rn(be.hi, zb.hi);
    float e2 = __fmaf_rn(be.hi, zb.hi, -p2);
    e2 = __fmaf_rn(be.hi, zb.lo, e2);
    e2 = __fmaf_rn(be.lo, zb.hi, e2);
    const dfl s = df_two_sum(p1, -p2);
    return df_two_sum(s.hi, __fadd_rn(s.lo, __fsub_rn(e1, e2)));
}


// Running double-float sum, folded into FP64 every HP_FOLD terms so the
// double-float rounding never accumulates over more than HP_FOLD additions.
constexpr int HP_FOLD = 64;

struct DfAcc {
    dfl s{0.0f, 0.0f};
    double d = 0.0;
    __device__ __forceinline__ void add(dfl t) { s = df_add(s, t); }
    __device__ __forceinline__ void fold()
    {
        d += (double)s.hi + (double)s.lo;
        s = dfl{0.0f, 0.0f};
    }
};

// FP64 moment terms (tier 2), with the CUDA double exp/log1p.
__device__ __forceinline__ void f64_terms(double u, double &t1, double &t2)
{
    const double au = fabs(u);
    t1 = au + log1p(exp(-2.0 * au));      // log cosh u + ln 2
    t2 = u * exp(-0.5 * u * u);
}

// ----------------------------------------------------------- pass kernel --
// TIER 1: double-float from the split standardised residuals (zhi + zlo by
// position); TIER 2: FP64 from the residual data R by original index.
// The work of one instance, for the global warp index w0 of nw warps.
template <int TIER>
__device__ __forceinline__ void hp_instance(const HpParams &P, const float2 *s_exp,
                                            const float4 *s_log, int64_t w0, int64_t nw)
{
    const int lane = threadIdx.x & 31;
    int cbeg = 0;
    int64_t npair;
    bool with_vars = true;
    if (P.mode == 1) {
        const DevState *st = P.state;
        if (st->resolved || st->tier != TIER) return;
        cbeg = st->pass_begin;
        const int cend = st->pass_end;
        if (cend <= cbeg) return;
        npair = (int64_t)(cend - cbeg) * P.p;
        with_vars = P.with_vars != 0;
    } else {
        npair = (int64_t)P.p * (P.p - 1) / 2;
    }
    const int64_t nitems = npair + (with_vars ? P.p : 0);
    const int64_t nunits = nitems * P.nsplit;
    // one warp per work unit; its lanes stride the unit's samples
    const int64_t first = (w0 + nw - P.woff % nw) % nw;
    for (int64_t unit = first; unit < nunits; unit += nw) {
        // work unit = (item q, sample range sp); each range writes its own
        // partial record, summed in range order by the consumer
        const int64_t q = unit / P.nsplit;
        const int sp = (int)(unit % P.nsplit);
        const int s0 = (int)((int64_t)sp * P.sps);
        const int n = (int)std::min<int64_t>(P.n, (int64_t)s0 + P.sps);
        double *momp = P.mom + (size_t)sp * P.mom_sstride;
        double *hzp = P.hz + (size_t)sp * P.p * 2;
        if (q >= npair) {
            // moments of the standardised variable at position a
            const int a = (int)(q - npair);
            double v[2];
            if (TIER == 1) {
                const float *zh = P.zhi + (int64_t)a * P.ldz, *zl = P.zlo + (int64_t)a * P.ldz;
                DfAcc A1, A2;
                int cnt = 0;
                for (int s = s0 + lane; s < n; s += 32) {
                    dfl t1, t2;
                    df_terms(dfl{zh[s], zl[s]}, t1, t2, s_exp, s_log);
                    A1.add(t1);
                    A2.add(t2);
                    if (++cnt == HP_FOLD) {
                        A1.fold();
                        A2.fold();
                        cnt = 0;
                    }
                }
                A1.fold();
                A2.fold();
                v[0] = A1.d;
                v[1] = A2.d;
            } else {
                const int oa = P.U[a];
                const double inv = 1.0 / sqrt(P.C[(int64_t)oa * P.ldc + oa]);
                const double *ra = P.R + (int64_t)oa * P.ldr;
                double s1 = 0.0, s2 = 0.0;
                for (int s = s0 + lane; s < n; s += 32) {
                    double t1, t2;
                    f64_terms(ra[s] * inv, t1, t2);
                    s1 += t1;
                    s2 += t2;
                }
                v[0] = s1;
                v[1] = s2;
            }
            v[0] = warp_sum_xor(v[0]);
            v[1] = warp_sum_xor(v[1]);
            if (lane == 0) {
                hzp[(size_t)a * 2 + 0] = v[0];
                hzp[(size_t)a * 2 + 1] = v[1];
            }
            continue;
        }
        int a, b, cidx = 0;
        if (P.mode == 1) {
            cidx = cbeg + (int)(q / P.p);
            a = P.state->cand[cidx];
            b = (int)(q % P.p);
            // a lower bound I32(a, b) >= 0 proves I(a, b) >= 0: min(0, I)^2 = 0
            // exactly, so the entry needs no moments (marked by a negative sum)
            if (a == b || (P.I32 && P.I32[(size_t)a * P.p + b] >= 0.0f)) {
                if (lane == 0 && sp == 0) {   // the marker lives in range 0
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
        double rho;
        if (TIER == 1)
            rho = P.C[(int64_t)lo * P.ldc + hi] * P.isd[a] * P.isd[b];
        else
            rho = P.C[(int64_t)lo * P.ldc + hi] /
                  (sqrt(P.C[(int64_t)oa * P.ldc + oa]) * sqrt(P.C[(int64_t)ob * P.ldc + ob]));
        double s2v = 1.0 - rho * rho;
        if (!(s2v > 1e-12)) {
            if (lane == 0) set_status(P.status, ST_DEGENERATE);
            s2v = 1.0;
        }
        const double alpha = 1.0 / sqrt(s2v);   // residual of a given b: alpha z_a - rho alpha z_b
        double v[4];
        if (TIER == 1) {
            const dfl al = df_split(alpha), be = df_split(rho * alpha);
            const float *zah = P.zhi + (int64_t)a * P.ldz, *zal = P.zlo + (int64_t)a * P.ldz;
            const float *zbh = P.zhi + (int64_t)b * P.ldz, *zbl = P.zlo + (int64_t)b * P.ldz;
            DfAcc A1, A2, B1, B2;
            int cnt = 0;
            for (int s = s0 + lane; s < n; s += 32) {
                const dfl za{zah[s], zal[s]}, zb{zbh[s], zbl[s]};
                dfl t1, t2;
                df_terms(df_resid(al, be, za, zb), t1, t2, s_exp, s_log);
                A1.add(t1);
                A2.add(t2);
                df_terms(df_resid(al, be, zb, za), t1, t2, s_exp, s_log);
                B1.add(t1);
                B2.add(t2);
                if (++cnt == HP_FOLD) {
                    A1.fold();
                    A2.fold();
                    B1.fold();
                    B2.fold();
                    cnt = 0;
                }
            }
            A1.fold();
            A2.fold();
            B1.fold();
            B2.fold();
            v[0] = A1.d;
            v[1] = A2.d;
            v[2] = B1.d;
            v[3] = B2.d;
        } else {
            const double ia = 1.0 / sqrt(P.C[(int64_t)oa * P.ldc + oa]);
            const double ib = 1.0 / sqrt(P.C[(int64_t)ob * P.ldc + ob]);
            const double *ra = P.R + (int64_t)oa * P.ldr, *rb = P.R + (int64_t)ob * P.ldr;
            double ab1 = 0.0, ab2 = 0.0, ba1 = 0.0, ba2 = 0.0;
            for (int s = s0 + lane; s < n; s += 32) {
                const double za = ra[s] * ia, zb = rb[s] * ib;
                double t1, t2;
                f64_terms((za - rho * zb) * alpha, t1, t2);
                ab1 += t1;
                ab2 += t2;
                f64_terms((zb - rho * za) * alpha, t1, t2);
                ba1 += t1;
                ba2 += t2;
            }
            v[0] = ab1;
            v[1] = ab2;
            v[2] = ba1;
            v[3] = ba2;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = warp_sum_xor(v[k]);
        if (lane == 0) {
            if (P.mode == 1) {
                double *o = momp + ((size_t)cidx * P.p + b) * 4;
                o[0] = v[0];
                o[1] = v[1];
                o[2] = v[2];
                o[3] = v[3];
            } else {
                double *o = momp + ((size_t)a * P.p + b) * 2;
                o[0] = v[0];
                o[1] = v[1];
                o = momp + ((size_t)b * P.p + a) * 2;
                o[0] = v[2];
                o[1] = v[3];
            }
        }
    }
}

// Every warp of the grid works on every instance in turn, so the whole GPU
// serves whichever instances have work (in a batch usually a few).
template <int TIER>
__global__ void __launch_bounds__(HP_THREADS, 3) k_pairs_hp_b(const HpParams *__restrict__ Ps,
                                                             int count)
{
    __shared__ float2 s_exp[TIER == 1 ? EXP_TAB : 1];
    __shared__ float4 s_log[TIER == 1 ? LOG_TAB : 1];
    if (TIER == 1) {
        for (int k = threadIdx.x; k < EXP_TAB; k += blockDim.x) s_exp[k] = g_exp_tab[k];
        for (int k = threadIdx.x; k < LOG_TAB; k += blockDim.x) s_log[k] = g_log_tab[k];
        __syncthreads();
    }
    constexpr int WPB = HP_THREADS / 32;
    const int64_t w0 = (int64_t)blockIdx.x * WPB + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * WPB;
    for (int inst = 0; inst < count; ++inst) hp_instance<TIER>(Ps[inst], s_exp, s_log, w0, nw);
}

cudaError_t launch_pairs_hp_b(int tier, const HpParams *P, int count, int blocks, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    if (tier == 1)
        k_pairs_hp_b<1><<<blocks, HP_THREADS, 0, s>>>(P, count);
    else
        k_pairs_hp_b<2><<<blocks, HP_THREADS, 0, s>>>(P, count);
    return cudaGetLastError();
}

// Tables of the double-float exp and log: 2^(j/128), 1/c_k and log c_k from
// the host's FP64 libm (about 1 ulp of FP64), split into FP32 hi + lo.
cudaError_t df_tables_setup()
{
    float2 et[EXP_TAB];
    float4 lt[LOG_TAB];
    for (int j = 0; j < EXP_TAB; ++j) {
        const double v = exp2((double)j / EXP_TAB);
        const float h = (float)v;
        et[j] = make_float2(h, (float)(v - (double)h));
    }
    for (int k = 0; k < LOG_TAB; ++k) {
        const double c = 1.0 + (double)k / 256.0;
        const double inv = 1.0 / c, lg = log(c);
        const float ih = (float)inv, lh = (float)lg;
        lt[k] = make_float4(ih, (float)(inv - (double)ih), lh, (float)(lg - (double)lh));
    }
    cudaError_t e = cudaMemcpyToSymbol(g_exp_tab, et, sizeof(et));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(g_log_tab, lt, sizeof(lt));
}

// ------------------------------------------------------- refine + decide --
// Scores the candidates of the current pass from the re-computed moments and
// advances the step's decision:
//   tier 1 (df): each M carries the bound e = sum_j (2 |min(0, I)| epsI2 +
//     epsI2^2) over its computed entries.  Pass 1 covers the two candidates
//     with the highest FP32 upper bounds; pass 2 the others whose upper
//     bound still reaches the best lower bound M - e.  Candidates whose
//     intervals overlap the best one's go to tier 2; if none do, the step is
//     decided.  The last pass always decides or escalates, so every step
//     ends decided.
//   tier 2 (FP64): the argmax of the FP64 scores (ties to the smallest
//     original index), and a tie count when the top two are within
//     1e-9 max|M|.
__global__ void __launch_bounds__(256) k_refine_select_b(const RefineSelectParams *__restrict__ Ps)
{
    extern __shared__ double h64[];
    const RefineSelectParams P = Ps[blockIdx.x];
    DevState *st = P.state;
    if (st->resolved || st->tier != P.tier) return;
    const int cb = st->pass_begin, ce = st->pass_end, nc = st->ncand;
    const double invn = 1.0 / (double)P.n;
    const double eps = P.tier == 1 ? P.epsI : 0.0;
    for (int j = threadIdx.x; j < P.p; j += blockDim.x) {
        double s1 = 0.0, s2 = 0.0;
        for (int sp = 0; sp < P.nsplit; ++sp) {
            s1 += P.hz[((size_t)sp * P.p + j) * 2];
            s2 += P.hz[((size_t)sp * P.p + j) * 2 + 1];
        }
        h64[j] = neg_entropy_part(s1 * invn - LN2_D, s2 * invn);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = cb + w; c < ce; c += nw) {
        const int pc = st->cand[c];
        double acc = 0.0, err = 0.0;
        for (int j = lane; j < P.p; j += 32) {
            if (j == pc) continue;
            const size_t rec = ((size_t)c * P.p + j) * 4;
            if (P.mom[rec] < 0.0) continue;     // skipped entry (marker in range 0)
            double o[4] = {0.0, 0.0, 0.0, 0.0};
            for (int sp = 0; sp < P.nsplit; ++sp)
#pragma unroll
                for (int k = 0; k < 4; ++k) o[k] += P.mom[(size_t)sp * P.mom_sstride + rec + k];
            const double hcj = neg_entropy_part(o[0] * invn - LN2_D, o[1] * invn);
            const double hjc = neg_entropy_part(o[2] * invn - LN2_D, o[3] * invn);
            const double I = (h64[j] + hcj) - (h64[pc] + hjc);
            const double v = fmin(0.0, I);
            acc += v * v;
            err += 2.0 * fabs(v) * eps + eps * eps;
        }
        acc = warp_sum_xor(acc);
        err = warp_sum_xor(err);
        if (lane == 0) {
            st->mhp[c] = -acc;
            st->ehp[c] = err;
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    int best = 0;
    for (int c = 1; c < ce; ++c)
        if (better(st->mhp[c], P.U[st->cand[c]], st->mhp[best], P.U[st->cand[best]])) best = c;
    if (P.tier == 1)
        st->df_candidates += ce - cb;
    else
        st->fp64_candidates += ce - cb;
    if (P.hist)
        for (int c = cb; c < ce; ++c) P.hist[P.U[st->cand[c]]] = st->mhp[c];
    const double lb = st->mhp[best] - st->ehp[best];
    if (P.tier == 1) {
        // candidates never re-scored whose FP32 upper bound still reaches lb
        // (a prefix of the rest: they are sorted by upper bound)
        int cend = ce;
        while (cend < nc && !(lb > st->ub[cend])) ++cend;
        if (cend > ce && !P.last) {
            st->pass_begin = ce;       // undecided: pass 2 re-scores those
            st->pass_end = cend;
            return;
        }
        // candidates still not separated from the best one go to FP64: the
        // re-scored ones whose interval reaches lb and, after the last
        // double-float pass, any left whose upper bound reaches it
        int nk = cend - ce;
        for (int c = 0; c < ce; ++c)
            nk += (c == best || !(st->mhp[c] + st->ehp[c] < lb));
        if (nk == 1) {
            st->m_pos = st->cand[best];
            st->resolved = 1;
            return;
        }
        nk = 0;   // compact in place (the write index never passes the read index)
        for (int c = 0; c < cend; ++c)
            if (c >= ce || c == best || !(st->mhp[c] + st->ehp[c] < lb))
                st->cand[nk++] = st->cand[c];
        st->ncand = nk;
        st->pass_begin = 0;
        st->pass_end = nk;
        st->tier = 2;
        return;
    }
    double mx = 0.0, gap = INFINITY;
    for (int c = 0; c < ce; ++c) mx = fmax(mx, fabs(st->mhp[c]));
    for (int c = 0; c < ce; ++c)
        if (c != best) gap = fmin(gap, st->mhp[best] - st->mhp[c]);
    if (gap <= 1e-9 * mx) st->genuine_ties += 1;
    st->m_pos = st->cand[best];
    st->resolved = 1;
}

cudaError_t launch_refine_select_b(const RefineSelectParams *P, int count, int maxp, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    k_refine_select_b<<<count, 256, sizeof(double) * maxp, s>>>(P);
    return cudaGetLastError();
}

}  // namespace lg
