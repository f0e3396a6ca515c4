// kernels_refine.cu -- high-precision re-scoring of near-tied candidates.
//
// The FP32 pair-moment kernel gives every I(i, j) of Algorithm 1 with a known
// error bound; at steps where the top scores M(i) lie within that bound of
// each other the argmax is decided by re-scoring the candidates:
//
//   tier 1  double-float ("df"): every quantity carried as an unevaluated sum
//           hi + lo of two FP32 numbers (about 48 significant bits), the two
//           moment functions evaluated from tables by Taylor series, so the
//           work runs on the FP32 pipe.  Each I(i, j) carries a bound epsI2
//           on its error.
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

#include "conv.cuh"
#include "df.cuh"
#include "kernels.cuh"

namespace lg {

// Double-float moment terms by table and Taylor series.  With a = |u|,
//   t1 = log cosh u + ln 2 = a + phi(a),   phi(a) = log(1 + exp(-2a)),
//   t2 = u exp(-u^2/2)     = sign(u) psi(a),   psi(a) = a exp(-a^2/2).
// The tables hold phi, psi and their first two derivatives (double-float) at
// the nodes c_k = k/128, k <= 1152 (a <= 9).  At an FP32 point a = c_k + h
// (|h| <= 1/256, h exact by Sterbenz's lemma) each function is its Taylor
// polynomial to h^5: the h and h^2 terms in double-float, h^3 .. h^5 in FP32
// from derivatives written in tanh c (phi) or as Hermite polynomials times
// exp(-c^2/2) (psi); the h^6 remainder is below 1e-16.  The low part of the
// residual enters to second order through the derivative of that
// polynomial.  Beyond a = 9, phi(a) = exp(-2a) to 1e-16 and psi(a) < 3e-17
// come from the FP32 exponential.  A host emulation of these steps in FP32
// against 40-digit values shows at most 1e-14 absolute error per term, with
// no bias (an earlier route through exp and log1p by P. T. P. Tang's
// table-driven methods showed 3e-14).
constexpr int TT_STEP = 128;                  // nodes per unit of a
constexpr int TT_ROWS = 9 * TT_STEP + 1;      // c_k = k / 128, k <= 1152

__device__ float4 g_tt_pa[TT_ROWS];   // phi hi, lo; phi' hi, lo
__device__ float4 g_tt_pb[TT_ROWS];   // phi''/2 hi, lo; psi''/2 hi, lo
__device__ float4 g_tt_qa[TT_ROWS];   // psi hi, lo; psi' hi, lo
__device__ float4 g_tt_pc[TT_ROWS];   // phi'''/6, phi''''/24, phi^(5)/120, psi'''/6
__device__ float2 g_tt_qc[TT_ROWS];   // psi''''/24, psi^(5)/120

// The block's shared-memory copies of the tables.
struct TtTab {
    const float4 *pa, *pb, *qa, *pc;
    const float2 *qc;
};
constexpr size_t TT_SMEM = (size_t)TT_ROWS * (4 * sizeof(float4) + sizeof(float2));

// One function's value at c + h from its row: v0 (double-float value), v1
// (double-float first derivative), v2 (double-float half second derivative)
// and c3, c4, c5 (FP32 Taylor coefficients of h^3 .. h^5); al is the low
// part of the argument, entered to second order through the derivative of
// the polynomial.
__device__ __forceinline__ dfl tt_eval(float v0h, float v0l, float v1h, float v1l, float v2h,
                                       float v2l, float c3, float c4, float c5, float h,
                                       float qh, float ql, float al)
{
    float p1h = __fmul_rn(v1h, h), p1l = __fmaf_rn(v1h, h, -p1h);
    p1l = __fmaf_rn(v1l, h, p1l);
    float p2h = __fmul_rn(v2h, qh), p2l = __fmaf_rn(v2h, qh, -p2h);
    p2l = __fmaf_rn(v2h, ql, p2l);
    p2l = __fmaf_rn(v2l, qh, p2l);
    const float r = qh * h * (c3 + h * (c4 + h * c5));
    const float corr = (v1h + h * (2.0f * v2h + h * (3.0f * c3 + h * 4.0f * c4)) + v2h * al) * al;
    const dfl s1 = df_two_sum(v0h, p1h);
    const dfl s2 = df_two_sum(s1.hi, p2h);
    const float lo = __fadd_rn(__fadd_rn(__fadd_rn(s1.lo, s2.lo), __fadd_rn(v0l, p1l)),
                               __fadd_rn(p2l, __fadd_rn(r, corr)));
    return df_fast_two_sum(s2.hi, lo);
}

// The moment terms of one residual value u: t1 = (a + al) + f, t2 = g.
__device__ __forceinline__ void tt_terms(dfl u, const TtTab &T, float &a, float &al, dfl &f,
                                         dfl &g)
{
    const float sg = u.hi < 0.0f ? -1.0f : 1.0f;
    a = fabsf(u.hi);
    al = sg * u.lo;   // |u| = a + al
    const float kf = rintf(__fmul_rn(a, (float)TT_STEP));
    if (kf < (float)TT_ROWS) {
        const int k = (int)kf;
        const float h = __fsub_rn(a, __fmul_rn(kf, 1.0f / TT_STEP));   // exact
        const float qh = __fmul_rn(h, h), ql = __fmaf_rn(h, h, -qh);   // h^2
        const float4 A = T.pa[k], B = T.pb[k], Q = T.qa[k], C = T.pc[k];
        const float2 D = T.qc[k];
        f = tt_eval(A.x, A.y, A.z, A.w, B.x, B.y, C.x, C.y, C.z, h, qh, ql, al);
        const dfl v = tt_eval(Q.x, Q.y, Q.z, Q.w, B.z, B.w, C.w, D.x, D.y, h, qh, ql, al);
        g = dfl{sg * v.hi, sg * v.lo};
    } else {
        const float e = expf(-2.0f * a);
        f = dfl{e, -2.0f * e * al};
        g = dfl{sg * a * expf(-0.5f * a * a), 0.0f};
    }
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
    // adds (a + al) + f, the three parts of t1 from tt_terms
    __device__ __forceinline__ void add3(float a, float al, dfl f)
    {
        const dfl x = df_two_sum(s.hi, a);
        const dfl y = df_two_sum(x.hi, f.hi);
        s = df_fast_two_sum(y.hi, __fadd_rn(__fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)),
                                            __fadd_rn(al, f.lo)));
    }
    __device__ __forceinline__ void fold()
    {
        d += f32_to_f64(s.hi) + f32_to_f64(s.lo);   // exact conversions off the FP64 pipe
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
__device__ __forceinline__ void hp_instance(const HpParams &P, const TtTab &T, int64_t w0,
                                            int64_t nw)
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
                // the next iteration's sample is loaded before this one's work
                int s = s0 + lane;
                dfl zn{0.0f, 0.0f};
                if (s < n) zn = dfl{__ldg(zh + s), __ldg(zl + s)};
                for (; s < n; s += 32) {
                    const dfl z = zn;
                    if (s + 32 < n) zn = dfl{__ldg(zh + s + 32), __ldg(zl + s + 32)};
                    float ua, ual;
                    dfl f, g;
                    tt_terms(z, T, ua, ual, f, g);
                    A1.add3(ua, ual, f);
                    A2.add(g);
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
            // the next iteration's samples are loaded before this one's work
            int s = s0 + lane;
            dfl zan{0.0f, 0.0f}, zbn{0.0f, 0.0f};
            if (s < n) {
                zan = dfl{__ldg(zah + s), __ldg(zal + s)};
                zbn = dfl{__ldg(zbh + s), __ldg(zbl + s)};
            }
            for (; s < n; s += 32) {
                const dfl za = zan, zb = zbn;
                if (s + 32 < n) {
                    zan = dfl{__ldg(zah + s + 32), __ldg(zal + s + 32)};
                    zbn = dfl{__ldg(zbh + s + 32), __ldg(zbl + s + 32)};
                }
                float ua, ual;
                dfl f, g;
                tt_terms(df_resid(al, be, za, zb), T, ua, ual, f, g);
                A1.add3(ua, ual, f);
                A2.add(g);
                tt_terms(df_resid(al, be, zb, za), T, ua, ual, f, g);
                B1.add3(ua, ual, f);
                B2.add(g);
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

// Every warp of the grid works on every instance with work in turn, so the
// whole GPU serves whichever instances have work (in a batch usually a few).
// Each block first lists those instances (256 at a time, all threads testing
// at once); the double-float tier copies the Taylor tables into the block's
// shared memory before the first one, and not at all when there is none.
template <int TIER>
__device__ __forceinline__ bool hp_has_work(const HpParams &P)
{
    if (P.mode == 0) return true;
    const DevState *st = P.state;
    return !st->resolved && st->tier == TIER && st->pass_end > st->pass_begin;
}

template <int TIER>
__global__ void __launch_bounds__(HP_THREADS, TIER == 1 ? 2 : 3)
    k_pairs_hp_b(const HpParams *__restrict__ Ps, int count)
{
    extern __shared__ float4 tt_smem[];
    __shared__ int s_act[HP_THREADS];
    __shared__ int s_wcnt[HP_THREADS / 32];
    TtTab T{};
    bool tables = false;
    constexpr int WPB = HP_THREADS / 32;
    const int64_t w0 = (int64_t)blockIdx.x * WPB + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * WPB;
    for (int base = 0; base < count; base += HP_THREADS) {
        const int nact = block_active_list(
            base, count, [&](int k) { return hp_has_work<TIER>(Ps[k]); }, s_act, s_wcnt);
        if (nact == 0) continue;
        if (TIER == 1 && !tables) {
            float4 *pa = tt_smem, *pb = pa + TT_ROWS, *qa = pb + TT_ROWS, *pc = qa + TT_ROWS;
            float2 *qc = reinterpret_cast<float2 *>(pc + TT_ROWS);
            for (int k = threadIdx.x; k < TT_ROWS; k += blockDim.x) {
                pa[k] = g_tt_pa[k];
                pb[k] = g_tt_pb[k];
                qa[k] = g_tt_qa[k];
                pc[k] = g_tt_pc[k];
                qc[k] = g_tt_qc[k];
            }
            __syncthreads();
            T = TtTab{pa, pb, qa, pc, qc};
            tables = true;
        }
        for (int i = 0; i < nact; ++i) hp_instance<TIER>(Ps[s_act[i]], T, w0, nw);
        __syncthreads();   // s_act is rewritten by the next chunk
    }
}

cudaError_t launch_pairs_hp_b(int tier, const HpParams *P, int count, int blocks, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    if (tier == 1)
        k_pairs_hp_b<1><<<blocks, HP_THREADS, TT_SMEM, s>>>(P, count);
    else
        k_pairs_hp_b<2><<<blocks, HP_THREADS, 0, s>>>(P, count);
    return cudaGetLastError();
}

// Tables of the double-float tier from the host's FP64 libm (about 1 ulp of
// FP64, well inside the 48 bits of a double-float), written without
// cancellation: with e = exp(-2c), t = tanh c and s = 1 - t^2,
// t - 1 = -2e / (1 + e) and s = 4e / (1 + e)^2.  Derivatives of phi:
// phi' = t - 1, phi'' = s, phi''' = -2 t s, phi'''' = s (6 t^2 - 2),
// phi^(5) = 8 t s (2 - 3 t^2); of psi: psi^(m) = (-1)^m He_(m+1)(c) E with
// E = exp(-c^2/2) and the Hermite polynomials He_2 = c^2 - 1,
// He_3 = c^3 - 3c, He_4 = c^4 - 6c^2 + 3, He_5 = c^5 - 10c^3 + 15c,
// He_6 = c^6 - 15c^4 + 45c^2 - 15.
cudaError_t df_tables_setup()
{
    static float4 pa[TT_ROWS], pb[TT_ROWS], qa[TT_ROWS], pc[TT_ROWS];
    static float2 qc[TT_ROWS];
    auto hi = [](double v) { return (float)v; };
    auto lo = [](double v) { return (float)(v - (double)(float)v); };
    for (int k = 0; k < TT_ROWS; ++k) {
        const double c = (double)k / TT_STEP, c2 = c * c;
        const double e = exp(-2.0 * c);
        const double t = (1.0 - e) / (1.0 + e), s = 4.0 * e / ((1.0 + e) * (1.0 + e));
        const double phi = log1p(e), d1 = -2.0 * e / (1.0 + e), d2 = 0.5 * s;
        const double d3 = -2.0 * t * s, d4 = s * (6.0 * t * t - 2.0);
        const double d5 = 8.0 * t * s * (2.0 - 3.0 * t * t);
        const double E = exp(-0.5 * c2);
        const double psi = c * E, q1 = (1.0 - c2) * E, q2 = 0.5 * (c2 * c - 3.0 * c) * E;
        const double q3 = -(c2 * c2 - 6.0 * c2 + 3.0) * E;
        const double q4 = (c2 * c2 * c - 10.0 * c2 * c + 15.0 * c) * E;
        const double q5 = -(((c2 - 15.0) * c2 + 45.0) * c2 - 15.0) * E;
        pa[k] = make_float4(hi(phi), lo(phi), hi(d1), lo(d1));
        pb[k] = make_float4(hi(d2), lo(d2), hi(q2), lo(q2));
        qa[k] = make_float4(hi(psi), lo(psi), hi(q1), lo(q1));
        pc[k] = make_float4((float)(d3 / 6.0), (float)(d4 / 24.0), (float)(d5 / 120.0),
                            (float)(q3 / 6.0));
        qc[k] = make_float2((float)(q4 / 24.0), (float)(q5 / 120.0));
    }
    cudaError_t err;
    if ((err = cudaMemcpyToSymbol(g_tt_pa, pa, sizeof(pa))) != cudaSuccess) return err;
    if ((err = cudaMemcpyToSymbol(g_tt_pb, pb, sizeof(pb))) != cudaSuccess) return err;
    if ((err = cudaMemcpyToSymbol(g_tt_qa, qa, sizeof(qa))) != cudaSuccess) return err;
    if ((err = cudaMemcpyToSymbol(g_tt_pc, pc, sizeof(pc))) != cudaSuccess) return err;
    if ((err = cudaMemcpyToSymbol(g_tt_qc, qc, sizeof(qc))) != cudaSuccess) return err;
    return cudaFuncSetAttribute(k_pairs_hp_b<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TT_SMEM);
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
    // one candidate at a time over the whole block (its entries split over
    // all threads, fixed-order block sums): a pass often has only two
    __shared__ double s_acc[8], s_err[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = cb; c < ce; ++c) {
        const int pc = st->cand[c];
        double acc = 0.0, err = 0.0;
        for (int j = threadIdx.x; j < P.p; j += blockDim.x) {
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
            s_acc[w] = acc;
            s_err[w] = err;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double ta = 0.0, te = 0.0;
            for (int k = 0; k < nw; ++k) {
                ta += s_acc[k];
                te += s_err[k];
            }
            st->mhp[c] = -ta;
            st->ehp[c] = te;
        }
        __syncthreads();
    }
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
