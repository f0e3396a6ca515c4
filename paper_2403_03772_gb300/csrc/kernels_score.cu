// kernels_score.cu -- Algorithm 1's scores and the argmax: the entropies of
// the pair moments combined into I(i, j) and M(i) (k_score_b), and the
// selection of the step's variable with its candidate set for re-scoring
// (k_select_b).
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace lg {

// ------------------------------------------------------------------------
// Score: I(i, j) and M(i) (Algorithm 1, deterministic FP64 combine)
// ------------------------------------------------------------------------
//
// I(i, j) = (h(z_j) + h(r_i^j)) - (h(z_i) + h(r_j^i)) with h = H - H(nu);
// M(i) = -sum_{j != i} min(0, I(i, j))^2 (with a shard set, over the entries
// the rank owns: partial M and E, summed over ranks by the caller), summed by each lane over j in
// ascending order and across lanes by a fixed xor tree.  E(i) bounds |M(i) -
// M_exact(i)| given |I - I_exact| <= eps per entry: a fixed epsI for steps
// scored in double-float, else the moment-error model of ErrModel.
constexpr int SCORE_RPB = 2, SCORE_WPR = 4;   // rows per block, warps per row

// One launch covers every instance: prefix[k] is the first block of instance
// k (ceil(p / SCORE_RPB) blocks each).
__global__ void __launch_bounds__(256, 3) k_score_b(const ScoreParams *__restrict__ Ps,
                                                   const int *__restrict__ prefix, int count)
{
    extern __shared__ double hsh[];   // h(z_j), j < p; then their error bounds (float)
    const int inst = find_instance(prefix, count, blockIdx.x);
    const ScoreParams P = Ps[inst];
    const int rb = blockIdx.x - prefix[inst];   // row block of the instance
    float *wsh = reinterpret_cast<float *>(hsh + P.p);
    const bool df = P.mom2 != nullptr;
    dfl *hd = reinterpret_cast<dfl *>(wsh + P.p + (P.p & 1));   // h(z_j) as double-floats
    // the block's constants, by one thread (an FP64 division and the FP64 ->
    // double-float splits are dozens of FP64-pipe instructions per thread)
    __shared__ double s_invn;
    __shared__ float s_cst[10];   // c1, b1, c2 as (hi, lo); epsI and the model's d1, d2, da
    if (threadIdx.x == 0) {
        const double invn0 = 1.0 / (double)P.n;
        s_invn = invn0;
        if (df) {
            const dfl c1 = df_split(P.a1 * invn0), b1 = df_split(P.b1),
                      c2 = df_split(P.a2 * invn0);
            s_cst[0] = c1.hi;
            s_cst[1] = c1.lo;
            s_cst[2] = b1.hi;
            s_cst[3] = b1.lo;
            s_cst[4] = c2.hi;
            s_cst[5] = c2.lo;
            s_cst[6] = (float)P.epsI;
            s_cst[7] = (float)P.model.d1;
            s_cst[8] = (float)P.model.d2;
            s_cst[9] = (float)P.model.da;
        }
    }
    for (int j = threadIdx.x; j < P.p; j += blockDim.x) {
        if (df && P.hvar) {
            // computed once for the step by k_hvar_b (no FP64 work per block)
            const float4 v = P.hvar[j];
            hd[j] = dfl{v.x, v.y};
            wsh[j] = v.z;
        } else {
            score_var(P, j, 1.0 / (double)P.n, hsh[j], wsh[j]);
            if (df) hd[j] = df_split(hsh[j]);
        }
    }
    __syncthreads();
    const double invn = s_invn;
    // SCORE_WPR warps per row i: warp wr of the row takes j = 32 wr + lane +
    // 32 SCORE_WPR k; the row's partial sums are added in warp order.
    __shared__ double racc[8], rerr[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wr = warp % SCORE_WPR;
    const int i = rb * SCORE_RPB + warp / SCORE_WPR;
    double acc = 0.0, err = 0.0;
    if (i < P.p && df) {
        // FP32-scored step: double-float combine, FP32 bounds
        const dfl c1{s_cst[0], s_cst[1]}, b1{s_cst[2], s_cst[3]}, c2{s_cst[4], s_cst[5]};
        dfl accd{0.0f, 0.0f};
        float errf = 0.0f;
        const int oi = P.U[i];
        const float wi = wsh[i];
        // the model's FP32 constants, converted once per block (not per entry)
        const float epsI = s_cst[6], md1 = s_cst[7], md2 = s_cst[8], mda = s_cst[9];
        for (int j = wr * 32 + lane; j < P.p; j += 32 * SCORE_WPR) {
            if (j == i) continue;
            if (P.shard_n > 1 && shard_owner(i, j, P.p, P.shard_n) != P.shard_rank) continue;
            float mf[4];
            const dfl I = score_entry_df(P, i, j, hd, c1, b1, c2, mf);
            float eps = epsI;
            if (P.use_model) {
                float ra;
                if (P.ra) {
                    ra = P.ra[(size_t)i * P.p + j] * 1.01f;   // from the pair kernel
                } else {
                    const int oj = P.U[j];
                    const double rho =
                        P.C[(int64_t)min(oi, oj) * P.ldc + max(oi, oj)] * P.isd[i] * P.isd[j];
                    ra = rsqrtf(fmaxf((float)fma(-rho, rho, 1.0), 1e-12f)) * 1.01f;
                }
                const float e1 = md1 + mda * ra;
                const float e2 = md2 + mda * ra;
                eps = h_err(mf[0], mf[1], e1, e2) + h_err(mf[2], mf[3], e1, e2) + wi + wsh[j];
            }
            const bool neg = I.hi < 0.0f;
            if (neg) accd = df_add(accd, df_mul(I, I));
            const float Ilo = __fadd_rd(I.hi, I.lo);   // I rounded down
            if (Ilo < eps) {
                const float v = neg ? -Ilo : 0.0f;
                errf += 2.0f * v * eps + eps * eps;
            }
            if (P.Iout) P.Iout[(size_t)i * P.p + j] = (double)I.hi + (double)I.lo;
            if (P.epsOut) P.epsOut[(size_t)i * P.p + j] = eps;
            if (P.I32) P.I32[(size_t)i * P.p + j] = __fsub_rd(Ilo, eps);
        }
        acc = (double)accd.hi + (double)accd.lo;
        err = (double)errf * (1.0 + 1e-5);   // FP32 sum of a bound: cover its rounding
    } else if (i < P.p) {
        for (int j = wr * 32 + lane; j < P.p; j += 32 * SCORE_WPR) {
            if (j == i) continue;
            double I, eps;
            score_entry(P, i, j, hsh, wsh, invn, I, eps);
            const double v = fmin(0.0, I);
            acc += v * v;
            if (I < eps) err += 2.0 * fabs(v) * eps + eps * eps;
            if (P.Iout) P.Iout[(size_t)i * P.p + j] = I;
            if (P.epsOut) P.epsOut[(size_t)i * P.p + j] = eps;
            if (P.I32) P.I32[(size_t)i * P.p + j] = __double2float_rd(I - eps);
        }
    }
    acc = warp_sum_xor(acc);
    err = warp_sum_xor(err);
    if (lane == 0) {
        racc[warp] = acc;
        rerr[warp] = err;
    }
    __syncthreads();
    if (lane == 0 && wr == 0 && i < P.p) {
        double m = 0.0, e = 0.0;
        for (int k = 0; k < SCORE_WPR; ++k) {
            m += racc[warp + k];
            e += rerr[warp + k];
        }
        P.M[i] = -m;
        P.E[i] = e;
        if (P.hist) P.hist[P.U[i]] = -m;
    }
}

// The variable terms of an FP32-scored step, once per step: h(z_j) (from the
// regress kernel's split sums, FP64) as a double-float and its error bound,
// read by every block of k_score_b.
__global__ void __launch_bounds__(256) k_hvar_b(const ScoreParams *__restrict__ Ps, int count)
{
    const int inst = blockIdx.y;
    if (inst >= count) return;
    const ScoreParams &P = Ps[inst];
    if (!P.mom2 || !P.hvar) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.p) return;
    double h;
    float w;
    score_var(P, j, 1.0 / (double)P.n, h, w);
    const dfl d = df_split(h);
    P.hvar[j] = make_float4(d.hi, d.lo, w, 0.0f);
}

int score_blocks(int p) { return (p + SCORE_RPB - 1) / SCORE_RPB; }

cudaError_t launch_score_b(const ScoreParams *P, const int *prefix, int count, int total_blocks,
                           int maxp, cudaStream_t s)
{
    if (count <= 0 || total_blocks <= 0) return cudaSuccess;
    k_hvar_b<<<dim3((maxp + 255) / 256, count), 256, 0, s>>>(P, count);
    k_score_b<<<total_blocks, 32 * SCORE_RPB * SCORE_WPR,
                (sizeof(double) + sizeof(float) + sizeof(dfl)) * maxp + 32, s>>>(P, prefix, count);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// Select: argmax of M (ties to the smallest original index) and the set of
// candidates whose score intervals [M - E, M + E] reach the leader's.
//
// With prior ancestry knowledge, only the allowed positions take part: q is
// allowed when no other remaining variable is a known ancestor of U[q], and,
// if some remaining variables have every other one known not to be their
// ancestor (known exogenous), only those are.  No allowed position at all
// (contradictory knowledge) sets ST_ARG and lets every position take part.
// ------------------------------------------------------------------------

__device__ __forceinline__ void prior_allow(const SelectParams &P)
{
    const int tid = threadIdx.x;
    int exo_any = 0;
    for (int q = tid; q < P.p; q += blockDim.x) {
        const int8_t *row = P.prior + (int64_t)P.U[q] * P.ldp;
        bool anc = false, exo = true;
        for (int r = 0; r < P.p; ++r) {
            if (r == q) continue;
            const int8_t v = row[P.U[r]];
            anc |= v == 1;
            exo &= v == 0;
        }
        const uint8_t f = (uint8_t)((anc ? 0 : 1) | (exo && !anc ? 2 : 0));
        P.allow[q] = f;
        exo_any |= (f & 2) != 0;
    }
    exo_any = __syncthreads_or(exo_any);
    int any = 0;
    for (int q = tid; q < P.p; q += blockDim.x) {
        const uint8_t ok = exo_any ? (uint8_t)((P.allow[q] >> 1) & 1) : (uint8_t)(P.allow[q] & 1);
        P.allow[q] = ok;
        any |= ok;
    }
    any = __syncthreads_or(any);
    if (!any) {
        if (tid == 0) set_status(&P.state->status, ST_ARG);
        for (int q = tid; q < P.p; q += blockDim.x) P.allow[q] = 1;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_select_b(const SelectParams *__restrict__ Ps)
{
    const SelectParams P = Ps[blockIdx.x];
    __shared__ double sm[32];
    __shared__ int su[32], sp[32];
    __shared__ int s_top, s_cnt;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (P.prior) prior_allow(P);
    double bm = -INFINITY;
    int bu = 0x7fffffff, bp = -1;
    for (int q = tid; q < P.p; q += blockDim.x) {
        if (P.prior && !P.allow[q]) continue;
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
        if ((!P.prior || P.allow[q]) && P.M[q] + P.E[q] >= thr)
            P.scratch[atomicAdd(&s_cnt, 1)] = q;
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
    // rank by upper bound M + E descending, ties to the smaller original index
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
        st->cand[rank] = q;
        st->ub[rank] = ub;
    }
    if (tid == 0) {
        st->m_pos = top;
        st->ncand = cnt;
        st->resolved = 0;
        st->tier = P.tier;
        st->pass_begin = 0;
        st->pass_end = P.tier == 1 ? min(2, cnt) : cnt;
        st->refined_steps += 1;
        if (cnt > st->cand_max) st->cand_max = cnt;
    }
}

cudaError_t launch_select_b(const SelectParams *P, int count, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    k_select_b<<<count, 1024, 0, s>>>(P);
    return cudaGetLastError();
}

// The condition of a step's conditional re-score block (graphs captured with
// conditional_rescore): 1 iff the select kernel left candidates.  A kernel of
// its own, so that the select kernel stays free of device-side graph calls.
__global__ void k_set_rescore_cond(const DevState *__restrict__ st,
                                   const unsigned long long *__restrict__ cond)
{
    cudaGraphSetConditional(*cond, st->resolved ? 0u : 1u);
}

cudaError_t launch_set_rescore_cond(const DevState *st, const unsigned long long *cond,
                                    cudaStream_t s)
{
    k_set_rescore_cond<<<1, 1, 0, s>>>(st, cond);
    return cudaGetLastError();
}

}  // namespace lg
