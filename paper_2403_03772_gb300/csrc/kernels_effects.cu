// kernels_effects.cu -- what is read off the estimated graph (Sec. 4.2):
// total causal effects, the time-unrolled VarLiNGAM graph, influence
// rankings, edge statistics over bootstrap resamples, and the sparse
// (adaptive-lasso + BIC) adjacency.  FP64 throughout.

#include "kernels.cuh"

namespace lg {

// pos[order[k]] = k; status ST_ARG unless order is a permutation of 0..d-1.
__global__ void k_inverse_perm(const int32_t *order, int d, int32_t *pos, uint32_t *status)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < d; k += gridDim.x * blockDim.x) {
        const int v = order[k];
        if (v < 0 || v >= d) {
            set_status(status, ST_ARG);
            continue;
        }
        if (atomicExch(&pos[v], k) != -1) set_status(status, ST_ARG);
    }
}

// L[i][j] = -B[i][j], so that L permuted by the order is the unit lower
// triangular I - B_p (the diagonal is never read).  B must vanish on and
// above the order: B[i][j] != 0 with pos[j] >= pos[i] sets ST_ARG.
__global__ void k_effects_prep(const double *B, int d, const int32_t *pos, double *L,
                               uint32_t *status)
{
    const int64_t total = (int64_t)d * d;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q / d), j = (int)(q % d);
        const double b = B[q];
        if (b != 0.0 && pos[j] >= pos[i]) set_status(status, ST_ARG);
        if (!isfinite(b)) set_status(status, ST_NONFINITE);
        L[q] = -b;
    }
}

// T = I - W, W = -(strictly lower part of (I - B_p)^-1) scattered to the
// original indices by the unit-lower-inverse kernel.
__global__ void k_identity_minus(const double *W, int d, double *T)
{
    const int64_t total = (int64_t)d * d;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q / d), j = (int)(q % d);
        T[q] = (i == j ? 1.0 : 0.0) - W[q];
    }
}

cudaError_t launch_total_effects_prep(const double *B, const int32_t *order, int d, int32_t *pos,
                                      double *L, uint32_t *status, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(pos, 0xff, sizeof(int32_t) * d, s);
    if (e != cudaSuccess) return e;
    k_inverse_perm<<<(d + 255) / 256, 256, 0, s>>>(order, d, pos, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int blocks = (int)std::min<int64_t>(4096, ((int64_t)d * d + 255) / 256);
    k_effects_prep<<<blocks, 256, 0, s>>>(B, d, pos, L, status);
    return cudaGetLastError();
}

cudaError_t launch_identity_minus(const double *W, int d, double *T, cudaStream_t s)
{
    const int blocks = (int)std::min<int64_t>(4096, ((int64_t)d * d + 255) / 256);
    k_identity_minus<<<blocks, 256, 0, s>>>(W, d, T);
    return cudaGetLastError();
}

// Time-unrolled VarLiNGAM graph over the slices x(t - lags) .. x(t):
// block (s, s') of the (lags+1) d square matrix is B0 for s' = s and
// B_{s - s'} for 1 <= s - s' <= lags, zero otherwise; `order` of the window
// lists the slices oldest first, each in the instantaneous order order0.
__global__ void k_var_window(const double *B0, const double *Bt, int d, int lags,
                             const int32_t *order0, double *A, int32_t *order)
{
    const int q = (lags + 1) * d;
    const int64_t total = (int64_t)q * q;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / q), c = (int)(e % q);
        const int s = r / d, s2 = c / d, i = r % d, j = c % d;
        double v = 0.0;
        if (s2 == s)
            v = B0[(int64_t)i * d + j];
        else if (s2 < s && s - s2 <= lags)
            v = Bt[((int64_t)(s - s2 - 1) * d + i) * d + j];
        A[e] = v;
        if (e < q) order[e] = (int)(e / d) * d + order0[e % d];
    }
}

cudaError_t launch_var_window(const double *B0, const double *Bt, int d, int lags,
                              const int32_t *order0, double *A, int32_t *order, cudaStream_t s)
{
    const int64_t q = (int64_t)(lags + 1) * d;
    const int blocks = (int)std::min<int64_t>(4096, (q * q + 255) / 256);
    k_var_window<<<blocks, 256, 0, s>>>(B0, Bt, d, lags, order0, A, order);
    return cudaGetLastError();
}

// Influence from the total effects: block b < d sums |T[i][b]| over i != b
// (exerted by node b), block d + b sums |T[b][j]| over j != b (received);
// fixed-order block sums.
__global__ void __launch_bounds__(256) k_influence(const double *T, int d, double *exert,
                                                   double *receive)
{
    __shared__ double sh[32];
    const bool col = (int)blockIdx.x < d;
    const int b = col ? (int)blockIdx.x : (int)blockIdx.x - d;
    double acc = 0.0;
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
        if (k == b) continue;
        acc += fabs(col ? T[(int64_t)k * d + b] : T[(int64_t)b * d + k]);
    }
    const double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) (col ? exert : receive)[b] = tot;
}

// rank_out[r] = the node of rank r by descending score, equal scores to the
// smaller index (a counting rank, O(d^2)).
__global__ void k_rank_desc(const double *score, int d, int32_t *rank_out)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d; j += gridDim.x * blockDim.x) {
        const double v = score[j];
        int r = 0;
        for (int k = 0; k < d; ++k) {
            const double w = score[k];
            r += (w > v) || (w == v && k < j);
        }
        rank_out[r] = j;
    }
}

cudaError_t launch_influence(const double *T, int d, double *exert, double *receive,
                             int32_t *rank_exert, int32_t *rank_receive, cudaStream_t s)
{
    k_influence<<<2 * d, 256, 0, s>>>(T, d, exert, receive);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_rank_desc<<<(d + 127) / 128, 128, 0, s>>>(exert, d, rank_exert);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_rank_desc<<<(d + 127) / 128, 128, 0, s>>>(receive, d, rank_receive);
    return cudaGetLastError();
}

// Edge statistics over `count` adjacency matrices (device pointers in Bs):
// prob[i][j] = fraction with |B[i][j]| > threshold, mean[i][j] = their mean
// (summed in resample order).
__global__ void k_edge_stats(const double *const *Bs, int count, int64_t dd, double threshold,
                             double *prob, double *mean, uint32_t *status)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < dd;
         q += (int64_t)gridDim.x * blockDim.x) {
        int hits = 0;
        double sum = 0.0;
        for (int k = 0; k < count; ++k) {
            const double b = Bs[k][q];
            if (!isfinite(b)) set_status(status, ST_NONFINITE);
            hits += fabs(b) > threshold;
            sum += b;
        }
        prob[q] = (double)hits / (double)count;
        mean[q] = sum / (double)count;
    }
}

cudaError_t launch_edge_stats(const double *const *Bs, int count, int d, double threshold,
                              double *prob, double *mean, uint32_t *status, cudaStream_t s)
{
    const int64_t dd = (int64_t)d * d;
    const int blocks = (int)std::min<int64_t>(4096, (dd + 255) / 256);
    k_edge_stats<<<blocks, 256, 0, s>>>(Bs, count, dd, threshold, prob, mean, status);
    return cudaGetLastError();
}

}  // namespace lg

namespace lg {

// ----------------------------------------------------- sparse adjacency ---
// Cp[a][b] = C[order[a]][order[b]]: the covariance in causal-order positions,
// so a variable's predecessors are the leading block of its row.
__global__ void k_permute_sym(const double *C, const int32_t *order, int d, double *Cp)
{
    const int64_t total = (int64_t)d * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(e / d), b = (int)(e % d);
        Cp[e] = C[(int64_t)order[a] * d + order[b]];
    }
}

// Adaptive lasso path of each variable on its predecessors by homotopy (the
// lasso form of LARS; Osborne, Presnell and Turlach 2000; Efron et al. 2004).
// The variable at order position k has the q = k predecessors at positions
// 0..k-1.  With D_j = |b_ols_j|^gamma (0 when b_ols_j = 0: that coefficient
// stays 0), beta = b / D solves a plain lasso on Ct = D Cp_PP D,
// ct = D Cp_Pk, whose minimiser is piecewise linear in lam.  State: the
// active positions A (in joining order), their signs s and
// Ginv = Ct_AA^-1, kept by bordering on a join and by the Schur complement on
// a drop.  Per event:
//   beta_A = Ginv (ct_A - lam s), d = Ginv s (one refinement step each),
//   rho = ct - Ct_:A beta_A, a = Ct_:A d,
// then lam decreases to the nearest of: an inactive |rho_j| reaching lam (j
// joins with the sign of rho_j; at once if it is already there), an active
// beta_j reaching 0 (j leaves; not in the event right after it joined, and
// it does not re-join in the event right after it left), or the next grid
// value lam_i = lam_max eps^(i/(L-1)), lam_max = (1 + 1e-9) max |ct|, where
// the path point b = D beta is scored by BIC = n log(RSS/n) + df log n and
// the first minimum kept.  Ties: grid before join before drop, then the
// smaller position (joins) or the earlier joined (drops).
//
// One block per row, rows strided over the grid; per-block workspace of
// HL_VEC vectors of qmax doubles, qmax ints and the qmax x qmax inverse.
constexpr int HL_THREADS = 256;
constexpr int HL_VEC = 10;

struct HlKey {       // event candidate: the smaller (step, rank) wins
    double step;
    int rank;        // 0 grid, 1 + position for a join, 1 + qmax + slot for a drop
};

__device__ __forceinline__ HlKey hl_min(HlKey x, HlKey y)
{
    return (y.step < x.step || (y.step == x.step && y.rank < x.rank)) ? y : x;
}

__device__ HlKey hl_block_min(HlKey v, HlKey *sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        HlKey u;
        u.step = __shfl_xor_sync(0xffffffffu, v.step, o);
        u.rank = __shfl_xor_sync(0xffffffffu, v.rank, o);
        v = hl_min(v, u);
    }
    if (lane == 0) sh[w] = v;
    __syncthreads();
    HlKey r = sh[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) r = hl_min(r, sh[i]);
    __syncthreads();
    return r;
}

// Block-wide sum returned to every thread (fixed order: warp xor trees, then
// the per-warp totals in warp order).
__device__ double hl_block_sum(double v, double *sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum_xor(v);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    __syncthreads();
    return t;
}

// y[t] = sum_u M[t][u] x[u], t, u < m (M row-major, stride ld): a warp per
// row, lanes over u, fixed xor-tree sums.
__device__ void hl_matvec(const double *M, int64_t ld, const double *x, double *y, int m)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int t = w; t < m; t += nw) {
        const double *row = M + (int64_t)t * ld;
        double s = 0.0;
        for (int u = lane; u < m; u += 32) s += row[u] * x[u];
        s = warp_sum_xor(s);
        if (lane == 0) y[t] = s;
    }
    __syncthreads();
}

// y[t] = sum_u Ct(A_t, A_u) x[u] (Ct from the permuted covariance).
__device__ void hl_gram_vec(const double *Cp, int64_t d, const double *Dv, const int *A,
                            const double *x, double *y, int m)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int t = w; t < m; t += nw) {
        const int jt = A[t];
        const double *row = Cp + (int64_t)jt * d;
        double s = 0.0;
        for (int u = lane; u < m; u += 32) s += row[A[u]] * Dv[A[u]] * x[u];
        s = warp_sum_xor(s) * Dv[jt];
        if (lane == 0) y[t] = s;
    }
    __syncthreads();
}

// x = Ginv rhs with one step of iterative refinement (r = rhs - G x).
__device__ void hl_solve(const double *Gi, int64_t ld, const double *Cp, int64_t d,
                         const double *Dv, const int *A, const double *rhs, double *x,
                         double *t1, double *t2, int m)
{
    hl_matvec(Gi, ld, rhs, x, m);
    hl_gram_vec(Cp, d, Dv, A, x, t1, m);
    for (int t = threadIdx.x; t < m; t += blockDim.x) t1[t] = rhs[t] - t1[t];
    __syncthreads();
    hl_matvec(Gi, ld, t1, t2, m);
    for (int t = threadIdx.x; t < m; t += blockDim.x) x[t] += t2[t];
    __syncthreads();
}

__global__ void __launch_bounds__(HL_THREADS) k_lasso_homotopy(
    const double *Cp, const double *Bols, const int32_t *order, int d, int n, double gamma,
    int L, double eps, double *ws, int64_t ws_stride, int *iws, double *B, uint32_t *status)
{
    __shared__ HlKey s_red[HL_THREADS / 32];
    __shared__ double s_sum[HL_THREADS / 32];
    __shared__ int s_m, s_left, s_fresh, s_gi;
    __shared__ double s_lam, s_best_bic;
    const int64_t qmax = d;
    double *wb = ws + (int64_t)blockIdx.x * ws_stride;
    double *ct = wb, *Dv = ct + qmax, *rho = Dv + qmax, *av = rho + qmax, *best = av + qmax;
    double *bA = best + qmax, *dA = bA + qmax, *sA = dA + qmax, *t1 = sA + qmax, *t2 = t1 + qmax;
    double *Gi = t2 + qmax;   // qmax x qmax
    int *A = iws + (int64_t)blockIdx.x * qmax;
    const double logn = log((double)n);

    for (int k = blockIdx.x; k < d; k += gridDim.x) {
        const int q = k, ok = order[k];
        const double *crow = Cp + (int64_t)k * d;   // Cp[k][j] = C(pos j, pos k)
        const double ckk = crow[k];
        // weights, scaled correlations, lam_top and its (first) position
        HlKey top{0.0, 0x7fffffff};
        for (int j = threadIdx.x; j < q; j += blockDim.x) {
            const double bo = Bols[(int64_t)ok * d + order[j]];
            const double dj = bo != 0.0 ? pow(fabs(bo), gamma) : 0.0;
            Dv[j] = dj;
            ct[j] = crow[j] * dj;
            best[j] = 0.0;
            const double v = fabs(ct[j]);
            top = hl_min(top, HlKey{-v, j});   // the largest |ct|, first position
        }
        __syncthreads();
        top = hl_block_min(top, s_red);
        const double lam_top = -top.step;
        const double lam_max = lam_top * (1.0 + 1e-9);
        if (q == 0 || !(lam_max > 0.0)) {
            for (int j = threadIdx.x; j < d; j += blockDim.x) B[(int64_t)ok * d + j] = 0.0;
            __syncthreads();
            continue;
        }
        if (threadIdx.x == 0) {
            // grid values above the first join: b = 0, RSS/n = C_kk
            int gi = 0;
            s_best_bic = INFINITY;
            while (gi < L && lam_max * pow(eps, (double)gi / (double)(L - 1)) >= lam_top) {
                const double bic = (double)n * log(fmax(ckk, 1e-300));
                if (bic < s_best_bic) s_best_bic = bic;
                ++gi;
            }
            s_gi = gi;
            const int f = top.rank;
            A[0] = f;
            sA[0] = ct[f] > 0.0 ? 1.0 : -1.0;
            Gi[0] = 1.0 / (Dv[f] * Dv[f] * Cp[(int64_t)f * d + f]);
            s_m = 1;
            s_lam = lam_top;
            s_left = -1;
            s_fresh = f;
        }
        __syncthreads();
        const int max_events = 20 * q + 100;
        for (int ev = 0; ev < max_events; ++ev) {
            const int m = s_m, gi = s_gi, left = s_left, fresh = s_fresh;
            const double lam = s_lam;
            if (gi >= L) break;
            // beta_A and the direction d
            for (int t = threadIdx.x; t < m; t += blockDim.x) av[t] = ct[A[t]] - lam * sA[t];
            __syncthreads();
            hl_solve(Gi, qmax, Cp, d, Dv, A, av, bA, t1, t2, m);
            hl_solve(Gi, qmax, Cp, d, Dv, A, sA, dA, t1, t2, m);
            // correlations and their rates: a warp per position j
            {
                const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
                for (int j = w; j < q; j += nw) {
                    const double *row = Cp + (int64_t)j * d;
                    double sb = 0.0, sd = 0.0;
                    for (int u = lane; u < m; u += 32) {
                        const double c = row[A[u]] * Dv[A[u]];
                        sb += c * bA[u];
                        sd += c * dA[u];
                    }
                    sb = warp_sum_xor(sb) * Dv[j];
                    sd = warp_sum_xor(sd) * Dv[j];
                    if (lane == 0) {
                        rho[j] = ct[j] - sb;
                        av[j] = sd;
                    }
                }
            }
            __syncthreads();
            // the next event
            const double lam_g = lam_max * pow(eps, (double)gi / (double)(L - 1));
            HlKey e{lam - lam_g, 0};
            for (int j = threadIdx.x; j < q; j += blockDim.x) {
                if (Dv[j] == 0.0 || j == left) continue;
                bool act = false;
                for (int u = 0; u < m; ++u) act |= A[u] == j;
                if (act) continue;
                if (fabs(rho[j]) >= lam) {
                    e = hl_min(e, HlKey{0.0, 1 + j});
                    continue;
                }
                const double n1 = lam - rho[j], d1 = 1.0 - av[j];
                const double n2 = lam + rho[j], d2 = 1.0 + av[j];
                if (d1 > 0.0) e = hl_min(e, HlKey{n1 / d1, 1 + j});
                if (d2 > 0.0) e = hl_min(e, HlKey{n2 / d2, 1 + j});
            }
            for (int t = threadIdx.x; t < m; t += blockDim.x) {
                if (A[t] == fresh || dA[t] == 0.0) continue;
                const double dl = -bA[t] / dA[t];
                if (dl > 1e-12 * lam) e = hl_min(e, HlKey{dl, 1 + q + t});
            }
            e = hl_block_min(e, s_red);
            if (e.rank == 0) {
                // path point at lam_g
                for (int t = threadIdx.x; t < m; t += blockDim.x) av[t] = ct[A[t]] - lam_g * sA[t];
                __syncthreads();
                hl_solve(Gi, qmax, Cp, d, Dv, A, av, bA, t1, t2, m);
                for (int t = threadIdx.x; t < m; t += blockDim.x) t1[t] = bA[t] * Dv[A[t]];   // b
                __syncthreads();
                // RSS/n = C_kk - 2 b'C_Pk + b'C_PP b, df = nonzeros
                double s1 = 0.0, s2 = 0.0, nz = 0.0;
                {
                    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5,
                              nw = blockDim.x >> 5;
                    for (int t = w; t < m; t += nw) {
                        const double *row = Cp + (int64_t)A[t] * d;
                        double s = 0.0;
                        for (int u = lane; u < m; u += 32) s += row[A[u]] * t1[u];
                        s = warp_sum_xor(s);
                        if (lane == 0) {
                            s1 += t1[t] * crow[A[t]];
                            s2 += t1[t] * s;
                            nz += t1[t] != 0.0 ? 1.0 : 0.0;
                        }
                    }
                }
                s1 = hl_block_sum(s1, s_sum);
                s2 = hl_block_sum(s2, s_sum);
                nz = hl_block_sum(nz, s_sum);
                const double rss = ckk - 2.0 * s1 + s2;
                const double bic = (double)n * log(fmax(rss, 1e-300)) + nz * logn;
                const bool better = bic < s_best_bic;
                __syncthreads();
                if (better) {
                    for (int j = threadIdx.x; j < q; j += blockDim.x) best[j] = 0.0;
                    __syncthreads();
                    for (int t = threadIdx.x; t < m; t += blockDim.x) best[A[t]] = t1[t];
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    if (better) s_best_bic = bic;
                    s_lam = lam_g;
                    s_gi = gi + 1;
                    s_left = s_fresh = -1;
                }
            } else if (e.rank <= q) {
                // join of position j: border Ginv with c = Ct(A, j)
                const int j = e.rank - 1;
                for (int t = threadIdx.x; t < m; t += blockDim.x)
                    t2[t] = Cp[(int64_t)A[t] * d + j] * Dv[A[t]] * Dv[j];
                __syncthreads();
                hl_matvec(Gi, qmax, t2, t1, m);   // u = Ginv c
                double cu = 0.0;
                for (int t = threadIdx.x; t < m; t += blockDim.x) cu += t2[t] * t1[t];
                cu = hl_block_sum(cu, s_sum);
                const double sig = Dv[j] * Dv[j] * Cp[(int64_t)j * d + j] - cu;
                if (!(sig > 0.0)) {
                    if (threadIdx.x == 0) set_status(status, ST_DEGENERATE);
                    __syncthreads();
                    break;
                }
                const double is = 1.0 / sig;
                for (int64_t e2 = threadIdx.x; e2 < (int64_t)m * m; e2 += blockDim.x) {
                    const int t = (int)(e2 / m), v = (int)(e2 % m);
                    Gi[t * qmax + v] += t1[t] * t1[v] * is;
                }
                for (int t = threadIdx.x; t < m; t += blockDim.x) {
                    Gi[t * qmax + m] = -t1[t] * is;
                    Gi[(int64_t)m * qmax + t] = -t1[t] * is;
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    Gi[(int64_t)m * qmax + m] = is;
                    A[m] = j;
                    sA[m] = rho[j] - e.step * av[j] > 0.0 ? 1.0 : -1.0;
                    s_m = m + 1;
                    s_lam = lam - e.step;
                    s_left = -1;
                    s_fresh = j;
                }
            } else {
                // drop of slot t0: Schur complement, then close the gap
                const int t0 = e.rank - 1 - q;
                const double g0 = Gi[(int64_t)t0 * qmax + t0];
                for (int64_t e2 = threadIdx.x; e2 < (int64_t)m * m; e2 += blockDim.x) {
                    const int t = (int)(e2 / m), v = (int)(e2 % m);
                    if (t == t0 || v == t0) continue;
                    Gi[t * qmax + v] -= Gi[t * qmax + t0] * Gi[(int64_t)t0 * qmax + v] / g0;
                }
                __syncthreads();
                for (int v = threadIdx.x; v < m; v += blockDim.x)   // rows up
                    for (int t = t0; t + 1 < m; ++t) Gi[t * qmax + v] = Gi[(t + 1) * qmax + v];
                __syncthreads();
                for (int t = threadIdx.x; t + 1 < m; t += blockDim.x)   // columns left
                    for (int v = t0; v + 1 < m; ++v) Gi[t * qmax + v] = Gi[t * qmax + v + 1];
                __syncthreads();
                if (threadIdx.x == 0) {
                    const int j = A[t0];
                    for (int t = t0; t + 1 < m; ++t) {
                        A[t] = A[t + 1];
                        sA[t] = sA[t + 1];
                    }
                    s_m = m - 1;
                    s_lam = lam - e.step;
                    s_left = j;
                    s_fresh = -1;
                }
            }
            __syncthreads();
            if (ev + 1 == max_events && threadIdx.x == 0)
                set_status(status, ST_DEGENERATE);   // no end of the path: numerical trouble
        }
        __syncthreads();
        for (int j = threadIdx.x; j < d; j += blockDim.x) B[(int64_t)ok * d + j] = 0.0;
        __syncthreads();
        for (int j = threadIdx.x; j < q; j += blockDim.x) B[(int64_t)ok * d + order[j]] = best[j];
        __syncthreads();
    }
}

// Blocks of the homotopy kernel and its workspace (doubles, ints) for d
// variables: at most 2 GB of workspace, at most two blocks per SM.
void prune_workspace(int d, int num_sms, int *blocks, size_t *dbl, size_t *ints)
{
    const size_t stride = (size_t)HL_VEC * d + (size_t)d * d;
    const size_t cap = ((size_t)2 << 30) / (stride * 8);
    const int b = (int)std::max<size_t>(1, std::min<size_t>({cap, (size_t)d, (size_t)2 * num_sms}));
    *blocks = b;
    *dbl = (size_t)b * stride;
    *ints = (size_t)b * d;
}

cudaError_t launch_prune(const double *C, const double *Bols, const int32_t *order, int d, int n,
                         double gamma, int L, double eps, int blocks, double *Cp, double *ws,
                         int *iws, double *B, uint32_t *status, cudaStream_t s)
{
    const int pb = (int)std::min<int64_t>(4096, ((int64_t)d * d + 255) / 256);
    k_permute_sym<<<pb, 256, 0, s>>>(C, order, d, Cp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t stride = (int64_t)HL_VEC * d + (int64_t)d * d;
    k_lasso_homotopy<<<blocks, HL_THREADS, 0, s>>>(Cp, Bols, order, d, n, gamma, L, eps, ws,
                                                   stride, iws, B, status);
    return cudaGetLastError();
}

}  // namespace lg
