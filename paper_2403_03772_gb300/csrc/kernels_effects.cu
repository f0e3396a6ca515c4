// kernels_effects.cu -- what is read off the estimated graph (Sec. 4.2):
// total causal effects, the time-unrolled VarLiNGAM graph, influence
// rankings, and edge statistics over bootstrap resamples.  FP64 throughout.

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

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Adaptive lasso of each variable on its predecessors (one warp per
// variable, position k in the order, q = k predecessors at positions 0..k-1):
//   min_b 1/2 b'C_PP b - b'C_Pk + lam sum_j w_j |b_j|,  w_j = |b_ols_j|^-gamma,
// cyclic coordinate descent over j = 0..q-1 with g = C_PP b kept up to date
// (one column update per changed coordinate), warm-started along
// lam_i = lam_max eps^(i/(L-1)), lam_max = (1 + 1e-9) max_j |C_jk| / w_j; a
// lam's sweeps stop once the largest change
// |db_j| sqrt(C_jj) <= tol sqrt(C_kk).  The lam of smallest BIC =
// n log(RSS/n) + df log n (first minimum) gives row order[k] of B.
// Scratch per row: b, g, best, w (4 q doubles at ws + 4 k d).
__global__ void __launch_bounds__(128) k_adaptive_lasso(const double *Cp, const double *Bols,
                                                        const int32_t *order, int d, int n,
                                                        double gamma, int L, double eps,
                                                        double tol, int max_sweeps, double *ws,
                                                        double *B)
{
    const int lane = threadIdx.x & 31;
    const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (k >= d) return;
    const int q = k, ok = order[k];
    double *b = ws + (int64_t)4 * k * d, *g = b + d, *best = g + d, *w = best + d;
    const double *crow_k = Cp + (int64_t)k * d;   // C[P][k] = Cp[k][0..q)
    const double ckk = crow_k[k];
    // adaptive weights from the least-squares row, lam_max
    double lmax = 0.0;
    for (int j = lane; j < q; j += 32) {
        const double bo = Bols[(int64_t)ok * d + order[j]];
        const double wj = bo != 0.0 ? pow(fabs(bo), -gamma) : INFINITY;
        w[j] = wj;
        b[j] = 0.0;
        g[j] = 0.0;
        best[j] = 0.0;
        if (isfinite(wj)) lmax = fmax(lmax, fabs(crow_k[j]) / wj);
    }
    // 1e-9 above the exact boundary: rounding cannot leave a tiny coefficient
    // (counted as an edge by BIC) at the first grid point
    lmax = warp_max(lmax) * (1.0 + 1e-9);
    __syncwarp();
    if (q == 0 || !(lmax > 0.0)) {
        for (int j = lane; j < d; j += 32) B[(int64_t)ok * d + j] = 0.0;
        return;
    }
    const double stop = tol * sqrt(ckk), logn = log((double)n);
    double best_bic = INFINITY;
    for (int i = 0; i < L; ++i) {
        const double lam = lmax * pow(eps, (double)i / (double)(L - 1));
        for (int sweep = 0; sweep < max_sweeps; ++sweep) {
            double big = 0.0;
            for (int j = 0; j < q; ++j) {
                const double wj = w[j];
                if (!isfinite(wj)) continue;
                const double cjj = Cp[(int64_t)j * d + j];
                const double bj = b[j];
                const double r = crow_k[j] - (g[j] - cjj * bj);
                const double t = lam * wj;
                const double nb = (fabs(r) > t ? copysign(fabs(r) - t, r) : 0.0) / cjj;
                const double db = nb - bj;
                big = fmax(big, fabs(db) * sqrt(cjj));
                if (db != 0.0) {
                    __syncwarp();
                    if (lane == 0) b[j] = nb;
                    const double *cj = Cp + (int64_t)j * d;
                    for (int l = lane; l < q; l += 32) g[l] += db * cj[l];
                    __syncwarp();
                }
            }
            if (big <= stop) break;
        }
        // BIC of this lam: RSS/n = C_kk - 2 b'C_Pk + b'g, fixed-order lane sums
        double s1 = 0.0, s2 = 0.0;
        int nz = 0;
        for (int j = lane; j < q; j += 32) {
            const double bj = b[j];
            s1 += bj * crow_k[j];
            s2 += bj * g[j];
            nz += bj != 0.0;
        }
        s1 = warp_sum_xor(s1);
        s2 = warp_sum_xor(s2);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nz += __shfl_xor_sync(0xffffffffu, nz, o);
        const double rss = ckk - 2.0 * s1 + s2;
        const double bic = (double)n * log(fmax(rss, 1e-300)) + (double)nz * logn;
        if (bic < best_bic) {
            best_bic = bic;
            for (int j = lane; j < q; j += 32) best[j] = b[j];
        }
        __syncwarp();
    }
    for (int j = lane; j < d; j += 32) B[(int64_t)ok * d + j] = 0.0;
    __syncwarp();
    for (int j = lane; j < q; j += 32) B[(int64_t)ok * d + order[j]] = best[j];
}

cudaError_t launch_prune(const double *C, const double *Bols, const int32_t *order, int d, int n,
                         double gamma, int L, double eps, double tol, double *Cp, double *ws,
                         double *B, cudaStream_t s)
{
    const int blocks = (int)std::min<int64_t>(4096, ((int64_t)d * d + 255) / 256);
    k_permute_sym<<<blocks, 256, 0, s>>>(C, order, d, Cp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_adaptive_lasso<<<(d + 3) / 4, 128, 0, s>>>(Cp, Bols, order, d, n, gamma, L, eps, tol,
                                                  100000, ws, B);
    return cudaGetLastError();
}

}  // namespace lg
