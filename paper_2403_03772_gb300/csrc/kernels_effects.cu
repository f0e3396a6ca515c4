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
