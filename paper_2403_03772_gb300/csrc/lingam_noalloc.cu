// lingam_noalloc.cu -- first-step scores without any device allocation.
//
// Who needs this: callers that must not allocate device memory while they
// run.  Examples are code called from inside a custom device-memory allocator
// or pool (calling cudaMalloc there would re-enter the allocator), host
// applications or plugins whose framework reserves nearly all device memory
// up front and hands out nothing else, and latency-bound services that ban
// cudaMalloc/cudaFree on their serving path because those calls can
// synchronise the whole device.  The regular entry points keep their
// workspace in a context (lingam_create allocates it); this one keeps its
// scratch in a fixed array compiled into the library instead.
//
// What it computes: the scores M(i) = -sum_j min(0, I(i, j))^2 of the first
// ordering step of Algorithm 1 (the same quantity lingam_step_measures
// returns in M_out), in FP64 throughout, for at most NOALLOC_MAX_D variables.
//
// The scratch array lives in device memory of every GPU that loads this
// library, for as long as the process runs (~66 KB).  Host code cannot use
// the array's name as a device address; every call looks the address up with
// cudaGetSymbolAddress while the caller's device is current.  The lookup is
// repeated on each call rather than cached: a device reset (cudaDeviceReset,
// or a reset of the primary context) unloads the module, and the next load
// may place the array elsewhere, so a cached address could go stale.  Once
// the module is loaded on a device the lookup allocates nothing.  Under
// CUDA's lazy module loading the module is loaded by the first call on each
// device, and that load can allocate device memory for the code and the
// array: a caller that must not allocate makes one call on each device before
// entering its no-allocation region.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "../../include/lingam.h"
#include "common.cuh"

namespace {

constexpr int NOALLOC_MAX_D = 64;
// layout of the scratch array (in doubles):
//   [0, D*D*2)        pair moment sums, entry (i, j) at (i*D + j)*2
//   [D*D*2, +D*2)     variable moment sums
//   then one double holding the status word and one holding the done counter
constexpr int NA_MOM = 0;
constexpr int NA_HZ = NOALLOC_MAX_D * NOALLOC_MAX_D * 2;
constexpr int NA_STATUS = NA_HZ + NOALLOC_MAX_D * 2;
constexpr int NA_DONE = NA_STATUS + 1;
constexpr int NA_DOUBLES = NA_DONE + 1;

// One copy per GPU that loads the library; every call on that GPU shares it.
static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

__device__ __forceinline__ void terms64(double u, double &t1, double &t2)
{
    const double au = fabs(u);
    t1 = au + log1p(exp(-2.0 * au));   // log cosh u + ln 2
    t2 = u * exp(-0.5 * u * u);
}

// One warp per work item (an unordered pair, or one variable), lanes over
// samples; every item computes its own means, variances and covariance from
// X, so the kernel needs no other preparation.  The last block to finish
// combines the moments into I(i, j) and M(i) and resets the done counter.
__global__ void __launch_bounds__(256) k_step_scores_noalloc(const double *__restrict__ X,
                                                             int n, int d, int64_t ld,
                                                             double *scratch, double *M_out)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int npairs = d * (d - 1) / 2;
    const int nitems = npairs + d;
    unsigned int *status = reinterpret_cast<unsigned int *>(scratch + NA_STATUS);
    const double invn = 1.0 / (double)n;
    for (int q = gw; q < nitems; q += nw) {
        if (q >= npairs) {
            const int a = q - npairs;
            double s = 0.0, ss = 0.0;
            for (int i = lane; i < n; i += 32) s += X[(int64_t)i * ld + a];
            const double mu = lg::warp_sum_xor(s) * invn;
            for (int i = lane; i < n; i += 32) {
                const double c = X[(int64_t)i * ld + a] - mu;
                ss += c * c;
            }
            const double var = lg::warp_sum_xor(ss) * invn;
            if (!isfinite(var)) {
                if (lane == 0) atomicOr(status, lg::ST_NONFINITE);
                continue;
            }
            if (!(var > 0.0)) {
                if (lane == 0) atomicOr(status, lg::ST_DEGENERATE);
                continue;
            }
            const double isd = 1.0 / sqrt(var);
            double m1 = 0.0, m2 = 0.0;
            for (int i = lane; i < n; i += 32) {
                double t1, t2;
                terms64((X[(int64_t)i * ld + a] - mu) * isd, t1, t2);
                m1 += t1;
                m2 += t2;
            }
            m1 = lg::warp_sum_xor(m1);
            m2 = lg::warp_sum_xor(m2);
            if (lane == 0) {
                scratch[NA_HZ + a * 2] = m1;
                scratch[NA_HZ + a * 2 + 1] = m2;
            }
            continue;
        }
        // pair index q -> (a, b), a < b
        int a = 0, r = q;
        while (r >= d - 1 - a) {
            r -= d - 1 - a;
            ++a;
        }
        const int b = a + 1 + r;
        double sa = 0.0, sb = 0.0;
        for (int i = lane; i < n; i += 32) {
            sa += X[(int64_t)i * ld + a];
            sb += X[(int64_t)i * ld + b];
        }
        const double ma = lg::warp_sum_xor(sa) * invn, mb = lg::warp_sum_xor(sb) * invn;
        double vaa = 0.0, vbb = 0.0, vab = 0.0;
        for (int i = lane; i < n; i += 32) {
            const double ca = X[(int64_t)i * ld + a] - ma, cb = X[(int64_t)i * ld + b] - mb;
            vaa += ca * ca;
            vbb += cb * cb;
            vab += ca * cb;
        }
        vaa = lg::warp_sum_xor(vaa) * invn;
        vbb = lg::warp_sum_xor(vbb) * invn;
        vab = lg::warp_sum_xor(vab) * invn;
        const double ia = 1.0 / sqrt(vaa), ib = 1.0 / sqrt(vbb);
        const double rho = vab * ia * ib;
        double s2 = 1.0 - rho * rho;
        if (!(vaa > 0.0) || !(vbb > 0.0) || !(s2 > 1e-12)) {
            if (lane == 0) atomicOr(status, lg::ST_DEGENERATE);
            s2 = 1.0;
        }
        const double isd = 1.0 / sqrt(s2);
        double ab1 = 0.0, ab2 = 0.0, ba1 = 0.0, ba2 = 0.0;
        for (int i = lane; i < n; i += 32) {
            const double za = (X[(int64_t)i * ld + a] - ma) * ia;
            const double zb = (X[(int64_t)i * ld + b] - mb) * ib;
            double t1, t2;
            terms64((za - rho * zb) * isd, t1, t2);
            ab1 += t1;
            ab2 += t2;
            terms64((zb - rho * za) * isd, t1, t2);
            ba1 += t1;
            ba2 += t2;
        }
        ab1 = lg::warp_sum_xor(ab1);
        ab2 = lg::warp_sum_xor(ab2);
        ba1 = lg::warp_sum_xor(ba1);
        ba2 = lg::warp_sum_xor(ba2);
        if (lane == 0) {
            double *o = scratch + NA_MOM + ((size_t)a * NOALLOC_MAX_D + b) * 2;
            o[0] = ab1;
            o[1] = ab2;
            o = scratch + NA_MOM + ((size_t)b * NOALLOC_MAX_D + a) * 2;
            o[0] = ba1;
            o[1] = ba2;
        }
    }
    // last block: I(i, j) and M(i)
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int *done = reinterpret_cast<unsigned int *>(scratch + NA_DONE);
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const volatile double *vs = scratch;
    const int w = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    for (int i = w; i < d; i += nwb) {
        const double hi = lg::neg_entropy_part(vs[NA_HZ + i * 2] * invn - lg::LN2_D,
                                               vs[NA_HZ + i * 2 + 1] * invn);
        double acc = 0.0;
        for (int j = lane; j < d; j += 32) {
            if (j == i) continue;
            const double hj = lg::neg_entropy_part(vs[NA_HZ + j * 2] * invn - lg::LN2_D,
                                                   vs[NA_HZ + j * 2 + 1] * invn);
            const size_t eij = NA_MOM + ((size_t)i * NOALLOC_MAX_D + j) * 2;
            const size_t eji = NA_MOM + ((size_t)j * NOALLOC_MAX_D + i) * 2;
            const double hij = lg::neg_entropy_part(vs[eij] * invn - lg::LN2_D, vs[eij + 1] * invn);
            const double hji = lg::neg_entropy_part(vs[eji] * invn - lg::LN2_D, vs[eji + 1] * invn);
            const double I = (hj + hij) - (hi + hji);
            const double v = fmin(0.0, I);
            acc += v * v;
        }
        acc = lg::warp_sum_xor(acc);
        if (lane == 0) M_out[i] = -acc;
    }
    if (threadIdx.x == 0) *reinterpret_cast<unsigned int *>(scratch + NA_DONE) = 0u;
}

// Device address of the scratch array on the current device.
cudaError_t scratch_address(double **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = reinterpret_cast<double *>(p);
    return cudaSuccess;
}

}  // namespace

extern "C" {

lingam_status lingam_step_scores_noalloc(const double *X, int64_t n, int64_t d, int64_t ld,
                                         double *M_out, lingam_stream_t stream)
{
    if (!X || !M_out) return LINGAM_ERR_ARG;
    if (d < 2 || d > NOALLOC_MAX_D) return LINGAM_ERR_ARG;   // fixed-size scratch
    if (n < 2 || n > ((int64_t)1 << 30) || ld < d) return LINGAM_ERR_ARG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    double *scratch = nullptr;
    if (e == cudaSuccess) e = scratch_address(&scratch);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the status word and the done counter must start at zero
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch + NA_STATUS, 0, 2 * sizeof(double), s);
    if (e == cudaSuccess) {
        const int items = (int)(d * (d - 1) / 2 + d);
        int nsm = 1;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const int blocks = std::max(1, std::min((items + 7) / 8, 4 * std::max(1, nsm)));
        k_step_scores_noalloc<<<blocks, 256, 0, s>>>(X, (int)n, (int)d, ld, scratch, M_out);
        e = cudaGetLastError();
    }
    unsigned int st = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&st, scratch + NA_STATUS, sizeof(st), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return LINGAM_ERR_CUDA;
    }
    if (st & lg::ST_NONFINITE) return LINGAM_ERR_NONFINITE;
    if (st & lg::ST_DEGENERATE) return LINGAM_ERR_DEGENERATE;
    return LINGAM_OK;
}

}  // extern "C"
