// common.cuh -- device helpers shared by the sm_103a kernels of the library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lg {

// ---------------------------------------------------------------- status ---
// Bits of the device status word (mapped to lingam_status by the host).
enum : uint32_t {
    ST_NONFINITE = 1u,
    ST_DEGENERATE = 2u,
    ST_TIMEOUT = 4u,
    ST_ARG = 8u,
};

// Device-resident state of one ordering run.  A step whose FP32 scores do
// not separate the argmax re-scores its candidates in double-float (tier 1),
// then the still-undecided ones in FP64 (tier 2).  The candidate arrays hold
// up to d entries (every remaining variable), so no candidate is ever dropped.
struct DevState {
    uint32_t status;
    int32_t m_pos;          // position (in U) chosen at the current step
    int32_t ncand;          // candidates of the current tier (1 = decided in FP32)
    int32_t refined_steps;
    int32_t genuine_ties;
    int32_t cand_max;
    int32_t pass_begin;     // candidate index range of the current re-score pass
    int32_t pass_end;
    int32_t resolved;       // 1 once the step's argmax is decided
    int32_t fp64_candidates;  // candidates re-scored in FP64 over the run
    int32_t tier;           // 1: next re-score in double-float, 2: in FP64
    int32_t df_candidates;  // candidates re-scored in double-float over the run
    int32_t *cand;          // [d] candidate positions, by upper bound M + E descending
    double *ub;             // [d] M + E of each candidate (FP32 scores)
    double *mhp;            // [d] re-scored M of each candidate
    double *ehp;            // [d] bound on |mhp - M| (0 in FP64)
};

// Argmax order of Algorithm 1: larger M first, equal M to the smaller
// original index.
__device__ __forceinline__ bool better(double m, int u, double bm, int bu)
{
    return (m > bm) || (m == bm && u < bu);
}

// ------------------------------------------------ entropy approximation ----
// Maximum-entropy approximation of differential entropy (Hyvarinen 1998), the
// measure behind the pairwise likelihood ratio of Hyvarinen & Smith (2013)
// cited in Sec. 1:  H(u) = H(nu) - K1 (E log cosh u - GAMMA)^2
//                               - K2 (E u exp(-u^2/2))^2.
// H(nu) cancels in I(i, j), so only h = H - H(nu) is formed.
constexpr double K1 = 79.047;
constexpr double K2 = 7.4129;
constexpr double GAMMA = 0.37457;
constexpr double LN2_D = 0.69314718055994530942;
constexpr double LOG2E_D = 1.44269504088896340736;

__host__ __device__ inline double neg_entropy_part(double m1, double m2)
{
    double a = m1 - GAMMA;
    return -K1 * a * a - K2 * m2 * m2;
}

// --------------------------------------------------------------- helpers ---
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void set_status(uint32_t *status, uint32_t bit)
{
    atomicOr(status, bit);
}

// -------------------------------------------------------- pair sharding ---
// Rank that owns the entries (i, j) and (j, i) of a step with p remaining
// variables when the pair space is split over nranks.  The positions are cut
// into blocks of SHARD_BLOCK; the unordered block pairs (a <= b), taken row
// by row over the upper triangle, are cut into nranks contiguous ranges of
// about p (p - 1) / nranks ordered pairs each (a block pair goes to the range
// holding its midpoint).  Every pair-kernel tile lies inside one block pair
// (tile sides divide SHARD_BLOCK), and a tile and its transpose have the
// same owner.
constexpr int SHARD_BLOCK = 16;
__host__ __device__ inline int shard_owner(int i, int j, int p, int nranks)
{
    constexpr int64_t B = SHARD_BLOCK;
    if (p < 2 || nranks < 2) return 0;
    int64_t a = i / SHARD_BLOCK, b = j / SHARD_BLOCK;
    if (a > b) {
        const int64_t t = a;
        a = b;
        b = t;
    }
    const int64_t P = p;
    const int64_t sa = P - B * a < B ? P - B * a : B;   // size of block a (the last is short)
    const int64_t sb = P - B * b < B ? P - B * b : B;
    // ordered pairs before block pair (a, b): the full rows a' < a (each
    // s(s - 1) + 2 s (p - B a' - s) with s = B), then within row a the
    // diagonal block and the full blocks a + 1 .. b - 1
    int64_t cum = a * (2 * B * P - B * B - B) - B * B * a * (a - 1);
    if (b > a) cum += sa * (sa - 1) + 2 * sa * B * (b - a - 1);
    const int64_t w = a == b ? sa * (sa - 1) : 2 * sa * sb;
    const int64_t r = ((int64_t)nranks * (2 * cum + w)) / (2 * P * (P - 1));
    return (int)(r < nranks - 1 ? r : nranks - 1);
}

// ------------------------------------------------------------- mbarrier ---
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Global timer in nanoseconds (for waits bounded in time).
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the phase with the given parity to complete.  Returns
// false after ~2^22 polls with back-off (well over a second), so a kernel
// never spins forever; the caller then records ST_TIMEOUT and winds down.
// (A variant whose polls carried a suspend-time hint was measured slower: it
// woke the waiting warps late.)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    for (uint32_t it = 0; it < (1u << 22); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 64) __nanosleep(256);
    }
    return false;
}

// ------------------------------------------------------------------ TMA ----
// 2-D tiled bulk tensor load global -> shared, completion counted on `bar`.
// x is the innermost coordinate (elements); it must be a multiple of 16 bytes
// worth of elements -- callers pass multiples of the chunk length.
__device__ __forceinline__ void tma_load_2d(void *smem_dst, const CUtensorMap *map, int32_t x,
                                            int32_t y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ------------------------------------------------------ hardware approx ----
// MUFU approximations exposed by PTX (flush-to-zero forms).
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Error-free sum (Knuth TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// ------------------------------------------------------------ reductions ---
__device__ __forceinline__ double warp_sum_xor(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Neumaier's compensated running sum in FP32 (the rounding error of every
// addition is carried in c; value() adds the two in FP64).
struct CompSum {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float t = __fadd_rn(s, x);
        c = __fadd_rn(c, fabsf(s) >= fabsf(x) ? __fadd_rn(__fsub_rn(s, t), x)
                                              : __fadd_rn(__fsub_rn(x, t), s));
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Instance of a flattened batched grid: prefix[k] is the first block of
// instance k (prefix has count + 1 entries, ascending); returns the largest
// k with prefix[k] <= b.
__device__ __forceinline__ int find_instance(const int *prefix, int count, int b)
{
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Instances of a batched launch with work, found by the whole block at once
// instead of one instance after another in every warp: thread t tests
// instance base + t; the ones with has(k) true are listed in ascending order
// in list[] (blockDim.x entries), their number returned to every thread.
// wcnt holds blockDim.x / 32 ints.  Every thread of the block must call it.
template <class F>
__device__ __forceinline__ int block_active_list(int base, int count, F has, int *list, int *wcnt)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int k = base + (int)threadIdx.x;
    const bool act = k < count && has(k);
    const unsigned m = __ballot_sync(0xffffffffu, act);
    if (lane == 0) wcnt[w] = __popc(m);
    __syncthreads();
    int off = 0, total = 0;
    for (int i = 0; i < nwarp; ++i) {
        off += i < w ? wcnt[i] : 0;
        total += wcnt[i];
    }
    if (act) list[off + __popc(m & ((1u << lane) - 1u))] = k;
    __syncthreads();
    return total;
}

// Block-wide sum in a fixed order (warp xor trees, then warp 0 over the
// per-warp totals); the result is valid in warp 0.
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum_xor(v);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (w == 0) t = warp_sum_xor(t);
    __syncthreads();
    return t;
}

}  // namespace lg
