// kernels_gram_tc.cu -- covariance (Gram) on the 5th-generation tensor cores
// with near-FP64 accuracy, for the mixed-precision form.
//
// GB300's FP64 pipe is slow (about 1.7 FMA per clock per SM), so the FP64
// SIMT Gram C = R R^T / n costs ~16 ms at d = 1000, n = 10000.  Here every
// variable's centred column is cut into periods of 64 samples; within a
// period, relative to a power-of-two scale 2^e at least the period's largest
// magnitude, each value is written as six 7-bit signed digits:
//     x / 2^e = 2^-7 sum_k t_k,   t_k = sigma_k 2^(-7k),  |sigma_k| <= 127,
// each t_k exactly representable in BF16.  A product of two columns is then
//     2^(e_i + e_j - 14) sum_{k,l} t_ik t_jl,
// and the terms with k + l <= 5 are formed by tcgen05.mma (kind::f16, BF16
// operands, FP32 accumulation in tensor memory).  Terms of level k + l = 0, 1
// and 2 go to separate accumulators, levels 3..5 share a fourth.  After every
// period the four accumulators are read with tcgen05.ld, scaled by the
// period's 2^(e_i + e_j) and added in FP64.  Per-period scales keep a large
// value from costing digits elsewhere in its column.  The tensor cores do
// not add in exact IEEE FP32 (draining every 128 samples instead of 64 gave
// 2.5x the error), so the accuracy is measured: about 4e-11 of
// sqrt(C_ii C_jj) on heavy-tailed and skewed data (d <= 300, n <= 1e5).
//
// CTA tile: 128 x 128 entries of C (tile row <= tile column), one slice of
// the samples; 128 threads.  Per chunk of 64 samples one thread issues 12 TMA
// loads (six digit planes of the row block and six of the column block, 128
// rows x 128 bytes each, 128-byte swizzle) and 84 MMAs of 128 x 128 x 16.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "conv.cuh"
#include "kernels.cuh"

namespace lg {

namespace {

constexpr int TC_SLICES = 6;
constexpr int TC_TILE = 128;
constexpr int TC_KC = 64;           // samples per TMA chunk (128 bytes of BF16)
constexpr int TC_DRAIN = 64;        // samples per scale period and FP64 drain
constexpr int TC_THREADS = 128;
constexpr uint32_t TC_PLANE_BYTES = TC_TILE * TC_KC * 2;          // 16 KB
constexpr uint32_t TC_STAGE_BYTES = 2 * TC_SLICES * TC_PLANE_BYTES;  // 192 KB
constexpr uint32_t TC_TMEM_COLS = 512;                            // 4 accumulators x 128

// ---------------------------------------------------------- PTX wrappers ---
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A * B^T, A and B K-major BF16 tiles described by smem descriptors.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                         uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on `bar` once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

}  // namespace

// Shared-memory descriptor of a K-major tile with 128-byte rows, 128-byte
// swizzle, 8-row groups 1024 bytes apart (tcgen05 descriptor format).
__host__ __device__ inline uint64_t tc_smem_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);        // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused, 16 B)
    d |= (uint64_t)(1024u >> 4) << 32;               // stride byte offset
    d |= (uint64_t)1 << 46;                          // descriptor version
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}

// Instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t tc_instr_desc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// ------------------------------------------------------------- slicing ----
// One block per padded variable row, one warp per drain period of TC_DRAIN
// samples: the period's scale exponent e (max |x| < 2^e over the period, so
// a large value elsewhere in the column costs no digits here) and the six
// digit planes of its samples, zero beyond n and for rows beyond d.
__global__ void __launch_bounds__(256) k_gram_slices(const double *__restrict__ R, int64_t ldr,
                                                     int n, int d, int d_pad, int64_t ldk,
                                                     __nv_bfloat16 *__restrict__ S,
                                                     int *__restrict__ expo)
{
    const int i = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int periods = (int)((ldk + TC_DRAIN - 1) / TC_DRAIN);
    for (int p = warp; p < periods; p += blockDim.x >> 5) {
        double x[TC_DRAIN / 32];
        double m = 0.0;
#pragma unroll
        for (int v = 0; v < TC_DRAIN / 32; ++v) {
            const int64_t s = (int64_t)p * TC_DRAIN + v * 32 + lane;
            x[v] = (i < d && s < n) ? R[(int64_t)i * ldr + s] : 0.0;
            m = fmax(m, fabs(x[v]));
        }
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        int e = 0;
        if (m > 0.0) frexp(m, &e);                  // m = f 2^e, f in [0.5, 1)
        if (lane == 0) expo[(int64_t)p * d_pad + i] = e;
#pragma unroll
        for (int v = 0; v < TC_DRAIN / 32; ++v) {
            const int64_t s = (int64_t)p * TC_DRAIN + v * 32 + lane;
            if (s >= ldk) continue;
            // The digits of r = x 2^-e (|r| < 1) in base 128, sign apart, are
            // the 7-bit groups of F = floor(|r| 2^(7 TC_SLICES)): the steps
            // r <- 128 r - trunc(128 r), each exact in FP64, peel exactly
            // these.  F comes from the bits of x with integer shifts (no FP64
            // arithmetic): |x| = M 2^(E - 1075) for the 53-bit significand M.
            const unsigned long long b = (unsigned long long)__double_as_longlong(x[v]);
            int E = (int)((b >> 52) & 0x7ff);
            unsigned long long M = b & ((1ull << 52) - 1);
            if (E > 0) M |= 1ull << 52;
            else E = 1;                              // subnormal or zero
            const int sh = 1075 - 7 * TC_SLICES + e - E;
            const unsigned long long F = sh >= 0 ? (sh < 64 ? M >> sh : 0ull)
                                                 : (sh > -64 ? M << -sh : 0ull);
            const int sgn = (b >> 63) ? -1 : 1;
#pragma unroll
            for (int k = 0; k < TC_SLICES; ++k) {
                const int dg = (int)((F >> (7 * (TC_SLICES - 1 - k))) & 127u);   // <= 127
                const float scale = __int_as_float((127 - 7 * k) << 23);       // 2^-7k
                S[((int64_t)k * d_pad + i) * ldk + s] =
                    __float2bfloat16_rn((float)(sgn * dg) * scale);
            }
        }
    }
}

// ----------------------------------------------------------- MMA kernel ----
struct TcGramParams {
    int d, d_pad, n;
    int64_t ldk;
    int ksplit, chunks_per_split;   // in TC_KC chunks
    double *part;                   // [ksplit][d][d] partial sums (units of 2^-14)
    const int *expo;                // [periods][d_pad] scale exponents per drain period
    uint32_t *status;
};

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap tmS, const TcGramParams P)
{
    extern __shared__ uint8_t smem_raw[];
    // 1024-byte aligned operand area (128-byte swizzle atoms)
    uint8_t *base = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *planesA = base;                                   // 6 x 16 KB
    uint8_t *planesB = base + TC_SLICES * TC_PLANE_BYTES;      // 6 x 16 KB
    __shared__ uint64_t full_bar, mma_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ int s_ecol[TC_TILE];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nt = P.d_pad / TC_TILE;
    int t = blockIdx.x, bi = 0;
    while (t >= nt - bi) {
        t -= nt - bi;
        ++bi;
    }
    const int bj = bi + t;
    const int nchunks = (int)(P.ldk / TC_KC);
    const int c0 = blockIdx.y * P.chunks_per_split;
    const int c1 = min(nchunks, c0 + P.chunks_per_split);

    if (threadIdx.x == 0) {
        mbar_init(&full_bar, 1);
        mbar_init(&mma_bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&tmem_base, TC_TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    constexpr uint32_t IDESC = tc_instr_desc(TC_TILE, TC_TILE);
    const int row = bi * TC_TILE + warp * 32 + lane;   // this thread's TMEM lane = C row
    bool first_drain = true;
    int period_chunk = 0;                              // chunks since the last drain

    for (int c = c0; c < c1; ++c) {
        const uint32_t par = (uint32_t)((c - c0) & 1);
        if (threadIdx.x == 0) {
            mbar_arrive_expect_tx(&full_bar, TC_STAGE_BYTES);
            const int x = c * TC_KC;
#pragma unroll
            for (int k = 0; k < TC_SLICES; ++k) {
                tma_load_2d(planesA + k * TC_PLANE_BYTES, &tmS, x, k * P.d_pad + bi * TC_TILE,
                            &full_bar);
                tma_load_2d(planesB + k * TC_PLANE_BYTES, &tmS, x, k * P.d_pad + bj * TC_TILE,
                            &full_bar);
            }
        }
        // every exit decision below is taken by the whole block together
        if (!mbar_wait_bounded(&full_bar, par)) {
            set_status(P.status, ST_TIMEOUT);
            abort_flag = 1;
        }
        __syncthreads();
        if (abort_flag) break;
        if (threadIdx.x == 0) {
            tc_fence_after();
            const uint32_t sa = smem_u32(planesA), sb = smem_u32(planesB);
#pragma unroll
            for (int ks = 0; ks < TC_KC / 16; ++ks) {
#pragma unroll
                for (int k = 0; k < TC_SLICES; ++k) {
#pragma unroll
                    for (int l = 0; l + k < TC_SLICES; ++l) {
                        const int level = min(k + l, 3);
                        const uint32_t acc = tmem + (uint32_t)(level * TC_TILE);
                        const uint64_t ad = tc_smem_desc(sa + k * TC_PLANE_BYTES + ks * 32);
                        const uint64_t bd = tc_smem_desc(sb + l * TC_PLANE_BYTES + ks * 32);
                        // the first product of each level in a drain period overwrites
                        const bool first = period_chunk == 0 && ks == 0 &&
                                           ((level < 3 && k == 0) || (level == 3 && k == 0 && l == 3));
                        mma_bf16(acc, ad, bd, IDESC, first ? 0u : 1u);
                    }
                }
            }
            mma_commit(&mma_bar);
        }
        if (!mbar_wait_bounded(&mma_bar, par)) {
            set_status(P.status, ST_TIMEOUT);
            abort_flag = 1;
        }
        __syncthreads();
        if (abort_flag) break;
        tc_fence_after();
        ++period_chunk;
        const bool drain = period_chunk * TC_KC >= TC_DRAIN || c == c1 - 1;
        if (drain) {
            // the period's scales: entry (row, col) of this period's products
            // is worth 2^(e_row + e_col) in the partial's units
            const int64_t pe = (int64_t)(c / (TC_DRAIN / TC_KC)) * P.d_pad;
            s_ecol[threadIdx.x] = P.expo[pe + bj * TC_TILE + threadIdx.x];
            __syncthreads();
            const int erow = P.expo[pe + bi * TC_TILE + warp * 32 + lane];
            double *out = P.part + (size_t)blockIdx.y * P.d * P.d;
            const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
            for (int cb = 0; cb < TC_TILE / 32; ++cb) {
                float a0[32], a1[32], a2[32], a3[32];
                tmem_ld32(lane_addr + 0 * TC_TILE + cb * 32, a0);
                tmem_ld32(lane_addr + 1 * TC_TILE + cb * 32, a1);
                tmem_ld32(lane_addr + 2 * TC_TILE + cb * 32, a2);
                tmem_ld32(lane_addr + 3 * TC_TILE + cb * 32, a3);
                if (row < P.d) {
                    double *o = out + (size_t)row * P.d + bj * TC_TILE + cb * 32;
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const int col = bj * TC_TILE + cb * 32 + q;
                        if (col < P.d) {
                            // exact conversions off the FP64 pipe; the scale
                            // 2^k by one multiply (ldexp where 2^k is not a
                            // normal double)
                            const double sum = ((f32_to_f64(a0[q]) + f32_to_f64(a1[q])) +
                                                f32_to_f64(a2[q])) + f32_to_f64(a3[q]);
                            const int k = erow + s_ecol[cb * 32 + q];
                            const double v =
                                (k >= -1022 && k <= 1023)
                                    ? sum * __longlong_as_double((long long)(k + 1023) << 52)
                                    : ldexp(sum, k);
                            o[q] = first_drain ? v : o[q] + v;
                        }
                    }
                }
            }
            first_drain = false;
            period_chunk = 0;
            tc_fence_before();
        }
        __syncthreads();       // operands free and accumulators read before the next MMAs
        tc_fence_after();
    }
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TC_TMEM_COLS);
}

// C[i][j] = 2^-14 / n * sum over splits (upper-tile entry, so C is exactly
// symmetric).
__global__ void k_gram_tc_reduce(const double *__restrict__ part, int ksplit, int n, int d,
                                 double *__restrict__ C, int64_t ldc, double *ref_var)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
    if (j >= d) return;
    int a = i, b = j;
    if (i / TC_TILE > j / TC_TILE || (i / TC_TILE == j / TC_TILE && i > j)) {
        a = j;
        b = i;
    }
    double s = 0.0;
    for (int z = 0; z < ksplit; ++z) s += part[(size_t)z * d * d + (size_t)a * d + b];
    const double v = ldexp(s, -14) / (double)n;
    C[(int64_t)i * ldc + j] = v;
    if (i == j && ref_var) ref_var[i] = v;
}

size_t gram_tc_smem_bytes() { return (size_t)TC_STAGE_BYTES + 1024; }

cudaError_t gram_tc_setup()
{
    return cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)gram_tc_smem_bytes());
}

int gram_tc_dpad(int d) { return (d + TC_TILE - 1) / TC_TILE * TC_TILE; }
int64_t gram_tc_ldk(int n) { return ((int64_t)n + TC_KC - 1) / TC_KC * TC_KC; }
int64_t gram_tc_expo_count(int n, int d)
{
    return (gram_tc_ldk(n) + TC_DRAIN - 1) / TC_DRAIN * gram_tc_dpad(d);
}

int gram_tc_ksplit(int n, int d, int num_sms)
{
    const int nt = gram_tc_dpad(d) / TC_TILE;
    const int tiles = nt * (nt + 1) / 2;
    const int periods = (int)((gram_tc_ldk(n) + TC_DRAIN - 1) / TC_DRAIN);
    int ks = std::max(1, num_sms / std::max(1, tiles));
    return std::max(1, std::min(ks, periods));
}

cudaError_t launch_gram_tc(const CUtensorMap *tmS, const double *R, int64_t ldr, int n, int d,
                           __nv_bfloat16 *S, int *expo, double *part, int ksplit, double *C,
                           int64_t ldc, double *ref_var, uint32_t *status, cudaStream_t s)
{
    const int d_pad = gram_tc_dpad(d);
    const int64_t ldk = gram_tc_ldk(n);
    k_gram_slices<<<d_pad, 256, 0, s>>>(R, ldr, n, d, d_pad, ldk, S, expo);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nt = d_pad / TC_TILE;
    const int nchunks = (int)(ldk / TC_KC);
    // whole drain periods per split; with periods = ceil(chunks / 2) the used
    // splits never exceed ksplit (the partial buffer holds ksplit planes)
    const int periods = (nchunks * TC_KC + TC_DRAIN - 1) / TC_DRAIN;
    const int per_split_periods = (periods + ksplit - 1) / ksplit;
    TcGramParams P{};
    P.d = d;
    P.d_pad = d_pad;
    P.n = n;
    P.ldk = ldk;
    P.ksplit = ksplit;
    P.chunks_per_split = std::max(1, per_split_periods * (TC_DRAIN / TC_KC));
    P.part = part;
    P.expo = expo;
    P.status = status;
    const int used_splits = (nchunks + P.chunks_per_split - 1) / P.chunks_per_split;
    k_gram_tc<<<dim3(nt * (nt + 1) / 2, used_splits), TC_THREADS, gram_tc_smem_bytes(), s>>>(*tmS,
                                                                                            P);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_gram_tc_reduce<<<dim3((d + 127) / 128, d), 128, 0, s>>>(part, used_splits, n, d, C, ldc,
                                                              ref_var);
    return cudaGetLastError();
}

}  // namespace lg
