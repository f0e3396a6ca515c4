// lingam_abi.cu -- host orchestration and the extern "C" entry points
// declared in include/lingam.h.
//
// An ordering run is a batch of instances (a single call is a batch of one).
// Per instance: pack + centre the data (FP64 columns), FP64 covariance, then
// the d-1 steps of the DirectLiNGAM loop (Sec. 2.2), each running Algorithm 1
// on the device:
//   pair moments -> score I, M -> select (argmax + near-tie candidates)
//   -> FP64 re-score passes (no-ops unless candidates) -> regress-out +
//   standardise + variable moments -> rank-1 covariance downdate.
// All instances advance through global step t together: every kernel of a
// step is one launch over the instances still running, reading per-instance
// parameters from a device array.  p = d - t of every instance is known when
// the loop is captured, which variables remain is only known on the device,
// so the whole loop is captured once per batch shape into one CUDA graph and
// replayed; the host sees the device only at launch and at the final copies.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/lingam.h"
#include "kernels.cuh"

using namespace lg;

namespace {

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

cudaError_t ensure(Buf &b, size_t bytes, bool zero = false)
{
    if (bytes == 0) bytes = 256;
    if (b.bytes >= bytes) return cudaSuccess;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) return e;
    b.bytes = bytes;
    if (zero) return cudaMemset(b.p, 0, bytes);
    return cudaSuccess;
}

void release(Buf &b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

template <typename T>
T *ptr(Buf &b)
{
    return reinterpret_cast<T *>(b.p);
}

int64_t roundup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

// The mixed form computes the covariance of a single-instance run on the
// tensor cores (kernels_gram_tc.cu).
constexpr bool TC_GRAM_ENABLED = true;

// Steps with at most P_HP remaining variables are scored entirely in
// double-float (FP64 in the FP64 form): cheap there, and the scores of late
// steps are small enough that FP32 rounding would dominate them.
constexpr int P_HP = 32;

// Bound on the error of one double-float I(i, j) (kernels_refine.cu).  The
// terms carry at most about 3e-14 absolute error and the sums fold into FP64
// every 64 samples.  Measured against FP64 on GB300 over all 1e6 first-step
// entries of the d=1000, n=10000 workload: max 7.5e-15; the bound keeps a
// factor of about 130 above that.
constexpr double DF_EPS_I = 1.0e-12;

// With the tensor-core covariance (single-instance MIXED runs; about 4e-11
// relative error) the standardised columns and rho themselves carry that
// error, which moved I by up to 1.4e-10 on the test workloads: the
// double-float bound there is 1e-9.
constexpr double DF_EPS_I_TC = 1.0e-9;

struct InstSpec {
    int64_t n, d;
    bool operator==(const InstSpec &o) const { return n == o.n && d == o.d; }
};

// Device layout of one instance inside the plan arena.
struct InstDev {
    int64_t n = 0, d = 0, ldr = 0;
    double *R = nullptr, *C = nullptr, *Cpart = nullptr, *mom = nullptr, *hzpart = nullptr;
    double *M = nullptr, *E = nullptr, *hist = nullptr, *ref_var = nullptr, *fmom = nullptr;
    double *fhz = nullptr, *lcoef = nullptr, *isd0 = nullptr, *isd1 = nullptr;
    float *I32 = nullptr;
    float *ra = nullptr;      // [d][d] 1 / sqrt(1 - rho^2) of the step's pairs (pair kernel)
    float4 *hvar = nullptr;   // [d] variable entropy terms of the step (k_hvar_b)
    int32_t *U0 = nullptr, *U1 = nullptr, *order = nullptr, *scratch = nullptr, *rows = nullptr;
    uint8_t *allow = nullptr;   // positions the prior knowledge allows at the step
    DevState *state = nullptr;
    int zrow = 0;
    int ksplit = 1;
    size_t mom_elems = 0, hz_elems = 0, fmom_elems = 0, fhz_elems = 0;
    // tensor-core covariance (mixed form): digit planes, scale exponents, map
    __nv_bfloat16 *S = nullptr;
    int *expo = nullptr;
    int tc_ksplit = 0;
    CUtensorMap tmS{};
};

// Sample-split decisions of one global step (shared by sizing and capture).
struct StepSplit {
    std::vector<int> pair_nsplit, pair_cps, reg_nsplit, reg_sps;
    std::vector<int> hp0_nsplit, hp1_nsplit;   // sample ranges of the high-precision kernel
    int cfg = 0;           // pair-kernel tile configuration of the step
};

enum LaunchKind {
    K_GRAM, K_IOTA, K_REG_INIT, K_PAIR, K_HP_ALL, K_SCORE, K_SELECT, K_HP_PASS, K_REFINE,
    K_REGRESS, K_DOWNDATE, K_FINISH, K_EVENT, K_FILL_NAN, K_GRAM_TC, K_ZLO, K_FORK, K_JOIN,
    K_COND_BEGIN, K_COND_END, K_SET_COND
};

// Batched MIXED calls compute the instances' tensor-core covariances on up
// to this many streams at once (fork/join in the step graph), each stream
// with its own digit-plane scratch: one instance's launches (at most a few
// dozen CTAs for d <= 400) leave most of the GPU idle.
constexpr int GRAM_STREAMS = 8;

// Timing events per ordering step when profiling: before the pair moments,
// after them, after score + select, after the FP64 passes, after regress-out.
constexpr int EV_PER_STEP = 5;

struct Launch {
    LaunchKind kind;
    size_t off = 0, off2 = 0;
    int count = 0, a = 0, b = 0, c = 0;
    int x = 0;   // K_SCORE of a sharded call: p of the step whose partial M, E are exchanged;
                 // K_GRAM_TC: 1 + the side stream it runs on (0: the call's stream)
};

struct Plan {
    std::vector<InstSpec> spec;
    int prec = -1, profile = -1, scores = -1, lcoef = -1, rows = -1;
    bool partial = false;   // graph holds only the first step's scores
    cudaGraphExec_t exec = nullptr;
    int nodes = 0;
    Buf arena, zarena, zloarena, params;
    std::vector<InstDev> inst;
    int64_t ldz = 0, zrows = 0;
    int maxd = 0;
    CUtensorMap tmI[PAIR_NCFG]{}, tmJ[PAIR_NCFG]{};   // per tile configuration
    std::vector<cudaEvent_t> pev;
    std::vector<double> punits;
    std::vector<Launch> eager;   // sharded calls: the launches, run in order with the
                                 // exchange after each sharded score (no graph)
    Buf conds;                   // [maxd] conditional handles of the steps' re-score blocks
    int cond_nodes = 0, cond_bodies = 0;   // kernel nodes inside them, and their number
    int nside = 0;               // side streams of the covariance fork (ctx-owned handles)
    cudaStream_t side[GRAM_STREAMS]{};
    cudaEvent_t ev_side[GRAM_STREAMS]{}, ev_fork = nullptr;
};

}  // namespace

struct lingam_ctx {
    int device = 0;
    int num_sms = 0;
    lingam_opts opts{};
    std::string err;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr, g0 = nullptr, g1 = nullptr;
    Plan plan;
    // host-input staging and the buffers of the adjacency / VAR paths
    Buf xstage, aR, aC, aCpart, aL, aW, aPiv, aM, aBt, aRef, aStatus;
    // buffers of the graph read-outs (total effects, influence, edge stats)
    Buf eIn, eIn2, eL, eW, eT, ePos, eOrd, ePtr, eOut, eStatus;
    lingam_stats stats{};
    lingam_tuning tune[2]{};   // pair-kernel choices: [0] accurate (FP32), [1] fast (MIXED)
    Buf prior;                 // prior ancestry knowledge [prior_d][prior_d] int8, or none
    int64_t prior_d = 0;
    const uint32_t *gate = nullptr;   // input gate flag (lingam_set_input_gate), or none
    uint64_t gate_ns = 0;
    // pair sharding (lingam_set_shard): this rank's slice of the pair space
    int shard_rank = 0, shard_n = 1;
    lingam_allreduce_fn allreduce = nullptr;
    void *allreduce_user = nullptr;
    std::vector<double> xbuf;         // host buffer of the exchange
    // side streams of the batched covariance (made on first use)
    cudaStream_t side[GRAM_STREAMS]{};
    cudaStream_t sbody = nullptr;   // captures the bodies of conditional nodes
    bool no_cond = false;           // conditional nodes failed to capture here: plain graphs
    cudaEvent_t ev_side[GRAM_STREAMS]{}, ev_fork = nullptr;
};

static std::string g_create_error;

#define CK(expr)                                                                 \
    do {                                                                         \
        cudaError_t _e = (expr);                                                 \
        if (_e != cudaSuccess) return fail_cuda(ctx, _e, #expr, __LINE__);       \
    } while (0)

static lingam_status fail(lingam_ctx *ctx, lingam_status st, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return st;
}

static lingam_status fail_cuda(lingam_ctx *ctx, cudaError_t e, const char *what, int line)
{
    char buf[512];
    snprintf(buf, sizeof buf, "CUDA error %d (%s) at lingam_abi.cu:%d in %s", (int)e,
             cudaGetErrorString(e), line, what);
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return fail(ctx, LINGAM_ERR_OOM, buf);
    return fail(ctx, LINGAM_ERR_CUDA, buf);
}

static lingam_status status_to_code(lingam_ctx *ctx, uint32_t st)
{
    if (st & ST_NONFINITE) return fail(ctx, LINGAM_ERR_NONFINITE, "input contains NaN or Inf");
    if (st & ST_TIMEOUT) return fail(ctx, LINGAM_ERR_TIMEOUT, "a bounded device wait expired");
    if (st & ST_DEGENERATE)
        return fail(ctx, LINGAM_ERR_DEGENERATE,
                    "degenerate data: zero residual variance or |rho| = 1 between variables");
    if (st & ST_ARG) return fail(ctx, LINGAM_ERR_ARG, "invalid argument seen on the device");
    return LINGAM_OK;
}

// ------------------------------------------------------------ planning -----

// Whole step scored by the high-precision kernel (every pair): always in the
// FP64 and DF forms, and at the small late steps of the others.
static bool step_hp(int prec, int p)
{
    return prec == LINGAM_PREC_FP64 || prec == LINGAM_PREC_DF || p <= P_HP;
}

// Tier of such a step: 2 (FP64) in the FP64 form, else 1 (double-float).
static int step_hp_tier(int prec) { return prec == LINGAM_PREC_FP64 ? 2 : 1; }

static int pair_nchunks(int64_t n) { return (int)((n + PAIR_S - 1) / PAIR_S); }

static int pair_tiles(int p, int cfg)
{
    const PairCfg &G = PAIR_CFGS[cfg];
    return ((p + G.ti() - 1) / G.ti()) * ((p + G.tj() - 1) / G.tj());
}

// Tuning table of the FP32 pair kernel of a precision form.
static const lingam_tuning &tuning_of(const lingam_ctx *ctx, int prec)
{
    return ctx->tune[prec == LINGAM_PREC_MIXED ? 1 : 0];
}

// Bucket of the table that covers p.
static int tune_bucket(const lingam_tuning &tb, int p)
{
    for (int b = 0; b < tb.count; ++b)
        if (p <= tb.p_max[b]) return b;
    return tb.count - 1;
}

// Untuned defaults: the 8 x 16 tile, splits aiming at 4 CTAs per SM.
static void default_tuning(lingam_tuning &tb, int prec)
{
    tb = lingam_tuning{};
    tb.count = 1;
    tb.precision = prec;
    tb.p_max[0] = INT32_MAX;
    tb.tile[0] = 0;
    tb.ctas_per_sm[0] = 4;
}

// Sample splits of the pair and regress kernels at global step t: enough CTAs
// in total to fill the GPU, never more splits than chunks.  The pair kernel's
// tile configuration and split target come from the tuning table at the
// largest p of the step.
// Sample ranges per work item of the high-precision kernel (one warp per
// item and range): about 64 units per SM (many items are skipped at run
// time, and units differ in length), each range at least 2048 samples.
static int hp_splits(const lingam_ctx *ctx, int64_t items, int64_t n, int count)
{
    (void)count;   // the pass serves instances in turn with the whole grid
    const int64_t target = (int64_t)ctx->num_sms * 64;
    int64_t s = (target + std::max<int64_t>(items, 1) - 1) / std::max<int64_t>(items, 1);
    s = std::min<int64_t>(s, std::max<int64_t>(1, n / 2048));
    return (int)std::max<int64_t>(1, std::min<int64_t>(s, 64));
}

static StepSplit step_splits(const lingam_ctx *ctx, const std::vector<InstSpec> &spec, int prec,
                             int t)
{
    const int K = (int)spec.size();
    StepSplit ss;
    ss.hp0_nsplit.assign(K, 1);
    ss.hp1_nsplit.assign(K, 1);
    ss.pair_nsplit.assign(K, 1);
    ss.pair_cps.assign(K, 1);
    ss.reg_nsplit.assign(K, 1);
    ss.reg_sps.assign(K, 1);
    int pmax = 0;
    for (int k = 0; k < K; ++k) pmax = std::max(pmax, (int)spec[k].d - t);
    const lingam_tuning &tb = tuning_of(ctx, prec);
    const int b = tune_bucket(tb, pmax);
    ss.cfg = tb.tile[b];
    int64_t tiles = 0, cols = 0;
    for (int k = 0; k < K; ++k) {
        const int p = (int)spec[k].d - t;
        if (p < 2 && !(t == 0 && p == 1)) continue;
        if (p >= 2 && !step_hp(prec, p)) tiles += pair_tiles(p, ss.cfg);
        cols += std::max(1, p - 1);
    }
    // a sharded rank runs about 1 / shard_n of the tiles: split its samples finer
    if (ctx->shard_n > 1) tiles = (tiles + ctx->shard_n - 1) / ctx->shard_n;
    const int64_t target_pair = (int64_t)ctx->num_sms * std::max(1, tb.ctas_per_sm[b]);
    const int64_t target = (int64_t)ctx->num_sms * 4;
    const int ns_reg = cols > 0 ? (int)std::max<int64_t>(1, (target + cols - 1) / cols) : 1;
    for (int k = 0; k < K; ++k) {
        const int64_t n = spec[k].n;
        pair_split(tiles, target_pair, pair_nchunks(n), &ss.pair_cps[k], &ss.pair_nsplit[k]);
        const int nr = std::max(1, std::min<int>(ns_reg, (int)std::max<int64_t>(1, n / 1024)));
        const int sps = (int)((n + nr - 1) / nr);
        ss.reg_sps[k] = sps;
        ss.reg_nsplit[k] = (int)((n + sps - 1) / sps);
        const int64_t p = std::max<int64_t>(2, spec[k].d - t);
        // mode 0 items: every pair and variable; mode 1: about two candidates'
        // rows plus the variables
        ss.hp0_nsplit[k] = hp_splits(ctx, p * (p - 1) / 2 + p, n, K);
        ss.hp1_nsplit[k] = hp_splits(ctx, 3 * p, n, K);
    }
    return ss;
}

static int hp_sps(int64_t n, int nsplit) { return (int)((n + nsplit - 1) / nsplit); }

static lingam_status make_tensor_maps(lingam_ctx *ctx, Plan &pl)
{
    if (!g_encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return fail(ctx, LINGAM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    cuuint64_t dims[2] = {(cuuint64_t)pl.ldz, (cuuint64_t)pl.zrows};
    cuuint64_t strides[1] = {(cuuint64_t)(pl.ldz * sizeof(float))};
    cuuint32_t elem[2] = {1, 1};
    for (int c = 0; c < PAIR_NCFG; ++c) {
        cuuint32_t boxI[2] = {(cuuint32_t)PAIR_S, (cuuint32_t)PAIR_CFGS[c].ti()};
        cuuint32_t boxJ[2] = {(cuuint32_t)PAIR_S, (cuuint32_t)PAIR_CFGS[c].tj()};
        CUresult r = g_encode(&pl.tmI[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, pl.zarena.p, dims,
                              strides, boxI, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(ctx, LINGAM_ERR_CUDA, "tensor map encode failed (rows)");
        r = g_encode(&pl.tmJ[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, pl.zarena.p, dims, strides,
                     boxJ, elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(ctx, LINGAM_ERR_CUDA, "tensor map encode failed (cols)");
    }
    return LINGAM_OK;
}

static void destroy_plan(Plan &pl)
{
    if (pl.exec) cudaGraphExecDestroy(pl.exec);
    pl.exec = nullptr;
    for (cudaEvent_t e : pl.pev) cudaEventDestroy(e);
    pl.pev.clear();
    release(pl.arena);
    release(pl.zarena);
    release(pl.zloarena);
    release(pl.params);
    release(pl.conds);
    pl.inst.clear();
    pl.spec.clear();
    pl.prec = pl.profile = pl.scores = pl.lcoef = pl.rows = -1;
    pl.partial = false;
    pl.eager.clear();
}

// Lay out and allocate the arenas of a batch (no graph yet).
static lingam_status layout_plan(lingam_ctx *ctx, Plan &pl, const std::vector<InstSpec> &spec,
                                 int prec, bool scores, bool lcoef, bool rows)
{
    const int K = (int)spec.size();
    pl.spec = spec;
    pl.prec = prec;
    pl.scores = scores;
    pl.lcoef = lcoef;
    pl.rows = rows;
    pl.inst.assign(K, InstDev{});
    pl.maxd = 0;
    int64_t maxn = 0;
    for (auto &s : spec) {
        pl.maxd = std::max<int>(pl.maxd, (int)s.d);
        maxn = std::max(maxn, s.n);
    }
    for (int k = 0; k < K; ++k) {
        pl.inst[k].n = spec[k].n;
        pl.inst[k].d = spec[k].d;
        pl.inst[k].ldr = roundup(spec[k].n, 32);
        pl.inst[k].ksplit = gram_ksplit((int)spec[k].n, (int)spec[k].d, ctx->num_sms);
        pl.inst[k].mom_elems = (size_t)spec[k].d * spec[k].d * 2;
        pl.inst[k].fmom_elems = (size_t)spec[k].d * spec[k].d * 4;
        pl.inst[k].fhz_elems = (size_t)spec[k].d * 2;
    }
    for (int t = 0; t + 1 < std::max(2, pl.maxd); ++t) {
        StepSplit ss = step_splits(ctx, spec, prec, t);
        for (int k = 0; k < K; ++k) {
            const int64_t p = spec[k].d - t;
            if (t == 0)
                pl.inst[k].hz_elems = std::max(
                    pl.inst[k].hz_elems, (size_t)ss.reg_nsplit[k] * (size_t)spec[k].d * 2);
            if (p < 2) continue;
            if (!step_hp(prec, (int)p))
                pl.inst[k].mom_elems =
                    std::max(pl.inst[k].mom_elems, (size_t)ss.pair_nsplit[k] * p * p * 2);
            else
                pl.inst[k].mom_elems =
                    std::max(pl.inst[k].mom_elems, (size_t)ss.hp0_nsplit[k] * p * p * 2);
            const size_t hs = (size_t)std::max(ss.hp0_nsplit[k], ss.hp1_nsplit[k]);
            pl.inst[k].fhz_elems = std::max(pl.inst[k].fhz_elems, hs * p * 2);
            pl.inst[k].fmom_elems = std::max(pl.inst[k].fmom_elems,
                                             (size_t)ss.hp1_nsplit[k] * spec[k].d * p * 4);
            pl.inst[k].hz_elems =
                std::max(pl.inst[k].hz_elems, (size_t)ss.reg_nsplit[k] * (size_t)p * 2);
        }
    }
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (size_t)roundup((int64_t)std::max<size_t>(bytes, 8), 256);
        return o;
    };
    struct Off {
        size_t R, C, Cpart, mom, hz, M, E, hist, ref, fmom, fhz, lcoef, U, order, scratch, rows,
            state, isd, I32, ra, hvar, S, expo, cand, cdbl, allow;
    };
    std::vector<Off> o(K);
    // MIXED form: tensor-core covariance for every instance.  The BF16 digit
    // planes and exponents are scratch of one instance's launches at a time:
    // a batch runs its instances' covariances on W side streams, instance k
    // on stream k mod W in order, so W regions sized for the largest
    // instance serve them all (region k mod W).
    const bool tc = TC_GRAM_ENABLED && prec == LINGAM_PREC_MIXED;
    size_t tcS = 0, tcE = 0, maxS = 0, maxE = 0;
    const int W = (tc && K > 1) ? std::min(K, GRAM_STREAMS) : 1;   // scratch regions
    if (tc) {
        for (int k = 0; k < K; ++k) {
            maxS = std::max(maxS, (size_t)6 * gram_tc_dpad((int)spec[k].d) *
                                      gram_tc_ldk((int)spec[k].n) * 2);
            maxE = std::max(maxE, (size_t)gram_tc_expo_count((int)spec[k].n, (int)spec[k].d) * 4);
        }
        maxS = (size_t)roundup((int64_t)maxS, 1024);
        maxE = (size_t)roundup((int64_t)maxE, 256);
        tcS = take(maxS * W);
        tcE = take(maxE * W);
    }
    pl.nside = W > 1 ? W : 0;
    for (int k = 0; k < pl.nside; ++k) {   // the context's side streams, made once
        if (!ctx->side[k]) CK(cudaStreamCreateWithFlags(&ctx->side[k], cudaStreamNonBlocking));
        if (!ctx->ev_side[k])
            CK(cudaEventCreateWithFlags(&ctx->ev_side[k], cudaEventDisableTiming));
        pl.side[k] = ctx->side[k];
        pl.ev_side[k] = ctx->ev_side[k];
    }
    if (pl.nside > 0) {
        if (!ctx->ev_fork) CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
        pl.ev_fork = ctx->ev_fork;
    }
    for (int k = 0; k < K; ++k) {
        const int64_t n = spec[k].n, d = spec[k].d, ldr = pl.inst[k].ldr;
        o[k].R = take((size_t)d * ldr * 8);
        o[k].C = take((size_t)d * d * 8);
        pl.inst[k].tc_ksplit = tc ? gram_tc_ksplit((int)n, (int)d, ctx->num_sms) : 0;
        o[k].Cpart = take((size_t)std::max(pl.inst[k].ksplit, pl.inst[k].tc_ksplit) * d * d * 8);
        o[k].S = tcS + (size_t)(k % W) * maxS;
        o[k].expo = tcE + (size_t)(k % W) * maxE;
        o[k].mom = take(pl.inst[k].mom_elems * 8);
        o[k].hz = take(pl.inst[k].hz_elems * 8);
        o[k].M = take((size_t)d * 8);
        o[k].E = take((size_t)d * 8);
        o[k].hist = scores ? take((size_t)d * d * 8) : 0;
        o[k].ref = take((size_t)d * 8);
        o[k].fmom = take(pl.inst[k].fmom_elems * 8);
        o[k].fhz = take(pl.inst[k].fhz_elems * 8);
        o[k].lcoef = lcoef ? take((size_t)d * d * 8) : 0;
        o[k].U = take((size_t)2 * d * 4);
        o[k].order = take((size_t)d * 4);
        o[k].scratch = take((size_t)d * 4);
        o[k].rows = rows ? take((size_t)n * 4) : 0;
        o[k].state = take(sizeof(DevState));
        o[k].isd = take((size_t)2 * d * 8);
        o[k].I32 = take((size_t)d * d * 4);
        o[k].ra = take((size_t)d * d * 4);
        o[k].hvar = take((size_t)d * 16);
        o[k].cand = take((size_t)d * 4);
        o[k].cdbl = take((size_t)3 * d * 8);
        o[k].allow = take((size_t)d);

    }
    CK(ensure(pl.arena, off));
    CK(cudaMemset(pl.arena.p, 0, off));
    pl.ldz = roundup(std::max<int64_t>(maxn, PAIR_S), 64);
    pl.zrows = 0;
    for (int k = 0; k < K; ++k) {
        pl.inst[k].zrow = (int)pl.zrows;
        pl.zrows += spec[k].d;
    }
    CK(ensure(pl.zarena, (size_t)pl.zrows * pl.ldz * 4, true));
    // the padding of every z row (samples n .. ldz) must read as zeros: the
    // fast pair kernel runs a range's last chunk through its full-chunk path
    // and corrects for the padding exactly; a reused arena may hold old rows
    CK(cudaMemset(pl.zarena.p, 0, (size_t)pl.zrows * pl.ldz * 4));
    if (prec != LINGAM_PREC_FP64) CK(ensure(pl.zloarena, (size_t)pl.zrows * pl.ldz * 4, true));
    char *base = reinterpret_cast<char *>(pl.arena.p);
    for (int k = 0; k < K; ++k) {
        InstDev &I = pl.inst[k];
        const int64_t d = spec[k].d;
        I.R = reinterpret_cast<double *>(base + o[k].R);
        I.C = reinterpret_cast<double *>(base + o[k].C);
        I.Cpart = reinterpret_cast<double *>(base + o[k].Cpart);
        I.mom = reinterpret_cast<double *>(base + o[k].mom);
        I.hzpart = reinterpret_cast<double *>(base + o[k].hz);
        I.M = reinterpret_cast<double *>(base + o[k].M);
        I.E = reinterpret_cast<double *>(base + o[k].E);
        I.hist = scores ? reinterpret_cast<double *>(base + o[k].hist) : nullptr;
        I.ref_var = reinterpret_cast<double *>(base + o[k].ref);
        I.fmom = reinterpret_cast<double *>(base + o[k].fmom);
        I.fhz = reinterpret_cast<double *>(base + o[k].fhz);
        I.lcoef = lcoef ? reinterpret_cast<double *>(base + o[k].lcoef) : nullptr;
        I.U0 = reinterpret_cast<int32_t *>(base + o[k].U);
        I.U1 = I.U0 + d;
        I.order = reinterpret_cast<int32_t *>(base + o[k].order);
        I.scratch = reinterpret_cast<int32_t *>(base + o[k].scratch);
        I.rows = rows ? reinterpret_cast<int32_t *>(base + o[k].rows) : nullptr;
        I.state = reinterpret_cast<DevState *>(base + o[k].state);
        I.isd0 = reinterpret_cast<double *>(base + o[k].isd);
        I.isd1 = I.isd0 + d;
        I.I32 = reinterpret_cast<float *>(base + o[k].I32);
        I.ra = reinterpret_cast<float *>(base + o[k].ra);
        I.hvar = reinterpret_cast<float4 *>(base + o[k].hvar);
        I.allow = reinterpret_cast<uint8_t *>(base + o[k].allow);

        {   // candidate arrays of the device state
            DevState h{};
            h.cand = reinterpret_cast<int32_t *>(base + o[k].cand);
            h.ub = reinterpret_cast<double *>(base + o[k].cdbl);
            h.mhp = h.ub + d;
            h.ehp = h.mhp + d;
            CK(cudaMemcpy(I.state, &h, sizeof(DevState), cudaMemcpyHostToDevice));
        }
        if (I.tc_ksplit > 0) {
            I.S = reinterpret_cast<__nv_bfloat16 *>(base + o[k].S);
            I.expo = reinterpret_cast<int *>(base + o[k].expo);
            const int64_t ldk = gram_tc_ldk((int)I.n);
            const int dpad = gram_tc_dpad((int)I.d);
            cuuint64_t dims[2] = {(cuuint64_t)ldk, (cuuint64_t)6 * dpad};
            cuuint64_t strides[1] = {(cuuint64_t)(ldk * 2)};
            cuuint32_t box[2] = {64, 128}, elem[2] = {1, 1};
            if (!g_encode) {
                lingam_status st = make_tensor_maps(ctx, pl);   // loads the encoder
                if (st) return st;
            }
            CUresult r = g_encode(&I.tmS, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, I.S, dims, strides,
                                  box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return fail(ctx, LINGAM_ERR_CUDA, "tensor map encode failed (slices)");
        }
    }
    return make_tensor_maps(ctx, pl);
}

// First block of every instance in a flattened batched launch (count + 1
// entries, the last one the total).
static std::vector<int> block_prefix(const std::vector<int> &blocks)
{
    std::vector<int> pre(1, 0);
    for (int b : blocks) pre.push_back(pre.back() + b);
    return pre;
}

// Parameter arrays of every launch, gathered host-side and uploaded at once.
struct ParamBlob {
    std::vector<char> bytes;
    template <typename T>
    size_t add(const std::vector<T> &v)
    {
        size_t o = (size_t)roundup((int64_t)bytes.size(), 64);
        bytes.resize(o + sizeof(T) * std::max<size_t>(v.size(), 1));
        if (!v.empty()) memcpy(bytes.data() + o, v.data(), sizeof(T) * v.size());
        return o;
    }
};

// Issue one launch of a plan on stream s (captured into the plan's graph, or
// run directly by a sharded call); *nodes counts the kernel nodes.
static cudaError_t issue_launch(Plan &pl, const Launch &l, char *pb, cudaStream_t s, bool capture,
                                int *nodes)
{
    void *P = pb + l.off;
    cudaError_t e = cudaSuccess;
    switch (l.kind) {
    case K_GRAM: e = launch_gram_b((const GramParams *)P, l.count, l.a, l.b, s); ++*nodes; break;
    case K_IOTA: e = launch_iota_b((const IotaParams *)P, l.count, l.a, s); break;
    case K_REG_INIT:
        e = launch_regress_b((const RegressParams *)P, (const int *)(pb + l.off2), l.count,
                             true, l.a, s);
        break;
    case K_PAIR:
        e = launch_pair_b(l.c, l.b, &pl.tmI[l.b], &pl.tmJ[l.b], (const PairParams *)P,
                          (const int *)(pb + l.off2), l.count, l.a, s);
        break;
    case K_HP_ALL: e = launch_pairs_hp_b(l.c, (const HpParams *)P, l.count, l.a, s); break;
    case K_SCORE:
        e = launch_score_b((const ScoreParams *)P, (const int *)(pb + l.off2), l.count, l.b,
                           l.a, s);
        ++*nodes;   // k_hvar_b + k_score_b
        break;
    case K_SELECT: e = launch_select_b((const SelectParams *)P, l.count, s); break;
    case K_SET_COND:
        e = launch_set_rescore_cond(pl.inst[0].state, ptr<unsigned long long>(pl.conds) + l.a, s);
        break;
    case K_HP_PASS: e = launch_pairs_hp_b(l.c, (const HpParams *)P, l.count, l.a, s); break;
    case K_REFINE:
        e = launch_refine_select_b((const RefineSelectParams *)P, l.count, l.a, s);
        break;
    case K_REGRESS:
        e = launch_regress_b((const RegressParams *)P, (const int *)(pb + l.off2), l.count,
                             false, l.a, s);
        break;
    case K_DOWNDATE:
        e = launch_downdate_b((const DowndateParams *)P, (const int *)(pb + l.off2), l.count,
                              l.a, s);
        break;
    case K_FINISH: e = launch_finish_b((const FinishParams *)P, l.count, s); break;
    case K_EVENT:
        e = capture ? cudaEventRecordWithFlags(pl.pev[l.a], s, cudaEventRecordExternal)
                    : cudaEventRecord(pl.pev[l.a], s);
        --*nodes;
        break;
    case K_GRAM_TC: {
        InstDev &I = pl.inst[l.c];
        const cudaStream_t gs = l.x > 0 ? pl.side[l.x - 1] : s;
        e = launch_gram_tc(&I.tmS, I.R, I.ldr, (int)I.n, (int)I.d, I.S, I.expo, I.Cpart,
                           I.tc_ksplit, I.C, I.d, I.ref_var, &I.state->status, gs);
        *nodes += 2;
        break;
    }
    case K_FORK:   // the side streams start after everything before on s
        e = cudaEventRecord(pl.ev_fork, s);
        for (int k = 0; k < l.a && e == cudaSuccess; ++k)
            e = cudaStreamWaitEvent(pl.side[k], pl.ev_fork, 0);
        return e;
    case K_COND_BEGIN:   // captured by capture_plan; an eager run issues the body as is
    case K_COND_END:
        return cudaSuccess;
    case K_JOIN:   // s continues after everything issued on the side streams
        for (int k = 0; k < l.a && e == cudaSuccess; ++k) {
            e = cudaEventRecord(pl.ev_side[k], pl.side[k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, pl.ev_side[k], 0);
        }
        return e;
    case K_ZLO: e = launch_zlo_b((const ZloParams *)P, l.count, l.a, s); break;
    case K_FILL_NAN:
        e = launch_fill_nan(pl.inst[l.c].hist, (size_t)pl.inst[l.c].d * pl.inst[l.c].d, s);
        break;
    }
    ++*nodes;
    return e;
}

// Adds an if-node after the work captured so far on s (its condition: a new
// handle, 0 at every graph launch until a kernel sets it), makes it the
// point where the capture of s continues, and starts capturing its body on
// sb.
static cudaError_t begin_cond_body(cudaStream_t s, cudaStream_t sb, unsigned long long *handle)
{
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edata = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, &edata, &nd);
    if (e != cudaSuccess) return e;
    if (st != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    cudaGraphConditionalHandle h = 0;
    e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    e = cudaGraphAddNode(&node, g, deps, edata, nd, &np);
    if (e != cudaSuccess) return e;
    e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) return e;
    *handle = h;
    return cudaStreamBeginCaptureToGraph(sb, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal);
}

// Capture the covariance + ordering loop of the current plan into one graph.
// stop_after_score0 captures only the first step up to its scores (and writes
// I(i, j) of the single instance to Iout and the per-entry bounds to epsOut).
static lingam_status capture_plan(lingam_ctx *ctx, bool stop_after_score0, double *Iout,
                                  double *epsOut)
{
    Plan &pl = ctx->plan;
    const int K = (int)pl.inst.size();
    const int prec = pl.prec;
    const bool profile = ctx->opts.profile != 0 && !stop_after_score0;
    const bool sharded = ctx->shard_n > 1;
    cudaStream_t s = ctx->s;
    const double tie = ctx->opts.tie_scale > 0 ? ctx->opts.tie_scale : 1.0;
    // On request (opts.conditional_rescore) a single-instance graph puts each
    // step's re-score block (the low parts and the double-float and FP64
    // passes, no-ops unless candidates remain) under a conditional node that
    // a one-thread kernel after the select kernel sets: steps decided by
    // their FP32 scores skip those launches.  A batch keeps them (one
    // condition would have to summarise all its instances).  Off by default:
    // Nsight Compute does not profile the kernel nodes of a graph with
    // conditional nodes, and at d = 1000 the blocks cost more than they save.
    const bool use_cond = ctx->opts.conditional_rescore != 0 && pl.inst.size() == 1 &&
                          !sharded && !stop_after_score0 && !ctx->no_cond;
    if (use_cond) CK(ensure(pl.conds, (size_t)pl.maxd * sizeof(unsigned long long)));
    std::vector<unsigned long long> hconds(use_cond ? pl.maxd : 0, 0ull);
    // Moment-error model of the FP32 pair kernels and the regress kernel
    // (ErrModel): per-sample worst cases of the MUFU ex2/lg2 approximations
    // (relative 2^-22.5 / absolute 2^-22.6), the FP32 product of four 1 + y
    // and the accurate expf/log1pf (a few ulp), with compensated sums; the
    // residual a z_i - b z_j carries about 3 * 2^-24 a (|z_i| + |z_j|).
    // Those worst cases assume every per-sample error has the same sign; on
    // the calibration workloads (heavy and light tails, skewed noise, VAR
    // innovations, n = 1e6, a near-collinear chain) the largest error was
    // 0.18 of the resulting bound, so the terms are scaled by 0.45: the bound
    // stays 2.5x above every error seen, and a GPU test keeps it above 2x.
    const double s6 = 0.45 * tie;
    ErrModel em{};
    if (prec == LINGAM_PREC_MIXED)
        em = ErrModel{2.0e-7 * s6, 1.2e-7 * s6, 3.0e-7 * s6, 1.5e-7 * s6, 1.0e-7 * s6};
    else
        em = ErrModel{1.5e-7 * s6, 1.0e-7 * s6, 3.0e-7 * s6, 1.5e-7 * s6, 1.0e-7 * s6};
    const int pmode = prec == LINGAM_PREC_MIXED ? PAIR_FAST : PAIR_ACCURATE;
    const double a1 = pmode == PAIR_FAST ? LN2_D : 1.0;
    const double a2 = pmode == PAIR_FAST ? 1.0 / KSC : 1.0;
    const int last_t = stop_after_score0 ? 0 : pl.maxd - 2;
    float *zbase = ptr<float>(pl.zarena);
    float *zlobase = prec == LINGAM_PREC_FP64 ? nullptr : ptr<float>(pl.zloarena);

    ParamBlob blob;
    std::vector<Launch> L;
    for (int k = 0; k < K; ++k)
        if (pl.inst[k].hist) {
            Launch lf{K_FILL_NAN};
            lf.c = k;
            L.push_back(lf);
        }
    {
        std::vector<GramParams> g(K);
        std::vector<IotaParams> io(K);
        int maxks = 1;
        for (int k = 0; k < K; ++k) {
            InstDev &I = pl.inst[k];
            g[k] = GramParams{I.R, I.ldr, (int)I.n, (int)I.d, I.ksplit, I.Cpart, I.C, I.d, I.ref_var};
            io[k] = IotaParams{I.U0, (int)I.d, I.state};
            maxks = std::max(maxks, I.ksplit);
        }
        if (pl.inst[0].tc_ksplit > 0) {
            // one tensor-core covariance per instance; a batch spreads them
            // over the side streams (instance k on stream k mod nside, which
            // owns scratch region k mod nside)
            if (pl.nside > 0) {
                Launch lf{K_FORK};
                lf.a = pl.nside;
                L.push_back(lf);
            }
            for (int k = 0; k < K; ++k) {
                Launch lt{K_GRAM_TC};
                lt.c = k;
                lt.x = pl.nside > 0 ? 1 + k % pl.nside : 0;
                L.push_back(lt);
            }
            if (pl.nside > 0) {
                Launch lj{K_JOIN};
                lj.a = pl.nside;
                L.push_back(lj);
            }
        } else {
            Launch lg_{K_GRAM};
            lg_.off = blob.add(g);
            lg_.count = K;
            lg_.a = pl.maxd;
            lg_.b = maxks;
            L.push_back(lg_);
        }
        Launch li{K_IOTA};
        li.off = blob.add(io);
        li.count = K;
        li.a = pl.maxd;
        L.push_back(li);
    }
    std::vector<int> nsplit_hz(K, 1);
    auto regress_params = [&](InstDev &I, int t, int p, int32_t *Uc, int32_t *Un, int sps,
                              bool init) {
        RegressParams P{};
        P.isd_out = init ? I.isd0 : ((t & 1) ? I.isd0 : I.isd1);
        P.R = I.R;
        P.ldr = I.ldr;
        P.z = zbase + (int64_t)I.zrow * pl.ldz;
        P.ldz = pl.ldz;
        P.C = I.C;
        P.ldc = I.d;
        P.U = Uc;
        P.Unext = Un;
        P.p = p;
        P.n = (int)I.n;
        P.sps = sps;
        P.state = I.state;
        P.order = I.order;
        P.t = t;
        P.hzpart = I.hzpart;
        P.ref_var = I.ref_var;
        P.lcoef = init ? nullptr : I.lcoef;
        P.ldl = I.d;
        P.status = &I.state->status;
        return P;
    };
    {
        StepSplit ss0 = step_splits(ctx, pl.spec, prec, 0);
        std::vector<RegressParams> r(K);
        int maxsplit = 1;
        for (int k = 0; k < K; ++k) {
            InstDev &I = pl.inst[k];
            r[k] = regress_params(I, 0, (int)I.d, I.U0, I.U1, ss0.reg_sps[k], true);
            nsplit_hz[k] = ss0.reg_nsplit[k];
            maxsplit = std::max(maxsplit, ss0.reg_nsplit[k]);
        }
        std::vector<int> nb(K);
        for (int k = 0; k < K; ++k)
            nb[k] = regress_blocks((int)pl.inst[k].d, (int)pl.inst[k].n, r[k].sps);
        const std::vector<int> pre = block_prefix(nb);
        Launch lr{K_REG_INIT};
        lr.off = blob.add(r);
        lr.off2 = blob.add(pre);
        lr.count = K;
        lr.a = pre.back();
        L.push_back(lr);
    }
    if (profile) {
        for (cudaEvent_t e : pl.pev) cudaEventDestroy(e);
        pl.pev.assign(EV_PER_STEP * (size_t)std::max(1, pl.maxd - 1), nullptr);
        for (auto &e : pl.pev) CK(cudaEventCreate(&e));
        pl.punits.assign((size_t)std::max(1, pl.maxd - 1), 0.0);
    }
    for (int t = 0; t <= last_t; ++t) {
        StepSplit ss = step_splits(ctx, pl.spec, prec, t);
        std::vector<PairParams> pp;
        std::vector<int> prefix(1, 0);
        std::vector<HpParams> fa, fd1, fd2, f64;
        std::vector<ZloParams> zl_all, zl_cond;   // low parts: every-pair steps / re-scores
        std::vector<ScoreParams> sc;
        std::vector<SelectParams> se;
        std::vector<RefineSelectParams> rd1, rd2, r64;
        std::vector<RegressParams> rg;
        std::vector<DowndateParams> dd;
        int maxp = 0, maxcols = 0, maxsplit = 1;
        int xp = 0;   // p of a sharded FP32-scored step (its partial scores are exchanged)
        double units = 0;
        for (int k = 0; k < K; ++k) {
            InstDev &I = pl.inst[k];
            const int p = (int)I.d - t;
            if (p < 2) continue;
            const int n = (int)I.n;
            maxp = std::max(maxp, p);
            units += (double)p * (p - 1) * n;
            int32_t *Uc = (t & 1) ? I.U1 : I.U0;
            int32_t *Un = (t & 1) ? I.U0 : I.U1;
            double *isd = (t & 1) ? I.isd1 : I.isd0;
            double *hist_row = I.hist ? I.hist + (size_t)t * I.d : nullptr;
            const bool hp = step_hp(prec, p);
            const double eps2 = (I.tc_ksplit > 0 ? DF_EPS_I_TC : DF_EPS_I) * tie;
            const int hp_tier = step_hp_tier(prec);
            auto hpp = [&](int mode, int with_vars, double *mom) {
                HpParams F{};
                // entries whose FP32 I clears the FP32 bound need no re-score
                // a sharded rank holds only its own entries' bounds, and every rank
                // must re-score identically: no skipping by the FP32 bounds then
                F.I32 = (mode == 1 && !hp && !sharded) ? I.I32 : nullptr;
                F.R = I.R;
                F.ldr = I.ldr;
                F.zhi = zbase + (int64_t)I.zrow * pl.ldz;
                F.zlo = zlobase ? zlobase + (int64_t)I.zrow * pl.ldz : nullptr;
                F.ldz = pl.ldz;
                F.isd = isd;
                F.C = I.C;
                F.ldc = I.d;
                F.U = Uc;
                F.p = p;
                F.n = n;
                F.mode = mode;
                F.with_vars = with_vars;
                F.state = I.state;
                F.mom = mom;
                F.hz = I.fhz;
                F.status = &I.state->status;
                F.nsplit = mode == 0 ? ss.hp0_nsplit[k] : ss.hp1_nsplit[k];
                F.sps = hp_sps(n, F.nsplit);
                F.mom_sstride = mode == 0 ? (int64_t)p * p * 2 : (int64_t)I.d * p * 4;
                return F;
            };
            if (zlobase) {
                ZloParams Z{};
                Z.R = I.R;
                Z.ldr = I.ldr;
                Z.zhi = zbase + (int64_t)I.zrow * pl.ldz;
                Z.zlo = zlobase + (int64_t)I.zrow * pl.ldz;
                Z.ldz = pl.ldz;
                Z.isd = isd;
                Z.U = Uc;
                Z.p = p;
                Z.n = n;
                Z.state = I.state;
                Z.always = hp ? 1 : 0;
                if (hp && hp_tier == 1) zl_all.push_back(Z);
                else if (!hp) zl_cond.push_back(Z);
            }
            ScoreParams S{};
            if (hp) {
                fa.push_back(hpp(0, 1, I.mom));
                S.mom = I.mom;
                S.nsplit = ss.hp0_nsplit[k];
                S.hz = I.fhz;
                S.nsplit_hz = ss.hp0_nsplit[k];
                S.a1 = 1.0;
                S.b1 = -LN2_D;
                S.a2 = 1.0;
                S.epsI = hp_tier == 1 ? eps2 : 0.0;
            } else {
                PairParams P{};
                P.C = I.C;
                P.ldc = I.d;
                P.U = Uc;
                P.p = p;
                P.n = n;
                P.tiles_i = (p + PAIR_CFGS[ss.cfg].ti() - 1) / PAIR_CFGS[ss.cfg].ti();
                P.tiles_j = (p + PAIR_CFGS[ss.cfg].tj() - 1) / PAIR_CFGS[ss.cfg].tj();
                P.nchunks = pair_nchunks(n);
                P.cps = ss.pair_cps[k];
                P.nsplit = ss.pair_nsplit[k];
                P.mom = reinterpret_cast<float2 *>(I.mom);
                P.status = &I.state->status;
                P.row0 = I.zrow;
                P.isd = isd;
                P.shard_rank = ctx->shard_rank;
                P.shard_n = ctx->shard_n;
                P.ra = I.ra;
                pp.push_back(P);
                prefix.push_back(prefix.back() + P.tiles_i * P.tiles_j * P.nsplit);
                S.mom2 = reinterpret_cast<const float2 *>(I.mom);
                S.nsplit = P.nsplit;
                S.hz = I.hzpart;
                S.nsplit_hz = nsplit_hz[k];
                S.a1 = a1;
                S.b1 = -LN2_D;
                S.a2 = a2;
                S.epsI = 0.0;
                S.use_model = 1;
                S.model = em;
                S.C = I.C;
                S.ldc = I.d;
                S.isd = isd;
                S.shard_rank = ctx->shard_rank;
                S.shard_n = ctx->shard_n;
                S.ra = I.ra;
                S.hvar = I.hvar;
                xp = p;
            }
            S.p = p;
            S.n = n;
            S.ha1 = 1.0;
            S.hb1 = -LN2_D;
            S.ha2 = 1.0;
            S.U = Uc;
            S.M = I.M;
            S.E = I.E;
            S.hist = hist_row;
            S.Iout = stop_after_score0 ? Iout : nullptr;
            S.epsOut = stop_after_score0 ? epsOut : nullptr;
            S.I32 = hp ? nullptr : I.I32;
            sc.push_back(S);
            // candidates of an FP32-scored step go to double-float first; a
            // step scored in double-float sends its near-ties to FP64
            se.push_back(SelectParams{I.M, I.E, Uc, p, I.state, I.scratch, hp ? 2 : 1,
                                      ctx->prior_d > 0 ? (const int8_t *)ctx->prior.p : nullptr,
                                      ctx->prior_d, I.allow});
            fd1.push_back(hpp(1, 1, I.fmom));
            fd2.push_back(hpp(1, 0, I.fmom));
            f64.push_back(hpp(1, 1, I.fmom));
            const double e2 = eps2;
            const int ns1 = ss.hp1_nsplit[k];
            const int64_t fst = (int64_t)I.d * p * 4;
            rd1.push_back(RefineSelectParams{I.fmom, I.fhz, p, n, ns1, fst, Uc, I.state, hist_row,
                                             1, e2, 0});
            rd2.push_back(RefineSelectParams{I.fmom, I.fhz, p, n, ns1, fst, Uc, I.state, hist_row,
                                             1, e2, 1});
            r64.push_back(RefineSelectParams{I.fmom, I.fhz, p, n, ns1, fst, Uc, I.state, hist_row,
                                             2, 0.0, 1});
            rg.push_back(regress_params(I, t, p, Uc, Un, ss.reg_sps[k], false));
            nsplit_hz[k] = ss.reg_nsplit[k];
            maxcols = std::max(maxcols, p - 1);
            maxsplit = std::max(maxsplit, ss.reg_nsplit[k]);
            dd.push_back(DowndateParams{I.C, I.d, Uc, p, I.state});
        }
        if (sc.empty()) break;
        // each instance of a high-precision launch starts at the warp after
        // the previous one's expected units (every unit of an every-pair
        // pass, two candidate rows of a re-score pass)
        for (std::vector<HpParams> *v : {&fa, &fd1, &fd2, &f64}) {
            int64_t off = 0;
            for (HpParams &F : *v) {
                F.woff = off;
                const int64_t items = F.mode == 0 ? (int64_t)F.p * (F.p - 1) / 2 + F.p
                                                  : 2 * (int64_t)F.p + (F.with_vars ? F.p : 0);
                off += items * F.nsplit;
            }
        }
        const int cnt = (int)sc.size();
        // re-score passes: 8 blocks per SM (64 warps, 24 resident) striding
        // over the units; one wave of resident blocks was measured slower on
        // the passes that have work, and a pass without work costs ~4 us
        const int hp_blocks = ctx->num_sms * 8;
        if (profile) {
            Launch ev{K_EVENT};
            ev.a = EV_PER_STEP * t;
            L.push_back(ev);
            pl.punits[t] = units;
        }
        if (!pp.empty()) {
            Launch l{K_PAIR};
            l.off = blob.add(pp);
            l.off2 = blob.add(prefix);
            l.count = (int)pp.size();
            l.a = prefix.back();
            l.b = ss.cfg;
            l.c = pmode;
            L.push_back(l);
        }
        if (!zl_all.empty()) {
            Launch l{K_ZLO};
            l.off = blob.add(zl_all);
            l.count = (int)zl_all.size();
            l.a = ctx->num_sms * 4;
            L.push_back(l);
        }
        if (!fa.empty()) {
            Launch l{K_HP_ALL};
            l.off = blob.add(fa);
            l.count = (int)fa.size();
            l.a = ctx->num_sms * 8;
            l.c = step_hp_tier(prec);
            L.push_back(l);
        }
        if (profile) {
            Launch ev{K_EVENT};
            ev.a = EV_PER_STEP * t + 1;
            L.push_back(ev);
        }
        std::vector<int> nbs, nbr, nbd;
        for (int q = 0; q < cnt; ++q) {
            nbs.push_back(score_blocks(sc[q].p));
            nbr.push_back(regress_blocks(rg[q].p - 1, rg[q].n, rg[q].sps));
            nbd.push_back(downdate_blocks(dd[q].p));
        }
        const std::vector<int> pres = block_prefix(nbs), prer = block_prefix(nbr),
                               pred = block_prefix(nbd);
        Launch ls{K_SCORE};
        ls.off = blob.add(sc);
        ls.off2 = blob.add(pres);
        ls.count = cnt;
        ls.a = maxp;
        ls.b = pres.back();
        ls.x = sharded && !stop_after_score0 ? xp : 0;
        L.push_back(ls);
        if (stop_after_score0) break;
        Launch lse{K_SELECT};
        lse.off = blob.add(se);
        lse.count = cnt;
        L.push_back(lse);
        if (use_cond) {
            Launch lsc{K_SET_COND};
            lsc.a = t;
            L.push_back(lsc);
        }
        if (profile) {
            Launch ev{K_EVENT};
            ev.a = EV_PER_STEP * t + 2;
            L.push_back(ev);
        }
        // re-score passes: double-float pass 1 and 2, then FP64; each is a
        // no-op unless the step's state routes candidates to it (as is the
        // low-part kernel the double-float passes read)
        if (use_cond) {
            Launch lc{K_COND_BEGIN};
            lc.a = t;
            L.push_back(lc);
        }
        if (!zl_cond.empty()) {
            Launch l{K_ZLO};
            l.off = blob.add(zl_cond);
            l.count = (int)zl_cond.size();
            l.a = ctx->num_sms * 4;
            L.push_back(l);
        }
        const std::vector<HpParams> *passes[3] = {&fd1, &fd2, &f64};
        const std::vector<RefineSelectParams> *decides[3] = {&rd1, &rd2, &r64};
        for (int q = 0; q < 3; ++q) {
            if (q < 2 && prec == LINGAM_PREC_FP64) continue;   // no double-float tier there
            Launch lf{K_HP_PASS};
            lf.off = blob.add(*passes[q]);
            lf.count = cnt;
            lf.a = hp_blocks;
            lf.c = q < 2 ? 1 : 2;
            L.push_back(lf);
            Launch lrs{K_REFINE};
            lrs.off = blob.add(*decides[q]);
            lrs.count = cnt;
            lrs.a = maxp;
            L.push_back(lrs);
        }
        if (use_cond) L.push_back(Launch{K_COND_END});
        if (profile) {
            Launch ev{K_EVENT};
            ev.a = EV_PER_STEP * t + 3;
            L.push_back(ev);
        }
        Launch lr{K_REGRESS};
        lr.off = blob.add(rg);
        lr.off2 = blob.add(prer);
        lr.count = cnt;
        lr.a = prer.back();
        L.push_back(lr);
        Launch ld{K_DOWNDATE};
        ld.off = blob.add(dd);
        ld.off2 = blob.add(pred);
        ld.count = cnt;
        ld.a = pred.back();
        L.push_back(ld);
        if (profile) {
            Launch ev{K_EVENT};
            ev.a = EV_PER_STEP * t + 4;
            L.push_back(ev);
        }
    }
    if (!stop_after_score0) {
        std::vector<FinishParams> fp(K);
        for (int k = 0; k < K; ++k) {
            InstDev &I = pl.inst[k];
            const int d = (int)I.d;
            fp[k] = FinishParams{((d - 1) & 1) ? I.U1 : I.U0, I.order, d,
                                 I.hist ? I.hist + (size_t)(d - 1) * d : nullptr};
        }
        Launch lf{K_FINISH};
        lf.off = blob.add(fp);
        lf.count = K;
        L.push_back(lf);
    }
    CK(ensure(pl.params, blob.bytes.size()));
    CK(cudaMemcpy(pl.params.p, blob.bytes.data(), blob.bytes.size(), cudaMemcpyHostToDevice));
    char *pb = reinterpret_cast<char *>(pl.params.p);

    if (sharded && !stop_after_score0) {
        // a sharded call runs the launches in order and exchanges the partial
        // scores after each sharded score launch (run_plan), so no graph
        if (pl.exec) cudaGraphExecDestroy(pl.exec);
        pl.exec = nullptr;
        pl.eager = L;
        pl.nodes = 0;
        for (const Launch &l : L)
            pl.nodes += (l.kind == K_EVENT || l.kind == K_FORK || l.kind == K_JOIN ||
                         l.kind == K_COND_BEGIN || l.kind == K_COND_END)
                            ? 0
                            : (l.kind == K_GRAM_TC ? 3 : 1);
        pl.profile = profile ? 1 : 0;
        pl.partial = false;
        return LINGAM_OK;
    }
    if (use_cond && !ctx->sbody) CK(cudaStreamCreateWithFlags(&ctx->sbody, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    int nodes = 0, cnodes = 0, bodies = 0;
    cudaError_t e = cudaSuccess;
    cudaStream_t cur = s;   // the body of a conditional node is captured on sbody
    for (const Launch &l : L) {
        if (l.kind == K_COND_BEGIN) {
            e = begin_cond_body(s, ctx->sbody, &hconds[l.a]);
            if (e != cudaSuccess) break;
            cur = ctx->sbody;
            ++bodies;
            continue;
        }
        if (l.kind == K_COND_END) {
            cudaGraph_t body = nullptr;
            e = cudaStreamEndCapture(ctx->sbody, &body);
            cur = s;
            if (e != cudaSuccess) break;
            continue;
        }
        const int before = nodes;
        e = issue_launch(pl, l, pb, cur, true, &nodes);
        if (cur != s) cnodes += nodes - before;
        if (e != cudaSuccess) break;
    }
    if (cur != s) {   // a failure inside a body: end that capture too
        cudaGraph_t body = nullptr;
        cudaStreamEndCapture(ctx->sbody, &body);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(s, &g);
    cudaGraphExec_t ex = nullptr;
    if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        cudaGetLastError();
        if (use_cond) {   // no conditional nodes here: capture plain graphs from now on
            ctx->no_cond = true;
            return capture_plan(ctx, stop_after_score0, Iout, epsOut);
        }
        return fail_cuda(ctx, e != cudaSuccess ? e : e2, "graph capture", __LINE__);
    }
    if (use_cond)
        CK(cudaMemcpy(pl.conds.p, hconds.data(), hconds.size() * sizeof(unsigned long long),
                      cudaMemcpyHostToDevice));
    if (pl.exec) cudaGraphExecDestroy(pl.exec);
    pl.exec = ex;
    pl.nodes = nodes;
    pl.cond_nodes = cnodes;
    pl.cond_bodies = bodies;
    pl.profile = profile ? 1 : 0;
    pl.partial = stop_after_score0;
    return LINGAM_OK;
}

// Make ctx->plan match the batch shape (reusing arenas and graph when equal).
static lingam_status ensure_plan(lingam_ctx *ctx, const std::vector<InstSpec> &spec, bool scores,
                                 bool lcoef, bool rows, bool stop_after_score0 = false,
                                 double *Iout = nullptr, double *epsOut = nullptr)
{
    if (ctx->shard_n > 1 && (spec.size() != 1 || scores))
        return fail(ctx, LINGAM_ERR_ARG,
                    "a sharded context orders one instance per call and records no score history");
    Plan &pl = ctx->plan;
    const int prec = ctx->opts.precision;
    if (ctx->prior_d > 0 && !stop_after_score0)
        for (const InstSpec &sp : spec)
            if (sp.d != ctx->prior_d)
                return fail(ctx, LINGAM_ERR_ARG,
                            "prior knowledge is set for d = " + std::to_string(ctx->prior_d) +
                                " but an input has d = " + std::to_string(sp.d));
    const bool same_layout = pl.arena.p && pl.spec == spec && pl.prec == prec &&
                             pl.scores == (int)scores && pl.lcoef == (int)lcoef &&
                             pl.rows == (int)rows;
    ctx->stats.graph_build_ms = 0;
    if (same_layout && pl.exec && !pl.partial && !stop_after_score0 &&
        pl.profile == (ctx->opts.profile ? 1 : 0))
        return LINGAM_OK;
    CK(cudaEventRecord(ctx->g0, ctx->s));
    if (!same_layout) {
        destroy_plan(pl);
        lingam_status st = layout_plan(ctx, pl, spec, prec, scores, lcoef, rows);
        if (st) return st;
    }
    lingam_status st = capture_plan(ctx, stop_after_score0, Iout, epsOut);
    if (st) return st;
    CK(cudaEventRecord(ctx->g1, ctx->s));
    CK(cudaEventSynchronize(ctx->g1));
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->g0, ctx->g1);
    ctx->stats.graph_build_ms = ms;
    return LINGAM_OK;
}

// ---------------------------------------------------------- input side -----

static lingam_status check_args(lingam_ctx *ctx, const void *X, int64_t n, int64_t d, int64_t ld,
                                int layout)
{
    if (!ctx) return LINGAM_ERR_ARG;
    if (!X) return fail(ctx, LINGAM_ERR_ARG, "X is NULL");
    if (d < 1 || n < 2) return fail(ctx, LINGAM_ERR_ARG, "need d >= 1 and n >= 2");
    if (layout != LINGAM_ROW_MAJOR && layout != LINGAM_COL_MAJOR)
        return fail(ctx, LINGAM_ERR_ARG, "layout must be LINGAM_ROW_MAJOR or LINGAM_COL_MAJOR");
    if (layout == LINGAM_ROW_MAJOR && ld < d) return fail(ctx, LINGAM_ERR_ARG, "ld < d");
    if (layout == LINGAM_COL_MAJOR && ld < n) return fail(ctx, LINGAM_ERR_ARG, "ld < n");
    if (d > 6000) return fail(ctx, LINGAM_ERR_ARG, "d > 6000 is not supported");
    if (n > ((int64_t)1 << 30)) return fail(ctx, LINGAM_ERR_ARG, "n > 2^30 is not supported");
    if (d > n) return fail(ctx, LINGAM_ERR_DEGENERATE, "d > n: the covariance is singular");
    return LINGAM_OK;
}

static lingam_status check_perm(lingam_ctx *ctx, const int32_t *order, int64_t d)
{
    std::vector<char> seen((size_t)d, 0);
    for (int64_t k = 0; k < d; ++k) {
        if (order[k] < 0 || order[k] >= d || seen[order[k]])
            return fail(ctx, LINGAM_ERR_ARG, "order is not a permutation of 0..d-1");
        seen[order[k]] = 1;
    }
    return LINGAM_OK;
}

static bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device view of X; host data is copied into ctx->xstage at byte offset *off.
static lingam_status stage(lingam_ctx *ctx, const void *X, size_t bytes, size_t *off,
                           const void **dX)
{
    if (is_device_ptr(X)) {
        *dX = X;
        return LINGAM_OK;
    }
    char *dst = reinterpret_cast<char *>(ctx->xstage.p) + *off;
    CK(cudaMemcpyAsync(dst, X, bytes, cudaMemcpyHostToDevice, ctx->s));
    *dX = dst;
    *off += (size_t)roundup((int64_t)bytes, 256);
    return LINGAM_OK;
}

static size_t matrix_bytes(int64_t n, int64_t d, int64_t ld, int layout, size_t elem)
{
    return (layout == LINGAM_ROW_MAJOR ? (size_t)((n - 1) * ld + d) : (size_t)((d - 1) * ld + n)) *
           elem;
}

static lingam_status begin_call(lingam_ctx *ctx, cudaStream_t user)
{
    CK(cudaSetDevice(ctx->device));
    CK(cudaEventRecord(ctx->e0, user));
    CK(cudaStreamWaitEvent(ctx->s, ctx->e0, 0));
    return LINGAM_OK;
}

static lingam_status end_call(lingam_ctx *ctx, cudaStream_t user)
{
    CK(cudaEventRecord(ctx->e1, ctx->s));
    CK(cudaStreamWaitEvent(user, ctx->e1, 0));
    CK(cudaEventSynchronize(ctx->e1));
    return LINGAM_OK;
}

// Launch the plan graph and read back orders, scores and states.
// A sharded call: the plan's launches in order; after each sharded score
// launch the rank's partial M and E (p + p doubles) go to the caller's
// all-reduce, whose sums every rank then uses identically (select, re-score
// tiers, regress-out and downdate are replicated).  One exchange per step.
static lingam_status run_eager(lingam_ctx *ctx)
{
    Plan &pl = ctx->plan;
    char *pb = reinterpret_cast<char *>(pl.params.p);
    InstDev &I = pl.inst[0];
    int nodes = 0;
    for (const Launch &l : pl.eager) {
        CK(issue_launch(pl, l, pb, ctx->s, false, &nodes));
        if (l.kind != K_SCORE || l.x <= 0) continue;
        const int p = l.x;
        ctx->xbuf.resize((size_t)2 * p);
        CK(cudaMemcpyAsync(ctx->xbuf.data(), I.M, (size_t)p * 8, cudaMemcpyDeviceToHost, ctx->s));
        CK(cudaMemcpyAsync(ctx->xbuf.data() + p, I.E, (size_t)p * 8, cudaMemcpyDeviceToHost,
                           ctx->s));
        CK(cudaStreamSynchronize(ctx->s));
        const int rc = ctx->allreduce(ctx->xbuf.data(), (int64_t)2 * p, ctx->allreduce_user);
        if (rc != 0)
            return fail(ctx, LINGAM_ERR_CUDA,
                        "the all-reduce callback of the sharded ordering failed (returned " +
                            std::to_string(rc) + ")");
        CK(cudaMemcpyAsync(I.M, ctx->xbuf.data(), (size_t)p * 8, cudaMemcpyHostToDevice, ctx->s));
        CK(cudaMemcpyAsync(I.E, ctx->xbuf.data() + p, (size_t)p * 8, cudaMemcpyHostToDevice,
                           ctx->s));
    }
    return LINGAM_OK;
}

static lingam_status run_plan(lingam_ctx *ctx, int32_t *const *orders_out, double *scores_out,
                              std::vector<DevState> &hs)
{
    Plan &pl = ctx->plan;
    const int K = (int)pl.inst.size();
    CK(cudaEventRecord(ctx->g0, ctx->s));
    if (!pl.eager.empty()) {
        lingam_status st = run_eager(ctx);
        if (st) return st;
    } else {
        CK(cudaGraphLaunch(pl.exec, ctx->s));
    }
    CK(cudaEventRecord(ctx->g1, ctx->s));
    for (int k = 0; k < K; ++k)
        if (orders_out && orders_out[k])
            CK(cudaMemcpyAsync(orders_out[k], pl.inst[k].order, (size_t)pl.inst[k].d * 4,
                               cudaMemcpyDeviceToHost, ctx->s));
    if (scores_out && pl.inst[0].hist)
        CK(cudaMemcpyAsync(scores_out, pl.inst[0].hist,
                           (size_t)pl.inst[0].d * pl.inst[0].d * 8, cudaMemcpyDeviceToHost,
                           ctx->s));
    hs.assign(K, DevState{});
    for (int k = 0; k < K; ++k)
        CK(cudaMemcpyAsync(&hs[k], pl.inst[k].state, sizeof(DevState), cudaMemcpyDeviceToHost,
                           ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    float gms = 0;
    cudaEventElapsedTime(&gms, ctx->g0, ctx->g1);
    lingam_stats st{};
    st.graph_build_ms = ctx->stats.graph_build_ms;
    st.total_ms = gms;
    for (auto &h : hs) {
        st.refined_steps += h.refined_steps;
        st.genuine_ties += h.genuine_ties;
        st.candidates_max = std::max(st.candidates_max, h.cand_max);
        st.fp64_candidates += h.fp64_candidates;
        st.df_candidates += h.df_candidates;

    }
    st.graph_nodes = pl.nodes;
    st.cond_nodes = pl.exec ? pl.cond_nodes : 0;
    st.cond_bodies = pl.exec ? pl.cond_bodies : 0;
    if (pl.profile && !pl.pev.empty()) {
        double ph[4] = {0, 0, 0, 0}, units = 0;
        int64_t launches = 0;
        for (size_t t = 0; t < pl.punits.size(); ++t) {
            if (pl.punits[t] <= 0) continue;
            for (int k = 0; k < 4; ++k) {
                float ms = 0;
                if (cudaEventElapsedTime(&ms, pl.pev[EV_PER_STEP * t + k],
                                         pl.pev[EV_PER_STEP * t + k + 1]) == cudaSuccess)
                    ph[k] += ms;
            }
            units += pl.punits[t];
            ++launches;
        }
        cudaGetLastError();
        st.pair_ms = ph[0];
        st.score_ms = ph[1];
        st.refine_ms = ph[2];
        st.regress_ms = ph[3];
        st.pair_launches = launches;
        st.pair_units = units;
    }
    ctx->stats = st;
    return LINGAM_OK;
}

// Fill the single-instance plan from X (validate, stage, pack, centre).
static lingam_status load_single(lingam_ctx *ctx, const void *X, int64_t n, int64_t d, int64_t ld,
                                 int layout)
{
    InstDev &I = ctx->plan.inst[0];
    const int is64 = ctx->opts.precision == LINGAM_PREC_FP64;
    const size_t bytes = matrix_bytes(n, d, ld, layout, is64 ? 8 : 4);
    if (!is_device_ptr(X)) CK(ensure(ctx->xstage, bytes));
    size_t off = 0;
    const void *dX = nullptr;
    lingam_status st = stage(ctx, X, bytes, &off, &dX);
    if (st) return st;
    CK(cudaMemsetAsync(&I.state->status, 0, sizeof(uint32_t), ctx->s));
    if (ctx->gate) CK(launch_gate_wait(ctx->gate, ctx->gate_ns, &I.state->status, ctx->s));
    CK(launch_pack(dX, is64, layout, ld, (int)n, (int)d, I.R, I.ldr, &I.state->status, ctx->s));
    CK(launch_center(I.R, I.ldr, (int)n, (int)d, ctx->s));
    return LINGAM_OK;
}

extern "C" {

lingam_status lingam_create(lingam_ctx **out, int device, const lingam_opts *opts)
{
    if (!out) return LINGAM_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        g_create_error = std::string("no CUDA device: ") + cudaGetErrorString(e);
        return LINGAM_ERR_CUDA;
    }
    if (device < 0 || device >= ndev) {
        g_create_error = "device index out of range";
        return LINGAM_ERR_ARG;
    }
    if (opts && (opts->precision < 0 || opts->precision > LINGAM_PREC_DF)) {
        g_create_error = "precision must be 0, 1, 2 or 3";
        return LINGAM_ERR_ARG;
    }
    lingam_ctx *ctx = new (std::nothrow) lingam_ctx();
    if (!ctx) return LINGAM_ERR_OOM;
    ctx->device = device;
    if (opts) ctx->opts = *opts;
    default_tuning(ctx->tune[0], LINGAM_PREC_FP32);
    default_tuning(ctx->tune[1], LINGAM_PREC_MIXED);
    auto bad = [&](cudaError_t err) {
        g_create_error = std::string("CUDA error during create: ") + cudaGetErrorString(err);
        cudaGetLastError();
        delete ctx;
        return err == cudaErrorMemoryAllocation ? LINGAM_ERR_OOM : LINGAM_ERR_CUDA;
    };
    if ((e = cudaSetDevice(device)) != cudaSuccess) return bad(e);
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess) return bad(e);
    if (prop.major * 10 + prop.minor < 100) {
        g_create_error = "this library is built for sm_103a (Blackwell) GPUs";
        delete ctx;
        return LINGAM_ERR_CUDA;
    }
    ctx->num_sms = prop.multiProcessorCount;
    if ((e = cudaStreamCreateWithFlags(&ctx->s, cudaStreamNonBlocking)) != cudaSuccess) return bad(e);
    cudaEvent_t *evs[] = {&ctx->e0, &ctx->e1, &ctx->g0, &ctx->g1};
    for (cudaEvent_t *ev : evs)
        if ((e = cudaEventCreate(ev)) != cudaSuccess) return bad(e);
    if ((e = pair_kernel_setup()) != cudaSuccess) return bad(e);
    if ((e = gram_tc_setup()) != cudaSuccess) return bad(e);
    if ((e = df_tables_setup()) != cudaSuccess) return bad(e);
    *out = ctx;
    return LINGAM_OK;
}

lingam_status lingam_destroy(lingam_ctx *ctx)
{
    if (!ctx) return LINGAM_OK;
    cudaSetDevice(ctx->device);
    if (ctx->s) cudaStreamSynchronize(ctx->s);
    destroy_plan(ctx->plan);
    Buf *aux[] = {&ctx->xstage, &ctx->aR,   &ctx->aC,   &ctx->aCpart,  &ctx->aL,
                  &ctx->aW,     &ctx->aPiv, &ctx->aM,   &ctx->aBt,     &ctx->aRef,
                  &ctx->aStatus, &ctx->eIn, &ctx->eIn2, &ctx->eL,      &ctx->eW,
                  &ctx->eT,     &ctx->ePos, &ctx->eOrd, &ctx->ePtr,    &ctx->eOut,
                  &ctx->eStatus, &ctx->prior};
    for (Buf *b : aux) release(*b);
    cudaEvent_t evs[] = {ctx->e0, ctx->e1, ctx->g0, ctx->g1, ctx->ev_fork};
    for (cudaEvent_t ev : evs)
        if (ev) cudaEventDestroy(ev);
    for (int k = 0; k < GRAM_STREAMS; ++k) {
        if (ctx->ev_side[k]) cudaEventDestroy(ctx->ev_side[k]);
        if (ctx->side[k]) cudaStreamDestroy(ctx->side[k]);
    }
    if (ctx->sbody) cudaStreamDestroy(ctx->sbody);
    if (ctx->s) cudaStreamDestroy(ctx->s);
    delete ctx;
    return LINGAM_OK;
}

const char *lingam_last_error(const lingam_ctx *ctx)
{
    if (!ctx) return g_create_error.c_str();
    return ctx->err.c_str();
}

lingam_status lingam_set_precision(lingam_ctx *ctx, int32_t precision)
{
    if (!ctx) return LINGAM_ERR_ARG;
    if (precision < 0 || precision > LINGAM_PREC_DF) return fail(ctx, LINGAM_ERR_ARG, "bad precision");
    ctx->opts.precision = precision;
    return LINGAM_OK;
}

lingam_status lingam_causal_order(lingam_ctx *ctx, const void *X, int64_t n, int64_t d, int64_t ld,
                                  int32_t layout, int32_t *order_out, double *scores_out,
                                  lingam_stream_t stream)
{
    if (!ctx) return LINGAM_ERR_ARG;
    ctx->err.clear();
    if (!order_out) return fail(ctx, LINGAM_ERR_ARG, "order_out is NULL");
    lingam_status st = check_args(ctx, X, n, d, ld, layout);
    if (st) return st;
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    if ((st = begin_call(ctx, user))) return st;
    std::vector<InstSpec> spec{{n, d}};
    if ((st = ensure_plan(ctx, spec, scores_out != nullptr, false, false))) return st;
    if ((st = load_single(ctx, X, n, d, ld, layout))) return st;
    std::vector<DevState> hs;
    int32_t *outs[1] = {order_out};
    if ((st = run_plan(ctx, outs, scores_out, hs))) return st;
    if ((st = end_call(ctx, user))) return st;
    return status_to_code(ctx, hs[0].status);
}

lingam_status lingam_step_measures(lingam_ctx *ctx, const void *X, int64_t n, int64_t d,
                                   int64_t ld, int32_t layout, double *I_out, double *M_out,
                                   double *eps_out, lingam_stream_t stream)
{
    if (!ctx) return LINGAM_ERR_ARG;
    ctx->err.clear();
    if (d < 2) return fail(ctx, LINGAM_ERR_ARG, "step measures need d >= 2");
    lingam_status st = check_args(ctx, X, n, d, ld, layout);
    if (st) return st;
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    if ((st = begin_call(ctx, user))) return st;
    CK(ensure(ctx->aW, (size_t)d * d * 8));
    CK(ensure(ctx->aL, (size_t)d * d * 8));
    CK(cudaMemsetAsync(ctx->aW.p, 0, (size_t)d * d * 8, ctx->s));
    CK(cudaMemsetAsync(ctx->aL.p, 0, (size_t)d * d * 8, ctx->s));
    std::vector<InstSpec> spec{{n, d}};
    if ((st = ensure_plan(ctx, spec, false, false, false, true, ptr<double>(ctx->aW),
                          ptr<double>(ctx->aL))))
        return st;
    if ((st = load_single(ctx, X, n, d, ld, layout))) return st;
    std::vector<DevState> hs;
    if ((st = run_plan(ctx, nullptr, nullptr, hs))) return st;
    if (I_out) CK(cudaMemcpyAsync(I_out, ctx->aW.p, (size_t)d * d * 8, cudaMemcpyDeviceToHost, ctx->s));
    if (M_out)
        CK(cudaMemcpyAsync(M_out, ctx->plan.inst[0].M, (size_t)d * 8, cudaMemcpyDeviceToHost, ctx->s));
    if (eps_out)
        CK(cudaMemcpyAsync(eps_out, ctx->aL.p, (size_t)d * d * 8, cudaMemcpyDeviceToHost, ctx->s));
    if ((st = end_call(ctx, user))) return st;
    return status_to_code(ctx, hs[0].status);
}

// Least-squares adjacency on `order` into ctx->aW (device, d x d).  With
// keep_cov the covariance before elimination is left in ctx->eIn.
static lingam_status adjacency_core(lingam_ctx *ctx, const void *X, int64_t n, int64_t d,
                                    int64_t ld, int32_t layout, const int32_t *order,
                                    bool keep_cov, uint32_t **status_out)
{
    lingam_status st;
    const int di = (int)d, ni = (int)n;
    const int64_t ldr = roundup(n, 32);
    const int ks = gram_ksplit(ni, di, ctx->num_sms);
    CK(ensure(ctx->aR, (size_t)d * ldr * 8));
    CK(ensure(ctx->aC, (size_t)d * d * 8));
    CK(ensure(ctx->aCpart, (size_t)ks * d * d * 8));
    CK(ensure(ctx->aL, (size_t)d * d * 8));
    CK(ensure(ctx->aW, (size_t)d * d * 8));
    CK(ensure(ctx->aPiv, (size_t)d * 4));
    CK(ensure(ctx->aRef, (size_t)d * 8));
    CK(ensure(ctx->aStatus, 256));
    const size_t bytes = matrix_bytes(n, d, ld, layout, 4);
    if (!is_device_ptr(X)) CK(ensure(ctx->xstage, bytes));
    size_t off = 0;
    const void *dX = nullptr;
    if ((st = stage(ctx, X, bytes, &off, &dX))) return st;
    uint32_t *status = ptr<uint32_t>(ctx->aStatus);
    CK(cudaMemsetAsync(status, 0, 4, ctx->s));
    CK(cudaMemcpyAsync(ctx->aPiv.p, order, (size_t)d * 4, cudaMemcpyHostToDevice, ctx->s));
    CK(launch_pack(dX, 0, layout, ld, ni, di, ptr<double>(ctx->aR), ldr, status, ctx->s));
    CK(launch_center(ptr<double>(ctx->aR), ldr, ni, di, ctx->s));
    CK(launch_gram_f64(ptr<double>(ctx->aR), ldr, ni, di, ptr<double>(ctx->aCpart), ks,
                       ptr<double>(ctx->aC), d, ptr<double>(ctx->aRef), ctx->s));
    if (keep_cov) {
        CK(ensure(ctx->eIn, (size_t)d * d * 8));
        CK(cudaMemcpyAsync(ctx->eIn.p, ctx->aC.p, (size_t)d * d * 8, cudaMemcpyDeviceToDevice,
                           ctx->s));
    }
    for (int t = 0; t + 1 < di; ++t)
        CK(launch_ldl_step(ptr<double>(ctx->aC), d, ptr<int32_t>(ctx->aPiv), t, di,
                           ptr<double>(ctx->aL), d, ctx->s));
    CK(launch_unit_lower_inverse(ptr<double>(ctx->aL), d, ptr<int32_t>(ctx->aPiv), di,
                                 ptr<double>(ctx->aW), d, ctx->s));
    *status_out = status;
    return LINGAM_OK;
}

lingam_status lingam_fit_adjacency(lingam_ctx *ctx, const void *X, int64_t n, int64_t d, int64_t ld,
                                   int32_t layout, const int32_t *order, double *B_out,
                                   int32_t B_on_device, lingam_stream_t stream)
{
    if (!ctx) return LINGAM_ERR_ARG;
    ctx->err.clear();
    if (!order || !B_out) return fail(ctx, LINGAM_ERR_ARG, "order or B_out is NULL");
    lingam_status st = check_args(ctx, X, n, d, ld, layout);
    if (st) return st;
    if ((st = check_perm(ctx, order, d))) return st;
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    if ((st = begin_call(ctx, user))) return st;
    uint32_t *status = nullptr;
    if ((st = adjacency_core(ctx, X, n, d, ld, layout, order, false, &status))) return st;
    CK(cudaMemcpyAsync(B_out, ctx->aW.p, (size_t)d * d * 8,
                       B_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->s));
    uint32_t hst = 0;
    CK(cudaMemcpyAsync(&hst, status, 4, cudaMemcpyDeviceToHost, ctx->s));
    if ((st = end_call(ctx, user))) return st;
    return status_to_code(ctx, hst);
}

lingam_status lingam_prune_adjacency(lingam_ctx *ctx, const void *X, int64_t n, int64_t d,
                                     int64_t ld, int32_t layout, const int32_t *order,
                                     double gamma, int32_t n_lambda, double eps, double *B_out,
                                     int32_t B_on_device, lingam_stream_t stream)
{
    if (!ctx) return LINGAM_ERR_ARG;
    ctx->err.clear();
    if (!order || !B_out) return fail(ctx, LINGAM_ERR_ARG, "order or B_out is NULL");
    if (!(gamma > 0.0) || n_lambda < 2 || n_lambda > 1000 || !(eps > 0.0 && eps < 1.0))
        return fail(ctx, LINGAM_ERR_ARG, "need gamma > 0, 2 <= n_lambda <= 1000, 0 < eps < 1");
    lingam_status st = check_args(ctx, X, n, d, ld, layout);
    if (st) return st;
    if ((st = check_perm(ctx, order, d))) return st;
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    if ((st = begin_call(ctx, user))) return st;
    uint32_t *status = nullptr;
    if ((st = adjacency_core(ctx, X, n, d, ld, layout, order, true, &status))) return st;
    int hblocks = 1;
    size_t wdbl = 0, wint = 0;
    prune_workspace((int)d, ctx->num_sms, &hblocks, &wdbl, &wint);
    CK(ensure(ctx->eL, (size_t)d * d * 8));
    CK(ensure(ctx->eW, wdbl * 8));
    CK(ensure(ctx->ePos, wint * 4));
    CK(ensure(ctx->eT, (size_t)d * d * 8));
    CK(launch_prune(ptr<double>(ctx->eIn), ptr<double>(ctx->aW), ptr<int32_t>(ctx->aPiv), (int)d,
                    (int)n, gamma, n_lambda, eps, hblocks, ptr<double>(ctx->eL),
                    ptr<double>(ctx->eW), ptr<int>(ctx->ePos), ptr<double>(ctx->eT), status,
                    ctx->s));
    CK(cudaMemcpyAsync(B_out, ctx->eT.p, (size_t)d * d * 8,
                       B_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->s));
    uint32_t hst = 0;
    CK(cudaMemcpyAsync(&hst, status, 4, cudaMemcpyDeviceToHost, ctx->s));
    if ((st = end_call(ctx, user))) return st;
    return status_to_code(ctx, hst);
}

lingam_status varlingam_fit(lingam_ctx *ctx, const void *Xt, int64_t T, int64_t d, int64_t ld,
                            int32_t layout, int32_t lags, int32_t *order_out, double *B0_out,
                            double *Btau_out, lingam_stream_t stream)
{
    if (!ctx) return LINGAM_ERR_ARG;
    ctx->err.clear();
    if (!Xt || !order_out) return fail(ctx, LINGAM_ERR_ARG, "Xt or order_out is NULL");
    if (lags < 1 || d < 1) return fail(ctx, LINGAM_ERR_ARG, "need lags >= 1 and d >= 1");
    if (layout != LINGAM_ROW_MAJOR && layout != LINGAM_COL_MAJOR)
        return fail(ctx, LINGAM_ERR_ARG, "bad layout");
    if ((layout == LINGAM_ROW_MAJOR && ld < d) || (layout == LINGAM_COL_MAJOR && ld < T))
        return fail(ctx, LINGAM_ERR_ARG, "ld too small");
    const int64_t n = T - lags, nz = (int64_t)lags * d, q = nz + d;
    if (n <= q) return fail(ctx, LINGAM_ERR_DEGENERATE, "T - lags must exceed lags*d + d");
    if (q > 6000) return fail(ctx, LINGAM_ERR_ARG, "(lags+1)*d > 6000 is not supported");
    if (ctx->opts.precision == LINGAM_PREC_FP64)
        return fail(ctx, LINGAM_ERR_ARG, "varlingam_fit takes FP32 data; use FP32, MIXED or DF");
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    lingam_status st;
    if ((st = begin_call(ctx, user))) return st;
    const int ni = (int)n, di = (int)d, qi = (int)q;
    const int64_t ldr = roundup(n, 32);
    const int ks = gram_ksplit(ni, qi, ctx->num_sms);
    CK(ensure(ctx->aR, (size_t)q * ldr * 8));
    CK(ensure(ctx->aC, (size_t)q * q * 8));
    CK(ensure(ctx->aCpart, (size_t)ks * q * q * 8));
    CK(ensure(ctx->aL, (size_t)q * q * 8));
    CK(ensure(ctx->aW, (size_t)d * d * 8));
    CK(ensure(ctx->aPiv, (size_t)q * 4));
    CK(ensure(ctx->aM, (size_t)nz * d * 8));
    CK(ensure(ctx->aBt, (size_t)lags * d * d * 8));
    CK(ensure(ctx->aRef, (size_t)q * 8));
    CK(ensure(ctx->aStatus, 256));
    std::vector<InstSpec> spec{{n, d}};
    if ((st = ensure_plan(ctx, spec, false, true, false))) return st;
    InstDev &I = ctx->plan.inst[0];
    const size_t bytes = matrix_bytes(T, d, ld, layout, 4);
    if (!is_device_ptr(Xt)) CK(ensure(ctx->xstage, bytes));
    size_t off = 0;
    const void *dX = nullptr;
    if ((st = stage(ctx, Xt, bytes, &off, &dX))) return st;
    uint32_t *status = &I.state->status;
    CK(cudaMemsetAsync(status, 0, 4, ctx->s));
    const float *xf = reinterpret_cast<const float *>(dX);
    double *R = ptr<double>(ctx->aR);
    auto shifted = [&](int64_t shift) {
        return layout == LINGAM_ROW_MAJOR ? (const void *)(xf + shift * ld) : (const void *)(xf + shift);
    };
    // design [x(t-1) .. x(t-lags) | x(t)], t = lags..T-1, one column per variable
    for (int tau = 1; tau <= lags; ++tau)
        CK(launch_pack(shifted(lags - tau), 0, layout, ld, ni, di, R + (int64_t)(tau - 1) * d * ldr,
                       ldr, status, ctx->s));
    CK(launch_pack(shifted(lags), 0, layout, ld, ni, di, R + nz * ldr, ldr, status, ctx->s));
    CK(launch_center(R, ldr, ni, qi, ctx->s));     // centring = the intercept
    CK(launch_gram_f64(R, ldr, ni, qi, ptr<double>(ctx->aCpart), ks, ptr<double>(ctx->aC), q,
                       ptr<double>(ctx->aRef), ctx->s));
    CK(launch_iota_plain(ptr<int32_t>(ctx->aPiv), qi, ctx->s));
    const int nsplit = std::max(1, std::min(ni / 1024, (ctx->num_sms * 4 + qi - 1) / qi));
    for (int t = 0; t < (int)nz; ++t) {
        CK(launch_ldl_step(ptr<double>(ctx->aC), q, ptr<int32_t>(ctx->aPiv), t, qi,
                           ptr<double>(ctx->aL), q, ctx->s));
        CK(launch_regress_cols(R, ldr, ptr<double>(ctx->aL), q, t, qi, ni, nsplit, ctx->s));
    }
    CK(launch_var_coefficients(ptr<double>(ctx->aL), q, (int)nz, di, ptr<double>(ctx->aM), ctx->s));
    // the innovations (columns nz..q-1) are the data of the ordering loop
    CK(cudaMemcpy2DAsync(I.R, I.ldr * 8, R + nz * ldr, ldr * 8, (size_t)n * 8, (size_t)d,
                         cudaMemcpyDeviceToDevice, ctx->s));
    std::vector<DevState> hs;
    int32_t *outs[1] = {order_out};
    if ((st = run_plan(ctx, outs, nullptr, hs))) return st;
    // B0 = I - L^{-1} along the order (L recorded by the regress-out steps)
    CK(launch_unit_lower_inverse(I.lcoef, d, I.order, di, ptr<double>(ctx->aW), d, ctx->s));
    CK(launch_var_transform(ptr<double>(ctx->aW), ptr<double>(ctx->aM), lags, di,
                            ptr<double>(ctx->aBt), ctx->s));
    if (B0_out)
        CK(cudaMemcpyAsync(B0_out, ctx->aW.p, (size_t)d * d * 8, cudaMemcpyDeviceToHost, ctx->s));
    if (Btau_out)
        CK(cudaMemcpyAsync(Btau_out, ctx->aBt.p, (size_t)lags * d * d * 8, cudaMemcpyDeviceToHost,
                           ctx->s));
    uint32_t hst = 0;
    CK(cudaMemcpyAsync(&hst, status, 4, cudaMemcpyDeviceToHost, ctx->s));
    if ((st = end_call(ctx, user))) return st;
    return status_to_code(ctx, hst | hs[0].status);
}

lingam_status lingam_causal_order_batch(lingam_ctx *ctx, const lingam_instance *inst,
                                        int32_t count, int32_t *const *orders_out,
                                        double *const *B_out, int32_t *failed_index,
                                        lingam_stream_t stream)
{
    if (!ctx) return LINGAM_ERR_ARG;
    ctx->err.clear();
    if (failed_index) *failed_index = -1;
    if (!inst || count < 1 || !orders_out)
        return fail(ctx, LINGAM_ERR_ARG, "need instances, count >= 1 and orders_out");
    if (ctx->opts.precision == LINGAM_PREC_FP64)
        return fail(ctx, LINGAM_ERR_ARG, "batched ordering takes FP32 data; use FP32, MIXED or DF");
    bool any_rows = false;
    std::vector<InstSpec> spec(count);
    for (int k = 0; k < count; ++k) {
        const lingam_instance &a = inst[k];
        char msg[160];
        snprintf(msg, sizeof msg, "instance %d: ", k);
        auto bad = [&](lingam_status s, const char *why) {
            if (failed_index) *failed_index = k;
            return fail(ctx, s, std::string(msg) + why);
        };
        if (!a.X || !orders_out[k]) return bad(LINGAM_ERR_ARG, "X or orders_out[k] is NULL");
        if (a.d < 1 || a.n < 2 || a.ld < a.d) return bad(LINGAM_ERR_ARG, "bad n, d or ld");
        if (a.d > 6000) return bad(LINGAM_ERR_ARG, "d > 6000 is not supported");
        if (a.d > a.n) return bad(LINGAM_ERR_DEGENERATE, "d > n");
        if (!a.rows && a.n > a.n_src) return bad(LINGAM_ERR_ARG, "n > n_src without rows");
        if (a.rows) {
            any_rows = true;
            for (int64_t s = 0; s < a.n; ++s)
                if (a.rows[s] < 0 || a.rows[s] >= a.n_src)
                    return bad(LINGAM_ERR_ARG, "row index out of range");
        }
        spec[k] = InstSpec{a.n, a.d};
    }
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    lingam_status st;
    if ((st = begin_call(ctx, user))) return st;
    if ((st = ensure_plan(ctx, spec, false, B_out != nullptr, any_rows))) return st;
    // stage every distinct host source once
    std::map<const void *, size_t> seen;
    size_t need = 0;
    for (int k = 0; k < count; ++k)
        if (!is_device_ptr(inst[k].X) && !seen.count(inst[k].X)) {
            seen[inst[k].X] = 0;
            need += (size_t)roundup((int64_t)matrix_bytes(inst[k].n_src, inst[k].d, inst[k].ld,
                                                          LINGAM_ROW_MAJOR, 4),
                                    256);
        }
    if (need) CK(ensure(ctx->xstage, need));
    std::map<const void *, const void *> dev;
    size_t off = 0;
    for (int k = 0; k < count; ++k) {
        const lingam_instance &a = inst[k];
        if (!dev.count(a.X)) {
            const void *dX = nullptr;
            if ((st = stage(ctx, a.X, matrix_bytes(a.n_src, a.d, a.ld, LINGAM_ROW_MAJOR, 4), &off,
                            &dX)))
                return st;
            dev[a.X] = dX;
        }
        InstDev &I = ctx->plan.inst[k];
        CK(cudaMemsetAsync(&I.state->status, 0, sizeof(uint32_t), ctx->s));
        const int32_t *rows = nullptr;
        if (a.rows) {
            CK(cudaMemcpyAsync(I.rows, a.rows, (size_t)a.n * 4, cudaMemcpyHostToDevice, ctx->s));
            rows = I.rows;
        }
        CK(launch_pack_gather((const float *)dev[a.X], a.ld, rows, (int)a.n, (int)a.d, I.R, I.ldr,
                              &I.state->status, ctx->s));
        CK(launch_center(I.R, I.ldr, (int)a.n, (int)a.d, ctx->s));
    }
    std::vector<DevState> hs;
    if ((st = run_plan(ctx, orders_out, nullptr, hs))) return st;
    if (B_out) {
        for (int k = 0; k < count; ++k) {
            if (!B_out[k]) continue;
            InstDev &I = ctx->plan.inst[k];
            CK(ensure(ctx->aW, (size_t)I.d * I.d * 8));
            CK(launch_unit_lower_inverse(I.lcoef, I.d, I.order, (int)I.d, ptr<double>(ctx->aW),
                                         I.d, ctx->s));
            CK(cudaMemcpyAsync(B_out[k], ctx->aW.p, (size_t)I.d * I.d * 8, cudaMemcpyDeviceToHost,
                               ctx->s));
        }
    }
    if ((st = end_call(ctx, user))) return st;
    for (int k = 0; k < count; ++k) {
        lingam_status sk = status_to_code(ctx, hs[k].status);
        if (sk) {
            if (failed_index) *failed_index = k;
            char msg[64];
            snprintf(msg, sizeof msg, "instance %d: ", k);
            ctx->err = msg + ctx->err;
            return sk;
        }
    }
    return LINGAM_OK;
}

lingam_status lingam_get_stats(const lingam_ctx *ctx, lingam_stats *out)
{
    if (!ctx || !out) return LINGAM_ERR_ARG;
    *out = ctx->stats;
    return LINGAM_OK;
}

// ------------------------------------------------ graph read-outs (Sec. 4.2)

// Device copy of a caller matrix of `bytes` (used in place when it already
// lives on the device).
static lingam_status device_view(lingam_ctx *ctx, const void *src, size_t bytes, Buf &stage,
                                 const void **out)
{
    if (is_device_ptr(src)) {
        *out = src;
        return LINGAM_OK;
    }
    CK(ensure(stage, bytes));
    CK(cudaMemcpyAsync(stage.p, src, bytes, cudaMemcpyHostToDevice, ctx->s));
    *out = stage.p;
    return LINGAM_OK;
}

// T = (I - B)^-1 for B strictly lower triangular in the device order dOrd.
static lingam_status effects_core(lingam_ctx *ctx, const double *dB, const int32_t *dOrd, int q,
                                  double *T_out, int on_device, uint32_t *status)
{
    CK(ensure(ctx->eL, (size_t)q * q * 8));
    CK(ensure(ctx->eW, (size_t)q * q * 8));
    CK(ensure(ctx->eT, (size_t)q * q * 8));
    CK(ensure(ctx->ePos, (size_t)q * 4));
    CK(launch_total_effects_prep(dB, dOrd, q, ptr<int32_t>(ctx->ePos), ptr<double>(ctx->eL), status,
                                 ctx->s));
    CK(launch_unit_lower_inverse(ptr<double>(ctx->eL), q, dOrd, q, ptr<double>(ctx->eW), q, ctx->s));
    CK(launch_identity_minus(ptr<double>(ctx->eW), q, ptr<double>(ctx->eT), ctx->s));
    if (T_out)
        CK(cudaMemcpyAsync(T_out, ctx->eT.p, (size_t)q * q * 8,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->s));
    return LINGAM_OK;
}

lingam_status lingam_total_effects(lingam_ctx *ctx, const double *B, int64_t d,
                                   const int32_t *order, double *T_out, int32_t T_on_device,
                                   lingam_stream_t stream)
{
    if (!ctx) return LINGAM_ERR_ARG;
    ctx->err.clear();
    if (!B || !order || !T_out) return fail(ctx, LINGAM_ERR_ARG, "B, order or T_out is NULL");
    if (d < 1 || d > 12000) return fail(ctx, LINGAM_ERR_ARG, "need 1 <= d <= 12000");
    lingam_status st = check_perm(ctx, order, d);
    if (st) return st;
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    if ((st = begin_call(ctx, user))) return st;
    CK(ensure(ctx->eStatus, 256));
    CK(ensure(ctx->eOrd, (size_t)d * 4));
    uint32_t *status = ptr<uint32_t>(ctx->eStatus);
    CK(cudaMemsetAsync(status, 0, 4, ctx->s));
    CK(cudaMemcpyAsync(ctx->eOrd.p, order, (size_t)d * 4, cudaMemcpyHostToDevice, ctx->s));
    const void *dB = nullptr;
    if ((st = device_view(ctx, B, (size_t)d * d * 8, ctx->eIn, &dB))) return st;
    if ((st = effects_core(ctx, (const double *)dB, ptr<int32_t>(ctx->eOrd), (int)d, T_out,
                           T_on_device, status)))
        return st;
    uint32_t hst = 0;
    CK(cudaMemcpyAsync(&hst, status, 4, cudaMemcpyDeviceToHost, ctx->s));
    if ((st = end_call(ctx, user))) return st;
    if (hst & ST_ARG) return fail(ctx, LINGAM_ERR_ARG, "B has an edge that does not follow order");
    return status_to_code(ctx, hst);
}

lingam_status varlingam_total_effects(lingam_ctx *ctx, const double *B0, const double *Btau,
                                      int64_t d, int32_t lags, const int32_t *order, double *T_out,
                                      int32_t T_on_device, lingam_stream_t stream)
{
    if (!ctx) return LINGAM_ERR_ARG;
    ctx->err.clear();
    if (!B0 || !Btau || !order || !T_out)
        return fail(ctx, LINGAM_ERR_ARG, "B0, Btau, order or T_out is NULL");
    if (d < 1 || lags < 1 || (lags + 1) * d > 12000)
        return fail(ctx, LINGAM_ERR_ARG, "need d >= 1, lags >= 1, (lags+1)*d <= 12000");
    lingam_status st = check_perm(ctx, order, d);
    if (st) return st;
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    if ((st = begin_call(ctx, user))) return st;
    const int q = (int)((lags + 1) * d);
    CK(ensure(ctx->eStatus, 256));
    CK(ensure(ctx->ePtr, (size_t)d * 4));
    CK(ensure(ctx->eOrd, (size_t)q * 4));
    CK(ensure(ctx->eOut, (size_t)q * q * 8));
    uint32_t *status = ptr<uint32_t>(ctx->eStatus);
    CK(cudaMemsetAsync(status, 0, 4, ctx->s));
    CK(cudaMemcpyAsync(ctx->ePtr.p, order, (size_t)d * 4, cudaMemcpyHostToDevice, ctx->s));
    const void *d0 = nullptr, *dt = nullptr;
    if ((st = device_view(ctx, B0, (size_t)d * d * 8, ctx->eIn, &d0))) return st;
    if ((st = device_view(ctx, Btau, (size_t)lags * d * d * 8, ctx->eIn2, &dt))) return st;
    CK(launch_var_window((const double *)d0, (const double *)dt, (int)d, lags,
                         ptr<int32_t>(ctx->ePtr), ptr<double>(ctx->eOut), ptr<int32_t>(ctx->eOrd),
                         ctx->s));
    if ((st = effects_core(ctx, ptr<double>(ctx->eOut), ptr<int32_t>(ctx->eOrd), q, T_out,
                           T_on_device, status)))
        return st;
    uint32_t hst = 0;
    CK(cudaMemcpyAsync(&hst, status, 4, cudaMemcpyDeviceToHost, ctx->s));
    if ((st = end_call(ctx, user))) return st;
    if (hst & ST_ARG) return fail(ctx, LINGAM_ERR_ARG, "B0 has an edge that does not follow order");
    return status_to_code(ctx, hst);
}

lingam_status lingam_influence(lingam_ctx *ctx, const double *T, int64_t q, double *exert_out,
                               double *receive_out, int32_t *exert_rank_out,
                               int32_t *receive_rank_out, lingam_stream_t stream)
{
    if (!ctx) return LINGAM_ERR_ARG;
    ctx->err.clear();
    if (!T) return fail(ctx, LINGAM_ERR_ARG, "T is NULL");
    if (q < 1 || q > 12000) return fail(ctx, LINGAM_ERR_ARG, "need 1 <= q <= 12000");
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    lingam_status st;
    if ((st = begin_call(ctx, user))) return st;
    CK(ensure(ctx->eOut, (size_t)q * 16 + 64));
    CK(ensure(ctx->ePos, (size_t)q * 8 + 64));
    const void *dT = nullptr;
    if ((st = device_view(ctx, T, (size_t)q * q * 8, ctx->eIn, &dT))) return st;
    double *ex = ptr<double>(ctx->eOut), *rc = ex + q;
    int32_t *rex = ptr<int32_t>(ctx->ePos), *rrc = rex + q;
    CK(launch_influence((const double *)dT, (int)q, ex, rc, rex, rrc, ctx->s));
    if (exert_out) CK(cudaMemcpyAsync(exert_out, ex, q * 8, cudaMemcpyDeviceToHost, ctx->s));
    if (receive_out) CK(cudaMemcpyAsync(receive_out, rc, q * 8, cudaMemcpyDeviceToHost, ctx->s));
    if (exert_rank_out)
        CK(cudaMemcpyAsync(exert_rank_out, rex, q * 4, cudaMemcpyDeviceToHost, ctx->s));
    if (receive_rank_out)
        CK(cudaMemcpyAsync(receive_rank_out, rrc, q * 4, cudaMemcpyDeviceToHost, ctx->s));
    return end_call(ctx, user);
}

lingam_status lingam_bootstrap_edge_stats(lingam_ctx *ctx, const double *const *B, int32_t count,
                                          int64_t d, double threshold, double *prob_out,
                                          double *mean_out, lingam_stream_t stream)
{
    if (!ctx) return LINGAM_ERR_ARG;
    ctx->err.clear();
    if (!B || count < 1 || !prob_out || !mean_out)
        return fail(ctx, LINGAM_ERR_ARG, "need B, count >= 1, prob_out and mean_out");
    if (d < 1 || d > 12000) return fail(ctx, LINGAM_ERR_ARG, "need 1 <= d <= 12000");
    if (!(threshold >= 0.0)) return fail(ctx, LINGAM_ERR_ARG, "threshold must be >= 0");
    for (int k = 0; k < count; ++k)
        if (!B[k]) return fail(ctx, LINGAM_ERR_ARG, "a B pointer is NULL");
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    lingam_status st;
    if ((st = begin_call(ctx, user))) return st;
    const size_t mat = (size_t)d * d * 8;
    std::vector<const double *> dptr(count);
    size_t host_mats = 0;
    for (int k = 0; k < count; ++k) host_mats += is_device_ptr(B[k]) ? 0 : 1;
    CK(ensure(ctx->eIn, std::max<size_t>(host_mats * mat, 256)));
    size_t h = 0;
    for (int k = 0; k < count; ++k) {
        if (is_device_ptr(B[k])) {
            dptr[k] = B[k];
        } else {
            char *dst = reinterpret_cast<char *>(ctx->eIn.p) + h * mat;
            CK(cudaMemcpyAsync(dst, B[k], mat, cudaMemcpyHostToDevice, ctx->s));
            dptr[k] = reinterpret_cast<const double *>(dst);
            ++h;
        }
    }
    CK(ensure(ctx->ePtr, (size_t)count * sizeof(void *)));
    CK(ensure(ctx->eOut, 2 * mat));
    CK(ensure(ctx->eStatus, 256));
    uint32_t *status = ptr<uint32_t>(ctx->eStatus);
    CK(cudaMemsetAsync(status, 0, 4, ctx->s));
    CK(cudaMemcpyAsync(ctx->ePtr.p, dptr.data(), (size_t)count * sizeof(void *),
                       cudaMemcpyHostToDevice, ctx->s));
    double *prob = ptr<double>(ctx->eOut), *mean = prob + (size_t)d * d;
    CK(launch_edge_stats(reinterpret_cast<const double *const *>(ctx->ePtr.p), count, (int)d,
                         threshold, prob, mean, status, ctx->s));
    CK(cudaMemcpyAsync(prob_out, prob, mat, cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaMemcpyAsync(mean_out, mean, mat, cudaMemcpyDeviceToHost, ctx->s));
    uint32_t hst = 0;
    CK(cudaMemcpyAsync(&hst, status, 4, cudaMemcpyDeviceToHost, ctx->s));
    if ((st = end_call(ctx, user))) return st;
    return status_to_code(ctx, hst);
}

static lingam_status check_tuning(lingam_ctx *ctx, const lingam_tuning &t)
{
    if (t.precision != LINGAM_PREC_FP32 && t.precision != LINGAM_PREC_MIXED)
        return fail(ctx, LINGAM_ERR_ARG, "tuning tables exist for the FP32 and MIXED forms only");
    if (t.count < 1 || t.count > 8) return fail(ctx, LINGAM_ERR_ARG, "tuning count must be 1..8");
    for (int b = 0; b < t.count; ++b) {
        if (t.tile[b] < 0 || t.tile[b] >= PAIR_NCFG)
            return fail(ctx, LINGAM_ERR_ARG, "tuning tile index out of range");
        if (t.ctas_per_sm[b] < 1 || t.ctas_per_sm[b] > 64)
            return fail(ctx, LINGAM_ERR_ARG, "tuning ctas_per_sm must be 1..64");
        if (b > 0 && t.p_max[b] <= t.p_max[b - 1])
            return fail(ctx, LINGAM_ERR_ARG, "tuning p_max must ascend");
    }
    return LINGAM_OK;
}

lingam_status lingam_set_tuning(lingam_ctx *ctx, const lingam_tuning *t)
{
    if (!ctx || !t) return LINGAM_ERR_ARG;
    ctx->err.clear();
    lingam_status st = check_tuning(ctx, *t);
    if (st) return st;
    CK(cudaSetDevice(ctx->device));
    ctx->tune[t->precision == LINGAM_PREC_MIXED ? 1 : 0] = *t;
    destroy_plan(ctx->plan);
    return LINGAM_OK;
}

lingam_status lingam_get_tuning(const lingam_ctx *ctx, int32_t precision, lingam_tuning *out)
{
    if (!ctx || !out) return LINGAM_ERR_ARG;
    if (precision != LINGAM_PREC_FP32 && precision != LINGAM_PREC_MIXED) return LINGAM_ERR_ARG;
    *out = ctx->tune[precision == LINGAM_PREC_MIXED ? 1 : 0];
    return LINGAM_OK;
}

lingam_status lingam_set_prior_knowledge(lingam_ctx *ctx, const int8_t *prior, int64_t d)
{
    if (!ctx) return LINGAM_ERR_ARG;
    if (!prior || d == 0) {
        ctx->prior_d = 0;
    } else {
        if (d < 1 || d > 6000) return fail(ctx, LINGAM_ERR_ARG, "prior knowledge: need 1 <= d <= 6000");
        for (int64_t k = 0; k < d * d; ++k)
            if (prior[k] < -1 || prior[k] > 1)
                return fail(ctx, LINGAM_ERR_ARG, "prior knowledge entries must be -1, 0 or 1");
        CK(cudaSetDevice(ctx->device));
        CK(ensure(ctx->prior, (size_t)(d * d)));
        CK(cudaMemcpyAsync(ctx->prior.p, prior, (size_t)(d * d), cudaMemcpyHostToDevice, ctx->s));
        CK(cudaStreamSynchronize(ctx->s));
        ctx->prior_d = d;
    }
    // the step graph holds the selection's parameters: capture it again
    if (ctx->plan.exec) cudaGraphExecDestroy(ctx->plan.exec);
    ctx->plan.exec = nullptr;
    return LINGAM_OK;
}

static_assert(PAIR_NCFG == LINGAM_PAIR_TILES, "the C ABI announces every configuration");

lingam_status lingam_set_shard(lingam_ctx *ctx, int32_t rank, int32_t nranks,
                               lingam_allreduce_fn allreduce, void *user)
{
    if (!ctx) return LINGAM_ERR_ARG;
    ctx->err.clear();
    if (nranks < 1 || rank < 0 || rank >= nranks)
        return fail(ctx, LINGAM_ERR_ARG, "need 0 <= rank < nranks");
    if (nranks > 1 && !allreduce) return fail(ctx, LINGAM_ERR_ARG, "a sharded context needs an all-reduce");
    ctx->shard_rank = nranks > 1 ? rank : 0;
    ctx->shard_n = nranks;
    ctx->allreduce = nranks > 1 ? allreduce : nullptr;
    ctx->allreduce_user = nranks > 1 ? user : nullptr;
    destroy_plan(ctx->plan);   // the graphs depend on the slice
    return LINGAM_OK;
}

int32_t lingam_shard_owner(int64_t i, int64_t j, int64_t p, int32_t nranks)
{
    if (nranks < 1 || p < 1 || p > INT32_MAX || i < 0 || j < 0 || i >= p || j >= p) return -1;
    return shard_owner((int)i, (int)j, (int)p, nranks);
}

lingam_status lingam_set_input_gate(lingam_ctx *ctx, const uint32_t *flag, double timeout_s)
{
    if (!ctx) return LINGAM_ERR_ARG;
    ctx->err.clear();
    if (!flag) {
        ctx->gate = nullptr;
        ctx->gate_ns = 0;
        return LINGAM_OK;
    }
    if (!(timeout_s > 0.0 && timeout_s <= 60.0))
        return fail(ctx, LINGAM_ERR_ARG, "the gate's timeout must be in (0, 60] seconds");
    if ((reinterpret_cast<uintptr_t>(flag) & 3u) != 0)
        return fail(ctx, LINGAM_ERR_ARG, "the gate flag must be 4-byte aligned");
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, flag) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, LINGAM_ERR_ARG, "the gate flag is not memory the device can read");
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged &&
        !(a.type == cudaMemoryTypeHost && a.devicePointer != nullptr))
        return fail(ctx, LINGAM_ERR_ARG,
                    "the gate flag must be device, managed or mapped host memory");
    ctx->gate = a.type == cudaMemoryTypeHost ? reinterpret_cast<const uint32_t *>(a.devicePointer)
                                             : flag;
    ctx->gate_ns = (uint64_t)(timeout_s * 1e9);
    return LINGAM_OK;
}

lingam_status lingam_pair_tile_info(int32_t tile, int32_t *out)
{
    if (!out || tile < 0 || tile >= PAIR_NCFG) return LINGAM_ERR_ARG;
    const PairCfg &G = PAIR_CFGS[tile];
    const int32_t v[9] = {G.wi, G.wj, G.wgi, G.wgj, G.stages, G.groups, G.fold, G.packed, G.sub};
    for (int k = 0; k < 9; ++k) out[k] = v[k];
    return LINGAM_OK;
}

// Times one pair-kernel launch of configuration cfg on the synthetic columns
// (minimum of three runs after a warm-up).
// `copies` identical instances in one launch (a batch of that many problems),
// each writing its own moments; the splits aim at the batch's total tiles as
// the plan's do.
static lingam_status time_pair(lingam_ctx *ctx, int mode, int cfg, const CUtensorMap *tI,
                               const CUtensorMap *tJ, PairParams P, int copies,
                               int64_t mom_per_copy, PairParams *dP, int *dprefix,
                               int ctas_target, cudaEvent_t a, cudaEvent_t b, double *ms_out)
{
    const int tiles = pair_tiles(P.p, cfg);
    P.tiles_i = (P.p + PAIR_CFGS[cfg].ti() - 1) / PAIR_CFGS[cfg].ti();
    P.tiles_j = (P.p + PAIR_CFGS[cfg].tj() - 1) / PAIR_CFGS[cfg].tj();
    pair_split((int64_t)tiles * copies, (int64_t)ctx->num_sms * ctas_target, P.nchunks, &P.cps,
               &P.nsplit);
    std::vector<PairParams> ps(copies, P);
    std::vector<int> prefix(copies + 1, 0);
    for (int k = 0; k < copies; ++k) {
        ps[k].mom = P.mom + (size_t)k * mom_per_copy;
        prefix[k + 1] = prefix[k] + tiles * P.nsplit;
    }
    const int total = prefix[copies];
    CK(cudaMemcpyAsync(dP, ps.data(), sizeof(PairParams) * copies, cudaMemcpyHostToDevice, ctx->s));
    CK(cudaMemcpyAsync(dprefix, prefix.data(), sizeof(int) * (copies + 1), cudaMemcpyHostToDevice,
                       ctx->s));
    CK(launch_pair_b(mode, cfg, tI, tJ, dP, dprefix, copies, total, ctx->s));
    double best = 1e30;
    for (int r = 0; r < 3; ++r) {
        CK(cudaEventRecord(a, ctx->s));
        CK(launch_pair_b(mode, cfg, tI, tJ, dP, dprefix, copies, total, ctx->s));
        CK(cudaEventRecord(b, ctx->s));
        CK(cudaEventSynchronize(b));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, a, b));
        best = std::min(best, (double)ms);
    }
    *ms_out = best;
    return LINGAM_OK;
}

lingam_status lingam_autotune(lingam_ctx *ctx, int64_t n, int64_t d, int32_t instances,
                              lingam_tuning *out)
{
    if (!ctx) return LINGAM_ERR_ARG;
    ctx->err.clear();
    const int prec = ctx->opts.precision;
    if (prec != LINGAM_PREC_FP32 && prec != LINGAM_PREC_MIXED)
        return fail(ctx, LINGAM_ERR_ARG, "autotune needs the FP32 or MIXED form");
    if (n < 2 || d < 2 || d > 6000) return fail(ctx, LINGAM_ERR_ARG, "need n >= 2, 2 <= d <= 6000");
    if (instances < 1) return fail(ctx, LINGAM_ERR_ARG, "need instances >= 1");
    CK(cudaSetDevice(ctx->device));
    destroy_plan(ctx->plan);
    const int mode = prec == LINGAM_PREC_MIXED ? PAIR_FAST : PAIR_ACCURATE;
    const int nprobe = (int)std::min<int64_t>(n, 131072);
    lingam_tuning tb{};
    tb.precision = prec;
    tb.n_probe = nprobe;
    // buckets (32, 64], (64, 128], ... up to the one holding d; probes capped at 2048
    for (int edge = 64; tb.count < 8; edge *= 2) {
        const bool last = edge >= d || tb.count == 7;
        tb.p_max[tb.count] = last ? INT32_MAX : edge;
        tb.p_probe[tb.count] = (int)std::min<int64_t>(std::min<int64_t>(edge, d), 2048);
        ++tb.count;
        if (last) break;
    }
    int pmax = 0;
    for (int b = 0; b < tb.count; ++b) pmax = std::max(pmax, tb.p_probe[b]);
    pmax = std::max(pmax, 2);
    const int64_t ldz = roundup(std::max<int64_t>(nprobe, PAIR_S), 64);
    const int nch = pair_nchunks(nprobe);
    // copies of the probe instance per launch: the batch size, within 2 GB of
    // moment output
    int copies = 1;
    int64_t mom_per_copy = 0;
    for (int cp = std::min(instances, 4096); cp >= 1; cp = (cp > 1 ? std::max(1, cp / 2) : 0)) {
        int64_t per = 0;
        for (int b = 0; b < tb.count; ++b)
            for (int c = 0; c < PAIR_NCFG; ++c)
                for (int m = 1; m <= 4; m *= 2) {
                    int cps = 1, ns = 1;
                    pair_split((int64_t)pair_tiles(tb.p_probe[b], c) * cp,
                               (int64_t)ctx->num_sms * pair_ctas_per_sm(mode, c) * m, nch, &cps,
                               &ns);
                    per = std::max<int64_t>(per, (int64_t)ns * tb.p_probe[b] * tb.p_probe[b] * 2);
                }
        copies = cp;
        mom_per_copy = per;
        if ((double)per * cp * sizeof(float2) <= 2.0e9 || cp == 1) break;
    }
    const int64_t mom_elems = mom_per_copy * copies;
    Buf z, C, U, isd, mom, status, dP, dpre;
    auto cleanup = [&]() {
        release(z);
        release(C);
        release(U);
        release(isd);
        release(mom);
        release(status);
        release(dP);
        release(dpre);
    };
    cudaEvent_t a = nullptr, b = nullptr;
    lingam_status st = [&]() -> lingam_status {
        CK(ensure(z, (size_t)pmax * ldz * 4));
        CK(ensure(C, (size_t)pmax * pmax * 8, true));      // rho = 0 for every pair
        CK(ensure(U, (size_t)pmax * 4));
        CK(ensure(isd, (size_t)pmax * 8));
        CK(ensure(mom, (size_t)mom_elems * sizeof(float2)));
        CK(ensure(status, 256, true));
        CK(ensure(dP, sizeof(PairParams) * copies));
        CK(ensure(dpre, sizeof(int) * (copies + 1)));
        CK(launch_fill_test_z(ptr<float>(z), ldz, pmax, nprobe, ctx->s));
        CK(launch_iota_plain(ptr<int32_t>(U), pmax, ctx->s));
        std::vector<double> ones(pmax, 1.0);
        CK(cudaMemcpyAsync(isd.p, ones.data(), pmax * 8, cudaMemcpyHostToDevice, ctx->s));
        CK(cudaStreamSynchronize(ctx->s));
        CUtensorMap tI[PAIR_NCFG], tJ[PAIR_NCFG];
        {
            Plan tmp;
            tmp.ldz = ldz;
            tmp.zrows = pmax;
            tmp.zarena = z;
            lingam_status s2 = make_tensor_maps(ctx, tmp);
            for (int c = 0; c < PAIR_NCFG; ++c) {
                tI[c] = tmp.tmI[c];
                tJ[c] = tmp.tmJ[c];
            }
            tmp.zarena = Buf{};
            if (s2) return s2;
        }
        CK(cudaEventCreate(&a));
        CK(cudaEventCreate(&b));
        for (int bk = 0; bk < tb.count; ++bk) {
            PairParams P{};
            P.C = ptr<double>(C);
            P.ldc = pmax;
            P.U = ptr<int32_t>(U);
            P.p = tb.p_probe[bk];
            P.n = nprobe;
            P.nchunks = nch;
            P.mom = ptr<float2>(mom);
            P.status = ptr<uint32_t>(status);
            P.row0 = 0;
            P.isd = ptr<double>(isd);
            double best = 1e30;
            for (int c = 0; c < PAIR_NCFG; ++c)
                for (int m = 1; m <= 4; m *= 2) {
                    const int target = pair_ctas_per_sm(mode, c) * m;
                    double ms = 0;
                    lingam_status s2 =
                        time_pair(ctx, mode, c, &tI[c], &tJ[c], P, copies, mom_per_copy,
                                  ptr<PairParams>(dP), ptr<int>(dpre), target, a, b, &ms);
                    if (s2) return s2;
                    if (ms < best) {
                        best = ms;
                        tb.tile[bk] = c;
                        tb.ctas_per_sm[bk] = target;
                        tb.ms[bk] = ms;
                    }
                }
        }
        uint32_t hst = 0;
        CK(cudaMemcpy(&hst, status.p, 4, cudaMemcpyDeviceToHost));
        if (hst) return status_to_code(ctx, hst);
        return LINGAM_OK;
    }();
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cleanup();
    if (st) return st;
    ctx->tune[mode == PAIR_FAST ? 1 : 0] = tb;
    if (out) *out = tb;
    return LINGAM_OK;
}

lingam_status lingam_peak_probe(lingam_ctx *ctx, int32_t which, double *ops_per_s,
                                double *sm_clock_mhz)
{
    if (!ctx || !ops_per_s || which < 0 || which > 3) return LINGAM_ERR_ARG;
    ctx->err.clear();
    CK(cudaSetDevice(ctx->device));
    const int blocks = ctx->num_sms * 4, iters = which == 3 ? 2000 : 20000;
    Buf cyc, ns, sink;
    CK(ensure(cyc, blocks * 8));
    CK(ensure(ns, blocks * 8));
    CK(ensure(sink, 64));
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    CK(launch_peak_probe(which, blocks, iters / 10, ptr<unsigned long long>(cyc),
                         ptr<unsigned long long>(ns), ptr<float>(sink), ctx->s));
    CK(cudaEventRecord(a, ctx->s));
    CK(launch_peak_probe(which, blocks, iters, ptr<unsigned long long>(cyc),
                         ptr<unsigned long long>(ns), ptr<float>(sink), ctx->s));
    CK(cudaEventRecord(b, ctx->s));
    CK(cudaEventSynchronize(b));
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    std::vector<unsigned long long> hc(blocks), hn(blocks);
    CK(cudaMemcpy(hc.data(), cyc.p, blocks * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hn.data(), ns.p, blocks * 8, cudaMemcpyDeviceToHost));
    double mhz = 0;
    for (int k = 0; k < blocks; ++k) mhz += hn[k] ? (double)hc[k] / (double)hn[k] * 1e3 : 0.0;
    mhz /= blocks;
    const double ops_per_thread = (double)iters * 8 * (which == 0 || which == 3 ? 2.0 : 1.0);
    *ops_per_s = ops_per_thread * blocks * 256 / (ms * 1e-3);
    if (sm_clock_mhz) *sm_clock_mhz = mhz;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    release(cyc);
    release(ns);
    release(sink);
    return LINGAM_OK;
}

}  // extern "C"
