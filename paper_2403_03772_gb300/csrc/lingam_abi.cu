// lingam_abi.cu -- host orchestration and the extern "C" entry points
// declared in include/lingam.h.
//
// One ordering run: pack + centre the data (FP64 columns), FP64 covariance,
// then the d-1 steps of the DirectLiNGAM loop (Sec. 2.2), each running
// Algorithm 1 on the device:
//   pair moments -> score I, M -> select (argmax + near-tie candidates)
//   -> FP64 re-score of candidates (no-op unless >= 2) -> regress-out +
//   standardise + variable moments -> rank-1 covariance downdate.
// p = d - t is known when the loop is captured, which variables remain is
// only known on the device, so the whole loop is captured once per shape into
// one CUDA graph and replayed; the host sees the device only at launch and at
// the final copy of the order.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <new>
#include <cstdio>
#include <cstring>
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

struct PairPlan {
    int tiles_i, tiles_j, nchunks, cps, nsplit;
};

struct Plan {
    int64_t n = -1, d = -1;
    int prec = -1, profile = -1;
    int scores = -1;
    int lcoef = -1;
    void *ws_epoch = nullptr;
    cudaGraphExec_t exec = nullptr;
    int nodes = 0;
};

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

}  // namespace

struct lingam_ctx {
    int device = 0;
    int num_sms = 0;
    lingam_opts opts{};
    std::string err;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;

    // workspace
    int64_t cap_n = 0, cap_d = 0;
    int64_t ldr = 0, ldz = 0;
    Buf xstage, R, z, C, Cpart, mom, hzpart, M, E, hist, U, order, state, ref_var, fmom, fhz,
        lcoef, W, piv, cscratch;
    size_t epoch = 0;
    Plan plan;
    CUtensorMap tmI{}, tmJ{};
    std::vector<cudaEvent_t> pev;
    std::vector<double> punits;
    lingam_stats stats{};
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

// ---------------------------------------------------------------- plans ----

static PairPlan pair_plan(const lingam_ctx *ctx, int p, int n)
{
    PairPlan q;
    q.tiles_i = (p + PAIR_TI - 1) / PAIR_TI;
    q.tiles_j = (p + PAIR_TJ - 1) / PAIR_TJ;
    q.nchunks = (n + PAIR_S - 1) / PAIR_S;
    const int tiles = q.tiles_i * q.tiles_j;
    const int target = ctx->num_sms * 2 * 2;   // two resident CTAs per SM, two waves
    int ns = std::max(1, std::min(q.nchunks, (target + tiles - 1) / tiles));
    q.cps = (q.nchunks + ns - 1) / ns;
    q.nsplit = (q.nchunks + q.cps - 1) / q.cps;
    return q;
}

static int regress_splits(const lingam_ctx *ctx, int cols, int n)
{
    const int target = ctx->num_sms * 4;
    int ns = std::max(1, (target + cols - 1) / std::max(1, cols));
    ns = std::min(ns, std::max(1, n / 1024));
    return ns;
}

static size_t mom_elems(const lingam_ctx *ctx, int64_t n, int64_t d)
{
    size_t mx = (size_t)d * d * 2;
    for (int64_t p = 2; p <= d; ++p) {
        PairPlan q = pair_plan(ctx, (int)p, (int)n);
        mx = std::max(mx, (size_t)q.nsplit * p * p * 2);
    }
    return mx;
}

static lingam_status make_tensor_maps(lingam_ctx *ctx, int64_t n, int64_t d)
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
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)d};
    cuuint64_t strides[1] = {(cuuint64_t)(ctx->ldz * sizeof(float))};
    cuuint32_t elem[2] = {1, 1};
    cuuint32_t boxI[2] = {(cuuint32_t)PAIR_S, (cuuint32_t)PAIR_TI};
    cuuint32_t boxJ[2] = {(cuuint32_t)PAIR_S, (cuuint32_t)PAIR_TJ};
    CUresult r = g_encode(&ctx->tmI, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ctx->z.p, dims, strides,
                          boxI, elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, LINGAM_ERR_CUDA, "tensor map encode failed (rows)");
    r = g_encode(&ctx->tmJ, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ctx->z.p, dims, strides, boxJ, elem,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, LINGAM_ERR_CUDA, "tensor map encode failed (cols)");
    return LINGAM_OK;
}

// Workspace for problems up to (n, d); reallocation invalidates the graph.
static lingam_status ensure_workspace(lingam_ctx *ctx, int64_t n, int64_t d)
{
    const bool grow = n > ctx->cap_n || d > ctx->cap_d;
    const int64_t N = grow ? std::max(n, ctx->cap_n) : ctx->cap_n;
    const int64_t D = grow ? std::max(d, ctx->cap_d) : ctx->cap_d;
    if (grow) {
        ctx->ldr = roundup(N, 32);
        ctx->ldz = roundup(N, 64);
        const int ks = gram_ksplit((int)N, (int)D, ctx->num_sms);
        // free first so that the new sizes fit
        Buf *all[] = {&ctx->R, &ctx->z, &ctx->C, &ctx->Cpart, &ctx->mom, &ctx->hzpart, &ctx->M,
                      &ctx->E, &ctx->hist, &ctx->U, &ctx->order, &ctx->state, &ctx->ref_var,
                      &ctx->fmom, &ctx->fhz, &ctx->lcoef, &ctx->W, &ctx->piv, &ctx->cscratch};
        for (Buf *b : all) release(*b);
        CK(ensure(ctx->R, (size_t)D * ctx->ldr * 8));
        CK(ensure(ctx->z, (size_t)D * ctx->ldz * 4, true));
        CK(ensure(ctx->C, (size_t)D * D * 8));
        CK(ensure(ctx->Cpart, (size_t)std::max(ks, 1) * D * D * 8));
        CK(ensure(ctx->mom, mom_elems(ctx, N, D) * 8));
        CK(ensure(ctx->hzpart, (size_t)regress_splits(ctx, 1, (int)N) * D * 2 * 8));
        CK(ensure(ctx->M, (size_t)D * 8));
        CK(ensure(ctx->E, (size_t)D * 8));
        CK(ensure(ctx->hist, (size_t)D * D * 8));
        CK(ensure(ctx->U, (size_t)2 * D * 4));
        CK(ensure(ctx->order, (size_t)D * 4));
        CK(ensure(ctx->state, sizeof(DevState), true));
        CK(ensure(ctx->ref_var, (size_t)D * 8));
        CK(ensure(ctx->fmom, (size_t)MAXC * D * 4 * 8));
        CK(ensure(ctx->fhz, (size_t)D * 2 * 8));
        CK(ensure(ctx->lcoef, (size_t)D * D * 8));
        CK(ensure(ctx->W, (size_t)D * D * 8));
        CK(ensure(ctx->piv, (size_t)D * 4));
        CK(ensure(ctx->cscratch, (size_t)D * 4));
        ctx->cap_n = N;
        ctx->cap_d = D;
        ctx->epoch++;
        lingam_status st = make_tensor_maps(ctx, N, D);
        if (st) return st;
    }
    return LINGAM_OK;
}

// Device copy of X (staging host input); returns the device pointer.
static lingam_status stage_input(lingam_ctx *ctx, const void *X, int64_t n, int64_t d, int64_t ld,
                                 int layout, size_t elem, const void **dX)
{
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, X);
    if (e != cudaSuccess) {
        cudaGetLastError();
        at.type = cudaMemoryTypeUnregistered;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
        *dX = X;
        return LINGAM_OK;
    }
    const size_t count = layout == LINGAM_ROW_MAJOR ? (size_t)((n - 1) * ld + d)
                                                    : (size_t)((d - 1) * ld + n);
    CK(ensure(ctx->xstage, count * elem));
    CK(cudaMemcpyAsync(ctx->xstage.p, X, count * elem, cudaMemcpyHostToDevice, ctx->s));
    *dX = ctx->xstage.p;
    return LINGAM_OK;
}

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
    if (n > (int64_t)1 << 30) return fail(ctx, LINGAM_ERR_ARG, "n > 2^30 is not supported");
    if (d > n) return fail(ctx, LINGAM_ERR_DEGENERATE, "d > n: the covariance is singular");
    return LINGAM_OK;
}

// Capture the covariance + ordering loop for (n, d) into one graph.
static lingam_status capture_order_graph(lingam_ctx *ctx, int64_t n64, int64_t d64, bool scores,
                                         int stop_after_score0, double *Iout, bool lcoef)
{
    const int n = (int)n64, d = (int)d64;
    const int prec = ctx->opts.precision;
    const bool profile = ctx->opts.profile != 0;
    cudaStream_t s = ctx->s;
    DevState *state = ptr<DevState>(ctx->state);
    uint32_t *status = &state->status;
    int32_t *U0 = ptr<int32_t>(ctx->U), *U1 = U0 + d;
    const int ks = gram_ksplit(n, d, ctx->num_sms);
    const double tie = ctx->opts.tie_scale > 0 ? ctx->opts.tie_scale : 1.0;
    // Bound on |I_fp32 - I_exact| per entry, used to pick the candidates that
    // are re-scored in FP64.  Measured against the FP64 oracle on GB300: max
    // 5.8e-7 (accurate FP32) and 3.4e-7 (fast + compensated) over ~5e4
    // entries; the bound keeps a margin above both.
    const double epsI = prec == LINGAM_PREC_FP64 ? 0.0
                        : prec == LINGAM_PREC_MIXED ? 2.0e-6 * tie
                                                    : 2.5e-6 * tie;
    // Steps with at most P64 remaining variables are scored entirely in FP64:
    // cheap there, and the scores of late steps are small enough that FP32
    // rounding would dominate them.
    const int P64 = 32;
    const int pmode = prec == LINGAM_PREC_MIXED ? PAIR_FAST : PAIR_ACCURATE;
    const double a1 = pmode == PAIR_FAST ? LN2_D : 1.0;
    const double a2 = pmode == PAIR_FAST ? 1.0 / KSC : 1.0;

    if (profile && !stop_after_score0) {
        for (cudaEvent_t e : ctx->pev) cudaEventDestroy(e);
        ctx->pev.assign(2 * (size_t)(d - 1), nullptr);
        for (auto &e : ctx->pev) CK(cudaEventCreate(&e));
        ctx->punits.assign((size_t)(d - 1), 0.0);
    }

    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    auto abort_capture = [&](cudaError_t e, const char *what, int line) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
        return fail_cuda(ctx, e, what, line);
    };
#define CKC(expr)                                                    \
    do {                                                             \
        cudaError_t _e = (expr);                                     \
        if (_e != cudaSuccess) return abort_capture(_e, #expr, __LINE__); \
    } while (0)

    CKC(launch_gram_f64(ptr<double>(ctx->R), ctx->ldr, n, d, ptr<double>(ctx->Cpart), ks,
                        ptr<double>(ctx->C), d, ptr<double>(ctx->ref_var), s));
    CKC(launch_iota(U0, d, state, s));
    {
        RegressParams P{};
        P.R = ptr<double>(ctx->R);
        P.ldr = ctx->ldr;
        P.z = ptr<float>(ctx->z);
        P.ldz = ctx->ldz;
        P.C = ptr<double>(ctx->C);
        P.ldc = d;
        P.U = U0;
        P.Unext = U1;
        P.p = d;
        P.n = n;
        const int ns = regress_splits(ctx, d, n);
        P.sps = (n + ns - 1) / ns;
        P.state = state;
        P.order = ptr<int32_t>(ctx->order);
        P.t = 0;
        P.hzpart = ptr<double>(ctx->hzpart);
        P.ref_var = ptr<double>(ctx->ref_var);
        P.status = status;
        CKC(launch_regress(P, true, (n + P.sps - 1) / P.sps, s));
    }
    int nsplit_hz = regress_splits(ctx, d, n);
    {
        const int sps = (n + nsplit_hz - 1) / nsplit_hz;
        nsplit_hz = (n + sps - 1) / sps;
    }
    int nodes = 3;
    const int last_t = stop_after_score0 ? 0 : d - 2;
    for (int t = 0; t <= last_t && d >= 2; ++t) {
        const int p = d - t;
        int32_t *Uc = (t & 1) ? U1 : U0;
        int32_t *Un = (t & 1) ? U0 : U1;
        double *hist_row = scores ? ptr<double>(ctx->hist) + (size_t)t * d : nullptr;

        ScoreParams S{};
        const bool step64 = prec == LINGAM_PREC_FP64 || p <= P64;
        if (step64) {
            F64Params F{};
            F.R = ptr<double>(ctx->R);
            F.ldr = ctx->ldr;
            F.C = ptr<double>(ctx->C);
            F.ldc = d;
            F.U = Uc;
            F.p = p;
            F.n = n;
            F.mode = 0;
            F.state = state;
            F.mom = ptr<double>(ctx->mom);
            F.hz = ptr<double>(ctx->fhz);
            F.status = status;
            if (profile && !stop_after_score0) CKC(cudaEventRecordWithFlags(ctx->pev[2 * t], s, cudaEventRecordExternal));
            CKC(launch_pairs_f64(F, ctx->num_sms * 8, s));
            if (profile && !stop_after_score0) {
                CKC(cudaEventRecordWithFlags(ctx->pev[2 * t + 1], s, cudaEventRecordExternal));
                ctx->punits[t] = (double)p * (p - 1) * n;
            }
            S.mom = F.mom;
            S.nsplit = 1;
            S.hz = F.hz;
            S.nsplit_hz = 1;
            S.a1 = 1.0;
            S.b1 = -LN2_D;
            S.a2 = 1.0;
        } else {
            PairPlan q = pair_plan(ctx, p, n);
            PairParams P{};
            P.C = ptr<double>(ctx->C);
            P.ldc = d;
            P.U = Uc;
            P.p = p;
            P.n = n;
            P.tiles_i = q.tiles_i;
            P.tiles_j = q.tiles_j;
            P.nchunks = q.nchunks;
            P.cps = q.cps;
            P.nsplit = q.nsplit;
            P.mom = ptr<double>(ctx->mom);
            P.status = status;
            if (profile && !stop_after_score0) CKC(cudaEventRecordWithFlags(ctx->pev[2 * t], s, cudaEventRecordExternal));
            CKC(launch_pair(pmode, &ctx->tmI, &ctx->tmJ, P, s));
            if (profile && !stop_after_score0) {
                CKC(cudaEventRecordWithFlags(ctx->pev[2 * t + 1], s, cudaEventRecordExternal));
                ctx->punits[t] = (double)p * (p - 1) * n;
            }
            S.mom = P.mom;
            S.nsplit = q.nsplit;
            S.hz = ptr<double>(ctx->hzpart);
            S.nsplit_hz = nsplit_hz;
            S.a1 = a1;
            S.b1 = -LN2_D;
            S.a2 = a2;
        }
        S.p = p;
        S.n = n;
        S.ha1 = 1.0;
        S.hb1 = -LN2_D;
        S.ha2 = 1.0;
        S.epsI = step64 ? 0.0 : epsI;
        S.U = Uc;
        S.M = ptr<double>(ctx->M);
        S.E = ptr<double>(ctx->E);
        S.hist = hist_row;
        S.Iout = (stop_after_score0 ? Iout : nullptr);
        CKC(launch_score(S, s));
        if (stop_after_score0) {
            nodes += 2;
            break;
        }

        SelectParams SP{ptr<double>(ctx->M), ptr<double>(ctx->E), Uc, p, state,
                        ptr<int32_t>(ctx->cscratch)};
        CKC(launch_select(SP, s));

        for (int pass = 1; pass <= 2; ++pass) {
            F64Params F{};
            F.R = ptr<double>(ctx->R);
            F.ldr = ctx->ldr;
            F.C = ptr<double>(ctx->C);
            F.ldc = d;
            F.U = Uc;
            F.p = p;
            F.n = n;
            F.mode = 1;
            F.pass = pass;
            F.state = state;
            F.mom = ptr<double>(ctx->fmom);
            F.hz = ptr<double>(ctx->fhz);
            F.status = status;
            CKC(launch_pairs_f64(F, ctx->num_sms * 4, s));
            RefineSelectParams RS{ptr<double>(ctx->fmom), ptr<double>(ctx->fhz), p, n, Uc, state,
                                  hist_row, pass};
            CKC(launch_refine_select(RS, s));
        }

        RegressParams P{};
        P.R = ptr<double>(ctx->R);
        P.ldr = ctx->ldr;
        P.z = ptr<float>(ctx->z);
        P.ldz = ctx->ldz;
        P.C = ptr<double>(ctx->C);
        P.ldc = d;
        P.U = Uc;
        P.Unext = Un;
        P.p = p;
        P.n = n;
        int ns = regress_splits(ctx, p - 1, n);
        P.sps = (n + ns - 1) / ns;
        ns = (n + P.sps - 1) / P.sps;
        P.state = state;
        P.order = ptr<int32_t>(ctx->order);
        P.t = t;
        P.hzpart = ptr<double>(ctx->hzpart);
        P.ref_var = ptr<double>(ctx->ref_var);
        P.lcoef = lcoef ? ptr<double>(ctx->lcoef) : nullptr;
        P.ldl = d;
        P.status = status;
        CKC(launch_regress(P, false, ns, s));
        nsplit_hz = ns;
        CKC(launch_downdate(ptr<double>(ctx->C), d, Uc, p, state, s));
        nodes += 9;
    }
    if (!stop_after_score0) {
        int32_t *Ulast = ((d - 1) & 1) ? U1 : U0;
        double *hist_row = scores ? ptr<double>(ctx->hist) + (size_t)(d - 1) * d : nullptr;
        CKC(launch_finish(Ulast, ptr<int32_t>(ctx->order), d, hist_row, s));
        nodes += 1;
    }
#undef CKC
    cudaGraph_t g = nullptr;
    CK(cudaStreamEndCapture(s, &g));
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    if (ctx->plan.exec) cudaGraphExecDestroy(ctx->plan.exec);
    ctx->plan.exec = ex;
    ctx->plan.nodes = nodes;
    return LINGAM_OK;
}

// Shared front half of every ordering call: validate, stage, pack, centre.
static lingam_status prepare(lingam_ctx *ctx, const void *X, int64_t n, int64_t d, int64_t ld,
                             int layout, cudaStream_t user)
{
    lingam_status st = check_args(ctx, X, n, d, ld, layout);
    if (st) return st;
    CK(cudaSetDevice(ctx->device));
    st = ensure_workspace(ctx, n, d);
    if (st) return st;
    CK(cudaEventRecord(ctx->e0, user));
    CK(cudaStreamWaitEvent(ctx->s, ctx->e0, 0));
    const int is64 = ctx->opts.precision == LINGAM_PREC_FP64;
    const void *dX = nullptr;
    st = stage_input(ctx, X, n, d, ld, layout, is64 ? 8 : 4, &dX);
    if (st) return st;
    DevState *state = ptr<DevState>(ctx->state);
    CK(cudaMemsetAsync(&state->status, 0, sizeof(uint32_t), ctx->s));
    CK(launch_pack(dX, is64, layout, ld, (int)n, (int)d, ptr<double>(ctx->R), ctx->ldr,
                   &state->status, ctx->s));
    CK(launch_center(ptr<double>(ctx->R), ctx->ldr, (int)n, (int)d, ctx->s));
    return LINGAM_OK;
}

static lingam_status finish_call(lingam_ctx *ctx, cudaStream_t user, DevState *hs)
{
    CK(cudaMemcpyAsync(hs, ctx->state.p, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaEventRecord(ctx->e1, ctx->s));
    CK(cudaStreamWaitEvent(user, ctx->e1, 0));
    CK(cudaEventSynchronize(ctx->e1));
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
    if (opts && (opts->precision < 0 || opts->precision > 2)) {
        g_create_error = "precision must be 0, 1 or 2";
        return LINGAM_ERR_ARG;
    }
    lingam_ctx *ctx = new (std::nothrow) lingam_ctx();
    if (!ctx) return LINGAM_ERR_OOM;
    ctx->device = device;
    if (opts) ctx->opts = *opts;
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
    if ((e = cudaEventCreate(&ctx->e0)) != cudaSuccess) return bad(e);
    if ((e = cudaEventCreate(&ctx->e1)) != cudaSuccess) return bad(e);
    if ((e = pair_kernel_setup()) != cudaSuccess) return bad(e);
    *out = ctx;
    return LINGAM_OK;
}

lingam_status lingam_destroy(lingam_ctx *ctx)
{
    if (!ctx) return LINGAM_OK;
    cudaSetDevice(ctx->device);
    if (ctx->s) cudaStreamSynchronize(ctx->s);
    if (ctx->plan.exec) cudaGraphExecDestroy(ctx->plan.exec);
    for (cudaEvent_t e : ctx->pev) cudaEventDestroy(e);
    Buf *all[] = {&ctx->xstage, &ctx->R, &ctx->z, &ctx->C, &ctx->Cpart, &ctx->mom, &ctx->hzpart,
                  &ctx->M, &ctx->E, &ctx->hist, &ctx->U, &ctx->order, &ctx->state, &ctx->ref_var,
                  &ctx->fmom, &ctx->fhz, &ctx->lcoef, &ctx->W, &ctx->piv, &ctx->cscratch};
    for (Buf *b : all) release(*b);
    if (ctx->e0) cudaEventDestroy(ctx->e0);
    if (ctx->e1) cudaEventDestroy(ctx->e1);
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
    if (precision < 0 || precision > 2) return fail(ctx, LINGAM_ERR_ARG, "bad precision");
    ctx->opts.precision = precision;
    return LINGAM_OK;
}

// Run the captured ordering loop on the data already packed in ctx->R
// (columns 0..d-1, centred FP64).  Copies order (and scores) to the host.
static lingam_status run_order(lingam_ctx *ctx, int64_t n, int64_t d, int32_t *order_out,
                               double *scores_out, bool lcoef, cudaStream_t user)
{
    const bool scores = scores_out != nullptr;
    Plan &pl = ctx->plan;
    ctx->stats = lingam_stats{};
    lingam_status st;
    if (!pl.exec || pl.n != n || pl.d != d || pl.prec != ctx->opts.precision ||
        pl.profile != ctx->opts.profile || pl.scores != (int)scores || pl.lcoef != (int)lcoef ||
        pl.ws_epoch != (void *)ctx->epoch) {
        cudaEvent_t a, b;
        CK(cudaEventCreate(&a));
        CK(cudaEventCreate(&b));
        CK(cudaEventRecord(a, ctx->s));
        st = capture_order_graph(ctx, n, d, scores, 0, nullptr, lcoef);
        if (st) return st;
        CK(cudaEventRecord(b, ctx->s));
        CK(cudaEventSynchronize(b));
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        ctx->stats.graph_build_ms = ms;
        pl.n = n;
        pl.d = d;
        pl.prec = ctx->opts.precision;
        pl.profile = ctx->opts.profile;
        pl.scores = (int)scores;
        pl.lcoef = (int)lcoef;
        pl.ws_epoch = (void *)ctx->epoch;
    }
    if (scores) {
        // NaN marks variables already ordered
        std::vector<double> nanrow((size_t)d * d, __builtin_nan(""));
        CK(cudaMemcpyAsync(ctx->hist.p, nanrow.data(), nanrow.size() * 8, cudaMemcpyHostToDevice,
                           ctx->s));
        CK(cudaStreamSynchronize(ctx->s));
    }
    cudaEvent_t g0, g1;
    CK(cudaEventCreate(&g0));
    CK(cudaEventCreate(&g1));
    CK(cudaEventRecord(g0, ctx->s));
    CK(cudaGraphLaunch(pl.exec, ctx->s));
    CK(cudaEventRecord(g1, ctx->s));
    CK(cudaMemcpyAsync(order_out, ctx->order.p, (size_t)d * 4, cudaMemcpyDeviceToHost, ctx->s));
    if (scores)
        CK(cudaMemcpyAsync(scores_out, ctx->hist.p, (size_t)d * d * 8, cudaMemcpyDeviceToHost,
                           ctx->s));
    DevState hs{};
    st = finish_call(ctx, user, &hs);
    if (st) return st;
    float gms = 0;
    cudaEventElapsedTime(&gms, g0, g1);
    cudaEventDestroy(g0);
    cudaEventDestroy(g1);
    ctx->stats.total_ms = gms;
    ctx->stats.refined_steps = hs.refined_steps;
    ctx->stats.genuine_ties = hs.genuine_ties;
    ctx->stats.candidates_max = hs.cand_max;
    ctx->stats.fp64_candidates = hs.fp64_candidates;
    ctx->stats.graph_nodes = pl.nodes;
    if (ctx->opts.profile && !ctx->pev.empty()) {
        double tot = 0, units = 0;
        for (size_t t = 0; t + 1 < (size_t)d; ++t) {
            float ms = 0;
            if (cudaEventElapsedTime(&ms, ctx->pev[2 * t], ctx->pev[2 * t + 1]) == cudaSuccess) {
                tot += ms;
                units += ctx->punits[t];
            }
        }
        cudaGetLastError();
        ctx->stats.pair_ms = tot;
        ctx->stats.pair_launches = d - 1;
        ctx->stats.pair_units = units;
    }
    return status_to_code(ctx, hs.status);
}

lingam_status lingam_causal_order(lingam_ctx *ctx, const void *X, int64_t n, int64_t d, int64_t ld,
                                  int32_t layout, int32_t *order_out, double *scores_out,
                                  lingam_stream_t stream)
{
    if (!ctx) return LINGAM_ERR_ARG;
    ctx->err.clear();
    if (!order_out) return fail(ctx, LINGAM_ERR_ARG, "order_out is NULL");
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    lingam_status st = prepare(ctx, X, n, d, ld, layout, user);
    if (st) return st;
    if (d == 1) {
        DevState hs{};
        st = finish_call(ctx, user, &hs);
        if (st) return st;
        order_out[0] = 0;
        if (scores_out) scores_out[0] = 0.0;
        return status_to_code(ctx, hs.status);
    }
    return run_order(ctx, n, d, order_out, scores_out, false, user);
}

lingam_status lingam_step_measures(lingam_ctx *ctx, const void *X, int64_t n, int64_t d,
                                   int64_t ld, int32_t layout, double *I_out, double *M_out,
                                   lingam_stream_t stream)
{
    if (!ctx) return LINGAM_ERR_ARG;
    ctx->err.clear();
    if (d < 2) return fail(ctx, LINGAM_ERR_ARG, "step measures need d >= 2");
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    lingam_status st = prepare(ctx, X, n, d, ld, layout, user);
    if (st) return st;
    Buf Ib;
    CK(ensure(Ib, (size_t)d * d * 8));
    CK(cudaMemsetAsync(Ib.p, 0, (size_t)d * d * 8, ctx->s));
    // a one-off graph (not cached): covariance, standardise, step-0 scores
    ctx->plan.exec = nullptr;   // force re-capture for the next ordering call
    ctx->plan.n = -1;
    st = capture_order_graph(ctx, n, d, false, 1, ptr<double>(Ib), false);
    if (st) {
        release(Ib);
        return st;
    }
    CK(cudaGraphLaunch(ctx->plan.exec, ctx->s));
    if (I_out) CK(cudaMemcpyAsync(I_out, Ib.p, (size_t)d * d * 8, cudaMemcpyDeviceToHost, ctx->s));
    if (M_out) CK(cudaMemcpyAsync(M_out, ctx->M.p, (size_t)d * 8, cudaMemcpyDeviceToHost, ctx->s));
    DevState hs{};
    st = finish_call(ctx, user, &hs);
    cudaGraphExecDestroy(ctx->plan.exec);
    ctx->plan.exec = nullptr;
    release(Ib);
    if (st) return st;
    return status_to_code(ctx, hs.status);
}

lingam_status lingam_fit_adjacency(lingam_ctx *ctx, const void *X, int64_t n, int64_t d, int64_t ld,
                                   int32_t layout, const int32_t *order, double *B_out,
                                   int32_t B_on_device, lingam_stream_t stream)
{
    if (!ctx) return LINGAM_ERR_ARG;
    ctx->err.clear();
    if (!order || !B_out) return fail(ctx, LINGAM_ERR_ARG, "order or B_out is NULL");
    {
        std::vector<char> seen((size_t)std::max<int64_t>(d, 1), 0);
        for (int64_t k = 0; k < d; ++k) {
            if (order[k] < 0 || order[k] >= d || seen[order[k]])
                return fail(ctx, LINGAM_ERR_ARG, "order is not a permutation of 0..d-1");
            seen[order[k]] = 1;
        }
    }
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    const int32_t prec_save = ctx->opts.precision;
    ctx->opts.precision = LINGAM_PREC_FP32;   // adjacency input is FP32 data
    lingam_status st = prepare(ctx, X, n, d, ld, layout, user);
    ctx->opts.precision = prec_save;
    if (st) return st;
    const int di = (int)d, ni = (int)n;
    CK(ensure(ctx->lcoef, (size_t)d * d * 8));
    CK(ensure(ctx->W, (size_t)d * d * 8));
    CK(ensure(ctx->piv, (size_t)d * 4));
    CK(cudaMemcpyAsync(ctx->piv.p, order, (size_t)d * 4, cudaMemcpyHostToDevice, ctx->s));
    const int ks = gram_ksplit(ni, di, ctx->num_sms);
    CK(launch_gram_f64(ptr<double>(ctx->R), ctx->ldr, ni, di, ptr<double>(ctx->Cpart), ks,
                       ptr<double>(ctx->C), d, ptr<double>(ctx->ref_var), ctx->s));
    CK(cudaMemsetAsync(ctx->lcoef.p, 0, (size_t)d * d * 8, ctx->s));
    for (int t = 0; t + 1 < di; ++t)
        CK(launch_ldl_step(ptr<double>(ctx->C), d, ptr<int32_t>(ctx->piv), t, di,
                           ptr<double>(ctx->lcoef), d, ctx->s));
    CK(launch_unit_lower_inverse(ptr<double>(ctx->lcoef), d, ptr<int32_t>(ctx->piv), di,
                                 ptr<double>(ctx->W), d, ctx->s));
    CK(cudaMemcpyAsync(B_out, ctx->W.p, (size_t)d * d * 8,
                       B_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->s));
    DevState hs{};
    st = finish_call(ctx, user, &hs);
    if (st) return st;
    return status_to_code(ctx, hs.status);
}

lingam_status lingam_get_stats(const lingam_ctx *ctx, lingam_stats *out)
{
    if (!ctx || !out) return LINGAM_ERR_ARG;
    *out = ctx->stats;
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
    // warm-up, then timed
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
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
    CK(cudaSetDevice(ctx->device));
    lingam_status st = ensure_workspace(ctx, n, q);
    if (st) return st;
    CK(cudaEventRecord(ctx->e0, user));
    CK(cudaStreamWaitEvent(ctx->s, ctx->e0, 0));
    const void *dX = nullptr;
    st = stage_input(ctx, Xt, T, d, ld, layout, 4, &dX);
    if (st) return st;
    DevState *state = ptr<DevState>(ctx->state);
    CK(cudaMemsetAsync(&state->status, 0, sizeof(uint32_t), ctx->s));
    const float *xf = reinterpret_cast<const float *>(dX);
    double *R = ptr<double>(ctx->R);
    const int ni = (int)n, di = (int)d, qi = (int)q;
    // design [x(t-1) .. x(t-lags) | x(t)], t = lags..T-1, one column per variable
    auto shifted = [&](int64_t shift) {
        return layout == LINGAM_ROW_MAJOR ? (const void *)(xf + shift * ld) : (const void *)(xf + shift);
    };
    for (int tau = 1; tau <= lags; ++tau)
        CK(launch_pack(shifted(lags - tau), 0, layout, ld, ni, di, R + (int64_t)(tau - 1) * d * ctx->ldr,
                       ctx->ldr, &state->status, ctx->s));
    CK(launch_pack(shifted(lags), 0, layout, ld, ni, di, R + nz * ctx->ldr, ctx->ldr, &state->status,
                   ctx->s));
    CK(launch_center(R, ctx->ldr, ni, qi, ctx->s));     // centring = the intercept
    const int ks = gram_ksplit(ni, qi, ctx->num_sms);
    CK(launch_gram_f64(R, ctx->ldr, ni, qi, ptr<double>(ctx->Cpart), ks, ptr<double>(ctx->C), q,
                       ptr<double>(ctx->ref_var), ctx->s));
    CK(launch_iota_plain(ptr<int32_t>(ctx->piv), qi, ctx->s));
    const int nsplit = regress_splits(ctx, qi / 2, ni);
    for (int t = 0; t < (int)nz; ++t) {
        CK(launch_ldl_step(ptr<double>(ctx->C), q, ptr<int32_t>(ctx->piv), t, qi,
                           ptr<double>(ctx->lcoef), q, ctx->s));
        CK(launch_regress_cols(R, ctx->ldr, ptr<double>(ctx->lcoef), q, t, qi, ni, nsplit, ctx->s));
    }
    Buf Mb, Btb;
    CK(ensure(Mb, (size_t)nz * d * 8));
    CK(launch_var_coefficients(ptr<double>(ctx->lcoef), q, (int)nz, di, ptr<double>(Mb), ctx->s));
    // innovations E (columns nz..q-1) become the data of the ordering loop
    CK(cudaMemcpyAsync(R, R + nz * ctx->ldr, (size_t)d * ctx->ldr * 8, cudaMemcpyDeviceToDevice,
                       ctx->s));
    if (d == 1) {
        order_out[0] = 0;
    } else {
        st = run_order(ctx, n, d, order_out, nullptr, true, user);
        if (st) {
            release(Mb);
            return st;
        }
    }
    // B0 = I - L^{-1} along the order (L recorded by the regress-out steps)
    CK(cudaMemcpyAsync(ctx->piv.p, order_out, (size_t)d * 4, cudaMemcpyHostToDevice, ctx->s));
    CK(launch_unit_lower_inverse(ptr<double>(ctx->lcoef), d, ptr<int32_t>(ctx->piv), di,
                                 ptr<double>(ctx->W), d, ctx->s));
    CK(ensure(Btb, (size_t)lags * d * d * 8));
    CK(launch_var_transform(ptr<double>(ctx->W), ptr<double>(Mb), lags, di, ptr<double>(Btb),
                            ctx->s));
    if (B0_out)
        CK(cudaMemcpyAsync(B0_out, ctx->W.p, (size_t)d * d * 8, cudaMemcpyDeviceToHost, ctx->s));
    if (Btau_out)
        CK(cudaMemcpyAsync(Btau_out, Btb.p, (size_t)lags * d * d * 8, cudaMemcpyDeviceToHost, ctx->s));
    DevState hs{};
    st = finish_call(ctx, user, &hs);
    release(Mb);
    release(Btb);
    if (st) return st;
    return status_to_code(ctx, hs.status);
}

lingam_status lingam_causal_order_batch(lingam_ctx *ctx, const lingam_instance *inst,
                                        int32_t count, int32_t *const *orders_out,
                                        double *const *B_out, int32_t *failed_index,
                                        lingam_stream_t stream)
{
    (void)inst; (void)count; (void)orders_out; (void)B_out; (void)failed_index; (void)stream;
    return fail(ctx, LINGAM_ERR_ARG, "lingam_causal_order_batch: not built yet");
}

}  // extern "C"
