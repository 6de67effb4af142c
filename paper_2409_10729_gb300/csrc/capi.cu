// capi.cu -- host implementation of the C ABI declared in include/mfc.h.
//
// A context owns the device buffers of one problem and a stream.  A step of
// SSP-RK3 is: one step_begin kernel (dt from the device-resident wave speed),
// then for each of the three stages one fused sweep per direction; the last
// sweep of a stage applies the stage update, and the last sweep of stage 3
// reduces the wave speed of the new state.  The launches of one step are
// captured once into a CUDA graph and replayed.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#include "mfc.h"
#include "mfc_internal.cuh"

using namespace mfc5;

namespace {

enum KernelKind { K_STEP_BEGIN = 0, K_SWEEP_X, K_SWEEP_Y, K_SWEEP_Z, K_NKINDS };
const char* kKindNames[K_NKINDS] = {"step_begin", "sweep_x", "sweep_y", "sweep_z"};
constexpr int kMaxTimedLaunches = 16;

}  // namespace

struct mfc_ctx {
    mfc_params p;
    int ndim, neq, form;
    int n[3];
    long long ncell;
    double inv_dx[3];
    double dx[3], rdx[3];
    int periodic[3];
    Eos eos;
    int device;
    cudaStream_t stream;
    cudaStream_t cap_stream;
    double* qn;       // q^n, FP64 conservative
    void* sa;         // stage 1 output (FP64, or FP32 cons + p)
    void* sb;         // stage 2 output
    float* s0;        // mixed form: FP32 copy of q^n with p
    float* dinc;      // FP32 forms: RK increment D_k (q^(k) = q^n + D_k), neq fields
    void* acc;        // RHS accumulator
    double* tmp64;    // mixed form: FP64 RHS output staging (lazy)
    DevCtrl* ctrl;    // device
    DevCtrl* ctrl_h;  // pinned host mirror
    bool have_state;
    cudaGraphExec_t gexec;
    bool graph_ok;
    bool timing;
    cudaEvent_t ev[kMaxTimedLaunches + 1];
    double ktime[K_NKINDS];
    long long kcount[K_NKINDS];
    int last_cuda;
    bool have_gate;
    float* gate_w;     // gated form: network weights (device)
    // non-uniform directions (mfc_set_grid); null where uniform
    void* gtab[3];     // WENO5 tables of cells -1 .. n (FP64, or FP32 for the FP32 forms)
    double* gw[3];     // cell widths
    double* grw[3];    // RN(1/width)
    float* grw32[3];   // 1/width in FP32
    // block of a decomposed grid (mfc_create_block); zero otherwise
    int is_block;
    int blk_lo[3];     // global index of the block's first cell
    int nbr[3][2];     // 1 where side (d, s) borders another block
    long long hoff[6]; // halo layout: element offset of side (d, s) at 2 d + s, -1 if none
    long long htotal;  // halo buffer elements
    const void* halo_cur;  // halo buffer of the call in progress (sweeps read ghosts there)
    signed char* dec_dev;  // gated form: per-direction, per-cell decisions of mfc_gate_rhs (lazy)
    bool dec_on;           // the call in progress records decisions
    // MFC_TMA_YZ builds, FP32 forms: tensor maps of the stage inputs (s0, sa,
    // sb) for the y and z sweeps, tmap[2 b + d] (64-byte aligned host
    // allocation); tma_ok when all were encoded
    CUtensorMap* tmap;
    bool tma_ok;
};

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) {                   \
            ctx->last_cuda = (int)e_;              \
            return MFC_ECUDA;                      \
        }                                          \
    } while (0)

// Largest cell count a context accepts: 2^36 cells, beyond what any device
// holds in any form (the FP64 form alone needs 4 state arrays of neq doubles
// per cell), and small enough that every byte count and index of the library
// fits in 64 bits.
static const long long kMaxCells = 1LL << 36;

static int validate(const mfc_params* p) {
    if (!p || p->ndim < 1 || p->ndim > 3) return MFC_EINVAL;
    for (int d = 0; d < p->ndim; ++d) {
        if (p->n[d] < 1) return MFC_EINVAL;
        if (!(p->hi[d] > p->lo[d]) || !isfinite(p->hi[d] - p->lo[d])) return MFC_EINVAL;
        int b0 = p->bc[d][0], b1 = p->bc[d][1];
        if (b0 < 0 || b0 > 1 || b1 < 0 || b1 > 1 || b0 != b1) return MFC_EINVAL;
    }
    // cell count, checked step by step so that it cannot overflow
    long long ncell = 1;
    for (int d = 0; d < p->ndim; ++d) {
        if (ncell > kMaxCells / p->n[d]) return MFC_ENOMEM;
        ncell *= p->n[d];
    }
    if (p->nfluids != 0 && (p->nfluids < 2 || p->nfluids > MFC_MAX_FLUIDS)) return MFC_EINVAL;
    const int nf = params_nfluids(p->nfluids);
    for (int i = 0; i < nf; ++i)
        if (!(p->gamma[i] > 1.0) || !isfinite(p->gamma[i]) || !(p->pi_inf[i] >= 0.0) || !isfinite(p->pi_inf[i]))
            return MFC_EINVAL;
    if (nf > 2 && p->precision == MFC_GATED) return MFC_EINVAL;
    if (!(p->weno_eps > 0.0) || !isfinite(p->weno_eps)) return MFC_EINVAL;
    if (p->precision != MFC_FP64 && p->precision != MFC_MIXED && p->precision != MFC_FP64_FAST &&
        p->precision != MFC_GATED)
        return MFC_EINVAL;
    if (p->weno_order != 0 && p->weno_order != 3 && p->weno_order != 5) return MFC_EINVAL;
    if (p->weno_order == 3 && p->precision == MFC_GATED) return MFC_EINVAL;
    return MFC_OK;
}

static bool fp32_state(const mfc_ctx* c) { return c->form == FORM_MIXED || c->form == FORM_GATED; }
static size_t state_elem(const mfc_ctx* c) { return fp32_state(c) ? sizeof(float) : sizeof(double); }
static int state_fields(const mfc_ctx* c) { return fp32_state(c) ? c->neq + 1 : c->neq; }

static void free_all(mfc_ctx* c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    void* bufs[] = {c->qn, c->sa, c->sb, c->s0, c->dinc, c->acc, c->tmp64, c->ctrl, c->gate_w, c->dec_dev};
    for (void* b : bufs)
        if (b) cudaFree(b);
    for (int d = 0; d < 3; ++d) {
        void* g[] = {c->gtab[d], c->gw[d], c->grw[d], c->grw32[d]};
        for (void* b : g)
            if (b) cudaFree(b);
    }
    if (c->ctrl_h) cudaFreeHost(c->ctrl_h);
    free(c->tmap);
    for (int i = 0; i <= kMaxTimedLaunches; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
}

// cuTensorMapEncodeTiled, looked up through the runtime (no link against the
// driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = NULL;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* f = NULL;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
        else
            cudaGetLastError();
    }
    return fn;
}

// Tensor maps of an FP32 stage buffer [field][z][y][x] as a 4-D tensor
// (x, y, z, field) with boxes of 32 x-cells by kTmaCells cells along y or z.
// TMA needs 16-byte row strides: nx a multiple of 4.
static void setup_tma(mfc_ctx* ctx) {
    ctx->tma_ok = false;
    if (!MFC_TMA_YZ || !fp32_state(ctx) || ctx->ndim < 2 || ctx->n[0] % 4 != 0) return;
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return;
    ctx->tmap = (CUtensorMap*)aligned_alloc(64, 6 * sizeof(CUtensorMap));
    if (!ctx->tmap) return;
    memset(ctx->tmap, 0, 6 * sizeof(CUtensorMap));
    void* bufs[3] = {ctx->s0, ctx->sa, ctx->sb};
    const cuuint64_t dims[4] = {(cuuint64_t)ctx->n[0], (cuuint64_t)ctx->n[1], (cuuint64_t)ctx->n[2],
                                (cuuint64_t)state_fields(ctx)};
    const cuuint64_t strides[3] = {(cuuint64_t)ctx->n[0] * 4, (cuuint64_t)ctx->n[0] * ctx->n[1] * 4,
                                   (cuuint64_t)ctx->ncell * 4};
    const cuuint32_t ones[4] = {1, 1, 1, 1};
    const cuuint32_t box[2][4] = {{32, kTmaCells, 1, 1}, {32, 1, kTmaCells, 1}};
    for (int b = 0; b < 3; ++b)
        for (int d = 0; d < 2; ++d) {
            if (d == 1 && ctx->ndim < 3) continue;
            if (enc(&ctx->tmap[2 * b + d], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, bufs[b], dims, strides, box[d], ones,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return;
        }
    ctx->tma_ok = true;
}

extern "C" int mfc_create(const mfc_params* params, void* cuda_stream, mfc_ctx** out) {
    if (!out) return MFC_EINVAL;
    *out = NULL;
    int st = validate(params);
    if (st) return st;
    mfc_ctx* ctx = (mfc_ctx*)calloc(1, sizeof(mfc_ctx));
    if (!ctx) return MFC_ENOMEM;
    ctx->p = *params;
    ctx->ndim = params->ndim;
    ctx->neq = 2 * params_nfluids(params->nfluids) + params->ndim;
    switch (params->precision) {
        case MFC_FP64: ctx->form = FORM_FP64_EXACT; break;
        case MFC_FP64_FAST: ctx->form = FORM_FP64_FAST; break;
        case MFC_GATED: ctx->form = FORM_GATED; break;
        default: ctx->form = FORM_MIXED; break;
    }
    ctx->ncell = 1;
    for (int d = 0; d < 3; ++d) {
        ctx->n[d] = d < ctx->ndim ? params->n[d] : 1;
        ctx->ncell *= ctx->n[d];
        ctx->inv_dx[d] = d < ctx->ndim ? (double)ctx->n[d] / (params->hi[d] - params->lo[d]) : 0.0;
        ctx->dx[d] = d < ctx->ndim ? (params->hi[d] - params->lo[d]) / (double)ctx->n[d] : 1.0;
        ctx->rdx[d] = 1.0 / ctx->dx[d];
        ctx->periodic[d] = d < ctx->ndim ? params->bc[d][0] == MFC_BC_PERIODIC : 0;
    }
    ctx->eos = make_eos(params->gamma, params->pi_inf, params_nfluids(params->nfluids));
    ctx->stream = (cudaStream_t)cuda_stream;

    if (cudaGetDevice(&ctx->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        free_all(ctx);
        free(ctx);
        return MFC_ECUDA;
    }
    size_t nc = (size_t)ctx->ncell;
    size_t sfield = state_fields(ctx), selem = state_elem(ctx);
    bool ok = cudaMalloc((void**)&ctx->qn, nc * ctx->neq * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&ctx->sa, nc * sfield * selem) == cudaSuccess &&
              cudaMalloc(&ctx->sb, nc * sfield * selem) == cudaSuccess &&
              cudaMalloc(&ctx->acc, nc * ctx->neq * selem) == cudaSuccess &&
              cudaMalloc((void**)&ctx->ctrl, sizeof(DevCtrl)) == cudaSuccess &&
              cudaMallocHost((void**)&ctx->ctrl_h, sizeof(DevCtrl)) == cudaSuccess;
    if (ok && fp32_state(ctx))
        ok = cudaMalloc((void**)&ctx->s0, nc * sfield * sizeof(float)) == cudaSuccess &&
             cudaMalloc((void**)&ctx->dinc, nc * ctx->neq * sizeof(float)) == cudaSuccess;
    if (ok && ctx->form == FORM_GATED)
        ok = cudaMalloc((void**)&ctx->gate_w, kGateParams * sizeof(float)) == cudaSuccess;
    for (int i = 0; ok && i <= kMaxTimedLaunches; ++i) ok = cudaEventCreate(&ctx->ev[i]) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_all(ctx);
        free(ctx);
        return MFC_ENOMEM;
    }
    setup_tma(ctx);
    memset(ctx->ctrl_h, 0, sizeof(DevCtrl));
    if (cudaMemcpyAsync(ctx->ctrl, ctx->ctrl_h, sizeof(DevCtrl), cudaMemcpyHostToDevice, ctx->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        free_all(ctx);
        free(ctx);
        return MFC_ECUDA;
    }
    *out = ctx;
    return MFC_OK;
}

extern "C" int mfc_destroy(mfc_ctx* ctx) {
    if (!ctx) return MFC_OK;
    cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
    free(ctx);
    return MFC_OK;
}

static SweepArgs base_args(mfc_ctx* ctx) {
    SweepArgs a;
    memset(&a, 0, sizeof(a));
    for (int d = 0; d < 3; ++d) {
        a.n[d] = ctx->n[d];
        a.inv_dx[d] = ctx->inv_dx[d];
        a.dx[d] = ctx->dx[d];
        a.rdx[d] = ctx->rdx[d];
        a.inv_dx32[d] = (float)ctx->inv_dx[d];
    }
    a.ncell = ctx->ncell;
    a.eos = ctx->eos;
    a.eps = ctx->p.weno_eps;
    a.order = ctx->p.weno_order == 3 ? 3 : 5;
    a.ctrl = ctx->ctrl;
    a.acc = ctx->acc;
    a.qn = ctx->qn;
    a.gate_w = ctx->gate_w;
    a.dinc = ctx->dinc;
    for (int d = 0; d < 3; ++d) {
        a.cw[d] = ctx->gw[d];
        a.crw[d] = ctx->grw[d];
        a.crw32[d] = ctx->grw32[d];
    }
    return a;
}

static cudaError_t launch_sweep(mfc_ctx* ctx, int dir, int mode, SweepArgs a, cudaStream_t s) {
    a.periodic = ctx->periodic[dir];
    a.tab = ctx->gtab[dir];
    if (ctx->is_block && ctx->halo_cur) {
        const char* h = static_cast<const char*>(ctx->halo_cur);
        const size_t el = state_elem(ctx);
        if (ctx->nbr[dir][0]) a.hlo = h + ctx->hoff[2 * dir] * el;
        if (ctx->nbr[dir][1]) a.hhi = h + ctx->hoff[2 * dir + 1] * el;
        a.hplane = ctx->ncell / ctx->n[dir];
    }
    if (ctx->dec_on) a.gate_dec = ctx->dec_dev + (long long)dir * ctx->ncell;
    if (ctx->tma_ok && dir >= 1 && !ctx->gtab[dir]) {
        const int bi = a.qin == ctx->s0 ? 0 : (a.qin == ctx->sa ? 1 : (a.qin == ctx->sb ? 2 : -1));
        if (bi >= 0) a.tmap = &ctx->tmap[2 * bi + dir - 1];
    }
    switch (ctx->form) {
        case FORM_FP64_EXACT: return launch_sweep_fp64x(ctx->ndim, dir, mode, a, s);
        case FORM_FP64_FAST: return launch_sweep_fp64(ctx->ndim, dir, mode, a, s);
        case FORM_GATED: return launch_sweep_gated(ctx->ndim, dir, mode, a, s);
        default: return launch_sweep_mixed(ctx->ndim, dir, mode, a, s);
    }
}

// The stage input/output buffers of stage k (1..3).
static void stage_buffers(mfc_ctx* ctx, int k, SweepArgs& a) {
    const void* in0 = fp32_state(ctx) ? (const void*)ctx->s0 : (const void*)ctx->qn;
    a.stage = k;
    a.qin = k == 1 ? in0 : (k == 2 ? ctx->sa : ctx->sb);
    a.qout = k == 1 ? ctx->sa : (k == 2 ? ctx->sb : (void*)ctx->qn);
    a.qout2 = (k == 3 && fp32_state(ctx)) ? (void*)ctx->s0 : NULL;
}

// Enqueue the launches of one step on stream s; with `timed`, bracket each
// launch with events ev[i], ev[i+1] (recorded for later accumulation).
static cudaError_t enqueue_step(mfc_ctx* ctx, cudaStream_t s, bool timed, int* kinds, int* nl) {
    int L = 0;
    cudaError_t e;
    if (timed && (e = cudaEventRecord(ctx->ev[0], s)) != cudaSuccess) return e;
    if ((e = launch_step_begin(ctx->ctrl, s)) != cudaSuccess) return e;
    if (timed) {
        kinds[L++] = K_STEP_BEGIN;
        if ((e = cudaEventRecord(ctx->ev[L], s)) != cudaSuccess) return e;
    }
    for (int k = 1; k <= 3; ++k) {
        SweepArgs a = base_args(ctx);
        stage_buffers(ctx, k, a);
        for (int d = 0; d < ctx->ndim; ++d) {
            int mode = d == ctx->ndim - 1 ? SW_LAST_RK : (d == 0 ? SW_FIRST : SW_MID);
            if ((e = launch_sweep(ctx, d, mode, a, s)) != cudaSuccess) return e;
            if (timed) {
                kinds[L++] = K_SWEEP_X + d;
                if ((e = cudaEventRecord(ctx->ev[L], s)) != cudaSuccess) return e;
            }
        }
    }
    if (nl) *nl = L;
    return cudaSuccess;
}

static int ensure_graph(mfc_ctx* ctx) {
    if (ctx->graph_ok) return MFC_OK;
    // the sweeps' launch shapes come from occupancy queries, made here once
    // rather than inside the capture
    SweepArgs dry = base_args(ctx);
    dry.dry = 1;
    for (int d = 0; d < ctx->ndim; ++d)
        CK(launch_sweep(ctx, d, d == ctx->ndim - 1 ? SW_LAST_RK : (d == 0 ? SW_FIRST : SW_MID), dry, ctx->stream));
    cudaGraph_t g = NULL;
    CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_step(ctx, ctx->cap_stream, false, NULL, NULL);
    cudaError_t e2 = cudaStreamEndCapture(ctx->cap_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        ctx->last_cuda = (int)(e != cudaSuccess ? e : e2);
        cudaGetLastError();
        return MFC_ECUDA;
    }
    e = cudaGraphInstantiate(&ctx->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        ctx->last_cuda = (int)e;
        return MFC_ECUDA;
    }
    ctx->graph_ok = true;
    return MFC_OK;
}

static int after_state_change(mfc_ctx* ctx) {
    if (fp32_state(ctx))
        CK(launch_make_mixed_state(ctx->ndim, ctx->qn, ctx->s0, ctx->ncell, ctx->eos, ctx->stream));
    CK(launch_wavespeed(ctx->ndim, ctx->qn, ctx->n, ctx->gw, ctx->grw, ctx->ncell, ctx->dx, ctx->rdx, ctx->eos,
                        ctx->ctrl, ctx->stream));
    ctx->have_state = true;
    return MFC_OK;
}


extern "C" int mfc_set_state(mfc_ctx* ctx, const double* q, int on_device) {
    if (!ctx || !q) return MFC_EINVAL;
    size_t bytes = (size_t)ctx->ncell * ctx->neq * sizeof(double);
    CK(on_device ? cudaMemcpyAsync(ctx->qn, q, bytes, cudaMemcpyDeviceToDevice, ctx->stream)
                 : host_copy(ctx->qn, q, bytes, true, ctx->stream));
    int st = after_state_change(ctx);
    if (st) return st;
    if (!on_device) CK(cudaStreamSynchronize(ctx->stream));
    return MFC_OK;
}

extern "C" int mfc_set_state_prim(mfc_ctx* ctx, const double* w, int on_device) {
    if (!ctx || !w) return MFC_EINVAL;
    size_t bytes = (size_t)ctx->ncell * ctx->neq * sizeof(double);
    CK(on_device ? cudaMemcpyAsync(ctx->qn, w, bytes, cudaMemcpyDeviceToDevice, ctx->stream)
                 : host_copy(ctx->qn, w, bytes, true, ctx->stream));
    CK(launch_prim_to_cons(ctx->ndim, ctx->qn, ctx->ncell, ctx->eos, ctx->stream));
    int st = after_state_change(ctx);
    if (st) return st;
    if (!on_device) CK(cudaStreamSynchronize(ctx->stream));
    return MFC_OK;
}

extern "C" int mfc_get_state(mfc_ctx* ctx, double* q, int on_device) {
    if (!ctx || !q) return MFC_EINVAL;
    if (!ctx->have_state) return MFC_ESTATE;
    size_t bytes = (size_t)ctx->ncell * ctx->neq * sizeof(double);
    CK(on_device ? cudaMemcpyAsync(q, ctx->qn, bytes, cudaMemcpyDeviceToDevice, ctx->stream)
                 : host_copy(q, ctx->qn, bytes, false, ctx->stream));
    if (!on_device) CK(cudaStreamSynchronize(ctx->stream));
    return MFC_OK;
}

static int read_ctrl(mfc_ctx* ctx) {
    CK(cudaMemcpyAsync(ctx->ctrl_h, ctx->ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MFC_OK;
}

// Host-set part of the control block: t, cfl, dt_fixed, status.
static int write_ctrl_params(mfc_ctx* ctx, double cfl, double dt_fixed) {
    ctx->ctrl_h->t = 0.0;
    ctx->ctrl_h->cfl = cfl;
    ctx->ctrl_h->dt_fixed = dt_fixed;
    ctx->ctrl_h->status = 0;
    ctx->ctrl_h->gated = ctx->ctrl_h->fallback = ctx->ctrl_h->cells = ctx->ctrl_h->flat = 0;
    size_t off = offsetof(DevCtrl, t);
    CK(cudaMemcpyAsync((char*)ctx->ctrl + off, (char*)ctx->ctrl_h + off, sizeof(DevCtrl) - off,
                       cudaMemcpyHostToDevice, ctx->stream));
    return MFC_OK;
}

static bool has_neighbours(const mfc_ctx* ctx) {
    for (int d = 0; d < 3; ++d)
        if (ctx->nbr[d][0] || ctx->nbr[d][1]) return true;
    return false;
}

static int rhs_impl(mfc_ctx* ctx, double* rhs, int on_device) {
    if (!ctx->have_state || (ctx->form == FORM_GATED && !ctx->have_gate)) return MFC_ESTATE;
    int st = write_ctrl_params(ctx, 0.0, 0.0);
    if (st) return st;
    double* out = on_device ? rhs : NULL;
    if (!out) {
        if (!fp32_state(ctx)) {
            out = (double*)ctx->acc;  // the last sweep reads and writes each cell in place
        } else {
            if (!ctx->tmp64 && cudaMalloc((void**)&ctx->tmp64, (size_t)ctx->ncell * ctx->neq * sizeof(double)) !=
                                   cudaSuccess) {
                cudaGetLastError();
                return MFC_ENOMEM;
            }
            out = ctx->tmp64;
        }
    }
    SweepArgs a = base_args(ctx);
    a.qin = fp32_state(ctx) ? (const void*)ctx->s0 : (const void*)ctx->qn;
    a.qout = out;
    a.stage = 0;
    for (int d = 0; d < ctx->ndim; ++d) {
        int mode = d == ctx->ndim - 1 ? SW_LAST_RHS : (d == 0 ? SW_FIRST : SW_MID);
        CK(launch_sweep(ctx, d, mode, a, ctx->stream));
    }
    if (!on_device)
        CK(host_copy(rhs, out, (size_t)ctx->ncell * ctx->neq * sizeof(double), false, ctx->stream));
    st = read_ctrl(ctx);
    if (st) return st;
    return ctx->ctrl_h->status ? MFC_ENONPHYSICAL : MFC_OK;
}

extern "C" int mfc_rhs(mfc_ctx* ctx, double* rhs, int on_device) {
    if (!ctx || !rhs) return MFC_EINVAL;
    if (has_neighbours(ctx)) return MFC_ESTATE;   // a block's ghosts: mfc_block_rhs
    return rhs_impl(ctx, rhs, on_device);
}

extern "C" int mfc_gate_rhs(mfc_ctx* ctx, double* rhs, signed char* decisions, int on_device) {
    if (!ctx || !rhs || !decisions) return MFC_EINVAL;
    if (ctx->form != FORM_GATED) return MFC_EINVAL;
    if (has_neighbours(ctx)) return MFC_ESTATE;
    const size_t nb = (size_t)ctx->ndim * ctx->ncell;
    if (!ctx->dec_dev && cudaMalloc((void**)&ctx->dec_dev, nb) != cudaSuccess) {
        cudaGetLastError();
        return MFC_ENOMEM;
    }
    ctx->dec_on = true;
    int st = rhs_impl(ctx, rhs, on_device);
    ctx->dec_on = false;
    if (st != MFC_OK && st != MFC_ENONPHYSICAL) return st;
    CK(on_device ? cudaMemcpyAsync(decisions, ctx->dec_dev, nb, cudaMemcpyDeviceToDevice, ctx->stream)
                 : host_copy(decisions, ctx->dec_dev, nb, false, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return st;
}

extern "C" int mfc_max_wavespeed(mfc_ctx* ctx, double* s) {
    if (!ctx || !s) return MFC_EINVAL;
    if (!ctx->have_state) return MFC_ESTATE;
    int st = write_ctrl_params(ctx, 0.0, 0.0);
    if (st) return st;
    CK(launch_wavespeed(ctx->ndim, ctx->qn, ctx->n, ctx->gw, ctx->grw, ctx->ncell, ctx->dx, ctx->rdx, ctx->eos,
                        ctx->ctrl, ctx->stream));
    st = read_ctrl(ctx);
    if (st) return st;
    unsigned long long bits = ctx->ctrl_h->S_bits;
    memcpy(s, &bits, sizeof(double));
    return ctx->ctrl_h->status ? MFC_ENONPHYSICAL : MFC_OK;
}

static int run_steps(mfc_ctx* ctx, double cfl, double dt_fixed, int nsteps, double* t_out) {
    if (!ctx->have_state || (ctx->form == FORM_GATED && !ctx->have_gate)) return MFC_ESTATE;
    if (has_neighbours(ctx)) return MFC_ESTATE;   // a block steps stage by stage (mfc_block_stage)
    int st = write_ctrl_params(ctx, cfl, dt_fixed);
    if (st) return st;
    if (ctx->timing) {
        for (int n = 0; n < nsteps; ++n) {
            int kinds[kMaxTimedLaunches], nl = 0;
            CK(enqueue_step(ctx, ctx->stream, true, kinds, &nl));
            CK(cudaEventSynchronize(ctx->ev[nl]));
            for (int i = 0; i < nl; ++i) {
                float ms = 0.0f;
                CK(cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]));
                ctx->ktime[kinds[i]] += ms;
                ctx->kcount[kinds[i]] += 1;
            }
        }
    } else {
        st = ensure_graph(ctx);
        if (st) return st;
        for (int n = 0; n < nsteps; ++n) CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
    }
    st = read_ctrl(ctx);
    if (st) return st;
    if (t_out) *t_out = ctx->ctrl_h->t;
    return ctx->ctrl_h->status ? MFC_ENONPHYSICAL : MFC_OK;
}

extern "C" int mfc_step_rk3(mfc_ctx* ctx, double cfl, int nsteps, double* t_advanced) {
    if (!ctx || nsteps < 0 || !(cfl > 0.0) || !isfinite(cfl)) return MFC_EINVAL;
    return run_steps(ctx, cfl, 0.0, nsteps, t_advanced);
}

extern "C" int mfc_step_rk3_dt(mfc_ctx* ctx, double dt, int nsteps) {
    if (!ctx || nsteps < 0 || !(dt > 0.0) || !isfinite(dt)) return MFC_EINVAL;
    return run_steps(ctx, 0.0, dt, nsteps, NULL);
}

extern "C" int mfc_set_grid(mfc_ctx* ctx, int dir, const double* edges) {
    if (!ctx || !edges || dir < 0 || dir >= ctx->ndim) return MFC_EINVAL;
    if (ctx->is_block) return MFC_EINVAL;
    if (ctx->form == FORM_GATED || ctx->p.weno_order == 3 || ctx->eos.nf != 2) return MFC_EINVAL;
    const int n = ctx->n[dir];
    std::vector<double> tab, width;
    if (!build_grid_tables(edges, n, ctx->periodic[dir], tab, width)) return MFC_EINVAL;
    std::vector<double> rw(n);
    std::vector<float> rw32(n), tab32;
    for (int j = 0; j < n; ++j) {
        rw[j] = 1.0 / width[j];
        rw32[j] = (float)rw[j];
    }
    const bool fp32 = fp32_state(ctx);
    if (fp32) tab32.assign(tab.begin(), tab.end());
    // the new tables go into new buffers first: on failure the context keeps
    // its current grid (and the captured step its buffers)
    const size_t tb = tab.size() * (fp32 ? sizeof(float) : sizeof(double));
    void* nt = nullptr;
    double *nw = nullptr, *nrw = nullptr;
    float* nrw32 = nullptr;
    auto free_new = [&]() {
        void* b[] = {nt, nw, nrw, nrw32};
        for (void* x : b)
            if (x) cudaFree(x);
    };
    if (cudaMalloc(&nt, tb) != cudaSuccess || cudaMalloc((void**)&nw, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&nrw, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&nrw32, n * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        free_new();
        return MFC_ENOMEM;
    }
    cudaError_t e = cudaMemcpy(nt, fp32 ? (const void*)tab32.data() : (const void*)tab.data(), tb,
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(nw, width.data(), n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(nrw, rw.data(), n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(nrw32, rw32.data(), n * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        ctx->last_cuda = (int)e;
        free_new();
        return MFC_ECUDA;
    }
    // the captured step refers to the old buffers; the wave speed of the
    // current state changes with the widths
    if (ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = NULL;
    }
    ctx->graph_ok = false;
    void* old[] = {ctx->gtab[dir], ctx->gw[dir], ctx->grw[dir], ctx->grw32[dir]};
    for (void* b : old)
        if (b) cudaFree(b);
    ctx->gtab[dir] = nt;
    ctx->gw[dir] = nw;
    ctx->grw[dir] = nrw;
    ctx->grw32[dir] = nrw32;
    if (ctx->have_state) {
        CK(launch_wavespeed(ctx->ndim, ctx->qn, ctx->n, ctx->gw, ctx->grw, ctx->ncell, ctx->dx, ctx->rdx, ctx->eos,
                            ctx->ctrl, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return MFC_OK;
}

extern "C" int mfc_set_mlp_weights(mfc_ctx* ctx, const float* w, int n) {
    if (!ctx || !w || n != kGateParams) return MFC_EINVAL;
    if (ctx->form != FORM_GATED) return MFC_EINVAL;
    for (int k = 0; k < n; ++k)
        if (!isfinite(w[k])) return MFC_EINVAL;
    CK(cudaMemcpyAsync(ctx->gate_w, w, kGateParams * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->have_gate = true;
    return MFC_OK;
}

extern "C" int mfc_gate_stats(mfc_ctx* ctx, long long* gated, long long* fallback, long long* cells) {
    if (!ctx) return MFC_EINVAL;
    if (gated) *gated = (long long)ctx->ctrl_h->gated;
    if (fallback) *fallback = (long long)ctx->ctrl_h->fallback;
    if (cells) *cells = (long long)ctx->ctrl_h->cells;
    return MFC_OK;
}

extern "C" int mfc_gate_flat(mfc_ctx* ctx, long long* flat) {
    if (!ctx || !flat) return MFC_EINVAL;
    *flat = (long long)ctx->ctrl_h->flat;
    return MFC_OK;
}

extern "C" int mfc_gate_samples(mfc_ctx* ctx, float* X, float* Y, long long capacity, float tau, long long* count) {
    if (!ctx || !X || !Y || !(tau > 0.f) || ctx->eos.nf != 2) return MFC_EINVAL;
    if (!ctx->have_state) return MFC_ESTATE;
    long long need = 2LL * ctx->ndim * ctx->ncell;
    if (capacity < need) return MFC_EINVAL;
    CK(launch_gate_samples(ctx->ndim, ctx->qn, ctx->n, ctx->periodic, ctx->eos, ctx->p.weno_eps, tau, X, Y,
                           ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (count) *count = need;
    return MFC_OK;
}

extern "C" int mfc_launches_per_step(mfc_ctx* ctx, int* launches) {
    if (!ctx || !launches) return MFC_EINVAL;
    *launches = 1 + 3 * ctx->ndim;
    return MFC_OK;
}

extern "C" int mfc_set_timing(mfc_ctx* ctx, int enable) {
    if (!ctx) return MFC_EINVAL;
    ctx->timing = enable != 0;
    for (int k = 0; k < K_NKINDS; ++k) {
        ctx->ktime[k] = 0.0;
        ctx->kcount[k] = 0;
    }
    return MFC_OK;
}

extern "C" int mfc_kernel_time(mfc_ctx* ctx, int index, const char** name, double* ms, long long* launches) {
    if (!ctx || index < 0 || index >= K_NKINDS) return MFC_EINVAL;
    if (name) *name = kKindNames[index];
    if (ms) *ms = ctx->ktime[index];
    if (launches) *launches = ctx->kcount[index];
    return MFC_OK;
}

extern "C" int mfc_alu_peak(int fp64, double* tflops) {
    if (!tflops) return MFC_EINVAL;
    cudaError_t e = run_fma_probe(fp64 != 0, tflops, (cudaStream_t)0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MFC_ECUDA;
    }
    return MFC_OK;
}

// ---- block decomposition (Sec. III-A) ---------------------------------------

extern "C" int mfc_create_block(const mfc_params* global, const mfc_block* block, void* cuda_stream,
                                mfc_ctx** out) {
    if (!out) return MFC_EINVAL;
    *out = NULL;
    if (!block) return MFC_EINVAL;
    int st = validate(global);
    if (st) return st;
    mfc_params pb = *global;
    int lo[3], n[3], nbr[3][2];
    double dx[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = d < global->ndim ? block->lo[d] : 0;
        n[d] = d < global->ndim ? block->n[d] : 1;
        const int N = d < global->ndim ? global->n[d] : 1;
        if (lo[d] < 0 || n[d] < 1 || lo[d] > N - n[d]) return MFC_EINVAL;
        const bool periodic = d < global->ndim && global->bc[d][0] == MFC_BC_PERIODIC;
        // a side borders another block unless it is a non-periodic domain
        // boundary, or the block spans a periodic direction (its own wrap)
        nbr[d][0] = d < global->ndim && (lo[d] > 0 || (periodic && n[d] < N));
        nbr[d][1] = d < global->ndim && (lo[d] + n[d] < N || (periodic && n[d] < N));
        if ((nbr[d][0] || nbr[d][1]) && n[d] < 3) return MFC_EINVAL;   // three ghost layers from one neighbour
        if (d < global->ndim) {
            dx[d] = (global->hi[d] - global->lo[d]) / (double)N;
            pb.n[d] = n[d];
            pb.lo[d] = global->lo[d] + lo[d] * dx[d];
            pb.hi[d] = global->lo[d] + (lo[d] + n[d]) * dx[d];
            if (!(pb.hi[d] > pb.lo[d])) return MFC_EINVAL;
        }
    }
    mfc_ctx* ctx = NULL;
    st = mfc_create(&pb, cuda_stream, &ctx);
    if (st) return st;
    // the grid spacing is the global grid's, bit for bit
    for (int d = 0; d < global->ndim; ++d) {
        ctx->inv_dx[d] = (double)global->n[d] / (global->hi[d] - global->lo[d]);
        ctx->dx[d] = dx[d];
        ctx->rdx[d] = 1.0 / dx[d];
    }
    ctx->is_block = 1;
    long long off = 0;
    for (int d = 0; d < 3; ++d) {
        ctx->blk_lo[d] = lo[d];
        for (int sd = 0; sd < 2; ++sd) {
            ctx->nbr[d][sd] = nbr[d][sd];
            ctx->hoff[2 * d + sd] = nbr[d][sd] ? off : -1;
            if (nbr[d][sd]) off += (long long)state_fields(ctx) * 3 * (ctx->ncell / ctx->n[d]);
        }
    }
    ctx->htotal = off;
    *out = ctx;
    return MFC_OK;
}

extern "C" int mfc_halo_layout(mfc_ctx* ctx, long long* offset, long long* total, int* elem_bytes) {
    if (!ctx) return MFC_EINVAL;
    if (offset)
        for (int i = 0; i < 6; ++i) offset[i] = ctx->is_block ? ctx->hoff[i] : -1;
    if (total) *total = ctx->htotal;
    if (elem_bytes) *elem_bytes = (int)state_elem(ctx);
    return MFC_OK;
}

// The state stage k (1..3) reads: q^n (or its FP32 copy) for k = 1.
static const void* stage_input(mfc_ctx* ctx, int k) {
    SweepArgs a;
    memset(&a, 0, sizeof(a));
    stage_buffers(ctx, k, a);
    return a.qin;
}

extern "C" int mfc_block_pack(mfc_ctx* ctx, int stage, void* out) {
    if (!ctx || stage < 1 || stage > 3 || (!out && ctx->htotal > 0)) return MFC_EINVAL;
    if (!ctx->have_state) return MFC_ESTATE;
    const void* q = stage_input(ctx, stage);
    const int el = (int)state_elem(ctx);
    for (int d = 0; d < 3; ++d)
        for (int sd = 0; sd < 2; ++sd)
            if (ctx->nbr[d][sd])
                CK(launch_pack_side(q, static_cast<char*>(out) + ctx->hoff[2 * d + sd] * el, el,
                                    state_fields(ctx), ctx->ncell, ctx->n, d, sd, ctx->stream));
    return MFC_OK;
}

extern "C" int mfc_block_begin_step(mfc_ctx* ctx, double dt) {
    if (!ctx || !(dt > 0.0) || !isfinite(dt)) return MFC_EINVAL;
    if (!ctx->have_state || (ctx->form == FORM_GATED && !ctx->have_gate)) return MFC_ESTATE;
    CK(launch_block_begin(ctx->ctrl, dt, ctx->stream));
    return MFC_OK;
}

extern "C" int mfc_block_stage(mfc_ctx* ctx, int stage, const void* halo) {
    if (!ctx || stage < 1 || stage > 3 || (!halo && ctx->htotal > 0)) return MFC_EINVAL;
    if (!ctx->have_state || (ctx->form == FORM_GATED && !ctx->have_gate)) return MFC_ESTATE;
    SweepArgs a = base_args(ctx);
    stage_buffers(ctx, stage, a);
    ctx->halo_cur = halo;
    cudaError_t e = cudaSuccess;
    for (int d = 0; d < ctx->ndim && e == cudaSuccess; ++d) {
        int mode = d == ctx->ndim - 1 ? SW_LAST_RK : (d == 0 ? SW_FIRST : SW_MID);
        e = launch_sweep(ctx, d, mode, a, ctx->stream);
    }
    ctx->halo_cur = NULL;
    CK(e);
    return MFC_OK;
}

extern "C" int mfc_block_wavespeed(mfc_ctx* ctx, double* s) {
    if (!ctx || !s) return MFC_EINVAL;
    if (!ctx->have_state) return MFC_ESTATE;
    int st = read_ctrl(ctx);
    if (st) return st;
    unsigned long long bits = ctx->ctrl_h->S_bits;
    memcpy(s, &bits, sizeof(double));
    const unsigned status = ctx->ctrl_h->status;
    if (status) {   // reported once: cleared for the steps that follow
        const unsigned zero = 0;
        CK(cudaMemcpyAsync(&ctx->ctrl->status, &zero, sizeof(zero), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return status ? MFC_ENONPHYSICAL : MFC_OK;
}

extern "C" int mfc_block_rhs(mfc_ctx* ctx, const void* halo, double* rhs, int on_device) {
    if (!ctx || !rhs || (!halo && ctx->htotal > 0)) return MFC_EINVAL;
    ctx->halo_cur = halo;
    int st = rhs_impl(ctx, rhs, on_device);
    ctx->halo_cur = NULL;
    return st;
}

extern "C" const char* mfc_strerror(int status) {
    switch (status) {
        case MFC_OK: return "ok";
        case MFC_EINVAL: return "invalid argument";
        case MFC_ENOMEM: return "out of memory";
        case MFC_ECUDA: return "CUDA runtime error";
        case MFC_ENONPHYSICAL: return "non-physical state (rho<=0, c^2<=0 or NaN)";
        case MFC_ESTATE: return "no state set";
        case MFC_ETOOBIG: return "problem too large for the fixed no-allocation scratch";
        default: return "unknown status";
    }
}

extern "C" int mfc_last_cuda_error(mfc_ctx* ctx) { return ctx ? ctx->last_cuda : 0; }
