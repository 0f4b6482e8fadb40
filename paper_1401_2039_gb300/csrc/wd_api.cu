// C ABI of libwd: operator handle, operator applications and the CGNR
// solve of the even-odd Schur system (arXiv:1401.2039, Fig. "dirac",
// Alg. "schur", Alg. "CGNR").
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "dslash.cuh"

namespace wd {
#define WD_DECL(P)                                                                         \
    cudaError_t launch_dslash_##P##_r18(const DslashLaunch &L, cudaStream_t s);            \
    cudaError_t launch_dslash_##P##_r12(const DslashLaunch &L, cudaStream_t s);
WD_DECL(f64) WD_DECL(f32) WD_DECL(f16) WD_DECL(bf16)
#undef WD_DECL
cudaError_t launch_dslash_df64_r18(const DslashLaunch &L, cudaStream_t s);
cudaError_t launch_dslash_df64f32_r18(const DslashLaunch &L, cudaStream_t s);

cudaError_t launch_dslash(const DslashLaunch &L, int prec, cudaStream_t s) {
    const bool r12 = L.gauge->recon == 12;
    switch (prec) {
    case WD_F64: return r12 ? launch_dslash_f64_r12(L, s) : launch_dslash_f64_r18(L, s);
    case WD_F32: return r12 ? launch_dslash_f32_r12(L, s) : launch_dslash_f32_r18(L, s);
    case WD_F16: return r12 ? launch_dslash_f16_r12(L, s) : launch_dslash_f16_r18(L, s);
    case WD_BF16: return r12 ? launch_dslash_bf16_r12(L, s) : launch_dslash_bf16_r18(L, s);
    case WD_DF64: return r12 ? cudaErrorInvalidValue : launch_dslash_df64_r18(L, s);
    case WD_DF64_F32: return r12 ? cudaErrorInvalidValue : launch_dslash_df64f32_r18(L, s);
    default: return cudaErrorInvalidValue;
    }
}
}  // namespace wd

using namespace wd;

static thread_local std::string g_last_error;

static int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

#define WD_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(e_ == cudaErrorMemoryAllocation ? WD_ERR_NOMEM : WD_ERR_CUDA,      \
                        std::string(#call) + ": " + cudaGetErrorString(e_));               \
    } while (0)

#define WD_TRY(call)                                                                       \
    do {                                                                                   \
        int rc_ = (call);                                                                  \
        if (rc_ != WD_OK) return rc_;                                                      \
    } while (0)

#include "op.cuh"

// ------------------------------------------------------------------ helpers
static int dev_alloc(wd_op *op, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(WD_ERR_NOMEM, std::string("cudaMalloc(") + std::to_string(bytes) +
                                      "): " + cudaGetErrorString(e));
    }
    op->allocations.push_back(*p);
    WD_CUDA(cudaMemset(*p, 0, bytes));
    return WD_OK;
}

static int fork(wd_op *op) {
    WD_CUDA(cudaEventRecord(op->ev_fork, op->user));
    WD_CUDA(cudaStreamWaitEvent(op->stream, op->ev_fork, 0));
    return WD_OK;
}

static int join(wd_op *op) {
    WD_CUDA(cudaEventRecord(op->ev_join, op->stream));
    WD_CUDA(cudaStreamWaitEvent(op->user, op->ev_join, 0));
    return WD_OK;
}

static Reduction reduction(wd_op *op, int fin) {
    return Reduction{op->partials, op->counter, op->sc, fin};
}

// out = scale * H_{p,q} in  (PLAIN) or  x + scale * H_{p,q} in  (XPAY), optional norm.
// twist t != 0: out = scale (1 - i t gamma5) H in  or  (1 + i t gamma5) x + scale H in.
// early: (hi only, double-float residuals) the same fields in FP32 arithmetic
static int dslash(wd_op *op, bool hi, int out_parity, int dagger, void *out, const void *in,
                  const void *x, double scale, const Reduction *red, double twist = 0.0,
                  long h_begin = 0, long h_end = -1, bool early = false) {
    DslashLaunch L;
    L.g = op->g;
    L.gauge = hi ? &op->gauge_hi : &op->gauge_lo;
    L.out_parity = out_parity;
    L.dagger = dagger;
    memcpy(L.phase, op->phase, sizeof(L.phase));
    L.out = out;
    L.in = in;
    L.x = x;
    L.scale = scale;
    L.epi = x ? EPI_XPAY : EPI_PLAIN;
    L.red = red;
    L.cfg = hi ? op->cfg[1] : red ? op->cfg[2] : op->cfg[0];
    L.twist = twist;
    L.h_begin = h_begin;
    L.h_end = h_end;
    int prec = hi ? op->hi_prec : op->prec;
    if (early && hi && prec == WD_DF64) {
        prec = WD_DF64_F32;
        // (128 threads, no register cap): measured 766 us per application
        // at 32^3 x 64 against 847-860 us under the 64- and 80-register caps
        L.cfg = 0;
    }
    WD_CUDA(launch_dslash(L, prec, op->stream));
    return WD_OK;
}

// out_p = A in_p - kappa^2 H_pq A^-1 H_qp in_p  (Mhat_p, Alg. "schur"), with
// A = 1 + i t gamma5, t = 2 kappa mu (A = 1 for the Wilson operator), so that
// A^-1 = (1 - i t gamma5) / (1 + t^2).  Mhat_p^dag: H^dag and -t.
static int schur(wd_op *op, bool hi, int p, int dagger, void *out, const void *in, void *tmp,
                 const Reduction *red, bool early = false) {
    const double t = op->twist(dagger);
    WD_TRY(dslash(op, hi, 1 - p, dagger, tmp, in, nullptr, 1.0 / (1.0 + t * t), nullptr, t, 0,
                  -1, early));
    WD_TRY(dslash(op, hi, p, dagger, out, tmp, in, -op->kappa * op->kappa, red, t, 0, -1, early));
    return WD_OK;
}

static int check_op(const wd_op *op) {
    if (!op) return fail(WD_ERR_ARG, "null operator handle");
    if (!op->gauge_loaded) return fail(WD_ERR_STATE, "no gauge field loaded (wd_op_set_gauge)");
    return WD_OK;
}

// Autotuner: time every launch configuration of one hopping-term variant on
// this operator's lattice (two warm-up and five timed launches each, CUDA
// events on the work stream) and keep the fastest.  Variant 0: the plain
// storage-precision hop; 1: the plain residual-arithmetic hop; 2: the
// storage-precision hop with xpay epilogue and fused norm (the reduction
// result is the same under every configuration).  WD_DSLASH_CFG=k forces
// configuration k, WD_TUNE=0 keeps configuration 0.
static int tune_dslash(wd_op *op, int variant) {
    const char *force = getenv("WD_DSLASH_CFG");
    const char *tune = getenv("WD_TUNE");
    const bool hi = variant == 1;
    const int prec = hi ? op->hi_prec : op->prec;
    const int n_cfg = prec == WD_DF64 ? N_DSLASH_DF_CFG : N_DSLASH_CFG;
    auto applies = [&](int k) { return prec == WD_DF64 || dslash_cfg_applies(k, prec); };
    if (force) {
        int k = atoi(force);
        op->cfg[variant] = (k >= 0 && k < n_cfg && applies(k)) ? k : 0;
        return WD_OK;
    }
    if (tune && tune[0] == '0') {
        op->cfg[variant] = 0;
        return WD_OK;
    }
    void *in = hi ? (void *)op->th : op->slot[0];
    void *out = hi ? (void *)op->axh : op->slot[1];
    Reduction red = reduction(op, FIN_STORE0);
    auto launch = [&](int parity) {
        if (variant == 2)   // out = out - kappa^2 H in, |out|^2 -> scratch
            return dslash(op, false, parity, 0, out, in, out, -op->kappa * op->kappa, &red);
        return dslash(op, hi, parity, 0, out, in, nullptr, 1.0, nullptr);
    };
    int best = 0;
    float best_ms = 1e30f;
    for (int k = 0; k < n_cfg; ++k) {
        op->tune_us[variant][k] = 0.0;
        if (!applies(k)) continue;   // the same kernel as an unstaged candidate
        op->cfg[variant] = k;
        for (int w = 0; w < 2; ++w) WD_TRY(launch(w & 1));
        WD_CUDA(cudaEventRecord(op->ev_t0, op->stream));
        for (int r = 0; r < 5; ++r) WD_TRY(launch(r & 1));
        WD_CUDA(cudaEventRecord(op->ev_t1, op->stream));
        WD_CUDA(cudaEventSynchronize(op->ev_t1));
        float ms = 0;
        WD_CUDA(cudaEventElapsedTime(&ms, op->ev_t0, op->ev_t1));
        op->tune_us[variant][k] = ms * 1e3 / 5;
        if (ms < best_ms) { best_ms = ms; best = k; }
    }
    op->cfg[variant] = best;
    return WD_OK;
}

// ------------------------------------------------------------------ C ABI
extern "C" {

int wd_op_set_solver(wd_op *op, double ru_delta, int stall_iters) {
    if (!op) return fail(WD_ERR_ARG, "null operator handle");
    if (!(ru_delta > 0.0 && ru_delta < 1.0) || stall_iters < 1)
        return fail(WD_ERR_ARG, "ru_delta must lie in (0, 1) and stall_iters be >= 1");
    op->ru_delta = ru_delta;
    op->stall_iters = stall_iters;
    return WD_OK;
}

int wd_op_set_recovery(wd_op *op, int mode, double inner_tol) {
    if (!op) return fail(WD_ERR_ARG, "null operator handle");
    if (mode != WD_RECOVER_RELIABLE && mode != WD_RECOVER_DEFECT)
        return fail(WD_ERR_ARG, "mode must be WD_RECOVER_RELIABLE or WD_RECOVER_DEFECT");
    if (mode == WD_RECOVER_DEFECT && !(inner_tol > 0.0 && inner_tol < 1.0))
        return fail(WD_ERR_ARG, "inner_tol must lie in (0, 1)");
    op->recovery = mode;
    if (mode == WD_RECOVER_DEFECT) op->dc_delta = inner_tol;
    return WD_OK;
}

int wd_op_recovery(const wd_op *op, double *inner_tol) {
    if (!op) return -1;
    if (inner_tol) *inner_tol = op->dc_delta;
    return op->recovery;
}

int wd_op_set_residual_precision(wd_op *op, int mode) {
    if (!op) return fail(WD_ERR_ARG, "null operator handle");
    if (mode != 0 && mode != 1) return fail(WD_ERR_ARG, "mode must be 0 (FP64) or 1 (double-float)");
    if (op->prec == WD_F64) {
        if (mode != 0) return fail(WD_ERR_ARG, "a WD_F64 operator computes its residuals in FP64");
        return WD_OK;
    }
    const int want = mode ? WD_DF64 : WD_F64;
    if (want == op->hi_prec) return WD_OK;
    WD_TRY(fork(op));
    if (op->gauge_loaded) {   // both forms are 8 bytes per real: convert in place
        const long n = (long)(4 * op->gauge_hi.dir_bytes / 8);
        for (int p = 0; p < 2; ++p)
            WD_CUDA(launch_f64_df64(op->gauge_hi.ptr[p], n, mode, op->stream));
    }
    op->hi_prec = want;
    op->gauge_hi.prec = want;
    if (op->gauge_loaded) WD_TRY(tune_dslash(op, 1));
    return join(op);
}

int wd_op_set_twisted_mass(wd_op *op, double mu) {
    if (!op) return fail(WD_ERR_ARG, "null operator handle");
    if (!std::isfinite(mu)) return fail(WD_ERR_ARG, "mu must be finite");
    if (mu == op->mu) return WD_OK;
    // the cached iteration graphs carry the old twist in their kernel arguments
    WD_CUDA(cudaStreamSynchronize(op->stream));
    for (auto &row : op->graphs)
        for (auto &ge : row)
            if (ge) {
                cudaGraphExecDestroy(ge);
                ge = nullptr;
            }
    op->mu = mu;
    return WD_OK;
}

double wd_op_twisted_mass(const wd_op *op) { return op ? op->mu : 0.0; }

int wd_dslash_tuning(const wd_op *op, int hi, double *us, int n, int *block, int *min_blocks,
                     int *sites_per_thread, int *staged) {
    if (!op || hi < 0 || hi > 2) return -1;
    const int k = op->cfg[hi];
    const bool df = hi == 1 && op->hi_prec == WD_DF64;
    const int n_cfg = df ? N_DSLASH_DF_CFG : N_DSLASH_CFG;
    for (int i = 0; us && i < n; ++i) us[i] = i < n_cfg ? op->tune_us[hi][i] : 0.0;
    const DslashCfg &C = df ? DSLASH_DF_CFGS[k] : DSLASH_CFGS[k];
    if (block) *block = C.block;
    if (min_blocks) *min_blocks = C.minb;
    if (sites_per_thread) *sites_per_thread = C.spt;
    if (staged) *staged = C.stage;
    return k;
}

const char *wd_status_string(int s) {
    switch (s) {
    case WD_OK: return "ok";
    case WD_ERR_ARG: return "invalid argument";
    case WD_ERR_DIMS: return "invalid lattice dimensions";
    case WD_ERR_CUDA: return "CUDA error";
    case WD_ERR_NOMEM: return "out of device memory";
    case WD_ERR_NOT_CONVERGED: return "solver did not converge";
    case WD_ERR_BREAKDOWN: return "solver breakdown";
    case WD_ERR_TIMEOUT: return "device wait timed out";
    case WD_ERR_STATE: return "call out of order";
    default: return "unknown status";
    }
}

const char *wd_last_error(void) { return g_last_error.c_str(); }

void *wd_op_stream(wd_op *op) { return op ? (void *)op->stream : nullptr; }

long wd_op_half_volume(const wd_op *op) { return op ? op->g.vh : 0; }

double wd_dslash_bytes(const wd_op *op) {
    if (!op) return 0.0;
    return (double)op->g.vh * (48.0 + 8.0 * op->recon) * (double)prec_bytes(op->prec);
}

void wd_op_destroy(wd_op *op) {
    if (!op) return;
    if (op->stream) cudaStreamSynchronize(op->stream);
    for (auto &row : op->graphs)
        for (auto &ge : row)
            if (ge) cudaGraphExecDestroy(ge);
    for (void *p : op->allocations) cudaFree(p);
    if (op->sc_host) cudaFreeHost(op->sc_host);
    if (op->host_consts) cudaFreeHost(op->host_consts);
    if (op->ev_t0) cudaEventDestroy(op->ev_t0);
    if (op->ev_t1) cudaEventDestroy(op->ev_t1);
    if (op->ev_fork) cudaEventDestroy(op->ev_fork);
    if (op->ev_join) cudaEventDestroy(op->ev_join);
    if (op->ev_x) cudaEventDestroy(op->ev_x);
    if (op->ev_xd) cudaEventDestroy(op->ev_xd);
    for (cudaEvent_t e : op->ev_b2)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : op->ev_b)
        if (e) cudaEventDestroy(e);
    if (op->copy_stream) {
        cudaStreamSynchronize(op->copy_stream);
        cudaStreamDestroy(op->copy_stream);
    }
    if (op->stream) cudaStreamDestroy(op->stream);
    delete op;
}

static int create_impl(wd_op *op) {
    WD_CUDA(cudaStreamCreateWithFlags(&op->stream, cudaStreamNonBlocking));
    WD_CUDA(cudaEventCreateWithFlags(&op->ev_fork, cudaEventDisableTiming));
    WD_CUDA(cudaEventCreateWithFlags(&op->ev_join, cudaEventDisableTiming));
    WD_CUDA(cudaEventCreate(&op->ev_t0));
    WD_CUDA(cudaEventCreate(&op->ev_t1));
    WD_CUDA(cudaStreamCreateWithFlags(&op->copy_stream, cudaStreamNonBlocking));
    WD_CUDA(cudaEventCreateWithFlags(&op->ev_x, cudaEventDisableTiming));
    WD_CUDA(cudaEventCreateWithFlags(&op->ev_xd, cudaEventDisableTiming));
    for (cudaEvent_t &e : op->ev_b) WD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));

    const Geom &g = op->g;
    // gauge fields
    op->gauge_lo.prec = op->prec;
    op->gauge_lo.recon = op->recon;
    op->gauge_lo.dir_bytes = field_bytes(op->prec, g.stride, op->recon);
    for (int p = 0; p < 2; ++p)
        WD_TRY(dev_alloc(op, &op->gauge_lo.ptr[p], 4 * op->gauge_lo.dir_bytes));
    op->hi_shared = (op->prec == WD_F64 && op->recon == 18);
    if (op->hi_shared) {
        op->gauge_hi = op->gauge_lo;
    } else {
        op->gauge_hi.prec = op->hi_prec;
        op->gauge_hi.recon = 18;
        op->gauge_hi.dir_bytes = field_bytes(op->hi_prec, g.stride, 18);
        for (int p = 0; p < 2; ++p)
            WD_TRY(dev_alloc(op, &op->gauge_hi.ptr[p], 4 * op->gauge_hi.dir_bytes));
    }
    // fields
    const size_t lo = op->lo_field_bytes(), hi = op->hi_field_bytes();
    void **lo_fields[] = {&op->fa[0], &op->fa[1], &op->fc[0], &op->fc[1], &op->ftmp,
                          &op->slot[0], &op->slot[1], &op->xl, &op->rl, &op->pl, &op->zl,
                          &op->apl, &op->tl};
    for (void **f : lo_fields) WD_TRY(dev_alloc(op, f, lo));
    double **hi_fields[] = {&op->hb[0], &op->hb[1], &op->bh, &op->xh, &op->rh, &op->axh,
                            &op->th, &op->xq};
    for (double **f : hi_fields) WD_TRY(dev_alloc(op, (void **)f, hi));
    const size_t canon = (size_t)2 * g.vh * 24 * sizeof(double);
    WD_TRY(dev_alloc(op, (void **)&op->stage_x, canon));
    WD_TRY(dev_alloc(op, (void **)&op->stage_b, canon));
    // reductions
    WD_TRY(dev_alloc(op, (void **)&op->partials, sizeof(df64) * reduction_blocks(g)));
    WD_TRY(dev_alloc(op, (void **)&op->counter, sizeof(unsigned int) * ARRIVE_WORDS));
    WD_TRY(dev_alloc(op, (void **)&op->sc, sizeof(SolverScalars)));
    WD_TRY(dev_alloc(op, (void **)&op->dev_consts, sizeof(double) * 4));
    // the solve's scalars and constants cross between host and device through
    // mapped pinned buffers, copied by the SMs (launch_copy_small)
    WD_CUDA(cudaHostAlloc((void **)&op->sc_host, sizeof(SolverScalars), cudaHostAllocMapped));
    WD_CUDA(cudaHostAlloc((void **)&op->host_consts, sizeof(double) * 4, cudaHostAllocMapped));
    WD_CUDA(cudaHostGetDevicePointer((void **)&op->sc_host_dev, op->sc_host, 0));
    WD_CUDA(cudaHostGetDevicePointer((void **)&op->host_consts_dev, op->host_consts, 0));
    WD_CUDA(cudaDeviceSynchronize());
    return WD_OK;
}

int wd_op_create(wd_op **out, const int dims[4], double kappa, const double phase[8],
                 int prec, int recon, void *stream) {
    if (!out || !dims || !phase) return fail(WD_ERR_ARG, "null argument to wd_op_create");
    *out = nullptr;
    long V = 1;
    for (int m = 0; m < 4; ++m) {
        if (dims[m] < 2 || dims[m] % 2)
            return fail(WD_ERR_DIMS, "every lattice extent must be even and >= 2");
        if (dims[m] > (1 << 14)) return fail(WD_ERR_DIMS, "lattice extent too large");
        V *= dims[m];
    }
    if (V > (1L << 31)) return fail(WD_ERR_DIMS, "lattice volume above 2^31 sites");
    if (prec < WD_F64 || prec > WD_BF16) return fail(WD_ERR_ARG, "unknown precision");
    if (recon != 18 && recon != 12) return fail(WD_ERR_ARG, "recon must be 18 or 12");
    if (!std::isfinite(kappa)) return fail(WD_ERR_ARG, "kappa must be finite");
    for (int i = 0; i < 8; ++i)
        if (!std::isfinite(phase[i])) return fail(WD_ERR_ARG, "phases must be finite");

    wd_op *op = new wd_op();
    op->g = make_geom(dims, pad_stride(V / 2));
    op->kappa = kappa;
    memcpy(op->phase, phase, sizeof(op->phase));
    op->prec = prec;
    op->recon = recon;
    op->hi_prec = prec == WD_F64 ? WD_F64 : WD_DF64;
    // measured best at 32^3 x 64: the fewer significand bits the storage
    // keeps, the sooner the iterated residual drifts from the true one
    op->ru_delta = prec == WD_F32 ? 0.01 : prec == WD_BF16 ? 0.3 : RU_DELTA_DEFAULT;
    op->user = (cudaStream_t)stream;
    int rc = create_impl(op);
    if (rc != WD_OK) {
        std::string msg = g_last_error;
        wd_op_destroy(op);
        g_last_error = msg;
        return rc;
    }
    *out = op;
    return WD_OK;
}

int wd_op_set_gauge(wd_op *op, const double *U) {
    if (!op || !U) return fail(WD_ERR_ARG, "null argument to wd_op_set_gauge");
    WD_TRY(fork(op));
    WD_CUDA(launch_pack_gauge(op->gauge_lo, op->g, U, op->stream));
    if (!op->hi_shared) WD_CUDA(launch_pack_gauge(op->gauge_hi, op->g, U, op->stream));
    WD_TRY(tune_dslash(op, 0));
    WD_TRY(tune_dslash(op, 2));
    if (!op->hi_shared) WD_TRY(tune_dslash(op, 1));
    else op->cfg[1] = op->cfg[0];
    WD_TRY(join(op));
    op->gauge_loaded = true;
    return WD_OK;
}

int wd_apply(wd_op *op, double *out, const double *in, int dagger) {
    WD_TRY(check_op(op));
    if (!out || !in) return fail(WD_ERR_ARG, "null spinor");
    if (dagger != 0 && dagger != 1) return fail(WD_ERR_ARG, "dagger must be 0 or 1");
    WD_TRY(fork(op));
    WD_CUDA(launch_pack_full(op->prec, op->g, op->fa[0], op->fa[1], in, op->stream));
    for (int p = 0; p < 2; ++p)   // out_p = A in_p - kappa H_pq in_q
        WD_TRY(dslash(op, false, p, dagger, op->fc[p], op->fa[1 - p], op->fa[p], -op->kappa,
                      nullptr, op->twist(dagger)));
    WD_CUDA(launch_unpack_full(op->prec, op->g, out, op->fc[0], op->fc[1], op->stream));
    return join(op);
}

int wd_apply_eo(wd_op *op, double *out, const double *in, int parity, int dagger) {
    WD_TRY(check_op(op));
    if (!out || !in) return fail(WD_ERR_ARG, "null spinor");
    if (parity != 0 && parity != 1) return fail(WD_ERR_ARG, "parity must be 0 or 1");
    if (dagger != 0 && dagger != 1) return fail(WD_ERR_ARG, "dagger must be 0 or 1");
    WD_TRY(fork(op));
    WD_CUDA(launch_pack_half(op->prec, op->g, op->fa[0], in, op->stream));
    WD_TRY(schur(op, false, parity, dagger, op->fc[0], op->fa[0], op->ftmp, nullptr));
    WD_CUDA(launch_unpack_half(op->prec, op->g, out, op->fc[0], op->stream));
    return join(op);
}

static int apply_eo_hi(wd_op *op, double *out, const double *in, int parity, int dagger,
                       bool early) {
    WD_TRY(check_op(op));
    if (!out || !in) return fail(WD_ERR_ARG, "null spinor");
    if (parity != 0 && parity != 1) return fail(WD_ERR_ARG, "parity must be 0 or 1");
    if (dagger != 0 && dagger != 1) return fail(WD_ERR_ARG, "dagger must be 0 or 1");
    WD_TRY(fork(op));
    WD_CUDA(launch_pack_half(op->hi_prec, op->g, op->xh, in, op->stream));
    WD_TRY(schur(op, true, parity, dagger, op->axh, op->xh, op->th, nullptr, early));
    WD_CUDA(launch_unpack_half(op->hi_prec, op->g, out, op->axh, op->stream));
    return join(op);
}

int wd_apply_eo_residual(wd_op *op, double *out, const double *in, int parity, int dagger) {
    return apply_eo_hi(op, out, in, parity, dagger, false);
}

int wd_apply_eo_residual_early(wd_op *op, double *out, const double *in, int parity,
                               int dagger) {
    return apply_eo_hi(op, out, in, parity, dagger, true);
}

int wd_dslash_eo(wd_op *op, double *out, const double *in, int out_parity, int dagger) {
    WD_TRY(check_op(op));
    if (!out || !in) return fail(WD_ERR_ARG, "null spinor");
    if (out_parity != 0 && out_parity != 1) return fail(WD_ERR_ARG, "parity must be 0 or 1");
    if (dagger != 0 && dagger != 1) return fail(WD_ERR_ARG, "dagger must be 0 or 1");
    WD_TRY(fork(op));
    WD_CUDA(launch_pack_half(op->prec, op->g, op->fa[0], in, op->stream));
    WD_TRY(dslash(op, false, out_parity, dagger, op->fc[0], op->fa[0], nullptr, 1.0, nullptr));
    WD_CUDA(launch_unpack_half(op->prec, op->g, out, op->fc[0], op->stream));
    return join(op);
}

int wd_field_load(wd_op *op, int slot, const double *half_in) {
    if (!op || !half_in) return fail(WD_ERR_ARG, "null argument");
    if (slot != 0 && slot != 1) return fail(WD_ERR_ARG, "slot must be 0 or 1");
    WD_TRY(fork(op));
    WD_CUDA(launch_pack_half(op->prec, op->g, op->slot[slot], half_in, op->stream));
    return join(op);
}

int wd_field_store(wd_op *op, int slot, double *half_out) {
    if (!op || !half_out) return fail(WD_ERR_ARG, "null argument");
    if (slot != 0 && slot != 1) return fail(WD_ERR_ARG, "slot must be 0 or 1");
    WD_TRY(fork(op));
    WD_CUDA(launch_unpack_half(op->prec, op->g, half_out, op->slot[slot], op->stream));
    return join(op);
}

int wd_dslash_resident(wd_op *op, int in_slot, int out_parity, int dagger) {
    WD_TRY(check_op(op));
    if (in_slot != 0 && in_slot != 1) return fail(WD_ERR_ARG, "slot must be 0 or 1");
    if (out_parity != 0 && out_parity != 1) return fail(WD_ERR_ARG, "parity must be 0 or 1");
    if (dagger != 0 && dagger != 1) return fail(WD_ERR_ARG, "dagger must be 0 or 1");
    WD_TRY(fork(op));
    WD_TRY(dslash(op, false, out_parity, dagger, op->slot[1 - in_slot], op->slot[in_slot],
                  nullptr, 1.0, nullptr));
    return join(op);
}

}  // extern "C"

// ------------------------------------------------------------------ solver
namespace {

struct SolveState {
    int p, q;
    double target;      // absolute FP64 residual norm to reach
    double nb;          // ||b||
    double scale;       // r_lo = scale * r_hi
    double r_hi;        // ||r_hi|| at the last refresh
    int ru;             // reliable updates
    double dslash_lo, dslash_hi, bytes, launches;
    int restarts;
    bool th_valid;      // th holds H_qp x_hi for the current x_hi
};

double field_b(const wd_op *op, int prec) { return (double)op->g.vh * 24 * prec_bytes(prec); }
double dslash_b(const wd_op *op, bool hi, bool xpay) {
    const int pr = hi ? WD_F64 : op->prec;
    const int rc = hi ? 18 : op->recon;
    return (double)op->g.vh * (48.0 + 8.0 * rc + (xpay ? 24.0 : 0.0)) * (double)prec_bytes(pr);
}

// One CGNR iteration on Mhat_p in storage precision, with the residual
// checkpoint at its end:
//   z = A^dag r; beta = |z|^2 / nz; nz = |z|^2; p = z + beta p;
//   Ap = A p; alpha = nz / |Ap|^2; x += alpha p; r -= alpha Ap; nr = |r|^2
// (Alg. "CGNR", rotated so that the host may refresh r between iterations).
// The step x += alpha p only feeds x, so it runs one iteration late, in the
// pass that reads p anyway (p = z + beta p), and the fold of a refresh
// settles the step still owed.
int cg_iteration(wd_op *op, int p) {
    Reduction rb = reduction(op, FIN_BETA), ra = reduction(op, FIN_ALPHA),
              rn = reduction(op, FIN_NR);
    WD_TRY(schur(op, false, p, 1, op->zl, op->rl, op->tl, &rb));
    WD_CUDA(launch_cg_update_px(op->prec, op->g, op->xl, op->pl, op->zl, op->sc, op->stream));
    WD_TRY(schur(op, false, p, 0, op->apl, op->pl, op->tl, &ra));
    WD_CUDA(launch_cg_update_r(op->prec, op->g, op->rl, op->apl, rn, op->stream));
    return WD_OK;
}

int graph_for(wd_op *op, int p, int lg, cudaGraphExec_t *out) {
    if (!op->graphs[p][lg]) {
        cudaGraph_t graph = nullptr;
        WD_CUDA(cudaStreamBeginCapture(op->stream, cudaStreamCaptureModeThreadLocal));
        int rc = WD_OK;
        for (int i = 0; i < (1 << lg) && rc == WD_OK; ++i) rc = cg_iteration(op, p);
        cudaError_t e = cudaStreamEndCapture(op->stream, &graph);
        if (rc != WD_OK) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        WD_CUDA(e);
        cudaError_t ei = cudaGraphInstantiate(&op->graphs[p][lg], graph, 0);
        cudaGraphDestroy(graph);
        WD_CUDA(ei);
    }
    *out = op->graphs[p][lg];
    return WD_OK;
}

int run_iterations(wd_op *op, int p, int n) {
    for (int lg = MAX_BATCH_LOG2; lg >= 0; --lg) {
        while (n >= (1 << lg)) {
            cudaGraphExec_t ge;
            WD_TRY(graph_for(op, p, lg, &ge));
            WD_CUDA(cudaGraphLaunch(ge, op->stream));
            n -= 1 << lg;
        }
    }
    return WD_OK;
}

int read_scalars(wd_op *op) {
    // by the SMs: a copy-engine read would queue behind a large host copy
    // (the next source's upload or the last solution's download)
    WD_CUDA(launch_copy_small(op->sc_host_dev, op->sc, sizeof(SolverScalars), op->stream));
    WD_CUDA(cudaStreamSynchronize(op->stream));
    return WD_OK;
}

// x_q = A^-1 b_q + kappa th on stream s, where th = A^-1 H_qp x_p is the
// first hop of the last residual-arithmetic refresh (A = 1 + i t gamma5)
int reconstruct_from_th(wd_op *op, SolveState &st, cudaStream_t s) {
    const double tw = op->twist(0);
    const void *bq = op->hb[st.q];
    if (tw != 0.0) {
        WD_CUDA(launch_twist_hi(op->hi_prec, op->g, op->xq, op->hb[st.q], -tw, 1.0 / (1.0 + tw * tw),
                                s));
        bq = op->xq;
        st.launches += 1;
        st.bytes += 2 * field_b(op, WD_F64);
    }
    WD_CUDA(launch_xpay_hi(op->hi_prec, op->g, op->xq, bq, op->kappa, op->th, s));
    st.bytes += 3 * field_b(op, WD_F64);
    st.launches += 1;
    return WD_OK;
}

// unpack x = (x_p, x_q) into x_out on stream s and, with x_host, queue its
// download on the copy stream behind it
int unpack_and_download(wd_op *op, SolveState &st, double *x_out, double *x_host,
                        cudaStream_t s) {
    double *xe = st.p == 0 ? op->xh : op->xq, *xo = st.p == 0 ? op->xq : op->xh;
    // a download of the previous solution from the same buffer may still run
    if (op->xd_pending) WD_CUDA(cudaStreamWaitEvent(s, op->ev_xd, 0));
    WD_CUDA(launch_unpack_full(op->hi_prec, op->g, x_out, xe, xo, s));
    st.launches += 1;
    if (x_host) {
        WD_CUDA(cudaEventRecord(op->ev_x, s));
        WD_CUDA(cudaStreamWaitEvent(op->copy_stream, op->ev_x, 0));
        WD_CUDA(cudaMemcpyAsync(x_host, x_out, (size_t)2 * op->g.vh * 24 * sizeof(double),
                                cudaMemcpyDeviceToHost, op->copy_stream));
        WD_CUDA(cudaEventRecord(op->ev_xd, op->copy_stream));
        op->xd_pending = true;
    }
    return WD_OK;
}

// r_hi = bhat - Mhat x_hi in residual arithmetic and ||r_hi||^2 -> scratch[0]
// (the Schur operator's first hop leaves th = A^-1 H_qp x_hi).  early: Mhat
// x_hi in FP32 arithmetic on the double-float fields, for a refresh whose
// residual is still large (relative rounding ~1e-7 of ||Mhat|| ||x||, small
// against ||r_hi||; the next double-float refresh recomputes r_hi from x_hi
// and so corrects it).  th is then not accurate enough for the
// reconstruction.
int true_residual(wd_op *op, SolveState &st, bool early = false) {
    Reduction r0 = reduction(op, FIN_STORE0);
    WD_TRY(schur(op, true, st.p, 0, op->axh, op->xh, op->th, nullptr, early));
    st.th_valid = !early;
    WD_CUDA(launch_xmy_norm(op->hi_prec, op->g, op->rh, op->bh, op->axh, r0, op->stream));
    st.dslash_hi += 2;
    st.launches += 3;
    st.bytes += dslash_b(op, true, false) + dslash_b(op, true, true) + 3 * field_b(op, WD_F64);
    return WD_OK;
}

int set_consts(wd_op *op, double scale, double inv_scale, double ratio) {
    op->host_consts[0] = scale;
    op->host_consts[1] = inv_scale;
    op->host_consts[2] = ratio;
    WD_CUDA(launch_copy_small(op->dev_consts, op->host_consts_dev, 3 * sizeof(double),
                              op->stream));
    return WD_OK;
}

// The t-slabs b arrives in from host memory: slab k holds the time slices
// [slab_t(k), slab_t(k + 1)), canonical sites [2 S slab_t(k), 2 S slab_t(k + 1))
// with S = Lx Ly Lz / 2 sites per slice and parity.
int slab_t(const wd_op *op, int k) {
    return (int)((long)op->g.L[3] * k / wd_op::B_SLABS);
}

// bhat_p = b_p + kappa H_pq b_q (Wilson operator) while b arrives slab by
// slab (event slab_ev[k] on the copy stream): each slab is packed as soon as it
// is in, and the hop computes the output slices whose neighbours in t have
// all arrived, so that most of the packing and of the hop overlap the
// upload.  Slice 0 needs slice Lt - 1 and goes last.
int prepare_from_slabs(wd_op *op, SolveState &st, const double *b, const cudaEvent_t *slab_ev) {
    const Geom &g = op->g;
    const long S = (long)g.hx * g.L[1] * g.L[2];
    const int T = g.L[3];
    int done = 1;   // output slices [1, done) are computed
    for (int k = 0; k < wd_op::B_SLABS; ++k) {
        const int ta = slab_t(op, k), tb = slab_t(op, k + 1);
        WD_CUDA(cudaStreamWaitEvent(op->stream, slab_ev[k], 0));
        WD_CUDA(launch_pack_full(op->hi_prec, g, op->hb[0], op->hb[1], b, op->stream,
                                 2 * S * ta, 2 * S * tb));
        const int hi = k + 1 == wd_op::B_SLABS ? T : tb - 1;
        if (hi > done) {
            WD_TRY(dslash(op, true, st.p, 0, op->bh, op->hb[st.q], op->hb[st.p], op->kappa,
                          nullptr, 0.0, S * done, S * hi));
            done = hi;
        }
    }
    WD_TRY(dslash(op, true, st.p, 0, op->bh, op->hb[st.q], op->hb[st.p], op->kappa, nullptr,
                  0.0, 0, S));
    st.launches += wd_op::B_SLABS + 1;
    return WD_OK;
}

// x_in: the initial guess (read once, at the start; nullptr: x = 0); x_out:
// the solution (written once, at the end); they may be the same array.  x_host (optional):
// host memory the solution is also copied to, on the handle's copy stream as
// soon as it is complete, so that the copy overlaps the final true residual.
// slab_ev (optional): b is still arriving, in the t-slabs of slab_t, slab k
// complete at event slab_ev[k].
int solve_impl(wd_op *op, const double *x_in, double *x_out, const double *b, double tol,
               int maxiter, int parity, wd_solve_info *info, double *x_host = nullptr,
               const cudaEvent_t *slab_ev = nullptr) {
    const bool b_slabs = slab_ev != nullptr;
    SolveState st{};
    st.p = parity;
    st.q = 1 - parity;
    const Geom &g = op->g;
    const double n_real = 24.0 * (double)g.vh;
    const bool mixed = op->prec != WD_F64;

    // Alg. schur: split b and the initial guess by parity,
    // bhat_p = b_p + kappa H_pq A^-1 b_q  (A = 1 + i t gamma5, t = 2 kappa mu)
    const double tw = op->twist(0);
    const double inv_norm = 1.0 / (1.0 + tw * tw);
    if (x_in) {
        double *xe = st.p == 0 ? op->xh : op->xq, *xo = st.p == 0 ? op->xq : op->xh;
        WD_CUDA(launch_pack_full(op->hi_prec, g, xe, xo, x_in, op->stream));
    } else {   // all-zero bytes are a zero in FP64 and in double-float
        WD_CUDA(cudaMemsetAsync(op->xh, 0, op->hi_field_bytes(), op->stream));
    }
    const bool pipelined = b_slabs && tw == 0.0;   // (slabs may be empty when Lt < 8)
    if (b_slabs && !pipelined)
        for (int k = 0; k < wd_op::B_SLABS; ++k)
            WD_CUDA(cudaStreamWaitEvent(op->stream, slab_ev[k], 0));
    if (!pipelined) WD_CUDA(launch_pack_full(op->hi_prec, g, op->hb[0], op->hb[1], b, op->stream));
    if (pipelined) {
        WD_TRY(prepare_from_slabs(op, st, b, slab_ev));
    } else if (tw != 0.0) {   // A^-1 b_q = (1 - i t gamma5) b_q / (1 + t^2)
        WD_CUDA(launch_twist_hi(op->hi_prec, g, op->axh, op->hb[st.q], -tw, inv_norm, op->stream));
        WD_TRY(dslash(op, true, st.p, 0, op->bh, op->axh, op->hb[st.p], op->kappa, nullptr));
        st.launches += 1;
        st.bytes += 2 * field_b(op, WD_F64);
    } else {
        WD_TRY(dslash(op, true, st.p, 0, op->bh, op->hb[st.q], op->hb[st.p], op->kappa, nullptr));
    }
    Reduction r1 = reduction(op, FIN_STORE1), r0 = reduction(op, FIN_STORE0),
              r2 = reduction(op, FIN_STORE2), r3 = reduction(op, FIN_STORE3);
    WD_CUDA(launch_norm2(op->hi_prec, g, op->hb[st.q], r1, op->stream));
    WD_CUDA(launch_norm2(op->hi_prec, g, op->hb[st.p], r0, op->stream));
    if (x_in) WD_CUDA(launch_norm2(op->hi_prec, g, op->xh, r2, op->stream));
    WD_CUDA(launch_norm2(op->hi_prec, g, op->bh, r3, op->stream));
    WD_TRY(read_scalars(op));
    if (!x_in) op->sc_host->scratch[2] = 0.0;
    const double nb2 = op->sc_host->scratch[0] + op->sc_host->scratch[1];
    st.nb = std::sqrt(nb2);
    st.target = tol * st.nb;
    st.dslash_hi += 1;
    // packs of b (and the guess), the bhat hop, the norms
    st.launches += x_in ? 7 : 5;
    st.bytes += dslash_b(op, true, true) + (x_in ? 8 : 5) * field_b(op, WD_F64);

    if (op->sc_host->scratch[2] == 0.0) {
        // zero initial guess: r = bhat exactly, no operator application
        WD_CUDA(launch_copy_field(op->rh, op->bh, op->hi_field_bytes(), op->stream));
        st.r_hi = std::sqrt(op->sc_host->scratch[3]);
        st.bytes += 2 * field_b(op, WD_F64);
    } else {
        WD_TRY(true_residual(op, st));
        WD_TRY(read_scalars(op));
        st.r_hi = std::sqrt(op->sc_host->scratch[0]);
    }

    int status = WD_OK;
    int iters = 0;
    if (st.nb == 0.0) {
        WD_CUDA(cudaMemsetAsync(op->xh, 0, op->hi_field_bytes(), op->stream));
        st.th_valid = false;
        st.r_hi = 0.0;
    } else if (st.r_hi > st.target) {
        // inner system: r_lo = scale r_hi, x_lo = 0, p = 0, nz = +inf
        st.scale = (mixed && st.r_hi > 0) ? std::sqrt(n_real) / st.r_hi : 1.0;
        WD_TRY(set_consts(op, st.scale, 1.0 / st.scale, 1.0));
        WD_CUDA(launch_convert_scaled(op->prec, op->rl, op->hi_prec, op->rh, g, op->dev_consts, 0,
                                      op->stream));
        WD_CUDA(cudaMemsetAsync(op->xl, 0, op->lo_field_bytes(), op->stream));
        WD_CUDA(cudaMemsetAsync(op->pl, 0, op->lo_field_bytes(), op->stream));
        SolverScalars init{};
        init.nz = INFINITY;
        *op->sc_host = init;
        WD_CUDA(launch_copy_small(op->sc, op->sc_host_dev, sizeof(SolverScalars), op->stream));
        WD_CUDA(cudaStreamSynchronize(op->stream));
        st.bytes += field_b(op, WD_F64) + field_b(op, op->prec) * 3;
        st.launches += 1;

        const double per_iter_bytes =
            2 * (dslash_b(op, false, false) + dslash_b(op, false, true)) +
            8 * field_b(op, op->prec);
        double r_max_lo = st.r_hi * st.scale;   // iterated residual at the last refresh
        double last_lognr = 2 * std::log(r_max_lo);
        int last_it = 0;
        int batch = 8;
        double best_lo = r_max_lo;              // smallest iterated residual since then
        int best_it = 0;
        for (;;) {
            int n = std::min(batch, maxiter - iters);
            if (n > 0) {
                WD_TRY(run_iterations(op, st.p, n));
                WD_TRY(read_scalars(op));
                iters = op->sc_host->iter;
                st.dslash_lo += 4.0 * n;
                st.launches += 8.0 * n;   // 4 hops, 2 norm finishes, 2 vector updates
                st.bytes += per_iter_bytes * n;
            }
            const SolverScalars &h = *op->sc_host;
            if (h.flags & 1) { status = WD_ERR_BREAKDOWN; break; }
            const double r_lo = std::sqrt(h.nr);
            if (r_lo < best_lo) { best_lo = r_lo; best_it = iters; }
            const bool want_conv = r_lo <= st.target * st.scale;
            // reliable update: the iterated residual fell by ru_delta; defect
            // correction: the inner solve reached its tolerance
            const bool defect = mixed && op->recovery == WD_RECOVER_DEFECT;
            const double delta = defect ? op->dc_delta : op->ru_delta;
            const bool want_ru = mixed && r_lo < delta * r_max_lo;
            const bool stalled = mixed && iters - best_it >= op->stall_iters;
            const bool out_of_iters = iters >= maxiter;
            if (want_conv || want_ru || stalled || out_of_iters) {
                // reliable update: fold x_lo into x_hi, recompute r_hi in FP64
                WD_CUDA(launch_fold_x(op->prec, op->hi_prec, g, op->xh, op->xl, op->pl, op->sc,
                                      op->dev_consts + 1, op->stream));
                st.th_valid = false;
                st.bytes += field_b(op, op->prec) * 3 + field_b(op, WD_F64) * 2;
                st.launches += 1;
                // the residual this refresh expects, r_lo / scale, is still
                // above EARLY_REFRESH_REL ||b||: FP32 arithmetic suffices
                const bool early = mixed && !want_conv && !out_of_iters &&
                                   r_lo > EARLY_REFRESH_REL * st.nb * st.scale;
                WD_TRY(true_residual(op, st, early));
                WD_TRY(read_scalars(op));
                st.r_hi = std::sqrt(op->sc_host->scratch[0]);
                st.ru += 1;
                if (!(st.r_hi == st.r_hi)) { status = WD_ERR_BREAKDOWN; break; }
                if (st.r_hi <= st.target) break;
                if (out_of_iters) { status = WD_ERR_NOT_CONVERGED; break; }
                const double new_scale = mixed ? std::sqrt(n_real) / st.r_hi : 1.0;
                const double ratio = new_scale / st.scale;
                WD_TRY(set_consts(op, new_scale, 1.0 / new_scale, ratio));
                WD_CUDA(launch_convert_scaled(op->prec, op->rl, op->hi_prec, op->rh, g,
                                              op->dev_consts, 0, op->stream));
                if (stalled || defect) {
                    // restart: p = 0 and nz = +inf make the next direction z itself.
                    // Defect correction restarts at every outer step: the inner
                    // CGNR solves Mhat e = r_hi from e = 0 (x_lo was folded
                    // into x_hi and cleared) in a fresh Krylov space.
                    WD_CUDA(cudaMemsetAsync(op->pl, 0, op->lo_field_bytes(), op->stream));
                    op->host_consts[3] = INFINITY;
                    WD_CUDA(launch_copy_small(&op->sc->nz, op->host_consts_dev + 3,
                                              sizeof(double), op->stream));
                    st.restarts += stalled ? 1 : 0;
                } else if (ratio != 1.0) {
                    WD_CUDA(launch_rescale_lo(op->prec, g, op->pl, op->sc, op->dev_consts + 2,
                                              op->stream));
                    st.launches += 1;
                }
                st.bytes += field_b(op, WD_F64) + field_b(op, op->prec) * 3;
                st.launches += 1;
                st.scale = new_scale;
                r_max_lo = st.r_hi * st.scale;
                last_lognr = 2 * std::log(r_max_lo);
                last_it = iters;
                best_lo = r_max_lo;
                best_it = iters;
                batch = 4;
                continue;
            }
            // predict the iterations to the next event from the convergence rate
            const double lognr = std::log(h.nr);
            const int di = iters - last_it;
            int next = 8;
            if (di > 0 && lognr < last_lognr) {
                const double rate = (lognr - last_lognr) / di;   // < 0
                double thr = 2 * std::log(st.target * st.scale);
                if (mixed) {
                    const double d = op->recovery == WD_RECOVER_DEFECT ? op->dc_delta : op->ru_delta;
                    thr = std::max(thr, 2 * std::log(d * r_max_lo));
                }
                next = (int)std::ceil((thr - lognr) / rate);
            }
            last_lognr = lognr;
            last_it = iters;
            batch = std::max(1, std::min(next, 1 << MAX_BATCH_LOG2));
        }
    }

    // reconstruction x_q = A^-1 (b_q + kappa H_qp x_p), then the true residual
    // of the full system: r_p = b_p - (A x_p - kappa H_pq x_q), r_q = b_q -
    // (A x_q - kappa H_qp x_p).  When x_p has not changed since the last
    // residual-arithmetic refresh, that refresh's first hop is still in th:
    // th = A^-1 H_qp x_p (the same kernel on the same input gives the same
    // bits, so recomputing it would check nothing).  Then
    // x_q = A^-1 b_q + kappa th and A x_q - kappa H_qp x_p = A (x_q - kappa th).
    const bool reuse = st.th_valid;
    if (reuse) {
        WD_TRY(reconstruct_from_th(op, st, op->stream));
    } else {
        WD_TRY(dslash(op, true, st.q, 0, op->xq, op->xh, op->hb[st.q], op->kappa, nullptr));
        st.dslash_hi += 1;
        st.bytes += dslash_b(op, true, true);
        if (tw != 0.0) {
            WD_CUDA(launch_twist_hi(op->hi_prec, g, op->xq, op->xq, -tw, inv_norm, op->stream));
            st.launches += 1;
            st.bytes += 2 * field_b(op, WD_F64);
        }
    }
    // x is complete: unpack it now (the residual below reads but never
    // writes xh and xq) and start its download if the caller wants it
    WD_TRY(unpack_and_download(op, st, x_out, x_host, op->stream));
    WD_TRY(dslash(op, true, st.p, 0, op->axh, op->xq, op->xh, -op->kappa, nullptr, tw));
    WD_CUDA(launch_xmy_norm(op->hi_prec, g, op->rh, op->hb[st.p], op->axh, r0, op->stream));
    if (reuse) {
        WD_CUDA(launch_xpay_hi(op->hi_prec, g, op->axh, op->xq, -op->kappa, op->th, op->stream));
        st.bytes += 3 * field_b(op, WD_F64);
        if (tw != 0.0) {
            WD_CUDA(launch_twist_hi(op->hi_prec, g, op->axh, op->axh, tw, 1.0, op->stream));
            st.launches += 1;
            st.bytes += 2 * field_b(op, WD_F64);
        }
    } else {
        WD_TRY(dslash(op, true, st.q, 0, op->axh, op->xh, op->xq, -op->kappa, nullptr, tw));
        st.dslash_hi += 1;
        st.bytes += dslash_b(op, true, true);
    }
    WD_CUDA(launch_xmy_norm(op->hi_prec, g, op->th, op->hb[st.q], op->axh, r1, op->stream));
    WD_TRY(read_scalars(op));
    st.dslash_hi += 1;
    st.launches += 6;
    st.bytes += dslash_b(op, true, true) + 6 * field_b(op, WD_F64) + 4 * field_b(op, WD_F64);
    const double rfull = std::sqrt(op->sc_host->scratch[0] + op->sc_host->scratch[1]);
    if (info) {
        info->iters = iters;
        info->reliable_updates = st.ru;
        info->true_rel_resid = st.nb > 0 ? rfull / st.nb : 0.0;
        info->dslash_lo = st.dslash_lo;
        info->dslash_hi = st.dslash_hi;
        info->bytes = st.bytes;
        info->launches = st.launches;
        info->restarts = st.restarts;
    }
    if (status == WD_OK && st.nb > 0 && rfull > st.target * 1.0000001) {
        // the Schur residual met the target but rounding of the
        // reconstruction did not: report it rather than hide it
        status = WD_ERR_NOT_CONVERGED;
    }
    if (status != WD_OK) fail(status, wd_status_string(status));
    return status;
}

}  // namespace

extern "C" int wd_solve_cg(wd_op *op, double *x, const double *b, double tol, int maxiter,
                           int parity, wd_solve_info *info) {
    auto t0 = std::chrono::steady_clock::now();
    WD_TRY(check_op(op));
    if (!x || !b) return fail(WD_ERR_ARG, "null spinor");
    if (parity != 0 && parity != 1) return fail(WD_ERR_ARG, "parity must be 0 or 1");
    if (!(tol > 0) || maxiter < 0) return fail(WD_ERR_ARG, "tol must be > 0, maxiter >= 0");
    if (info) memset(info, 0, sizeof(*info));
    WD_TRY(fork(op));
    int rc = solve_impl(op, x, x, b, tol, maxiter, parity, info);
    int rj = join(op);
    if (info)
        info->seconds =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return rc != WD_OK ? rc : rj;
}

// Queue the canonical field src (host) into dst (device) in the t-slabs of
// slab_t on the copy stream, recording ev[k] after slab k.
static int upload_slabs(wd_op *op, double *dst, const double *src, const cudaEvent_t *ev) {
    const size_t slice = (size_t)op->g.vh / op->g.L[3] * 2 * 24;   // doubles per time slice
    for (int k = 0; k < wd_op::B_SLABS; ++k) {
        const size_t d0 = slice * slab_t(op, k), d1 = slice * slab_t(op, k + 1);
        if (d1 > d0)
            WD_CUDA(cudaMemcpyAsync(dst + d0, src + d0, (d1 - d0) * sizeof(double),
                                    cudaMemcpyHostToDevice, op->copy_stream));
        WD_CUDA(cudaEventRecord(ev[k], op->copy_stream));
    }
    return WD_OK;
}

// Host-memory solve; with_guess = 0 starts from x = 0 without reading x_host.
// The copies go through the handle's staging buffers with cudaMemcpyAsync
// (DMA, 200 GB/s each way on GB300); the solution's copy runs on a second
// stream while the final true residual is computed.  Reading b and writing x
// from the layout kernels through the mapping of pinned host memory was
// measured slower (55.2 against 49.8 ms per solve at 32^3 x 64).
static int solve_host_impl(wd_op *op, double *x_host, const double *b_host, double tol,
                           int maxiter, int parity, int with_guess, wd_solve_info *info) {
    auto t0 = std::chrono::steady_clock::now();
    WD_TRY(check_op(op));
    if (!x_host || !b_host) return fail(WD_ERR_ARG, "null spinor");
    if (parity != 0 && parity != 1) return fail(WD_ERR_ARG, "parity must be 0 or 1");
    if (!(tol > 0) || maxiter < 0) return fail(WD_ERR_ARG, "tol must be > 0, maxiter >= 0");
    if (info) memset(info, 0, sizeof(*info));
    const size_t bytes = (size_t)2 * op->g.vh * 24 * sizeof(double);
    WD_TRY(fork(op));
    // b goes up in t-slabs on the copy stream; the solve packs each slab as
    // soon as its event fires
    WD_CUDA(cudaStreamWaitEvent(op->copy_stream, op->ev_fork, 0));
    WD_TRY(upload_slabs(op, op->stage_b, b_host, op->ev_b));
    if (with_guess)
        WD_CUDA(cudaMemcpyAsync(op->stage_x, x_host, bytes, cudaMemcpyHostToDevice, op->stream));
    // the solution's download starts inside the solve, once x is complete
    int rc = solve_impl(op, with_guess ? op->stage_x : nullptr, op->stage_x, op->stage_b, tol,
                        maxiter, parity, info, x_host, op->ev_b);
    WD_CUDA(cudaStreamSynchronize(op->copy_stream));
    int rj = join(op);
    if (info)
        info->seconds =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return rc != WD_OK ? rc : rj;
}

extern "C" int wd_solve_cg_host(wd_op *op, double *x_host, const double *b_host, double tol,
                                int maxiter, int parity, wd_solve_info *info) {
    return solve_host_impl(op, x_host, b_host, tol, maxiter, parity, 1, info);
}

extern "C" int wd_solve_cg_host_zero_guess(wd_op *op, double *x_host, const double *b_host,
                                           double tol, int maxiter, int parity,
                                           wd_solve_info *info) {
    return solve_host_impl(op, x_host, b_host, tol, maxiter, parity, 0, info);
}

// A stream of host-memory solves: source k + 1 goes up into the second
// staging buffer while solve k runs, and solution k comes down while solve
// k + 1 runs, so each step costs about one device solve.
extern "C" int wd_solve_cg_host_stream(wd_op *op, int n, double *const *x_host,
                                       const double *const *b_host, double tol, int maxiter,
                                       int parity, wd_solve_info *infos) {
    WD_TRY(check_op(op));
    if (n < 0 || (n > 0 && (!x_host || !b_host)))
        return fail(WD_ERR_ARG, "n must be >= 0 with n solution and source pointers");
    for (int k = 0; k < n; ++k)
        if (!x_host[k] || !b_host[k]) return fail(WD_ERR_ARG, "null spinor in the stream");
    if (parity != 0 && parity != 1) return fail(WD_ERR_ARG, "parity must be 0 or 1");
    if (!(tol > 0) || maxiter < 0) return fail(WD_ERR_ARG, "tol must be > 0, maxiter >= 0");
    if (n == 0) return WD_OK;
    if (!op->stage_b2) {
        WD_TRY(dev_alloc(op, (void **)&op->stage_b2, (size_t)2 * op->g.vh * 24 * sizeof(double)));
        for (cudaEvent_t &e : op->ev_b2)
            WD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    double *stage[2] = {op->stage_b, op->stage_b2};
    const cudaEvent_t *ev[2] = {op->ev_b, op->ev_b2};
    WD_TRY(fork(op));
    WD_CUDA(cudaStreamWaitEvent(op->copy_stream, op->ev_fork, 0));
    WD_TRY(upload_slabs(op, stage[0], b_host[0], ev[0]));
    int rc = WD_OK;
    for (int k = 0; k < n && rc == WD_OK; ++k) {
        auto t0 = std::chrono::steady_clock::now();
        // solve k - 1 has returned, so its staging buffer is free for k + 1
        if (k + 1 < n) rc = upload_slabs(op, stage[(k + 1) & 1], b_host[k + 1], ev[(k + 1) & 1]);
        wd_solve_info *info = infos ? &infos[k] : nullptr;
        if (info) memset(info, 0, sizeof(*info));
        if (rc == WD_OK)
            rc = solve_impl(op, nullptr, op->stage_x, stage[k & 1], tol, maxiter, parity, info,
                            x_host[k], ev[k & 1]);
        if (info)
            info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0)
                                .count();
    }
    cudaError_t e = cudaStreamSynchronize(op->copy_stream);
    int rj = join(op);
    if (rc != WD_OK) return rc;
    if (e != cudaSuccess) return fail(WD_ERR_CUDA, std::string("copy stream: ") + cudaGetErrorString(e));
    return rj;
}
