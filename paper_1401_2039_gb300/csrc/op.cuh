// The operator handle (struct wd_op of include/wd.h), shared by the
// translation units that implement the C ABI.
#pragma once

#include <vector>

#include "dslash.cuh"

// Defaults of the reliable-update scheme (Clark et al. 2010): refresh the
// FP64 residual whenever the iterated residual has fallen by delta since
// the last refresh; restart the Krylov direction when the iterated residual
// has not improved for stall_iters iterations.
constexpr double RU_DELTA_DEFAULT = 0.1;
constexpr int STALL_ITERS_DEFAULT = 200;
constexpr int MAX_BATCH_LOG2 = 5;  // graph batches of 1, 2, ..., 32 iterations
// Defect correction: each inner solve reduces its residual by this factor.
constexpr double DC_DELTA_DEFAULT = 0.1;
// Refreshes whose expected residual is above this fraction of ||b|| compute
// it in FP32 arithmetic (the next refreshes recompute it in double-float).
constexpr double EARLY_REFRESH_REL = 1e-5;

struct wd_op {
    using Geom = wd::Geom;
    using GaugeSet = wd::GaugeSet;
    using SolverScalars = wd::SolverScalars;
    Geom g{};
    double kappa = 0;
    double phase[8] = {};
    int prec = WD_F64, recon = 18;
    int hi_prec = WD_F64;          // residual arithmetic: WD_F64 or wd::WD_DF64 (double-float)
    cudaStream_t user = nullptr;   // caller's stream (nullptr = legacy)
    cudaStream_t stream = nullptr; // work stream owned by the handle
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // host-memory solves: the solution's download overlaps the final residual
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_x = nullptr;
    // the last queued download of stage_x (xd_pending: one was queued); the
    // next unpack into stage_x waits for it
    cudaEvent_t ev_xd = nullptr;
    bool xd_pending = false;
    // host-memory solves: b arrives in t-slabs, one event per slab
    static constexpr int B_SLABS = 8;
    cudaEvent_t ev_b[B_SLABS] = {};
    // streams of host-memory solves: the second staging buffer for b and its
    // slab events (created at the first such call)
    double *stage_b2 = nullptr;
    cudaEvent_t ev_b2[B_SLABS] = {};
    bool gauge_loaded = false;

    GaugeSet gauge_lo;             // storage precision, recon
    GaugeSet gauge_hi;             // FP64, 18 reals (shares gauge_lo when identical)
    bool hi_shared = false;

    // storage-precision fields
    void *fa[2] = {}, *fc[2] = {}, *ftmp = nullptr, *slot[2] = {};
    void *xl = nullptr, *rl = nullptr, *pl = nullptr, *zl = nullptr, *apl = nullptr,
         *tl = nullptr;
    // FP64 fields
    double *hb[2] = {}, *bh = nullptr, *xh = nullptr, *rh = nullptr, *axh = nullptr,
           *th = nullptr, *xq = nullptr;
    // canonical staging for the host-memory solve
    double *stage_x = nullptr, *stage_b = nullptr;

    // reductions
    wd::df64 *partials = nullptr;
    unsigned int *counter = nullptr;
    SolverScalars *sc = nullptr;      // device
    SolverScalars *sc_host = nullptr; // pinned mirror (mapped)
    SolverScalars *sc_host_dev = nullptr;   // its device address
    double *dev_consts = nullptr;     // [0] scale, [1] 1/scale, [2] ratio
    double *host_consts = nullptr;    // pinned staging of dev_consts (mapped)
    double *host_consts_dev = nullptr;      // its device address

    // solver parameters (FP32 inner iterations stay accurate over a deeper
    // residual drop than FP16/BF16 ones)
    double ru_delta = RU_DELTA_DEFAULT;
    // twisted mass mu of D = 1 + 2 i kappa mu gamma5 - kappa H (0: Wilson)
    double mu = 0.0;
    // t = 2 kappa mu of A = 1 + i t gamma5; the adjoint flips its sign
    double twist(int dagger) const { return (dagger ? -2.0 : 2.0) * kappa * mu; }
    int stall_iters = STALL_ITERS_DEFAULT;
    // accuracy recovery of the mixed-precision solve: WD_RECOVER_RELIABLE
    // (reliable updates, the Krylov direction kept across refreshes) or
    // WD_RECOVER_DEFECT (defect correction: every refresh restarts the inner
    // solve on the new residual), and the inner tolerance of the latter
    int recovery = WD_RECOVER_RELIABLE;
    double dc_delta = DC_DELTA_DEFAULT;

    // tuned launch configuration of the hopping term: [0] storage precision,
    // [1] residual arithmetic, [2] storage precision with xpay and fused norm
    int cfg[3] = {0, 0, 0};
    double tune_us[3][8] = {};
    cudaEvent_t ev_t0 = nullptr, ev_t1 = nullptr;

    // CUDA graphs of 2^k CGNR iterations, per solved parity
    cudaGraphExec_t graphs[2][MAX_BATCH_LOG2 + 1] = {};

    std::vector<void *> allocations;

    size_t lo_field_bytes() const { return wd::field_bytes(prec, g.stride, 24); }
    size_t hi_field_bytes() const { return wd::field_bytes(hi_prec, g.stride, 24); }
};

