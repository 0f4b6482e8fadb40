// Batched solves: many right-hand sides on one lattice and several lattices
// of different sizes, advanced in lockstep by persistent kernels.
//
// A batch holds P problems (an operator handle each, up to BT_MAX_PROB) with
// n_p right-hand sides each.  Every (problem, rhs) pair is one "system" with
// its own solver scalars (slot).  Fields of a problem store the n_p
// right-hand sides with the rhs index innermost: element (plane j, site h,
// rhs r) sits at ((j * stride + h) * n_p + r) * 16 bytes.  That is the
// single-field layout with plane stride stride * n_p and site index
// h * n_p + r, so the record loads of the single-field kernels apply as they
// are, consecutive threads (consecutive r, then h) read consecutive 16-byte
// words, and the n_p threads of one site read its eight links once from
// DRAM (the duplicates are served by the same warp request or by L1/L2).
//
// Work is cut into tiles of BT_BLOCK items that never straddle two
// problems; a persistent grid walks the tile table.  Reductions are
// deterministic: each tile sums its items per rhs in a fixed order, each
// block accumulates its tiles per slot in tile order, and the last block to
// finish adds the per-block partials per slot in block order.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <type_traits>

#include "batch_internal.cuh"

namespace wd {

// ------------------------------------------------------------------ vector kernels
// Element-wise kernels walk 16-byte chunks; chunk i of a problem belongs to
// rhs i % nrhs (planes hold stride * nrhs chunks, a multiple of nrhs).
// BT_R:  f = {r, Ap}: r -= a Ap, |r|^2
// BT_PX: f = {p, z, x}: x += a_x p (the step the last iteration still owes
//        x, deferred into this pass over p, as in the single-system
//        solver), then p = z + b p
enum BtOp { BT_R = 0, BT_PX = 1, BT_NORM = 2, BT_RESCALE = 3 };

// c + a b with one rounding where the type has a fused multiply-add
template <typename R> __device__ __forceinline__ R bt_fma(R a, R b, R c) { return fma(a, b, c); }
template <> __device__ __forceinline__ df64 bt_fma<df64>(df64 a, df64 b, df64 c) { return c + a * b; }

template <typename S, typename R, int OP>
__global__ void __launch_bounds__(BT_BLOCK) k_bt_vec(const __grid_constant__ BtArgs a) {
    using C = Chunk16<S, R>;
    __shared__ df64 wv[BT_BLOCK];
    __shared__ df64 wacc[BT_WARPS][BT_MAX_SLOTS];
    __shared__ df64 sacc[BT_MAX_SLOTS];
    constexpr bool RED = OP == BT_R || OP == BT_NORM;
    if (RED) bt_zero_sums(wacc);
    for (long t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const BtProb &P = a.p[bt_problem(a, t)];
        const long item0 = (t - P.tile0) * BT_BLOCK;
        const long i = item0 + threadIdx.x;
        df64 v = 0;
        if (i < P.nitems) {
            SolverScalars *s = &a.scalars[P.slot0 + (int)((unsigned)i % (unsigned)P.nrhs)];
            if (OP == BT_R) {           // f = {r, Ap}: r -= a Ap, |r|^2
                const R al = (R)s->alpha;
                R rv[C::K], av[C::K];
                C::load(P.f[0], i, rv);
                C::load(P.f[1], i, av);
                R sq = 0;
#pragma unroll
                for (int k = 0; k < C::K; ++k) {
                    rv[k] -= al * av[k];
                    sq += rv[k] * rv[k];
                }
                C::store(P.f[0], i, rv);
                v = to_df(sq);
            } else if (OP == BT_PX) {   // f = {p, z, x}: x += a_x p, p = z + b p
                const R ax = (R)s->alpha_x, be = (R)s->beta;
                R pv[C::K], zv[C::K], xv[C::K];
                C::load(P.f[0], i, pv);
                C::load(P.f[1], i, zv);
                C::load(P.f[2], i, xv);
#pragma unroll
                for (int k = 0; k < C::K; ++k) {
                    xv[k] = bt_fma(ax, pv[k], xv[k]);
                    pv[k] = zv[k] + be * pv[k];
                }
                C::store(P.f[2], i, xv);
                C::store(P.f[0], i, pv);
            } else if (OP == BT_NORM) { // f = {v}
                R vv[C::K];
                C::load(P.f[0], i, vv);
                R sq = 0;
#pragma unroll
                for (int k = 0; k < C::K; ++k) sq += vv[k] * vv[k];
                v = to_df(sq);
            } else {                    // f = {p}: p *= ratio[slot]
                const int slot = P.slot0 + (int)((unsigned)i % (unsigned)P.nrhs);
                const R ratio = (R)a.consts[2 * BT_MAX_SLOTS + slot];
                R pv[C::K];
                C::load(P.f[0], i, pv);
#pragma unroll
                for (int k = 0; k < C::K; ++k) pv[k] *= ratio;
                C::store(P.f[0], i, pv);
            }
        }
        if (RED) bt_warp_sums(v, P, item0, wv, wacc);
    }
    if (RED) {
        bt_block_sums(wacc, sacc, a.nslots);
        bt_finish(a, sacc);
    }
}

// High-precision (FP64 or double-float) kernels over 16-byte chunks:
//   XMY:  f = {out, x, y}: out = x - y, |out|^2
//   XPAY: f = {out, y, x}: out = y + scale x
enum BtOp64 { BT64_XMY = 0, BT64_XPAY = 1 };

template <typename H, int OP>
__global__ void __launch_bounds__(BT_BLOCK) k_bt_hi(const __grid_constant__ BtArgs a) {
    using C = Chunk16<H, H>;
    __shared__ df64 wv[BT_BLOCK];
    __shared__ df64 wacc[BT_WARPS][BT_MAX_SLOTS];
    __shared__ df64 sacc[BT_MAX_SLOTS];
    if (OP == BT64_XMY) bt_zero_sums(wacc);
    for (long t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const BtProb &P = a.p[bt_problem(a, t)];
        const long item0 = (t - P.tile0) * BT_BLOCK;
        const long i = item0 + threadIdx.x;
        df64 v = 0;
        if (i < P.nitems) {
            H xv[C::K], yv[C::K], d[C::K];
            C::load(P.f[1], i, xv);
            C::load(P.f[2], i, yv);
            H sq = 0;
#pragma unroll
            for (int k = 0; k < C::K; ++k) {
                if (OP == BT64_XMY) d[k] = xv[k] - yv[k];
                else d[k] = xv[k] + H(P.scale) * yv[k];
                sq += d[k] * d[k];
            }
            C::store(P.f[0], i, d);
            v = to_df(sq);
        }
        if (OP == BT64_XMY) bt_warp_sums(v, P, item0, wv, wacc);
    }
    if (OP == BT64_XMY) {
        bt_block_sums(wacc, sacc, a.nslots);
        bt_finish(a, sacc);
    }
}

// Conversions over (site, rhs) items, with per-slot constants:
//   CONV: f = {out (SO), in (SI)}: out = consts[0][slot] * in
//   FOLD: f = {x_hi (H), x_lo (SI), p (SI)}: x_lo += alpha_x[slot] p (the owed
//         step, with the FMA and rounding of BT_PX), then x_hi +=
//         consts[1][slot] * x_lo; x_lo = 0
template <typename H, typename T> __device__ __forceinline__ H widen(T v) { return H(v); }
template <> __device__ __forceinline__ df64 widen<df64, float>(float v) { return df64(v, 0.0f); }

template <typename SO, typename SI, int FOLD, typename H = double>
__global__ void __launch_bounds__(BT_BLOCK) k_bt_conv(const __grid_constant__ BtArgs a) {
    // intermediate: FP32 unless an FP64 field takes part (GB300's FP64
    // adder is too slow for per-element work); double-float fields convert
    // to and from FP32 on the FP32 pipes
    constexpr bool F64 = std::is_same<SI, double>::value ||
                         (FOLD ? std::is_same<H, double>::value : std::is_same<SO, double>::value);
    using T = std::conditional_t<F64, double, float>;
    for (long t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const BtProb &P = a.p[bt_problem(a, t)];
        const long i = (t - P.tile0) * BT_BLOCK + threadIdx.x;
        if (i >= P.nitems) continue;
        const int slot = P.slot0 + (int)((unsigned)i % (unsigned)P.nrhs);
        const long ss = P.g.stride * P.nrhs;
        T v[24];
        Rec<SI, 24>::template load_coherent<T>(P.f[1], ss, i, v);
        if constexpr (FOLD != 0) {
            H hi[24];
            T pv[24];
            Rec<H, 24>::template load_coherent<H>(P.f[0], ss, i, hi);
            Rec<SI, 24>::template load_coherent<T>(P.f[2], ss, i, pv);
            const H is = H(a.consts[BT_MAX_SLOTS + slot]);
            const T ax = (T)a.scalars[slot].alpha_x;
#pragma unroll
            for (int k = 0; k < 24; ++k) {
                T xl = bt_fma(ax, pv[k], v[k]);
                if constexpr (std::is_same<SI, __half>::value) xl = __half2float(__float2half_rn(xl));
                hi[k] += is * widen<H>(xl);
                v[k] = T(0);
            }
            Rec<H, 24>::store(P.f[0], ss, i, hi);
            Rec<SI, 24>::store(P.f[1], ss, i, v);
        } else {
            const T sc = (T)a.consts[slot];
#pragma unroll
            for (int k = 0; k < 24; ++k) v[k] *= sc;
            Rec<SO, 24>::store(P.f[0], ss, i, v);
        }
    }
}

// rescale also multiplies nz by ratio^2 (one thread per slot)
__global__ void k_bt_rescale_nz(SolverScalars *sc, const double *consts, int nslots) {
    const int s = threadIdx.x;
    if (s < nslots) {
        const double r = consts[2 * BT_MAX_SLOTS + s];
        sc[s].nz *= r * r;
    }
}

// item i of an [nrhs][V] enumeration: rhs r, lexicographic site lex and the
// site's parity.  32-bit arithmetic (volumes stay below 2^31) except for the
// rhs division of items past 2^32.
__device__ __forceinline__ void bt_item_site(const Geom &g, long i, long V, int &r, long &lex,
                                             int &par) {
    if (i < (1L << 32)) {
        const unsigned iu = (unsigned)i, Vu = (unsigned)V;
        r = (int)(iu / Vu);
        lex = (long)(iu - (unsigned)r * Vu);
    } else {
        r = (int)(i / V);
        lex = i - (long)r * V;
    }
    unsigned q = (unsigned)lex;
    unsigned s = q / (unsigned)g.L[0];
    par = (int)(q - s * (unsigned)g.L[0]);
    q = s / (unsigned)g.L[1];
    par += (int)(s - q * (unsigned)g.L[1]);
    s = q / (unsigned)g.L[2];
    par += (int)(q - s * (unsigned)g.L[2]) + (int)s;
    par &= 1;
}

// Canonical [nrhs][V][3][4] complex128 <-> batched FP64 parity fields.
template <typename H>
__global__ void k_bt_pack_full(Geom g, int nrhs, void *even, void *odd, const double *src) {
    const long i = (long)blockIdx.x * BT_BLOCK + threadIdx.x;
    const long V = 2 * g.vh;
    if (i >= V * nrhs) return;
    int r, par;
    long lex;
    bt_item_site(g, i, V, r, lex, par);
    double v[24];
    const double2 *s2 = (const double2 *)(src + i * 24);
    for (int k = 0; k < 12; ++k) { v[2 * k] = s2[k].x; v[2 * k + 1] = s2[k].y; }
    Rec<H, 24>::store(par ? odd : even, g.stride * nrhs, (lex >> 1) * nrhs + r, v);
}

template <typename H>
__global__ void k_bt_unpack_full(Geom g, int nrhs, double *dst, const void *even,
                                 const void *odd) {
    const long i = (long)blockIdx.x * BT_BLOCK + threadIdx.x;
    const long V = 2 * g.vh;
    if (i >= V * nrhs) return;
    int r, par;
    long lex;
    bt_item_site(g, i, V, r, lex, par);
    double v[24];
    Rec<H, 24>::template load_coherent<double>(par ? odd : even, g.stride * nrhs,
                                               (lex >> 1) * nrhs + r, v);
    double2 *d2 = (double2 *)(dst + i * 24);
    for (int k = 0; k < 12; ++k) d2[k] = make_double2(v[2 * k], v[2 * k + 1]);
}

// Canonical half spinors [nrhs][Vh][3][4] <-> a batched field of precision S.
template <typename S, int UNPACK>
__global__ void k_bt_half(Geom g, int nrhs, void *field, double *canon) {
    const long i = (long)blockIdx.x * BT_BLOCK + threadIdx.x;
    if (i >= g.vh * nrhs) return;
    const int r = (int)(i / g.vh);
    const long h = i - (long)r * g.vh;
    double v[24];
    double2 *c2 = (double2 *)(canon + i * 24);
    if (UNPACK) {
        Rec<S, 24>::template load_coherent<double>(field, g.stride * nrhs, h * nrhs + r, v);
        for (int k = 0; k < 12; ++k) c2[k] = make_double2(v[2 * k], v[2 * k + 1]);
    } else {
        for (int k = 0; k < 12; ++k) { v[2 * k] = c2[k].x; v[2 * k + 1] = c2[k].y; }
        Rec<S, 24>::store(field, g.stride * nrhs, h * nrhs + r, v);
    }
}

}  // namespace wd

// =================================================================== host side
#include "op.cuh"

using namespace wd;

static thread_local std::string g_bt_error;
static int bt_fail(int code, const std::string &m) {
    g_bt_error = m;
    return code;
}
#define BT_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return bt_fail(e_ == cudaErrorMemoryAllocation ? WD_ERR_NOMEM : WD_ERR_CUDA,    \
                           std::string(#call) + ": " + cudaGetErrorString(e_));             \
    } while (0)
#define BT_TRY(call)                                                                        \
    do {                                                                                    \
        int rc_ = (call);                                                                   \
        if (rc_ != WD_OK) return rc_;                                                       \
    } while (0)

namespace {

enum Fld { F_XL, F_RL, F_PL, F_ZL, F_APL, F_TL, F_HB0, F_HB1, F_BH, F_XH, F_RH, F_AXH, F_TH,
           F_XQ, F_IO0, F_IO1, N_FLD };
enum Items { IT_SITES, IT_LO_CHUNKS, IT_HI_CHUNKS, IT_HI_D2 };
enum Scale { SC_ONE, SC_KAPPA, SC_MKAPPA, SC_MKAPPA2 };

struct BtFields { void *f[N_FLD]; };

}  // namespace

struct wd_batch {
    int nprob = 0;
    wd_op *ops[BT_MAX_PROB] = {};
    int nrhs[BT_MAX_PROB] = {};
    int slot0[BT_MAX_PROB] = {};
    int nslots = 0;
    int prec = WD_F32, recon = 18;
    int hi_prec = WD_F64;       // residual arithmetic shared by the operators
    cudaStream_t user = nullptr, stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    BtFields fl[BT_MAX_PROB];
    df64 *partials = nullptr;
    unsigned int *counter = nullptr;
    SolverScalars *sc = nullptr, *sc_host = nullptr;
    double *consts = nullptr, *consts_host = nullptr;
    cudaGraphExec_t graphs[2][MAX_BATCH_LOG2 + 1] = {};
    long max_grid = 0;          // blocks the partials buffer holds (SMs x 32)
    unsigned vec_grid = 0;      // persistent grid of the element-wise kernels (SMs x 8)
    // autotuned configuration (BT_CFGS) of the storage-precision hop per
    // variant (BTV_PLAIN, BTV_XPAY_NORM), with every candidate's time and grid
    int cfg[2] = {0, 0};
    double tune_us[2][N_BT_CFG] = {};
    unsigned tune_grid[2][N_BT_CFG] = {};
    std::vector<void *> allocs;
};

namespace {

int bt_alloc(wd_batch *bt, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return bt_fail(WD_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    bt->allocs.push_back(*p);
    BT_CUDA(cudaMemset(*p, 0, bytes));
    return WD_OK;
}

long items_of(const wd_batch *bt, int p, int kind) {
    const wd_op *op = bt->ops[p];
    const long n = bt->nrhs[p];
    switch (kind) {
    case IT_SITES: return op->g.vh * n;
    case IT_LO_CHUNKS: return (long)(24 * prec_bytes(bt->prec) / 16) * op->g.stride * n;
    case IT_HI_CHUNKS: return 12L * op->g.stride * n;
    default: return 12L * op->g.stride * n;   // IT_HI_D2: double2 elements
    }
}

double scale_of(const wd_op *op, int mode) {
    switch (mode) {
    case SC_KAPPA: return op->kappa;
    case SC_MKAPPA: return -op->kappa;
    case SC_MKAPPA2: return -op->kappa * op->kappa;
    default: return 1.0;
    }
}

// Arguments of one batched launch: tile table, fields, per-problem scale.
BtArgs make_args(wd_batch *bt, int kind, int fin, std::initializer_list<int> fields,
                 int scale_mode, bool hi, int out_parity, int tile_items = BT_BLOCK) {
    BtArgs a;
    memset(&a, 0, sizeof(a));
    a.nprob = bt->nprob;
    long tile = 0;
    for (int p = 0; p < bt->nprob; ++p) {
        wd_op *op = bt->ops[p];
        BtProb &P = a.p[p];
        P.g = op->g;
        const GaugeSet &gs = hi ? op->gauge_hi : op->gauge_lo;
        P.gauge_out = (const char *)gs.ptr[out_parity];
        P.gauge_in = (const char *)gs.ptr[1 - out_parity];
        P.dir_bytes = gs.dir_bytes;
        int k = 0;
        for (int fid : fields) P.f[k++] = bt->fl[p].f[fid];
        P.scale = scale_of(op, scale_mode);
        memcpy(P.ph, op->phase, sizeof(P.ph));
        P.phase_on = phase_mask(op->phase);
        P.nrhs = bt->nrhs[p];
        P.div_nrhs = make_divisor((unsigned)P.nrhs);
        P.slot0 = bt->slot0[p];
        P.tile0 = tile;
        P.nitems = items_of(bt, p, kind);
        tile += (P.nitems + tile_items - 1) / tile_items;
    }
    a.ntiles = tile;
    a.parity = out_parity;
    a.fin = fin;
    a.nslots = bt->nslots;
    a.partials = bt->partials;
    a.counter = bt->counter;
    a.scalars = bt->sc;
    a.consts = bt->consts;
    a.max_grid = bt->max_grid;
    return a;
}

// grid of the element-wise kernels: persistent over SMs x 8 blocks of 128
unsigned grid_of(const wd_batch *bt, const BtArgs &a) {
    return (unsigned)std::max<long>(1, std::min<long>(a.ntiles, bt->vec_grid));
}

// items per tile of the storage-precision hop in configuration cfg
int bt_hop_block(int prec, int cfg) {
    if (prec != WD_F32 && prec != WD_F16) return 128;
    return BT_CFGS[cfg].block * (BT_CFGS[cfg].pair ? 2 : 1);
}

// whether configuration cfg can run this batch: pair items need FP32
// storage and an even number of right-hand sides in every problem
bool bt_cfg_applies(const wd_batch *bt, int cfg) {
    if (!BT_CFGS[cfg].pair) return true;
    if (bt->prec != WD_F32) return false;
    for (int p = 0; p < bt->nprob; ++p)
        if (bt->nrhs[p] % 2) return false;
    return true;
}

cudaError_t bt_launch_hop(int prec, int recon, int dagger, int variant, int cfg, const BtArgs &a,
                          cudaStream_t s, unsigned *grid_out = nullptr) {
    const bool r12 = recon == 12;
    switch (prec) {
    case WD_DF64:
        return r12 ? cudaErrorInvalidValue
                   : bt_launch_hop_df64_r18(dagger, variant, cfg, a, s, grid_out);
    case WD_F64:
        return r12 ? bt_launch_hop_f64_r12(dagger, variant, cfg, a, s, grid_out)
                   : bt_launch_hop_f64_r18(dagger, variant, cfg, a, s, grid_out);
    case WD_F32:
        return r12 ? bt_launch_hop_f32_r12(dagger, variant, cfg, a, s, grid_out)
                   : bt_launch_hop_f32_r18(dagger, variant, cfg, a, s, grid_out);
    case WD_F16:
        return r12 ? bt_launch_hop_f16_r12(dagger, variant, cfg, a, s, grid_out)
                   : bt_launch_hop_f16_r18(dagger, variant, cfg, a, s, grid_out);
    default: return cudaErrorInvalidValue;
    }
}

// out = scale * H_{p,q} in  or  x + scale * H_{p,q} in, for every system, in
// the variant's tuned configuration (cfg_override >= 0: that one)
int bt_hop(wd_batch *bt, bool hi, int out_parity, int dagger, int out, int in, int x,
           int scale_mode, int fin, int cfg_override = -1, unsigned *grid_out = nullptr) {
    const bool xpay = x >= 0, norm = fin != FIN_NONE;
    const int variant = !xpay ? BTV_PLAIN : norm ? BTV_XPAY_NORM : BTV_XPAY;
    const int prec = hi ? bt->hi_prec : bt->prec;
    const int recon = hi ? 18 : bt->recon;
    const int cfg = cfg_override >= 0 ? cfg_override
                                      : (variant == BTV_XPAY ? 0 : bt->cfg[variant]);
    const int tile = variant == BTV_XPAY ? 128 : bt_hop_block(prec, cfg);
    BtArgs a = xpay ? make_args(bt, IT_SITES, fin, {out, in, x}, scale_mode, hi, out_parity, tile)
                    : make_args(bt, IT_SITES, fin, {out, in}, scale_mode, hi, out_parity, tile);
    BT_CUDA(bt_launch_hop(prec, recon, dagger, variant, cfg, a, bt->stream, grid_out));
    return WD_OK;
}

int bt_schur(wd_batch *bt, bool hi, int p, int dagger, int out, int in, int tmp, int fin) {
    BT_TRY(bt_hop(bt, hi, 1 - p, dagger, tmp, in, -1, SC_ONE, FIN_NONE));
    BT_TRY(bt_hop(bt, hi, p, dagger, out, tmp, in, SC_MKAPPA2, fin));
    return WD_OK;
}

template <int OP>
int bt_vec(wd_batch *bt, bool hi, int fin, std::initializer_list<int> fields) {
    BtArgs a = make_args(bt, hi ? IT_HI_CHUNKS : IT_LO_CHUNKS, fin, fields, SC_ONE, false, 0);
    const int prec = hi ? bt->hi_prec : bt->prec;
    const unsigned gr = grid_of(bt, a);
    if (prec == WD_DF64) k_bt_vec<df64, df64, OP><<<gr, BT_BLOCK, 0, bt->stream>>>(a);
    else if (prec == WD_F64) k_bt_vec<double, double, OP><<<gr, BT_BLOCK, 0, bt->stream>>>(a);
    else if (prec == WD_F32) k_bt_vec<float, float, OP><<<gr, BT_BLOCK, 0, bt->stream>>>(a);
    else k_bt_vec<__half, float, OP><<<gr, BT_BLOCK, 0, bt->stream>>>(a);
    BT_CUDA(cudaGetLastError());
    return WD_OK;
}

template <int OP>
int bt_f64(wd_batch *bt, int fin, std::initializer_list<int> fields, int scale_mode) {
    BtArgs a = make_args(bt, IT_HI_D2, fin, fields, scale_mode, false, 0);
    if (bt->hi_prec == WD_DF64) k_bt_hi<df64, OP><<<grid_of(bt, a), BT_BLOCK, 0, bt->stream>>>(a);
    else k_bt_hi<double, OP><<<grid_of(bt, a), BT_BLOCK, 0, bt->stream>>>(a);
    BT_CUDA(cudaGetLastError());
    return WD_OK;
}

// lo <- consts[0] * hi  (FOLD = 0)   or   lo += alpha_x p, hi += consts[1] * lo,
// lo = 0  (FOLD = 1; the caller then zeroes alpha_x)
int bt_conv(wd_batch *bt, bool fold, int dst, int src) {
    BtArgs a = fold ? make_args(bt, IT_SITES, FIN_NONE, {dst, src, F_PL}, SC_ONE, false, 0)
                    : make_args(bt, IT_SITES, FIN_NONE, {dst, src}, SC_ONE, false, 0);
    const unsigned gr = grid_of(bt, a);
    cudaStream_t s = bt->stream;
    const bool df = bt->hi_prec == WD_DF64;
    if (fold) {
        if (bt->prec == WD_F64) k_bt_conv<double, double, 1><<<gr, BT_BLOCK, 0, s>>>(a);
        else if (bt->prec == WD_F32) {
            if (df) k_bt_conv<double, float, 1, df64><<<gr, BT_BLOCK, 0, s>>>(a);
            else k_bt_conv<double, float, 1><<<gr, BT_BLOCK, 0, s>>>(a);
        } else {
            if (df) k_bt_conv<double, __half, 1, df64><<<gr, BT_BLOCK, 0, s>>>(a);
            else k_bt_conv<double, __half, 1><<<gr, BT_BLOCK, 0, s>>>(a);
        }
    } else {
        if (bt->prec == WD_F64) k_bt_conv<double, double, 0><<<gr, BT_BLOCK, 0, s>>>(a);
        else if (bt->prec == WD_F32) {
            if (df) k_bt_conv<float, df64, 0><<<gr, BT_BLOCK, 0, s>>>(a);
            else k_bt_conv<float, double, 0><<<gr, BT_BLOCK, 0, s>>>(a);
        } else {
            if (df) k_bt_conv<__half, df64, 0><<<gr, BT_BLOCK, 0, s>>>(a);
            else k_bt_conv<__half, double, 0><<<gr, BT_BLOCK, 0, s>>>(a);
        }
    }
    BT_CUDA(cudaGetLastError());
    return WD_OK;
}

int bt_read(wd_batch *bt) {
    BT_CUDA(cudaMemcpyAsync(bt->sc_host, bt->sc, sizeof(SolverScalars) * bt->nslots,
                            cudaMemcpyDeviceToHost, bt->stream));
    BT_CUDA(cudaStreamSynchronize(bt->stream));
    return WD_OK;
}

int bt_write(wd_batch *bt) {
    BT_CUDA(cudaMemcpyAsync(bt->sc, bt->sc_host, sizeof(SolverScalars) * bt->nslots,
                            cudaMemcpyHostToDevice, bt->stream));
    BT_CUDA(cudaMemcpyAsync(bt->consts, bt->consts_host, sizeof(double) * 4 * BT_MAX_SLOTS,
                            cudaMemcpyHostToDevice, bt->stream));
    return WD_OK;
}

// one lockstep CGNR iteration for every system (see cg_iteration of the
// single-system solver)
int bt_iteration(wd_batch *bt, int p) {
    BT_TRY(bt_schur(bt, false, p, 1, F_ZL, F_RL, F_TL, FIN_BETA));
    BT_TRY(bt_vec<BT_PX>(bt, false, FIN_NONE, {F_PL, F_ZL, F_XL}));
    BT_TRY(bt_schur(bt, false, p, 0, F_APL, F_PL, F_TL, FIN_ALPHA));
    BT_TRY(bt_vec<BT_R>(bt, false, FIN_NR, {F_RL, F_APL}));
    return WD_OK;
}

int bt_run(wd_batch *bt, int p, int n) {
    for (int lg = MAX_BATCH_LOG2; lg >= 0; --lg) {
        while (n >= (1 << lg)) {
            if (!bt->graphs[p][lg]) {
                cudaGraph_t graph = nullptr;
                BT_CUDA(cudaStreamBeginCapture(bt->stream, cudaStreamCaptureModeThreadLocal));
                int rc = WD_OK;
                for (int i = 0; i < (1 << lg) && rc == WD_OK; ++i) rc = bt_iteration(bt, p);
                cudaError_t e = cudaStreamEndCapture(bt->stream, &graph);
                if (rc != WD_OK) {
                    if (graph) cudaGraphDestroy(graph);
                    return rc;
                }
                BT_CUDA(e);
                cudaError_t ei = cudaGraphInstantiate(&bt->graphs[p][lg], graph, 0);
                cudaGraphDestroy(graph);
                BT_CUDA(ei);
            }
            BT_CUDA(cudaGraphLaunch(bt->graphs[p][lg], bt->stream));
            n -= 1 << lg;
        }
    }
    return WD_OK;
}

// r_hi = bhat - Mhat x_hi for every system, |r_hi|^2 -> scratch[0]
int bt_true_residual(wd_batch *bt, int p) {
    BT_TRY(bt_schur(bt, true, p, 0, F_AXH, F_XH, F_TH, FIN_NONE));
    BT_TRY(bt_f64<BT64_XMY>(bt, FIN_STORE0, {F_RH, F_BH, F_AXH}, SC_ONE));
    return WD_OK;
}

int bt_solve_impl(wd_batch *bt, double *const *x, const double *const *b, double tol,
                  int maxiter, int par, wd_solve_info *info) {
    const int q = 1 - par;
    const bool mixed = bt->prec != WD_F64;
    const int S = bt->nslots;
    std::vector<double> nb(S), target(S), r_hi(S), scale(S, 1.0), rmax(S), best(S);
    std::vector<int> best_it(S, 0), conv_iter(S, 0);
    std::vector<char> active(S, 0);
    cudaStream_t st = bt->stream;
    // split b and x0 by parity into the FP64 batched fields
    for (int p = 0; p < bt->nprob; ++p) {
        const wd_op *op = bt->ops[p];
        const long n = 2 * op->g.vh * bt->nrhs[p];
        const unsigned gr = (unsigned)((n + BT_BLOCK - 1) / BT_BLOCK);
        double *xe = (double *)bt->fl[p].f[par == 0 ? F_XH : F_XQ];
        double *xo = (double *)bt->fl[p].f[par == 0 ? F_XQ : F_XH];
        if (bt->hi_prec == WD_DF64) {
            k_bt_pack_full<df64><<<gr, BT_BLOCK, 0, st>>>(op->g, bt->nrhs[p], bt->fl[p].f[F_HB0],
                                                          bt->fl[p].f[F_HB1], b[p]);
            k_bt_pack_full<df64><<<gr, BT_BLOCK, 0, st>>>(op->g, bt->nrhs[p], xe, xo, x[p]);
        } else {
            k_bt_pack_full<double><<<gr, BT_BLOCK, 0, st>>>(op->g, bt->nrhs[p], bt->fl[p].f[F_HB0],
                                                            bt->fl[p].f[F_HB1], b[p]);
            k_bt_pack_full<double><<<gr, BT_BLOCK, 0, st>>>(op->g, bt->nrhs[p], xe, xo, x[p]);
        }
    }
    BT_CUDA(cudaGetLastError());
    const int HBP = par == 0 ? F_HB0 : F_HB1, HBQ = par == 0 ? F_HB1 : F_HB0;
    BT_TRY(bt_hop(bt, true, par, 0, F_BH, HBQ, HBP, SC_KAPPA, FIN_NONE));
    BT_TRY(bt_vec<BT_NORM>(bt, true, FIN_STORE1, {HBQ}));
    BT_TRY(bt_vec<BT_NORM>(bt, true, FIN_STORE0, {HBP}));
    BT_TRY(bt_vec<BT_NORM>(bt, true, FIN_STORE2, {F_XH}));
    BT_TRY(bt_vec<BT_NORM>(bt, true, FIN_STORE3, {F_BH}));
    BT_TRY(bt_read(bt));
    bool any_guess = false;
    for (int s = 0; s < S; ++s) {
        nb[s] = std::sqrt(bt->sc_host[s].scratch[0] + bt->sc_host[s].scratch[1]);
        target[s] = tol * nb[s];
        any_guess |= bt->sc_host[s].scratch[2] != 0.0;
        r_hi[s] = std::sqrt(bt->sc_host[s].scratch[3]);
    }
    if (any_guess) {
        BT_TRY(bt_true_residual(bt, par));
        BT_TRY(bt_read(bt));
        for (int s = 0; s < S; ++s) r_hi[s] = std::sqrt(bt->sc_host[s].scratch[0]);
    } else {
        for (int p = 0; p < bt->nprob; ++p)
            BT_CUDA(cudaMemcpyAsync(bt->fl[p].f[F_RH], bt->fl[p].f[F_BH],
                                    field_bytes(WD_F64, bt->ops[p]->g.stride, 24) * bt->nrhs[p],
                                    cudaMemcpyDeviceToDevice, st));
    }
    int n_active = 0;
    for (int p = 0; p < bt->nprob; ++p)
        for (int r = 0; r < bt->nrhs[p]; ++r) {
            const int s = bt->slot0[p] + r;
            const double n_real = 24.0 * bt->ops[p]->g.vh;
            active[s] = nb[s] > 0 && r_hi[s] > target[s];
            n_active += active[s];
            scale[s] = (mixed && active[s]) ? std::sqrt(n_real) / r_hi[s] : 1.0;
            rmax[s] = best[s] = r_hi[s] * scale[s];
            SolverScalars z{};
            z.nz = INFINITY;
            z.frozen = !active[s];
            bt->sc_host[s] = z;
            bt->consts_host[s] = scale[s];
            bt->consts_host[BT_MAX_SLOTS + s] = 1.0 / scale[s];
            bt->consts_host[2 * BT_MAX_SLOTS + s] = 1.0;
        }
    BT_TRY(bt_write(bt));
    BT_TRY(bt_conv(bt, false, F_RL, F_RH));
    for (int p = 0; p < bt->nprob; ++p) {
        const size_t lo = field_bytes(bt->prec, bt->ops[p]->g.stride, 24) * bt->nrhs[p];
        BT_CUDA(cudaMemsetAsync(bt->fl[p].f[F_XL], 0, lo, st));
        BT_CUDA(cudaMemsetAsync(bt->fl[p].f[F_PL], 0, lo, st));
    }
    int iters = 0, ru = 0, status = WD_OK;
    bool th_valid = any_guess;
    // accuracy recovery of the first operator for every system: reliable
    // updates (refresh after a residual drop of ru_delta, Krylov directions
    // kept) or defect correction (after a drop of the inner tolerance, and
    // every system restarts its inner CGNR on the new residual)
    const bool defect = mixed && bt->ops[0]->recovery == WD_RECOVER_DEFECT;
    const double delta = defect ? bt->ops[0]->dc_delta : bt->ops[0]->ru_delta;
    int batch = 8;
    while (n_active > 0) {
        const int n = std::min(batch, maxiter - iters);
        if (n > 0) {
            BT_TRY(bt_run(bt, par, n));
            iters += n;
        }
        BT_TRY(bt_read(bt));
        bool trigger = iters >= maxiter;
        int next = 1 << MAX_BATCH_LOG2;
        for (int s = 0; s < S; ++s) {
            if (!active[s]) continue;
            const SolverScalars &h = bt->sc_host[s];
            if (h.flags & 1) { status = WD_ERR_BREAKDOWN; trigger = true; }
            const double r = std::sqrt(h.nr);
            if (r <= target[s] * scale[s] || (mixed && r < delta * rmax[s])) trigger = true;
            if (r < best[s]) { best[s] = r; best_it[s] = iters; }
        }
        if (status != WD_OK) break;
        if (trigger) {
            BT_TRY(bt_conv(bt, true, F_XH, F_XL));
            BT_TRY(bt_true_residual(bt, par));
            BT_TRY(bt_read(bt));
            th_valid = true;
            ru += 1;
            for (int s = 0; s < S; ++s) bt->sc_host[s].alpha_x = 0.0;   // settled by the fold
            for (int s = 0; s < S; ++s) {
                if (!active[s]) continue;
                r_hi[s] = std::sqrt(bt->sc_host[s].scratch[0]);
                if (!(r_hi[s] == r_hi[s])) { status = WD_ERR_BREAKDOWN; break; }
                double ratio = 1.0;
                if (r_hi[s] <= target[s]) {
                    active[s] = 0;
                    n_active -= 1;
                    bt->sc_host[s].frozen = 1;
                    conv_iter[s] = iters;
                } else {
                    int p = 0;
                    while (p + 1 < bt->nprob && s >= bt->slot0[p + 1]) ++p;
                    const double ns = mixed ? std::sqrt(24.0 * bt->ops[p]->g.vh) / r_hi[s] : 1.0;
                    ratio = ns / scale[s];
                    scale[s] = ns;
                    rmax[s] = best[s] = r_hi[s] * ns;
                    best_it[s] = iters;
                }
                bt->consts_host[s] = scale[s];
                bt->consts_host[BT_MAX_SLOTS + s] = 1.0 / scale[s];
                bt->consts_host[2 * BT_MAX_SLOTS + s] = ratio;
            }
            if (status != WD_OK) break;
            if (n_active == 0) break;
            if (iters >= maxiter) { status = WD_ERR_NOT_CONVERGED; break; }
            if (defect)   // restart: p = 0 and nz = +inf make the next direction z itself
                for (int s = 0; s < S; ++s)
                    if (active[s]) bt->sc_host[s].nz = INFINITY;
            BT_TRY(bt_write(bt));
            BT_TRY(bt_conv(bt, false, F_RL, F_RH));
            if (defect) {
                for (int p = 0; p < bt->nprob; ++p)
                    BT_CUDA(cudaMemsetAsync(bt->fl[p].f[F_PL], 0,
                                            field_bytes(bt->prec, bt->ops[p]->g.stride, 24) *
                                                bt->nrhs[p], st));
            } else {
                BT_TRY(bt_vec<BT_RESCALE>(bt, false, FIN_NONE, {F_PL}));
                k_bt_rescale_nz<<<1, BT_MAX_SLOTS, 0, st>>>(bt->sc, bt->consts, S);
                BT_CUDA(cudaGetLastError());
            }
            batch = 4;
            continue;
        }
        // next checkpoint: the earliest predicted event over the active systems
        for (int s = 0; s < S; ++s) {
            if (!active[s]) continue;
            const SolverScalars &h = bt->sc_host[s];
            const int k = h.iter;
            if (k < 2) { next = std::min(next, 8); continue; }
            const double l1 = std::log(h.hist[(k - 1) & 63]), l0 = std::log(h.hist[(k - 2) & 63]);
            const double rate = l1 - l0;
            double thr = 2 * std::log(target[s] * scale[s]);
            if (mixed) thr = std::max(thr, 2 * std::log(delta * rmax[s]));
            const int pred = rate < 0 ? (int)std::ceil((thr - l1) / rate) : 8;
            next = std::min(next, std::max(1, pred));
        }
        batch = std::max(1, std::min(next, 1 << MAX_BATCH_LOG2));
    }
    // reconstruction and the FP64 true residual of every full system
    if (th_valid) BT_TRY(bt_f64<BT64_XPAY>(bt, FIN_NONE, {F_XQ, HBQ, F_TH}, SC_KAPPA));
    else BT_TRY(bt_hop(bt, true, q, 0, F_XQ, F_XH, HBQ, SC_KAPPA, FIN_NONE));
    BT_TRY(bt_hop(bt, true, par, 0, F_AXH, F_XQ, F_XH, SC_MKAPPA, FIN_NONE));
    BT_TRY(bt_f64<BT64_XMY>(bt, FIN_STORE0, {F_RH, HBP, F_AXH}, SC_ONE));
    BT_TRY(bt_hop(bt, true, q, 0, F_AXH, F_XH, F_XQ, SC_MKAPPA, FIN_NONE));
    BT_TRY(bt_f64<BT64_XMY>(bt, FIN_STORE1, {F_TH, HBQ, F_AXH}, SC_ONE));
    for (int p = 0; p < bt->nprob; ++p) {
        const wd_op *op = bt->ops[p];
        const long n = 2 * op->g.vh * bt->nrhs[p];
        const unsigned gr = (unsigned)((n + BT_BLOCK - 1) / BT_BLOCK);
        const double *xe = (const double *)bt->fl[p].f[par == 0 ? F_XH : F_XQ];
        const double *xo = (const double *)bt->fl[p].f[par == 0 ? F_XQ : F_XH];
        if (bt->hi_prec == WD_DF64)
            k_bt_unpack_full<df64><<<gr, BT_BLOCK, 0, st>>>(op->g, bt->nrhs[p], x[p], xe, xo);
        else
            k_bt_unpack_full<double><<<gr, BT_BLOCK, 0, st>>>(op->g, bt->nrhs[p], x[p], xe, xo);
    }
    BT_CUDA(cudaGetLastError());
    BT_TRY(bt_read(bt));
    bool all_ok = true;
    for (int s = 0; s < S; ++s) {
        const double rf = std::sqrt(bt->sc_host[s].scratch[0] + bt->sc_host[s].scratch[1]);
        const double rel = nb[s] > 0 ? rf / nb[s] : 0.0;
        if (nb[s] > 0 && rf > target[s] * 1.0000001) all_ok = false;
        if (info) {
            info[s].iters = active[s] ? iters : conv_iter[s];
            info[s].reliable_updates = ru;
            info[s].true_rel_resid = rel;
        }
    }
    if (status == WD_OK && !all_ok) status = WD_ERR_NOT_CONVERGED;
    if (status != WD_OK) bt_fail(status, wd_status_string(status));
    return status;
}

}  // namespace

extern "C" {

const char *wd_batch_last_error(void) { return g_bt_error.c_str(); }

void wd_batch_destroy(wd_batch *bt) {
    if (!bt) return;
    if (bt->stream) cudaStreamSynchronize(bt->stream);
    for (auto &row : bt->graphs)
        for (auto &ge : row)
            if (ge) cudaGraphExecDestroy(ge);
    for (void *p : bt->allocs) cudaFree(p);
    if (bt->sc_host) cudaFreeHost(bt->sc_host);
    if (bt->consts_host) cudaFreeHost(bt->consts_host);
    if (bt->ev_fork) cudaEventDestroy(bt->ev_fork);
    if (bt->ev_join) cudaEventDestroy(bt->ev_join);
    if (bt->stream) cudaStreamDestroy(bt->stream);
    delete bt;
}

// Autotuner of the storage-precision batched hop: every configuration of
// BT_CFGS (threads per block, register cap; grid = the kernel's resident
// capacity) is timed on this batch's own lattices and right-hand sides, the
// plain hop and the norm-fused xpay hop of the Schur operator separately
// (two warm-up and five timed launches on the resident fields, CUDA events
// on the batch stream), and the fastest kept.  The per-system norms add in
// an order fixed by the configuration (tile size and grid), so solves with
// the same configuration repeat bit for bit.  WD_BATCH_CFG=k forces
// configuration k, WD_TUNE=0 keeps configuration 0.
static int bt_tune(wd_batch *bt) {
    if (bt->prec != WD_F32 && bt->prec != WD_F16) return WD_OK;
    const char *force = getenv("WD_BATCH_CFG");
    const char *tune = getenv("WD_TUNE");
    if (force || (tune && tune[0] == '0')) {
        const int k = force ? atoi(force) : 0;
        bt->cfg[0] = bt->cfg[1] = (k >= 0 && k < N_BT_CFG && bt_cfg_applies(bt, k)) ? k : 0;
        return WD_OK;
    }
    cudaEvent_t e0, e1;
    BT_CUDA(cudaEventCreate(&e0));
    BT_CUDA(cudaEventCreate(&e1));
    int rc = WD_OK;
    for (int v = 0; v < 2 && rc == WD_OK; ++v) {
        float best = 1e30f;
        for (int k = 0; k < N_BT_CFG && rc == WD_OK; ++k) {
            bt->tune_us[v][k] = 0.0;
            if (!bt_cfg_applies(bt, k)) continue;
            auto launch = [&](int par) {
                return v == BTV_PLAIN
                           ? bt_hop(bt, false, par, 0, F_IO1, F_IO0, -1, SC_ONE, FIN_NONE, k,
                                    &bt->tune_grid[v][k])
                           : bt_hop(bt, false, par, 0, F_IO1, F_IO0, F_IO1, SC_MKAPPA2, FIN_STORE0,
                                    k, &bt->tune_grid[v][k]);
            };
            for (int w = 0; w < 2 && rc == WD_OK; ++w) rc = launch(w & 1);
            if (rc != WD_OK) break;
            if (cudaEventRecord(e0, bt->stream) != cudaSuccess) { rc = bt_fail(WD_ERR_CUDA, "event"); break; }
            for (int r = 0; r < 5 && rc == WD_OK; ++r) rc = launch(r & 1);
            if (rc != WD_OK) break;
            float ms = 0;
            if (cudaEventRecord(e1, bt->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = bt_fail(WD_ERR_CUDA, "event timing of the batch autotuner");
                break;
            }
            bt->tune_us[v][k] = ms * 1e3 / 5;
            if (ms < best) { best = ms; bt->cfg[v] = k; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

static int batch_create_impl(wd_batch *bt) {
    BT_CUDA(cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking));
    BT_CUDA(cudaEventCreateWithFlags(&bt->ev_fork, cudaEventDisableTiming));
    BT_CUDA(cudaEventCreateWithFlags(&bt->ev_join, cudaEventDisableTiming));
    for (int p = 0; p < bt->nprob; ++p) {
        const wd_op *op = bt->ops[p];
        const size_t lo = field_bytes(bt->prec, op->g.stride, 24) * bt->nrhs[p];
        const size_t hi = field_bytes(WD_F64, op->g.stride, 24) * bt->nrhs[p];
        for (int f = 0; f < N_FLD; ++f) {
            const bool is_lo = f <= F_TL || f == F_IO0 || f == F_IO1;
            BT_TRY(bt_alloc(bt, &bt->fl[p].f[f], is_lo ? lo : hi));
        }
    }
    int dev = 0, sms = 1;
    BT_CUDA(cudaGetDevice(&dev));
    BT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    bt->max_grid = (long)sms * BT_BLOCKS_PER_SM_MAX;
    bt->vec_grid = (unsigned)sms * 8;
    BT_TRY(bt_alloc(bt, (void **)&bt->partials, sizeof(df64) * bt->max_grid * BT_MAX_SLOTS));
    BT_TRY(bt_alloc(bt, (void **)&bt->counter, sizeof(unsigned int) * ARRIVE_WORDS));
    BT_TRY(bt_alloc(bt, (void **)&bt->sc, sizeof(SolverScalars) * BT_MAX_SLOTS));
    BT_TRY(bt_alloc(bt, (void **)&bt->consts, sizeof(double) * 4 * BT_MAX_SLOTS));
    BT_CUDA(cudaMallocHost((void **)&bt->sc_host, sizeof(SolverScalars) * BT_MAX_SLOTS));
    BT_CUDA(cudaMallocHost((void **)&bt->consts_host, sizeof(double) * 4 * BT_MAX_SLOTS));
    BT_CUDA(cudaDeviceSynchronize());
    return bt_tune(bt);
}

int wd_batch_create(wd_batch **out, wd_op *const *ops, const int *nrhs, int nops) {
    if (!out || !ops || !nrhs) return bt_fail(WD_ERR_ARG, "null argument to wd_batch_create");
    *out = nullptr;
    if (nops < 1 || nops > BT_MAX_PROB)
        return bt_fail(WD_ERR_ARG, "a batch holds 1 to 8 operators");
    int slots = 0;
    for (int p = 0; p < nops; ++p) {
        if (!ops[p] || !ops[p]->gauge_loaded)
            return bt_fail(WD_ERR_STATE, "every operator needs its gauge field loaded");
        if (nrhs[p] < 1) return bt_fail(WD_ERR_ARG, "nrhs must be >= 1");
        if (ops[p]->mu != 0.0)
            return bt_fail(WD_ERR_ARG, "batches have no twisted mass (mu must be 0)");
        if (ops[p]->prec != ops[0]->prec || ops[p]->recon != ops[0]->recon ||
            ops[p]->hi_prec != ops[0]->hi_prec)
            return bt_fail(WD_ERR_ARG,
                           "operators of a batch share precision, recon and residual precision");
        slots += nrhs[p];
    }
    if (ops[0]->prec == WD_BF16) return bt_fail(WD_ERR_ARG, "batches support FP64/FP32/FP16");
    if (slots > BT_MAX_SLOTS) return bt_fail(WD_ERR_ARG, "at most 64 systems per batch");
    wd_batch *bt = new wd_batch();
    bt->nprob = nops;
    bt->prec = ops[0]->prec;
    bt->recon = ops[0]->recon;
    bt->hi_prec = ops[0]->hi_prec;
    bt->user = ops[0]->user;
    int s = 0;
    for (int p = 0; p < nops; ++p) {
        bt->ops[p] = ops[p];
        bt->nrhs[p] = nrhs[p];
        bt->slot0[p] = s;
        s += nrhs[p];
    }
    bt->nslots = s;
    int rc = batch_create_impl(bt);
    if (rc != WD_OK) {
        std::string m = g_bt_error;
        wd_batch_destroy(bt);
        g_bt_error = m;
        return rc;
    }
    *out = bt;
    return WD_OK;
}

static int bt_fork(wd_batch *bt) {
    BT_CUDA(cudaEventRecord(bt->ev_fork, bt->user));
    BT_CUDA(cudaStreamWaitEvent(bt->stream, bt->ev_fork, 0));
    return WD_OK;
}
static int bt_join(wd_batch *bt) {
    BT_CUDA(cudaEventRecord(bt->ev_join, bt->stream));
    BT_CUDA(cudaStreamWaitEvent(bt->user, bt->ev_join, 0));
    return WD_OK;
}

int wd_batch_dslash(wd_batch *bt, double *const *out, const double *const *in, int out_parity,
                    int dagger) {
    if (!bt || !out || !in) return bt_fail(WD_ERR_ARG, "null argument to wd_batch_dslash");
    if (out_parity != 0 && out_parity != 1) return bt_fail(WD_ERR_ARG, "parity must be 0 or 1");
    if (dagger != 0 && dagger != 1) return bt_fail(WD_ERR_ARG, "dagger must be 0 or 1");
    for (int p = 0; p < bt->nprob; ++p)
        if (bt->ops[p]->mu != 0.0)
            return bt_fail(WD_ERR_ARG, "batches have no twisted mass (mu must be 0)");
    BT_TRY(bt_fork(bt));
    for (int p = 0; p < bt->nprob; ++p) {
        const wd_op *op = bt->ops[p];
        const long n = op->g.vh * bt->nrhs[p];
        const unsigned gr = (unsigned)((n + BT_BLOCK - 1) / BT_BLOCK);
        void *f = bt->fl[p].f[F_IO0];
        double *c = (double *)in[p];
        if (bt->prec == WD_F64) k_bt_half<double, 0><<<gr, BT_BLOCK, 0, bt->stream>>>(op->g, bt->nrhs[p], f, c);
        else if (bt->prec == WD_F32) k_bt_half<float, 0><<<gr, BT_BLOCK, 0, bt->stream>>>(op->g, bt->nrhs[p], f, c);
        else k_bt_half<__half, 0><<<gr, BT_BLOCK, 0, bt->stream>>>(op->g, bt->nrhs[p], f, c);
    }
    BT_CUDA(cudaGetLastError());
    BT_TRY(bt_hop(bt, false, out_parity, dagger, F_IO1, F_IO0, -1, SC_ONE, FIN_NONE));
    for (int p = 0; p < bt->nprob; ++p) {
        const wd_op *op = bt->ops[p];
        const long n = op->g.vh * bt->nrhs[p];
        const unsigned gr = (unsigned)((n + BT_BLOCK - 1) / BT_BLOCK);
        void *f = bt->fl[p].f[F_IO1];
        if (bt->prec == WD_F64) k_bt_half<double, 1><<<gr, BT_BLOCK, 0, bt->stream>>>(op->g, bt->nrhs[p], f, out[p]);
        else if (bt->prec == WD_F32) k_bt_half<float, 1><<<gr, BT_BLOCK, 0, bt->stream>>>(op->g, bt->nrhs[p], f, out[p]);
        else k_bt_half<__half, 1><<<gr, BT_BLOCK, 0, bt->stream>>>(op->g, bt->nrhs[p], f, out[p]);
    }
    BT_CUDA(cudaGetLastError());
    return bt_join(bt);
}

int wd_batch_tuning(const wd_batch *bt, int variant, double *us, int n, int *block,
                    int *min_blocks, int *grid) {
    if (!bt || variant < 0 || variant > 1) return -1;
    const int k = bt->cfg[variant];
    for (int i = 0; us && i < n && i < N_BT_CFG; ++i) us[i] = bt->tune_us[variant][i];
    if (block) *block = BT_CFGS[k].block;
    if (min_blocks) *min_blocks = BT_CFGS[k].minb;
    if (grid) *grid = (int)bt->tune_grid[variant][k];
    return k;
}

int wd_batch_dslash_resident(wd_batch *bt, int out_parity, int dagger) {
    if (!bt) return bt_fail(WD_ERR_ARG, "null batch");
    BT_TRY(bt_fork(bt));
    BT_TRY(bt_hop(bt, false, out_parity, dagger, F_IO1, F_IO0, -1, SC_ONE, FIN_NONE));
    return bt_join(bt);
}

int wd_batch_solve(wd_batch *bt, double *const *x, const double *const *b, double tol,
                   int maxiter, int parity, wd_solve_info *info) {
    auto t0 = std::chrono::steady_clock::now();
    if (!bt || !x || !b) return bt_fail(WD_ERR_ARG, "null argument to wd_batch_solve");
    if (parity != 0 && parity != 1) return bt_fail(WD_ERR_ARG, "parity must be 0 or 1");
    if (!(tol > 0) || maxiter < 0) return bt_fail(WD_ERR_ARG, "tol must be > 0, maxiter >= 0");
    for (int p = 0; p < bt->nprob; ++p)
        if (bt->ops[p]->mu != 0.0)
            return bt_fail(WD_ERR_ARG, "batches have no twisted mass (mu must be 0)");
    if (info) memset(info, 0, sizeof(wd_solve_info) * bt->nslots);
    BT_TRY(bt_fork(bt));
    const int rc = bt_solve_impl(bt, x, b, tol, maxiter, parity, info);
    const int rj = bt_join(bt);
    const double secs =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info)
        for (int s = 0; s < bt->nslots; ++s) info[s].seconds = secs;
    return rc != WD_OK ? rc : rj;
}

int wd_solve_cg_multi(wd_op *const *ops, int nops, double *const *x, const double *const *b,
                      const int *nrhs, double tol, int maxiter, int parity,
                      wd_solve_info *info) {
    wd_batch *bt = nullptr;
    const int rc = wd_batch_create(&bt, ops, nrhs, nops);
    if (rc != WD_OK) return rc;
    const int rs = wd_batch_solve(bt, x, b, tol, maxiter, parity, info);
    const std::string err = g_bt_error;
    wd_batch_destroy(bt);
    g_bt_error = err;
    return rs;
}

}  // extern "C"
