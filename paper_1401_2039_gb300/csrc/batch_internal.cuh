// Internal declarations of the batched solver (batch.cu) shared with the
// translation units that instantiate its hopping-term kernels
// (batch_hop_*.cu): problem table, deterministic per-system reductions and
// the batched hopping term.
//
#pragma once

#include <type_traits>

#include "dslash_df.cuh"

namespace wd {

constexpr int BT_BLOCK = 128;       // block (and tile) size of the element-wise kernels
constexpr int BT_WARPS = BT_BLOCK / 32;
constexpr int BT_MAX_PROB = 8;
constexpr int BT_MAX_SLOTS = 64;
constexpr int BT_BLOCKS_PER_SM_MAX = 32;   // per-block partials are sized for this grid

struct BtProb {
    Geom g;                  // stride = plane stride of one right-hand side
    const char *gauge_out;   // links of the output parity
    const char *gauge_in;    // links of the input parity
    size_t dir_bytes;
    void *f[4];              // fields of this launch (meaning set by the kernel)
    double scale;            // per-problem coefficient
    double ph[8];            // boundary phases
    unsigned phase_on;       // bit mu set: direction mu's phase is not 1
    int nrhs;
    Divisor div_nrhs;        // by nrhs (item -> site)
    int slot0;               // first solver slot of the problem
    long tile0;              // first tile of the problem
    long nitems;             // work items of the problem
};

struct BtArgs {
    BtProb p[BT_MAX_PROB];
    int nprob;
    long ntiles;
    int parity;              // output parity of hopping terms
    int fin;                 // final operation applied per slot
    int nslots;
    df64 *partials;          // [grid][BT_MAX_SLOTS]
    unsigned int *counter;
    SolverScalars *scalars;  // [nslots]
    const double *consts;    // per-slot constants, [4][BT_MAX_SLOTS]
    long max_grid;           // blocks the partials buffer holds
};

__device__ __forceinline__ int bt_problem(const BtArgs &a, long t) {
    int pi = 0;
#pragma unroll 1
    for (int k = 1; k < a.nprob; ++k)
        if (t >= a.p[k].tile0) pi = k;
    return pi;
}

// Per-rhs sums of the items of a tile, without block barriers.  Each warp
// stages its 32 values (items item0 + 32 w + lane; the item's rhs is item %
// nrhs) in its own shared-memory row; lane j then adds the values of rhs j in
// lane order and accumulates them into the warp's slot row wacc[w][slot].
// bt_block_sums later adds the warps' rows in warp order, so every sum has a
// fixed order.  Values are double-float (the FP64 adder of GB300 is too slow
// for per-item work).
template <int BLOCK = BT_BLOCK>
__device__ __forceinline__ void bt_warp_sums(df64 v, const BtProb &P, long item0, df64 *wv,
                                             df64 (*wacc)[BT_MAX_SLOTS]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    wv[threadIdx.x] = v;
    __syncwarp();
    const int nr = P.nrhs;
    const long iw = item0 + 32 * w;
    const int base = (int)(iw % nr);
    for (int j = lane; j < nr; j += 32) {
        df64 s = 0;
        for (int l = (j - base + nr) % nr; l < 32; l += nr) s = s + wv[32 * w + l];
        wacc[w][P.slot0 + j] = wacc[w][P.slot0 + j] + s;
    }
    __syncwarp();
}

template <int BLOCK = BT_BLOCK>
__device__ __forceinline__ void bt_zero_sums(df64 (*wacc)[BT_MAX_SLOTS]) {
    for (int i = threadIdx.x; i < (BLOCK / 32) * BT_MAX_SLOTS; i += BLOCK)
        wacc[i / BT_MAX_SLOTS][i % BT_MAX_SLOTS] = df64(0.0f, 0.0f);
    __syncthreads();
}

// the block's slot sums: the warps' rows added in warp order
template <int BLOCK = BT_BLOCK>
__device__ __forceinline__ void bt_block_sums(df64 (*wacc)[BT_MAX_SLOTS], df64 *sacc, int nslots) {
    __syncthreads();
    for (int sl = threadIdx.x; sl < nslots; sl += BLOCK) {
        df64 t = wacc[0][sl];
#pragma unroll
        for (int w = 1; w < BLOCK / 32; ++w) t = t + wacc[w][sl];
        sacc[sl] = t;
    }
    __syncthreads();
}

// Grid-wide finish: per-block slot partials, then the last block adds them
// in block order (one warp per slot) and applies the final operation.
template <int BLOCK = BT_BLOCK>
__device__ __forceinline__ void bt_finish(const BtArgs &a, const df64 *sacc) {
    __shared__ bool last;
    for (int s = threadIdx.x; s < a.nslots; s += BLOCK)
        a.partials[(long)blockIdx.x * BT_MAX_SLOTS + s] = sacc[s];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = arrive_last(a.counter, gridDim.x, blockIdx.x);
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int s = warp; s < a.nslots; s += BLOCK / 32) {
        const df64 sum = warp_sum(strided_sum<32>(a.partials + s, gridDim.x, lane, BT_MAX_SLOTS));
        if (lane == 0) apply_final(&a.scalars[s], a.fin, (double)sum);
    }
}

// ------------------------------------------------------------------ hopping term
// N reals of storage S at record rec of a field with plane stride `plane`
// bytes, in 32-bit record arithmetic (records < 2^32)
template <typename S, int N, int KIND, typename R>
__device__ __forceinline__ void bt_load(const void *base, size_t plane, unsigned rec, R *r) {
    using Q = Rec<S, N>;
    uint32_t w[Q::WORDS];
    const char *p0 = (const char *)base + (size_t)rec * 16;
#pragma unroll
    for (int j = 0; j < Q::NF; ++j) {
        const uint4 v = KIND ? ld_stream_v4(p0 + j * plane) : ld_nc_v4(p0 + j * plane);
        w[4 * j] = v.x; w[4 * j + 1] = v.y; w[4 * j + 2] = v.z; w[4 * j + 3] = v.w;
    }
    if (Q::TAIL == 8) {
        const uint2 v = ld_stream_v2((const char *)base + Q::NF * plane + (size_t)rec * 8);
        w[4 * Q::NF] = v.x; w[4 * Q::NF + 1] = v.y;
    } else if (Q::TAIL == 4) {
        w[4 * Q::NF] = ld_stream_u32((const char *)base + Q::NF * plane + (size_t)rec * 4);
    }
    Words<S, R>::unpack(w, r, N);
}

// 12-real links: row 2 = conj(row0 x row1) in the arithmetic R
template <typename R> __device__ __forceinline__ void bt_rebuild_row2(R *U) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int k = (j + 1) % 3, l = (j + 2) % 3;
        const R xr = U[2 * k], xi = U[2 * k + 1], yr = U[6 + 2 * l], yi = U[6 + 2 * l + 1];
        const R zr = U[2 * l], zi = U[2 * l + 1], wr = U[6 + 2 * k], wi = U[6 + 2 * k + 1];
        R t = xr * yr;
        t -= xi * yi; t -= zr * wr; t += zi * wi;
        U[12 + 2 * j] = t;
        t = zr * wi;
        t += zi * wr; t -= xr * yi; t -= xi * yr;
        U[12 + 2 * j + 1] = t;
    }
}

template <typename S, typename R, int RECON, int MU, int DAG>
__device__ __forceinline__ void bt_hop_pair(const BtProb &P, const int c[4], long h, int r,
                                            Acc<R> *acc) {
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    const size_t splane = (size_t)P.g.stride * P.nrhs * 16, lplane = (size_t)P.g.stride * 16;
    const unsigned hu = (unsigned)h;
    {
        bool wrap;
        const unsigned hn = neighbour32<MU, +1>(P.g, hu, c, wrap);
        R psi[24];
        bt_load<S, 24, 0>(P.f[1], splane, hn * (unsigned)P.nrhs + (unsigned)r, psi);
        cx<Acc<R>> hs[2][3], u[2][3];
        project<MU, SF>(psi, hs);
        R U[18];
        bt_load<S, RECON, 1>(P.gauge_out + MU * P.dir_bytes, lplane, hu, U);
        if (RECON == 12) bt_rebuild_row2(U);
        su3_mul(U, hs, u);
        if (wrap && (P.phase_on >> MU & 1u)) phase_mul(u, (R)P.ph[2 * MU], (R)P.ph[2 * MU + 1]);
        if constexpr (std::is_same<Acc<R>, float>::value) accumulate_x2<MU, SF>(acc, u);
        else accumulate<MU, SF>(acc, u);
    }
    {
        bool wrap;
        const unsigned hn = neighbour32<MU, -1>(P.g, hu, c, wrap);
        R psi[24];
        bt_load<S, 24, 0>(P.f[1], splane, hn * (unsigned)P.nrhs + (unsigned)r, psi);
        cx<Acc<R>> hs[2][3], u[2][3];
        project<MU, SB>(psi, hs);
        R U[18];
        bt_load<S, RECON, 1>(P.gauge_in + MU * P.dir_bytes, lplane, hn, U);
        if (RECON == 12) bt_rebuild_row2(U);
        su3_adj_mul(U, hs, u);
        if (wrap && (P.phase_on >> MU & 1u)) phase_mul(u, (R)P.ph[2 * MU], -(R)P.ph[2 * MU + 1]);
        if constexpr (std::is_same<Acc<R>, float>::value) accumulate_x2<MU, SB>(acc, u);
        else accumulate<MU, SB>(acc, u);
    }
}

// ---- two right-hand sides per thread (FP32 storage and arithmetic)
// The pair item (site, rhs r, r + 1) shares the neighbour indices, the link
// loads and the row-2 rebuild.  Each projected half spinor, SU(3) product and
// accumulation is one packed FP32 pair operation over the two right-hand
// sides (lane 0: rhs r, lane 1: rhs r + 1), each lane rounded as the scalar
// operation of bt_hop_pair in the same order.
struct c2 {
    f2 re, im;
};

// acc += (1 + SGN gamma_MU) expanded from u, lane-wise as accumulate<MU, SGN>
template <int MU, int SGN>
__device__ __forceinline__ void accumulate2(f2 *acc, const c2 u[2][3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        f2 *q = acc + 8 * c;
        q[0] = f2_add(q[0], u[0][c].re); q[1] = f2_add(q[1], u[0][c].im);
        q[2] = f2_add(q[2], u[1][c].re); q[3] = f2_add(q[3], u[1][c].im);
        if (MU == 1) {          // spin 2 += SGN u1, spin 3 -= SGN u0
            if (SGN > 0) {
                q[4] = f2_add(q[4], u[1][c].re); q[5] = f2_add(q[5], u[1][c].im);
                q[6] = f2_sub(q[6], u[0][c].re); q[7] = f2_sub(q[7], u[0][c].im);
            } else {
                q[4] = f2_sub(q[4], u[1][c].re); q[5] = f2_sub(q[5], u[1][c].im);
                q[6] = f2_add(q[6], u[0][c].re); q[7] = f2_add(q[7], u[0][c].im);
            }
        } else if (MU == 3) {   // spin 2 += SGN u0, spin 3 += SGN u1
            if (SGN > 0) {
                q[4] = f2_add(q[4], u[0][c].re); q[5] = f2_add(q[5], u[0][c].im);
                q[6] = f2_add(q[6], u[1][c].re); q[7] = f2_add(q[7], u[1][c].im);
            } else {
                q[4] = f2_sub(q[4], u[0][c].re); q[5] = f2_sub(q[5], u[0][c].im);
                q[6] = f2_sub(q[6], u[1][c].re); q[7] = f2_sub(q[7], u[1][c].im);
            }
        } else {
            // MU 0: spin 2 += -SGN i u1, spin 3 += -SGN i u0;
            // MU 2: spin 2 += -SGN i u0, spin 3 += SGN i u1;  i v = (-v.im, v.re)
            const c2 v2 = MU == 0 ? u[1][c] : u[0][c];
            const c2 v3 = MU == 0 ? u[0][c] : u[1][c];
            constexpr bool n3 = MU == 0 ? SGN > 0 : SGN < 0;
            if (SGN > 0) { q[4] = f2_add(q[4], v2.im); q[5] = f2_sub(q[5], v2.re); }
            else         { q[4] = f2_sub(q[4], v2.im); q[5] = f2_add(q[5], v2.re); }
            if (n3) { q[6] = f2_add(q[6], v3.im); q[7] = f2_sub(q[7], v3.re); }
            else    { q[6] = f2_sub(q[6], v3.im); q[7] = f2_add(q[7], v3.re); }
        }
    }
}

// u[k][a] = sum_b U[a][b] h[k][b] (ADJ: conj(U[b][a])), the FMA chains of
// su3_mul / su3_adj_mul with the link entries broadcast to both lanes
template <int ADJ>
__device__ __forceinline__ void su3_mul2(const float *U, const c2 h[2][3], c2 u[2][3]) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        f2 hn[3];   // -h.im (U h) or -h.re (U^dag h): the negative products
#pragma unroll
        for (int b = 0; b < 3; ++b) hn[b] = f2_neg(ADJ ? h[k][b].re : h[k][b].im);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int e0 = ADJ ? a : 3 * a;
            const f2 ur = f2_bcast(U[2 * e0]), ui = f2_bcast(U[2 * e0 + 1]);
            f2 re = f2_mul(ur, h[k][0].re);
            f2 im = f2_mul(ur, h[k][0].im);
            if (ADJ) {
                re = f2_fma(ui, h[k][0].im, re);
                im = f2_fma(ui, hn[0], im);
            } else {
                re = f2_fma(ui, hn[0], re);
                im = f2_fma(ui, h[k][0].re, im);
            }
#pragma unroll
            for (int b = 1; b < 3; ++b) {
                const int e = ADJ ? 3 * b + a : 3 * a + b;
                const f2 vr = f2_bcast(U[2 * e]), vi = f2_bcast(U[2 * e + 1]);
                re = f2_fma(vr, h[k][b].re, re);
                re = f2_fma(vi, ADJ ? h[k][b].im : hn[b], re);
                im = f2_fma(vr, h[k][b].im, im);
                im = f2_fma(vi, ADJ ? hn[b] : h[k][b].re, im);
            }
            u[k][a] = {re, im};
        }
    }
}

// the half spinors of the two right-hand sides' neighbour records, paired
template <int MU, int SGN>
__device__ __forceinline__ void project2(const float *p0, const float *p1, c2 h[2][3]) {
    cx<float> a[2][3], b[2][3];
    project<MU, SGN>(p0, a);
    project<MU, SGN>(p1, b);
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            h[k][c] = {f2_pack(a[k][c].re, b[k][c].re), f2_pack(a[k][c].im, b[k][c].im)};
}

// u *= phase (pr, pi), lane-wise
__device__ __forceinline__ void phase_mul2(c2 u[2][3], float pr, float pi) {
    const f2 r = f2_bcast(pr), i = f2_bcast(pi), ni = f2_bcast(-pi);
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const f2 re = f2_fma(u[k][a].re, r, f2_mul(u[k][a].im, ni));
            const f2 im = f2_fma(u[k][a].re, i, f2_mul(u[k][a].im, r));
            u[k][a] = {re, im};
        }
}

// acc += the forward and backward hops of direction MU for the right-hand
// sides r and r + 1 of site h (FP32 storage)
template <int RECON, int MU, int DAG>
__device__ __forceinline__ void bt_hop_pair2(const BtProb &P, const int c[4], unsigned hu, int r,
                                             f2 *acc) {
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    const size_t splane = (size_t)P.g.stride * P.nrhs * 16, lplane = (size_t)P.g.stride * 16;
    {
        bool wrap;
        const unsigned hn = neighbour32<MU, +1>(P.g, hu, c, wrap);
        const unsigned rec = hn * (unsigned)P.nrhs + (unsigned)r;
        float p0[24], p1[24];
        bt_load<float, 24, 0>(P.f[1], splane, rec, p0);
        bt_load<float, 24, 0>(P.f[1], splane, rec + 1, p1);
        c2 hs[2][3], u[2][3];
        project2<MU, SF>(p0, p1, hs);
        float U[18];
        bt_load<float, RECON, 1>(P.gauge_out + MU * P.dir_bytes, lplane, hu, U);
        if (RECON == 12) bt_rebuild_row2(U);
        su3_mul2<0>(U, hs, u);
        if (wrap && (P.phase_on >> MU & 1u))
            phase_mul2(u, (float)P.ph[2 * MU], (float)P.ph[2 * MU + 1]);
        accumulate2<MU, SF>(acc, u);
    }
    {
        bool wrap;
        const unsigned hn = neighbour32<MU, -1>(P.g, hu, c, wrap);
        const unsigned rec = hn * (unsigned)P.nrhs + (unsigned)r;
        float p0[24], p1[24];
        bt_load<float, 24, 0>(P.f[1], splane, rec, p0);
        bt_load<float, 24, 0>(P.f[1], splane, rec + 1, p1);
        c2 hs[2][3], u[2][3];
        project2<MU, SB>(p0, p1, hs);
        float U[18];
        bt_load<float, RECON, 1>(P.gauge_in + MU * P.dir_bytes, lplane, hn, U);
        if (RECON == 12) bt_rebuild_row2(U);
        su3_mul2<1>(U, hs, u);
        if (wrap && (P.phase_on >> MU & 1u))
            phase_mul2(u, (float)P.ph[2 * MU], -(float)P.ph[2 * MU + 1]);
        accumulate2<MU, SB>(acc, u);
    }
}

// Per-rhs sums of a pair tile (2 BLOCK items, two per thread), with the
// staging and summation order of bt_warp_sums over each warp's 64 items.
template <int BLOCK>
__device__ __forceinline__ void bt_warp_sums2(df64 v0, df64 v1, const BtProb &P, long item0,
                                              df64 *wv, df64 (*wacc)[BT_MAX_SLOTS]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    wv[2 * threadIdx.x] = v0;
    wv[2 * threadIdx.x + 1] = v1;
    __syncwarp();
    const int nr = P.nrhs;
    const long iw = item0 + 64 * w;
    const int base = (int)(iw % nr);
    for (int j = lane; j < nr; j += 32) {
        df64 s = 0;
        for (int l = (j - base + nr) % nr; l < 64; l += nr) s = s + wv[64 * w + l];
        wacc[w][P.slot0 + j] = wacc[w][P.slot0 + j] + s;
    }
    __syncwarp();
}

// f[0] = out, f[1] = in, f[2] = x:  out = scale * H in  or  x + scale * H in.
// Tiles of BLOCK items (one per thread); MINB resident blocks per SM set the
// register cap, the parameter the autotuner picks per batch.  Double-float
// instances run the hop loop of dslash_df.cuh (unrolled, their code
// outgrows the instruction cache).
template <typename S, typename R, int RECON, int DAG, int XPAY, int NORM, int BLOCK, int MINB,
          int PAIR = 0>
__global__ void __launch_bounds__(BLOCK, MINB) k_dslash_batch(const __grid_constant__ BtArgs a) {
    __shared__ df64 wv[PAIR ? 2 * BLOCK : BLOCK];
    __shared__ df64 wacc[BLOCK / 32][BT_MAX_SLOTS];
    __shared__ df64 sacc[BT_MAX_SLOTS];
    if (NORM) bt_zero_sums<BLOCK>(wacc);
    if constexpr (PAIR) {
        static_assert(std::is_same<S, float>::value && std::is_same<R, float>::value,
                      "pair items: FP32 storage");
        // tiles of 2 BLOCK items; thread t takes items item0 + 2 t and + 1,
        // rhs r and r + 1 of one site (every nrhs of the batch is even)
        for (long t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
            const BtProb &P = a.p[bt_problem(a, t)];
            const long item0 = (t - P.tile0) * (2 * BLOCK);
            const long item = item0 + 2 * threadIdx.x;
            df64 v0 = 0, v1 = 0;
            if (item < P.nitems) {
                const int nr = P.nrhs;
                const unsigned hu = udiv((unsigned)item, P.div_nrhs);   // items < 2^31
                const int r = (int)((unsigned)item - hu * (unsigned)nr);
                int c[4];
                site_coords(P.g, hu, a.parity, c);
                f2 acc[24];
#pragma unroll
                for (int k = 0; k < 24; ++k) acc[k] = f2_pack(0.0f, 0.0f);
                bt_hop_pair2<RECON, 0, DAG>(P, c, hu, r, acc);
                bt_hop_pair2<RECON, 1, DAG>(P, c, hu, r, acc);
                bt_hop_pair2<RECON, 2, DAG>(P, c, hu, r, acc);
                bt_hop_pair2<RECON, 3, DAG>(P, c, hu, r, acc);
                const long ss = P.g.stride * nr;
                const float sc = (float)P.scale;
                float o0[24], o1[24];
                if (XPAY) {
                    float x0[24], x1[24];
                    Rec<float, 24>::template load<float, 0>(P.f[2], ss, item, x0);
                    Rec<float, 24>::template load<float, 0>(P.f[2], ss, item + 1, x1);
#pragma unroll
                    for (int k = 0; k < 24; ++k) {
                        float a0, a1;
                        f2_unpack(acc[k], a0, a1);
                        o0[k] = fmaf(sc, a0, x0[k]);
                        o1[k] = fmaf(sc, a1, x1[k]);
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < 24; ++k) {
                        float a0, a1;
                        f2_unpack(acc[k], a0, a1);
                        o0[k] = sc * a0;
                        o1[k] = sc * a1;
                    }
                }
                Rec<float, 24>::store(P.f[0], ss, item, o0);
                Rec<float, 24>::store(P.f[0], ss, item + 1, o1);
                if (NORM) {
                    float q0 = 0, q0b = 0, q1 = 0, q1b = 0;
#pragma unroll
                    for (int k = 0; k < 24; k += 2) {
                        sq_acc_x2(q0, q0b, o0[k], o0[k + 1]);
                        sq_acc_x2(q1, q1b, o1[k], o1[k + 1]);
                    }
                    v0 = to_df(q0 + q0b);
                    v1 = to_df(q1 + q1b);
                }
            }
            if (NORM) bt_warp_sums2<BLOCK>(v0, v1, P, item0, wv, wacc);
        }
        if (NORM) {
            bt_block_sums<BLOCK>(wacc, sacc, a.nslots);
            bt_finish<BLOCK>(a, sacc);
        }
        return;
    }
    for (long t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const BtProb &P = a.p[bt_problem(a, t)];
        const long item0 = (t - P.tile0) * BLOCK;
        const long item = item0 + threadIdx.x;
        df64 v = 0;
        if (item < P.nitems) {
            const int nr = P.nrhs;
            const unsigned hu = udiv((unsigned)item, P.div_nrhs);   // items < 2^31
            const long h = hu;
            const int r = (int)((unsigned)item - hu * (unsigned)nr);
            int c[4];
            site_coords(P.g, h, a.parity, c);
            Acc<R> acc[24];
#pragma unroll
            for (int k = 0; k < 24; ++k) acc[k] = 0;
            if constexpr (std::is_same<S, df64>::value) {
                df_hops<DAG>(P.g, P.gauge_out, P.gauge_in, P.dir_bytes, P.ph, P.f[1],
                             P.g.stride * nr, nr, r, h, c, acc, nullptr, P.phase_on);
            } else if constexpr (std::is_same<S, __half>::value) {
                const long ss = P.g.stride * nr;
                hop_pair_h2<RECON, 0, DAG>(P.g, P.gauge_out, P.gauge_in, P.dir_bytes, P.ph, P.f[1],
                                           ss, nr, r, c, h, acc, P.phase_on);
                hop_pair_h2<RECON, 1, DAG>(P.g, P.gauge_out, P.gauge_in, P.dir_bytes, P.ph, P.f[1],
                                           ss, nr, r, c, h, acc, P.phase_on);
                hop_pair_h2<RECON, 2, DAG>(P.g, P.gauge_out, P.gauge_in, P.dir_bytes, P.ph, P.f[1],
                                           ss, nr, r, c, h, acc, P.phase_on);
                hop_pair_h2<RECON, 3, DAG>(P.g, P.gauge_out, P.gauge_in, P.dir_bytes, P.ph, P.f[1],
                                           ss, nr, r, c, h, acc, P.phase_on);
            } else {
                bt_hop_pair<S, R, RECON, 0, DAG>(P, c, h, r, acc);
                bt_hop_pair<S, R, RECON, 1, DAG>(P, c, h, r, acc);
                bt_hop_pair<S, R, RECON, 2, DAG>(P, c, h, r, acc);
                bt_hop_pair<S, R, RECON, 3, DAG>(P, c, h, r, acc);
            }
            const long ss = P.g.stride * nr;
            const R sc = (R)P.scale;
            R o[24];
            if (XPAY) {
                R xv[24];
                Rec<S, 24>::template load<R, 0>(P.f[2], ss, item, xv);
                if constexpr (std::is_same<R, float>::value) {
#pragma unroll
                    for (int k = 0; k < 24; k += 2)
                        scale_add_x2(o[k], o[k + 1], acc[k], acc[k + 1], sc, xv[k], xv[k + 1]);
                } else {
#pragma unroll
                    for (int k = 0; k < 24; ++k) o[k] = settle(xv[k] + sc * acc[k]);
                }
            } else {
                if constexpr (std::is_same<R, float>::value) {
#pragma unroll
                    for (int k = 0; k < 24; k += 2) scale_x2(o[k], o[k + 1], acc[k], acc[k + 1], sc);
                } else {
#pragma unroll
                    for (int k = 0; k < 24; ++k) o[k] = settle(sc * acc[k]);
                }
            }
            Rec<S, 24>::store(P.f[0], ss, item, o);
            if (NORM) {
                if constexpr (std::is_same<R, float>::value) {
                    float sq = 0, sq1 = 0;
#pragma unroll
                    for (int k = 0; k < 24; k += 2) sq_acc_x2(sq, sq1, o[k], o[k + 1]);
                    v = to_df(sq + sq1);
                } else {
                    R sq = 0;
#pragma unroll
                    for (int k = 0; k < 24; ++k) sq += o[k] * o[k];
                    v = to_df(sq);
                }
            }
        }
        if (NORM) bt_warp_sums<BLOCK>(v, P, item0, wv, wacc);
    }
    if (NORM) {
        bt_block_sums<BLOCK>(wacc, sacc, a.nslots);
        bt_finish<BLOCK>(a, sacc);
    }
}

// Launch configurations of the batched hopping term in storage precision
// (FP32, FP16): threads per block (= items per tile) and minimum resident
// blocks per SM (the register cap).  The grid is the kernel's resident
// capacity on this GPU (SMs x blocks per SM), capped at the tile count.
// pair = 1: two right-hand sides per thread (FP32 storage, every nrhs even).
struct BtCfg { int block, minb, pair; };
constexpr int N_BT_CFG = 9;
constexpr BtCfg BT_CFGS[N_BT_CFG] = {{128, 4, 0}, {128, 5, 0}, {128, 6, 0}, {128, 8, 0},
                                     {256, 2, 0}, {128, 2, 1}, {128, 3, 1}, {128, 4, 1},
                                     {256, 2, 1}};

// Variants of a batched hop: plain (out = scale H in) or xpay with the fused
// per-system norm (the second hop of the Schur operator in the CGNR
// iteration); residual-arithmetic handles also use xpay without a norm.
enum BtVariant { BTV_PLAIN = 0, BTV_XPAY_NORM = 1, BTV_XPAY = 2 };

// Resident capacity of a kernel with `block` threads: SMs x blocks per SM.
template <typename K>
inline unsigned bt_resident_grid(K kernel, int block) {
    int dev = 0, sms = 1, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, block, 0) != cudaSuccess || per < 1)
        per = 1;
    cudaGetLastError();
    return (unsigned)(sms * per);
}

// One launch of a batched hop: persistent grid = the kernel's resident
// capacity on this device (looked up once per device), capped at the tile
// count and at the partials buffer.
template <typename S, typename R, int RECON, int DAG, int X, int N, int BLOCK, int MINB,
          int PAIR = 0>
cudaError_t bt_go(const BtArgs &a, cudaStream_t s, unsigned *grid_out) {
    const auto k = k_dslash_batch<S, R, RECON, DAG, X, N, BLOCK, MINB, PAIR>;
    static unsigned cap[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    unsigned res = (dev >= 0 && dev < 64) ? cap[dev] : 0u;
    if (!res) {
        res = bt_resident_grid(k, BLOCK);
        if (dev >= 0 && dev < 64) cap[dev] = res;
    }
    long g = a.ntiles < (long)res ? a.ntiles : (long)res;
    if (g > a.max_grid) g = a.max_grid;
    const unsigned grid = (unsigned)(g < 1 ? 1 : g);
    k<<<grid, BLOCK, 0, s>>>(a);
    if (grid_out) *grid_out = grid;
    return cudaGetLastError();
}

template <typename S, typename R, int RECON, int DAG, int X, int N>
cudaError_t bt_go_cfg(int cfg, const BtArgs &a, cudaStream_t s, unsigned *g) {
#define WD_BT_CFG(C)                                                                       \
    bt_go<S, R, RECON, DAG, X, N, BT_CFGS[C].block, BT_CFGS[C].minb, BT_CFGS[C].pair>(a, s, g)
    if constexpr (std::is_same<S, float>::value) {
        switch (cfg) {
        case 5: return WD_BT_CFG(5);
        case 6: return WD_BT_CFG(6);
        case 7: return WD_BT_CFG(7);
        case 8: return WD_BT_CFG(8);
        default: break;
        }
    } else if (cfg >= 5) {
        return cudaErrorInvalidValue;   // pair items: FP32 storage only
    }
    switch (cfg) {
    case 1: return WD_BT_CFG(1);
    case 2: return WD_BT_CFG(2);
    case 3: return WD_BT_CFG(3);
    case 4: return WD_BT_CFG(4);
    default: return WD_BT_CFG(0);
    }
#undef WD_BT_CFG
}

// Storage-precision hops (FP32, FP16): the plain and the norm-fused xpay
// variants in every configuration; xpay without a norm (not on the solver's
// storage-precision path) in one.
template <typename S, typename R, int RECON>
cudaError_t bt_launch_lo(int dagger, int variant, int cfg, const BtArgs &a, cudaStream_t s,
                         unsigned *g) {
    if (variant == BTV_XPAY)
        return dagger ? bt_go<S, R, RECON, 1, 1, 0, 128, 4>(a, s, g)
                      : bt_go<S, R, RECON, 0, 1, 0, 128, 4>(a, s, g);
    if (variant == BTV_XPAY_NORM)
        return dagger ? bt_go_cfg<S, R, RECON, 1, 1, 1>(cfg, a, s, g)
                      : bt_go_cfg<S, R, RECON, 0, 1, 1>(cfg, a, s, g);
    return dagger ? bt_go_cfg<S, R, RECON, 1, 0, 0>(cfg, a, s, g)
                  : bt_go_cfg<S, R, RECON, 0, 0, 0>(cfg, a, s, g);
}

// FP64 storage and double-float residual hops: one configuration each
// (FP64-pipe bound, and the double-float hop's register appetite).
template <typename S, typename R, int RECON, int MINB>
cudaError_t bt_launch_fixed(int dagger, int variant, const BtArgs &a, cudaStream_t s,
                            unsigned *g) {
#define WD_BT_V(D, X, N) bt_go<S, R, RECON, D, X, N, 128, MINB>(a, s, g)
    if (variant == BTV_XPAY) return dagger ? WD_BT_V(1, 1, 0) : WD_BT_V(0, 1, 0);
    if (variant == BTV_XPAY_NORM) return dagger ? WD_BT_V(1, 1, 1) : WD_BT_V(0, 1, 1);
    return dagger ? WD_BT_V(1, 0, 0) : WD_BT_V(0, 0, 0);
#undef WD_BT_V
}

// Per-precision launchers, one translation unit each (batch_hop_*.cu).
#define WD_BT_DECL(NAME)                                                                   \
    cudaError_t NAME(int dagger, int variant, int cfg, const BtArgs &a, cudaStream_t s,      \
                     unsigned *grid_out);
WD_BT_DECL(bt_launch_hop_f32_r18)
WD_BT_DECL(bt_launch_hop_f32_r12)
WD_BT_DECL(bt_launch_hop_f16_r18)
WD_BT_DECL(bt_launch_hop_f16_r12)
WD_BT_DECL(bt_launch_hop_f64_r18)
WD_BT_DECL(bt_launch_hop_f64_r12)
WD_BT_DECL(bt_launch_hop_df64_r18)
#undef WD_BT_DECL

}  // namespace wd
