// One layer with 16 input channels (16 or 1 output channels) of the
// parallel-transport network in a single kernel: the transports are
// computed on the CUDA cores straight into the
// tensor cores' shared-memory operand tiles, so the gathered operand (nine
// transports x 16 channels x 4 spins x re/im per (site, colour) row, 2.3 KB
// per row in BF16) never goes to HBM.
//
//   out_c'(x)[a][s'] = sum_{k, c, s} W[c', c, k][s', s] (T_k in_c)(x)[a][s]
//
// Work split.  A persistent CTA takes tiles of 128 consecutive sites.  For
// colour a the rows of the tile are the 128 sites, so one tile is three
// 128 x N FP32 accumulators in tensor memory (N = 128 output columns for 16
// output channels, 16 for one: re/im x channels x spins, padded), one per
// colour, all multiplied by the same weight matrix.  The
// reduction (1152 real columns: re/im x 9 transports x 16 channels x 4
// spins) runs in 18 chunks of 64 columns, chunk (k, g) = transport k,
// channels 8 g .. 8 g + 7, the 32 real-part and the 32 imaginary-part
// columns.  Per chunk
//   * 16 producer warps compute (T_k in_c)(x) for 128 sites x 8 channels
//     in FP32 (one (site, channel) item: the neighbour's 3 x 4 spinor
//     entries and one link, 36 complex multiply-adds), round to BF16 and
//     store the values in the K-major core-matrix layout of three 128 x 64
//     tiles;
//   * the N x 64 slice of the real block weight matrix arrives by cp.async
//     (295 KB in all for 16 output channels: it stays in L2);
//   * one lane of a seventeenth warp issues 3 x 4 tcgen05.mma (M = 128, N,
//     K = 16) into the three accumulators and commits them to the stage's
//     mbarrier.
// Chunks cycle through three 64 KB shared-memory stages; a stage is refilled
// once the commit of the chunk that last used it has arrived, so the
// transports of the next chunks overlap the MMAs of the current one.  After
// the last chunk of a tile the accumulators go through tcgen05.ld to the FP32
// output rows (x, a), which are the next layer's input rows.
//
// Bounded waits as in tc_gemm.cuh: every mbarrier wait polls at most
// spin_limit times; a wait that gives up sets err = 1, no further MMA is
// issued, a final commit drains the MMAs already issued (err = 2 if even
// that wait gives up) and only then is tensor memory freed.  `withhold`
// (tests only) makes the CTA issue no MMA, so that its first stage wait
// runs out with nothing in flight.
#pragma once

#include "tc_gemm.cuh"

namespace wd {

constexpr int PF_SITES = 128;                  // sites per tile = MMA rows
constexpr int PF_THREADS = 512;
constexpr int PF_CIN = 16;
constexpr int PF_KHALF = PF_CIN * 36;          // 576 columns per re/im part
constexpr int PF_NCHUNK = 18;                  // 9 transports x 2 channel groups
constexpr int PF_STAGES = 3;
constexpr int PF_TILE = PF_SITES * 64 * 2;     // 16 KB: one 128 x 64 BF16 operand tile
constexpr int PF_ITEMS = PF_SITES * 8 / PF_THREADS;         // (site, channel) items per thread

// output columns of a layer with COUT output channels: re/im x COUT x 4 spins,
// at least 16 (the smallest N of an M = 128 MMA)
template <int COUT> constexpr int pf_n() { return 8 * COUT < 16 ? 16 : 8 * COUT; }
template <int COUT> constexpr int pf_stage_bytes() { return 3 * PF_TILE + pf_n<COUT>() * 64 * 2; }
template <int COUT> constexpr int pf_smem_bytes() { return PF_STAGES * pf_stage_bytes<COUT>(); }
template <int COUT> constexpr uint32_t pf_tmem_cols() {
    return 3 * pf_n<COUT>() <= 32 ? 32 : 3 * pf_n<COUT>() <= 64 ? 64 : 3 * pf_n<COUT>() <= 128 ? 128
         : 3 * pf_n<COUT>() <= 256 ? 256 : 512;
}

struct PfArgs {
    PtcGeom g;
    const float *F;            // input rows (x, a): [Re (c, s)][Im (c, s)], 16 channels
    int ldf;
    const float2 *U;           // links [V][4][3][3], complex64
    const __nv_bfloat16 *B;    // real block weights [N][ldb], K = (re/im, k, c, s)
    int ldb;
    float *out;                // output rows (x, a), row stride ldo (>= N)
    int ldo;
    long ntiles;
    int *err;
    unsigned spin_limit;
    int withhold;              // tests: issue no MMA, so the first stage wait runs out
};

__device__ __forceinline__ void sts64(uint32_t addr, uint32_t a, uint32_t b) {
    asm volatile("st.shared.v2.b32 [%0], {%1, %2};" :: "r"(addr), "r"(a), "r"(b));
}
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Warp roles: warps 0 .. PF_PRODUCER_WARPS - 1 produce the operand tiles and
// run the epilogue; warp PF_PRODUCER_WARPS owns the tensor memory and one of
// its lanes issues the MMAs.  Hand-offs go through mbarriers, never a
// CTA-wide barrier, so producer warps run up to PF_STAGES chunks ahead of
// the tensor cores and hide each other's memory latency:
//   full[s]   producer warps -> MMA: stage s holds a chunk (16 arrivals)
//   empty[s]  MMA -> producers: the chunk's MMAs have read stage s (commit)
//   accf      MMA -> producers: the tile's accumulators are complete (commit)
//   acce      producers -> MMA: the epilogue has read the accumulators
// A wait that runs out sets `abort` in shared memory; every role checks it
// and leaves its loop, and the MMAs already issued are drained before the
// tensor memory is freed.
constexpr int PF_PRODUCER_WARPS = PF_THREADS / 32;
constexpr int PF_ALL_THREADS = PF_THREADS + 32;

template <int COUT>
__global__ void __launch_bounds__(PF_ALL_THREADS, 1) k_ptc_layer_fused(const __grid_constant__ PfArgs p) {
    constexpr int N = pf_n<COUT>();
    constexpr int STAGE = pf_stage_bytes<COUT>();
    constexpr uint32_t TMEM_COLS = pf_tmem_cols<COUT>();
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[PF_STAGES], empty[PF_STAGES];
    __shared__ __align__(8) uint64_t accf, acce, drain;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool mma_warp = warp == PF_PRODUCER_WARPS;

    if (mma_warp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_slot)), "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < PF_STAGES; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&full[b])), "r"(PF_PRODUCER_WARPS) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&empty[b])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&accf)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&acce)), "r"(PF_PRODUCER_WARPS) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&drain)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t smem0 = smem_u32(smem);
    // a bounded wait that, when it runs out, tells every role to stop
    auto wait = [&](uint64_t *bar, uint32_t parity) {
        if (abort_flag) return false;
        if (tc_wait(smem_u32(bar), parity, p.spin_limit)) return true;
        abort_flag = 1;
        return false;
    };

    if (mma_warp) {
        // ---- MMA issue (one lane)
        if (lane == 0) {
            long chunk = 0, it = 0;
            for (long tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x, ++it) {
                if (it > 0 && !wait(&acce, (uint32_t)((it - 1) & 1))) break;
                bool ok = true;
                for (int q = 0; q < PF_NCHUNK; ++q, ++chunk) {
                    const int st = (int)(chunk % PF_STAGES);
                    if (!wait(&full[st], (uint32_t)((chunk / PF_STAGES) & 1))) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    if (!p.withhold) {
                        const uint32_t sbase = smem0 + st * STAGE, sB = sbase + 3 * PF_TILE;
#pragma unroll
                        for (int a = 0; a < 3; ++a)
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint64_t ad = tc_smem_desc(sbase + a * PF_TILE + kk * 256, 128, 1024);
                                const uint64_t bd = tc_smem_desc(sB + kk * 256, 128, 1024);
                                const uint32_t acc = (q > 0 || kk > 0) ? 1u : 0u;
                                asm volatile(
                                    "{\n\t.reg .pred p;\n\t"
                                    "setp.ne.b32 p, %4, 0;\n\t"
                                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                                    :: "r"(tmem + (uint32_t)(a * N)), "l"(ad), "l"(bd),
                                       "r"(tc_idesc_bf16<N, TC_NT>()), "r"(acc)
                                    : "memory");
                            }
                        tc_commit(&empty[st]);
                    }
                }
                if (!ok) break;
                if (!p.withhold) tc_commit(&accf);
            }
        }
        __syncwarp();
    } else {
        // ---- producers: operand tiles, then the epilogue of each tile
        long chunk = 0, it = 0;
        const int cl = tid & 7;    // channel within the chunk's group of eight
        for (long tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x, ++it) {
            const long x0 = tile * PF_SITES;
            int co[PF_ITEMS][4];
            long xs[PF_ITEMS];
#pragma unroll
            for (int j = 0; j < PF_ITEMS; ++j) {
                xs[j] = x0 + (tid >> 3) + (PF_THREADS / 8) * j;
                lex_coords(p.g, xs[j] < p.g.V ? xs[j] : 0, co[j]);
            }
            bool ok = true;
            for (int q = 0; q < PF_NCHUNK; ++q, ++chunk) {
                const int st = (int)(chunk % PF_STAGES);
                const uint32_t sbase = smem0 + st * STAGE;
                const uint32_t sB = sbase + 3 * PF_TILE;
                if (chunk >= PF_STAGES &&
                    !wait(&empty[st], (uint32_t)(((chunk - PF_STAGES) / PF_STAGES) & 1))) {
                    ok = false;
                    break;
                }
                const int k = q >> 1, grp = q & 1;
                // weight slice: rows n, K columns (re: k*64 + grp*32 + 0..31, im: 576 + the same)
                for (int i = tid; i < N * 8; i += PF_THREADS) {
                    const int row = i >> 3, kg = i & 7;
                    const int col = (kg < 4 ? 0 : PF_KHALF) + k * 64 + grp * 32 + (kg & 3) * 8;
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                                 :: "r"(sB + (row >> 3) * 1024 + kg * 128 + (row & 7) * 16),
                                    "l"(p.B + (long)row * p.ldb + col) : "memory");
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
                // transported operand: items (site, channel 8 grp + cl), unrolled so
                // that both items' loads go out together on the read-only path
                // (96 registers, no spill; 1.80 -> 1.66 ms per network
                // application at 16^3 x 32 against one item after the other)
                const int c = grp * 8 + cl;
                const int mu = (k - 1) & 3;
                const bool fwd = k <= 4;
#pragma unroll
                for (int j = 0; j < PF_ITEMS; ++j) {
                    const long x = xs[j] < p.g.V ? xs[j] : 0;
                    long xn = x;
                    bool wrap = false;
                    if (k > 0) xn = ptc_neighbour(p.g, co[j], mu, fwd ? 1 : -1, wrap);
                    float4 in_re[3], in_im[3];
                    float2 u[9];
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        const float *row = p.F + (xn * 3 + b) * (long)p.ldf;
                        in_re[b] = __ldg(reinterpret_cast<const float4 *>(row + c * 4));
                        in_im[b] = __ldg(reinterpret_cast<const float4 *>(row + 4 * PF_CIN + c * 4));
                    }
                    if (k > 0) {
                        const float2 *Ul = p.U + ((fwd ? x : xn) * 4 + mu) * 9;
#pragma unroll
                        for (int e = 0; e < 9; ++e) u[e] = __ldg(Ul + e);
                    }
                    float2 v[3][4];
                    const float2 zero = make_float2(0.f, 0.f);
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        const float4 r = in_re[b], m = in_im[b];
                        float2 pin[4] = {make_float2(r.x, m.x), make_float2(r.y, m.y),
                                         make_float2(r.z, m.z), make_float2(r.w, m.w)};
                        if (k == 0) {
#pragma unroll
                            for (int s = 0; s < 4; ++s) v[b][s] = pin[s];
                        } else {
#pragma unroll
                            for (int a = 0; a < 3; ++a)
#pragma unroll
                                for (int s = 0; s < 4; ++s) {
                                    // forward: U[a][b]; backward: conj(U[b][a])
                                    const float2 w = fwd ? u[3 * a + b] : u[3 * b + a];
                                    const float wi = fwd ? w.y : -w.y;
                                    const float2 acc = b == 0 ? zero : v[a][s];
                                    v[a][s] = make_float2(acc.x + w.x * pin[s].x - wi * pin[s].y,
                                                          acc.y + w.x * pin[s].y + wi * pin[s].x);
                                }
                        }
                    }
                    if (wrap) {
                        const float pr = p.g.ph[2 * mu];
                        const float pi = fwd ? p.g.ph[2 * mu + 1] : -p.g.ph[2 * mu + 1];
#pragma unroll
                        for (int a = 0; a < 3; ++a)
#pragma unroll
                            for (int s = 0; s < 4; ++s)
                                v[a][s] = make_float2(v[a][s].x * pr - v[a][s].y * pi,
                                                      v[a][s].x * pi + v[a][s].y * pr);
                    }
                    if (xs[j] >= p.g.V) {
#pragma unroll
                        for (int a = 0; a < 3; ++a)
#pragma unroll
                            for (int s = 0; s < 4; ++s) v[a][s] = zero;
                    }
                    // K-major core-matrix layout: row = site, K column = cl * 4 + s
                    // (re) or 32 + cl * 4 + s (im): four BF16 values per 8-byte store
                    const int sl = (tid >> 3) + (PF_THREADS / 8) * j;
                    const uint32_t off = (sl >> 3) * 1024 + (sl & 7) * 16 + (cl >> 1) * 128 + (cl & 1) * 8;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const uint32_t sa = sbase + a * PF_TILE + off;
                        sts64(sa, pack_bf16x2(v[a][0].x, v[a][1].x), pack_bf16x2(v[a][2].x, v[a][3].x));
                        sts64(sa + 4 * 128, pack_bf16x2(v[a][0].y, v[a][1].y),
                              pack_bf16x2(v[a][2].y, v[a][3].y));
                    }
                }
                asm volatile("cp.async.wait_group 0;" ::: "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&full[st])) : "memory");
            }
            if (!ok) break;
            // epilogue: wait for the tile's accumulators, read them, hand TMEM back
            if (!wait(&accf, (uint32_t)(it & 1))) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            {
                // warp w reads TMEM lanes 32 (w % 4) .. +31 (sites); column blocks
                // of 16 are dealt round-robin over the warps sharing a lane quarter
                constexpr int NGROUPS = PF_PRODUCER_WARPS / 4;
                const int quarter = warp & 3, group = warp >> 2;
                const long x = x0 + 32 * quarter + lane;
                const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
#pragma unroll 1
                for (int c0 = 16 * group; c0 < 3 * N; c0 += 16 * NGROUPS) {
                    uint32_t r[16];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                          "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                          "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                        : "r"(tmem + lane_base + (uint32_t)c0));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (x < p.g.V) {
                        const int a = c0 / N, n0 = c0 - a * N;
                        float *orow = p.out + (x * 3 + a) * (long)p.ldo + n0;
#pragma unroll
                        for (int j = 0; j < 16; j += 4)
                            *reinterpret_cast<float4 *>(orow + j) =
                                make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                            __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(&acce)) : "memory");
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
    // every role has left its loop; drain the MMAs issued if a wait ran out
    __syncthreads();
    if (abort_flag) {
        if (mma_warp && lane == 0) {
            atomicExch(p.err, 1);
            tc_commit(&drain);
            if (!tc_wait(smem_u32(&drain), 0u, 64ull * p.spin_limit)) atomicExch(p.err, 2);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (mma_warp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS) : "memory");
}

}  // namespace wd
