// BF16 x BF16 -> FP32 GEMMs on the fifth-generation tensor cores (tcgen05).
//
//   NT:  D[M x N] = A[M x K] * B[N x K]^T   (A, B row-major, K contiguous):
//        the forward and input-gradient products of the network.
//   TN:  D[M x N] = A[K x M]^T * B[K x N]   (A, B row-major, M and N
//        contiguous): the weight gradient, a reduction over the K rows of
//        two activation-shaped matrices; gridDim.z splits those rows and
//        each split writes its own partial D (summed afterwards in a fixed
//        order, so the result does not depend on scheduling).
//
// One CTA of four warps computes a 128 x BN tile of D.  The reduction runs
// in steps of 64 through a ring of TC_STAGES shared-memory buffers: the four
// warps copy the A and B tiles of step i + TC_STAGES - 1 from global memory
// with cp.async (16-byte chunks, no register staging) while the tensor cores
// work on step i.  Tiles use the no-swizzle canonical layouts of 8 x 16-byte
// core matrices:
//   NT (K-major):  a core matrix is 8 rows (M or N) x 8 K values, 16 bytes
//                  per row; K-adjacent core matrices 128 bytes apart,
//                  8-row groups 1024 bytes apart;
//   TN (MN-major): a core matrix is 8 K rows x 8 M (or N) values, 16 bytes
//                  per K row; MN-adjacent core matrices 128 bytes apart,
//                  K-adjacent ones (rows / 8) * 128 bytes apart,
// so that every 16-byte chunk of a global row lands in one core-matrix row
// (no transposition in either form).  For each step one elected thread
// issues four 128 x BN x 16 tcgen05.mma that accumulate in tensor memory
// (TMEM, BN fp32 columns x 128 lanes) and a tcgen05.commit that arrives on
// the step buffer's mbarrier once the MMAs have consumed it; a buffer is
// refilled only after that arrival.  The epilogue moves the accumulator from
// TMEM to registers with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31,
// i.e. rows 32w..32w+31 of the tile) and stores it.
//
// Bounded waits.  Every wait on an mbarrier polls at most spin_limit times.
// When one gives up, the kernel records err = 1, issues no further MMA,
// then commits once more to a drain barrier, which arrives when every MMA
// this CTA issued has completed, and waits for that (MMAs need no other
// work to finish, so this wait ends; its own bound, 64 x spin_limit polls,
// is there only against a broken device, and err = 2 records that case).
// Only then is TMEM freed.  `withhold` (tests only) makes the CTA issue no
// MMA and no per-step commit at all: its first buffer wait runs out with
// nothing in flight and the call reports the timeout.
//
// Requirements (checked by the host launchers): NT: M % 128 == 0,
// N % BN == 0, K % 64 == 0; TN: M % 128 == 0, N % BN == 0, every split's row
// range a multiple of 64; rows 16-byte aligned; tc_gemm_smem_bytes<BN>()
// bytes of dynamic shared memory.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace wd {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;
constexpr int TC_THREADS = 128;
constexpr unsigned TC_SPIN_LIMIT = 1u << 26;   // default polls of an mbarrier before giving up

enum TcLayout { TC_NT = 0, TC_TN = 1 };

struct TcArgs {
    const __nv_bfloat16 *A;   // NT: [M][K] row stride lda;  TN: [K][M] row stride lda
    const __nv_bfloat16 *B;   // NT: [N][K] row stride ldb;  TN: [K][N] row stride ldb
    float *D;                 // [M][N] row stride ldd (TN: split s at D + s * d_split)
    int lda, ldb, ldd;
    long k_total;             // reduction extent
    long k_split;             // TN: reduction rows per split (gridDim.z splits)
    long d_split;             // TN: elements between the splits' partial outputs
    int *err;                 // 1: a wait gave up; 2: the drain wait gave up too
    unsigned spin_limit;      // polls per wait
    int withhold;             // tests: issue no MMA (see above)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor, no swizzle.  K-major: lbo = byte
// offset of K-adjacent core matrices, sbo = of MN-adjacent 8-row groups;
// MN-major: lbo = of K-adjacent core matrices, sbo = of MN-adjacent ones.
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);            // start address
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;         // leading byte offset
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;         // stride byte offset
    d |= (uint64_t)1 << 46;                              // descriptor version
    return d;                                            // base offset 0, no swizzle
}

// Instruction descriptor of kind::f16: BF16 A and B, FP32 D; both operands
// K-major (NT) or both MN-major (TN: the transpose bits of A and B).
template <int BN, int LAYOUT>
__host__ __device__ constexpr uint32_t tc_idesc_bf16() {
    return (1u << 4)                                // D format: F32
           | (1u << 7)                              // A format: BF16
           | (1u << 10)                             // B format: BF16
           | (LAYOUT == TC_TN ? (1u << 15) | (1u << 16) : 0u)   // A, B MN-major
           | ((uint32_t)(BN >> 3) << 17)            // N / 8
           | ((uint32_t)(TC_BM >> 4) << 24);        // M / 16
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t phase, unsigned long long limit) {
    for (unsigned long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done) : "r"(mbar), "r"(phase) : "memory");
        if (done) return true;
    }
    return false;
}

constexpr int TC_STAGES = 3;
constexpr int TC_TILE_A = TC_BM * TC_BK * 2;   // bytes of one A tile

template <int BN> __host__ __device__ constexpr int tc_gemm_smem_bytes() {
    return TC_STAGES * (TC_TILE_A + BN * TC_BK * 2);
}
// The transposed form is launched with more than its ring needs (96 KB at
// most): with either reading of a descriptor's two byte offsets, every
// shared-memory address an MMA can form from it lies inside the CTA's
// allocation.
constexpr int TC_TN_SMEM_BYTES = 160 * 1024;

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                 :: "r"(smem_u32(smem_dst)), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(bar)) : "memory");
}

template <int BN, int LAYOUT>
__global__ void __launch_bounds__(TC_THREADS, 1) k_gemm_bf16_tc(const TcArgs p) {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "tcgen05 N for M = 128");
    constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;
    constexpr int TILE_B = BN * TC_BK * 2;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *const sA = smem;                            // TC_STAGES A tiles
    uint8_t *const sB = smem + TC_STAGES * TC_TILE_A;    // TC_STAGES B tiles
    __shared__ __align__(8) uint64_t mbar[TC_STAGES + 1];   // [TC_STAGES]: the drain barrier
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long m0 = (long)blockIdx.x * TC_BM;
    const long n0 = (long)blockIdx.y * BN;
    long k_begin = 0, k_end = p.k_total;
    float *D = p.D;
    if (LAYOUT == TC_TN) {
        k_begin = (long)blockIdx.z * p.k_split;
        k_end = k_begin + p.k_split < p.k_total ? k_begin + p.k_split : p.k_total;
        D += (long)blockIdx.z * p.d_split;
    }

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_slot)), "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b <= TC_STAGES; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[b]))
                         : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // cp.async of the A and B tiles of reduction step `step` into buffer `buf`
    auto load_step = [&](int step, int buf) {
        const long k0 = k_begin + (long)step * TC_BK;
        uint8_t *a = sA + buf * TC_TILE_A, *b = sB + buf * TILE_B;
        if (LAYOUT == TC_NT) {
            for (int i = tid; i < TC_BM * 8; i += TC_THREADS) {
                const int r = i >> 3, c = i & 7;
                cp_async16(a + (r >> 3) * 1024 + c * 128 + (r & 7) * 16, p.A + (m0 + r) * p.lda + k0 + c * 8);
            }
            for (int i = tid; i < BN * 8; i += TC_THREADS) {
                const int r = i >> 3, c = i & 7;
                cp_async16(b + (r >> 3) * 1024 + c * 128 + (r & 7) * 16, p.B + (n0 + r) * p.ldb + k0 + c * 8);
            }
        } else {
            // row k of the step, 8-element group g along M (N): core matrix
            // (k / 8, g) at ((k / 8) * groups + g) * 128, row k % 8
            constexpr int GA = TC_BM / 8, GB = BN / 8;
            for (int i = tid; i < TC_BK * GA; i += TC_THREADS) {
                const int k = i / GA, g = i - k * GA;
                cp_async16(a + ((k >> 3) * GA + g) * 128 + (k & 7) * 16, p.A + (k0 + k) * p.lda + m0 + g * 8);
            }
            for (int i = tid; i < TC_BK * GB; i += TC_THREADS) {
                const int k = i / GB, g = i - k * GB;
                cp_async16(b + ((k >> 3) * GB + g) * 128 + (k & 7) * 16, p.B + (k0 + k) * p.ldb + n0 + g * 8);
            }
        }
    };

    const int nk = (int)((k_end - k_begin) / TC_BK);
#pragma unroll
    for (int st = 0; st < TC_STAGES - 1; ++st) {
        if (st < nk) load_step(st, st);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    uint32_t phase_bits = 0;   // bit b: parity of the next completion of mbar[b]
    bool ok = true;
    for (int i = 0; i < nk; ++i) {
        // step i's tiles have landed once at most TC_STAGES - 2 newer groups are pending
        asm volatile("cp.async.wait_group %0;" :: "n"(TC_STAGES - 2) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0 && !p.withhold) {
            const int b = i % TC_STAGES;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
                uint64_t ad, bd;
                if (LAYOUT == TC_NT) {
                    ad = tc_smem_desc(smem_u32(sA + b * TC_TILE_A) + kk * 256, 128, 1024);
                    bd = tc_smem_desc(smem_u32(sB + b * TILE_B) + kk * 256, 128, 1024);
                } else {   // 16 K rows = two K-adjacent core matrices per MMA
                    constexpr uint32_t LA = (TC_BM / 8) * 128, LB = (BN / 8) * 128;
                    ad = tc_smem_desc(smem_u32(sA + b * TC_TILE_A) + kk * 2 * LA, LA, 128);
                    bd = tc_smem_desc(smem_u32(sB + b * TILE_B) + kk * 2 * LB, LB, 128);
                }
                const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                    :: "r"(tmem), "l"(ad), "l"(bd), "r"(tc_idesc_bf16<BN, LAYOUT>()), "r"(acc)
                    : "memory");
            }
            tc_commit(&mbar[b]);
        }
        // refill the buffer step i - 1 read (its MMAs are queued ahead of step i's)
        const int nxt = i + TC_STAGES - 1;
        if (nxt < nk) {
            const int nb = nxt % TC_STAGES;
            if (i > 0) {
                ok = __syncthreads_and(
                         tc_wait(smem_u32(&mbar[nb]), (phase_bits >> nb) & 1u, p.spin_limit) ? 1 : 0) != 0;
                phase_bits ^= 1u << nb;
                if (!ok) break;   // no MMA is issued after a failed wait
            }
            load_step(nxt, nb);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (ok && nk > 0) {   // MMAs complete in order: the last step's arrival covers all
        const int lb = (nk - 1) % TC_STAGES;
        ok = __syncthreads_and(tc_wait(smem_u32(&mbar[lb]), (phase_bits >> lb) & 1u, p.spin_limit) ? 1 : 0) != 0;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
        float *drow = D + (m0 + 32 * warp + lane) * (long)p.ldd + n0;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t v[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                  "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                  "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(tmem + lane_base + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 16; j += 4)
                *reinterpret_cast<float4 *>(drow + c0 + j) =
                    make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]),
                                __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]));
        }
    } else {
        // drain: a commit arrives once every MMA this thread issued has
        // completed (at once if none is in flight); TMEM is freed after that
        if (tid == 0) {
            atomicExch(p.err, 1);
            tc_commit(&mbar[TC_STAGES]);
        }
        const bool drained = tc_wait(smem_u32(&mbar[TC_STAGES]), 0u, 64ull * p.spin_limit);
        if (!drained && tid == 0) atomicExch(p.err, 2);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(tmem), "r"(TMEM_COLS) : "memory");
}

}  // namespace wd
