// BF16 x BF16 -> FP32 GEMM on the fifth-generation tensor cores (tcgen05).
//
//   D[M x N] = A[M x K] * B[N x K]^T      (A, B row-major with K contiguous)
//
// One CTA of four warps computes a 128 x BN tile of D.  The K loop runs over
// steps of 64 through a ring of TC_STAGES shared-memory buffers: the four
// warps copy the A and B tiles of step i + TC_STAGES - 1 from global memory
// with cp.async (16-byte chunks, no register staging) into the K-major,
// no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix, core
// matrices adjacent in K 128 bytes apart, 8-row groups 1024 bytes apart)
// while the tensor cores work on step i, so the loads of later steps overlap
// the MMAs.  For each step one elected thread issues four 128 x BN x 16
// tcgen05.mma operations that accumulate in tensor memory (TMEM, BN fp32
// columns x 128 lanes) and a tcgen05.commit that arrives on the step
// buffer's mbarrier when the MMAs have consumed it; a buffer is refilled only
// after that arrival.  Every wait on an mbarrier is bounded and, if the bound
// is hit, the kernel records an error and skips the remaining work instead
// of hanging.  The epilogue moves the accumulator from TMEM to registers
// with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31, i.e. rows
// 32w..32w+31 of the tile) and stores it.
//
// Requirements (checked by the host launcher): M % 128 == 0, N % BN == 0,
// K % 64 == 0, 16-byte aligned rows; tc_gemm_smem_bytes<BN>() bytes of
// dynamic shared memory.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace wd {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;
constexpr int TC_THREADS = 128;
constexpr unsigned TC_SPIN_LIMIT = 1u << 26;   // polls of an mbarrier before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: K-major, no swizzle.
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);            // start address
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;         // leading (K) byte offset
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;         // stride (M/N) byte offset
    d |= (uint64_t)1 << 46;                              // descriptor version
    return d;                                            // base offset 0, no swizzle
}

// Instruction descriptor of kind::f16: BF16 A and B, FP32 D, both K-major.
template <int BN>
__host__ __device__ constexpr uint32_t tc_idesc_bf16() {
    return (1u << 4)                                // D format: F32
           | (1u << 7)                              // A format: BF16
           | (1u << 10)                             // B format: BF16
           | ((uint32_t)(BN >> 3) << 17)            // N / 8
           | ((uint32_t)(TC_BM >> 4) << 24);        // M / 16
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t phase) {
    for (unsigned it = 0; it < TC_SPIN_LIMIT; ++it) {
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

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                 :: "r"(smem_u32(smem_dst)), "l"(gmem_src) : "memory");
}

template <int BN>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_gemm_bf16_tc(const __nv_bfloat16 *__restrict__ A, const __nv_bfloat16 *__restrict__ B,
               float *__restrict__ D, int K, int lda, int ldb, int ldd, int *err) {
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "tcgen05 N for M = 128");
    constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;
    constexpr int TILE_B = BN * TC_BK * 2;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *const sA = smem;                            // TC_STAGES A tiles
    uint8_t *const sB = smem + TC_STAGES * TC_TILE_A;    // TC_STAGES B tiles
    __shared__ __align__(8) uint64_t mbar[TC_STAGES];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long m0 = (long)blockIdx.x * TC_BM;
    const long n0 = (long)blockIdx.y * BN;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_slot)), "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int b = 0; b < TC_STAGES; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar[b]))
                         : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // cp.async of the A and B tiles of K step `step` into ring buffer `buf`
    auto load_step = [&](int step, int buf) {
        const int k0 = step * TC_BK;
        uint8_t *a = sA + buf * TC_TILE_A, *b = sB + buf * TILE_B;
        for (int i = tid; i < TC_BM * 8; i += TC_THREADS) {
            const int r = i >> 3, c = i & 7;
            cp_async16(a + (r >> 3) * 1024 + c * 128 + (r & 7) * 16, A + (m0 + r) * lda + k0 + c * 8);
        }
        for (int i = tid; i < BN * 8; i += TC_THREADS) {
            const int r = i >> 3, c = i & 7;
            cp_async16(b + (r >> 3) * 1024 + c * 128 + (r & 7) * 16, B + (n0 + r) * ldb + k0 + c * 8);
        }
    };

    const int nk = K / TC_BK;
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
        if (tid == 0) {
            const int b = i % TC_STAGES;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
                const uint64_t ad = tc_smem_desc(smem_u32(sA + b * TC_TILE_A) + kk * 256, 128, 1024);
                const uint64_t bd = tc_smem_desc(smem_u32(sB + b * TILE_B) + kk * 256, 128, 1024);
                const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                    :: "r"(tmem), "l"(ad), "l"(bd), "r"(tc_idesc_bf16<BN>()), "r"(acc)
                    : "memory");
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                :: "r"(smem_u32(&mbar[b])) : "memory");
        }
        // refill the buffer step i - 1 read (its MMAs are queued ahead of step i's)
        const int nxt = i + TC_STAGES - 1;
        if (nxt < nk) {
            const int nb = nxt % TC_STAGES;
            if (i > 0) {
                ok = __syncthreads_and(
                         tc_wait(smem_u32(&mbar[nb]), (phase_bits >> nb) & 1u) ? 1 : 0) != 0;
                phase_bits ^= 1u << nb;
                if (!ok) break;
            }
            load_step(nxt, nb);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (ok && nk > 0) {   // MMAs complete in order: the last step's arrival covers all
        const int lb = (nk - 1) % TC_STAGES;
        ok = __syncthreads_and(tc_wait(smem_u32(&mbar[lb]), (phase_bits >> lb) & 1u) ? 1 : 0) != 0;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
        float *drow = D + (m0 + 32 * warp + lane) * (long)ldd + n0;
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
        if (tid == 0) atomicExch(err, 1);
        // give MMAs still in flight a bounded chance to retire before TMEM is freed
        if (nk > 0) {
            const int lb = (nk - 1) % TC_STAGES;
            tc_wait(smem_u32(&mbar[lb]), (phase_bits >> lb) & 1u);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                     :: "r"(tmem), "r"(TMEM_COLS) : "memory");
}

}  // namespace wd
