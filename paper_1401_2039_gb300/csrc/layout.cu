// Conversions between the canonical boundary layout (FP64 complex,
// array-of-structures, lexicographic sites) and the internal layout
// (structure-of-arrays planes, one array per parity, storage precision).
#include "wd_internal.cuh"

namespace wd {

constexpr int LAYOUT_BLOCK = 128;

inline unsigned layout_grid(long n) {
    long b = (n + LAYOUT_BLOCK - 1) / LAYOUT_BLOCK;
    return (unsigned)(b < 1 ? 1 : b);
}

__device__ __forceinline__ void load_canonical(const double *src, long site, double *v, int n) {
    const double2 *p = reinterpret_cast<const double2 *>(src + (long)site * n);
    for (int i = 0; i < n / 2; ++i) {
        double2 d = p[i];
        v[2 * i] = d.x;
        v[2 * i + 1] = d.y;
    }
}

// Spinor records (24 doubles, 12 chunks of 16 bytes) of a block's
// LAYOUT_BLOCK consecutive sites pass through shared memory: the canonical
// side moves the block's contiguous chunks with consecutive threads on
// consecutive chunks (coalesced), the internal side handles one record per
// thread.  Records are padded to 13 chunks in shared memory, so that the
// per-record accesses of 8 consecutive threads fall in distinct banks.
constexpr int SPIN_CHUNKS = 12, SPIN_PAD = 13;

__device__ __forceinline__ void canonical_block_in(const double *src, long first, long n,
                                                   double2 *sm) {
    const double2 *g = reinterpret_cast<const double2 *>(src) + first * SPIN_CHUNKS;
    const long left = n - first;
    const int avail = (int)((left < LAYOUT_BLOCK ? left : LAYOUT_BLOCK) * SPIN_CHUNKS);
#pragma unroll 4
    for (int c = threadIdx.x; c < avail; c += LAYOUT_BLOCK)
        sm[(c / SPIN_CHUNKS) * SPIN_PAD + c % SPIN_CHUNKS] = __ldcs(g + c);
}

__device__ __forceinline__ void canonical_block_out(double *dst, long first, long n,
                                                    const double2 *sm) {
    double2 *g = reinterpret_cast<double2 *>(dst) + first * SPIN_CHUNKS;
    const long left = n - first;
    const int avail = (int)((left < LAYOUT_BLOCK ? left : LAYOUT_BLOCK) * SPIN_CHUNKS);
#pragma unroll 4
    for (int c = threadIdx.x; c < avail; c += LAYOUT_BLOCK)
        __stcs(g + c, sm[(c / SPIN_CHUNKS) * SPIN_PAD + c % SPIN_CHUNKS]);
}

__device__ __forceinline__ void record_from_smem(const double2 *sm, double *v) {
    const double2 *p = sm + threadIdx.x * SPIN_PAD;
#pragma unroll
    for (int i = 0; i < SPIN_CHUNKS; ++i) {
        const double2 d = p[i];
        v[2 * i] = d.x;
        v[2 * i + 1] = d.y;
    }
}

__device__ __forceinline__ void record_to_smem(double2 *sm, const double *v) {
    double2 *p = sm + threadIdx.x * SPIN_PAD;
#pragma unroll
    for (int i = 0; i < SPIN_CHUNKS; ++i) p[i] = make_double2(v[2 * i], v[2 * i + 1]);
}

template <typename S>
__global__ void __launch_bounds__(LAYOUT_BLOCK) k_pack_half(Geom g, void *dst, const double *src) {
    __shared__ double2 sm[LAYOUT_BLOCK * SPIN_PAD];
    const long first = (long)blockIdx.x * LAYOUT_BLOCK, h = first + threadIdx.x;
    canonical_block_in(src, first, g.vh, sm);
    __syncthreads();
    if (h >= g.vh) return;
    double v[24];
    record_from_smem(sm, v);
    Rec<S, 24>::store(dst, g.stride, h, v);
}

template <typename S>
__global__ void __launch_bounds__(LAYOUT_BLOCK) k_unpack_half(Geom g, double *dst, const void *src) {
    __shared__ double2 sm[LAYOUT_BLOCK * SPIN_PAD];
    const long first = (long)blockIdx.x * LAYOUT_BLOCK, h = first + threadIdx.x;
    if (h < g.vh) {
        double v[24];
        Rec<S, 24>::template load_coherent<double>(src, g.stride, h, v);
        record_to_smem(sm, v);
    }
    __syncthreads();
    canonical_block_out(dst, first, g.vh, sm);
}

// parity of lexicographic site lex (32-bit arithmetic: volumes stay below 2^31;
// 64-bit division costs tens of instructions per site)
__device__ __forceinline__ int lex_parity(const Geom &g, long lex) {
    unsigned r = (unsigned)lex;
    unsigned q = r / (unsigned)g.L[0];
    int par = (int)(r - q * (unsigned)g.L[0]);
    r = q / (unsigned)g.L[1];
    par += (int)(q - r * (unsigned)g.L[1]);
    q = r / (unsigned)g.L[2];
    par += (int)(r - q * (unsigned)g.L[2]) + (int)q;
    return par & 1;
}

// canonical sites [lex0, lex1) of the full lattice
template <typename S>
__global__ void __launch_bounds__(LAYOUT_BLOCK) k_pack_full(Geom g, void *even, void *odd,
                                                            const double *src, long lex0,
                                                            long lex1) {
    __shared__ double2 sm[LAYOUT_BLOCK * SPIN_PAD];
    const long first = lex0 + (long)blockIdx.x * LAYOUT_BLOCK, lex = first + threadIdx.x;
    canonical_block_in(src, first, lex1, sm);
    __syncthreads();
    if (lex >= lex1) return;
    double v[24];
    record_from_smem(sm, v);
    Rec<S, 24>::store(lex_parity(g, lex) ? odd : even, g.stride, lex >> 1, v);
}

template <typename S>
__global__ void __launch_bounds__(LAYOUT_BLOCK) k_unpack_full(Geom g, double *dst, const void *even,
                                                              const void *odd) {
    __shared__ double2 sm[LAYOUT_BLOCK * SPIN_PAD];
    const long first = (long)blockIdx.x * LAYOUT_BLOCK, lex = first + threadIdx.x;
    if (lex < 2 * g.vh) {
        double v[24];
        Rec<S, 24>::template load_coherent<double>(lex_parity(g, lex) ? odd : even, g.stride,
                                                    lex >> 1, v);
        record_to_smem(sm, v);
    }
    __syncthreads();
    canonical_block_out(dst, first, 2 * g.vh, sm);
}

// One thread per (site, direction): the link's first RECON reals (row-major,
// so 12 keeps rows 0 and 1).
template <typename S, int RECON>
__global__ void k_pack_gauge(Geom g, char *even, char *odd, size_t dir_bytes, const double *U) {
    const long i = (long)blockIdx.x * LAYOUT_BLOCK + threadIdx.x;
    if (i >= 8 * g.vh) return;
    const long lex = i >> 2;
    const int mu = (int)(i & 3);
    double v[18];
    load_canonical(U, i, v, 18);
    char *base = (lex_parity(g, lex) ? odd : even) + mu * dir_bytes;
    Rec<S, RECON>::store(base, g.stride, lex >> 1, v);
}

#define WD_STORE_DISPATCH(prec, KERNEL, ...)                                              \
    switch (prec) {                                                                       \
    case WD_F64: KERNEL<double><<<grid, LAYOUT_BLOCK, 0, s>>>(__VA_ARGS__); break;        \
    case WD_F32: KERNEL<float><<<grid, LAYOUT_BLOCK, 0, s>>>(__VA_ARGS__); break;         \
    case WD_F16: KERNEL<__half><<<grid, LAYOUT_BLOCK, 0, s>>>(__VA_ARGS__); break;        \
    case WD_BF16: KERNEL<__nv_bfloat16><<<grid, LAYOUT_BLOCK, 0, s>>>(__VA_ARGS__); break;\
    case WD_DF64: KERNEL<df64><<<grid, LAYOUT_BLOCK, 0, s>>>(__VA_ARGS__); break;         \
    default: return cudaErrorInvalidValue;                                                \
    }

cudaError_t launch_pack_half(int prec, const Geom &g, void *dst, const double *src,
                             cudaStream_t s) {
    const unsigned grid = layout_grid(g.vh);
    WD_STORE_DISPATCH(prec, k_pack_half, g, dst, src);
    return cudaGetLastError();
}

cudaError_t launch_unpack_half(int prec, const Geom &g, double *dst, const void *src,
                               cudaStream_t s) {
    const unsigned grid = layout_grid(g.vh);
    WD_STORE_DISPATCH(prec, k_unpack_half, g, dst, src);
    return cudaGetLastError();
}

cudaError_t launch_pack_full(int prec, const Geom &g, void *dst_even, void *dst_odd,
                             const double *src, cudaStream_t s, long lex0, long lex1) {
    if (lex1 < 0) lex1 = 2 * g.vh;
    if (lex0 < 0 || lex1 > 2 * g.vh || lex0 > lex1) return cudaErrorInvalidValue;
    if (lex0 == lex1) return cudaSuccess;
    const unsigned grid = layout_grid(lex1 - lex0);
    WD_STORE_DISPATCH(prec, k_pack_full, g, dst_even, dst_odd, src, lex0, lex1);
    return cudaGetLastError();
}

cudaError_t launch_unpack_full(int prec, const Geom &g, double *dst, const void *src_even,
                               const void *src_odd, cudaStream_t s) {
    const unsigned grid = layout_grid(2 * g.vh);
    WD_STORE_DISPATCH(prec, k_unpack_full, g, dst, src_even, src_odd);
    return cudaGetLastError();
}

cudaError_t launch_pack_gauge(const GaugeSet &gs, const Geom &g, const double *U,
                              cudaStream_t s) {
    const unsigned grid = layout_grid(8 * g.vh);
    char *e = (char *)gs.ptr[0], *o = (char *)gs.ptr[1];
#define WD_G(S)                                                                              \
    if (gs.recon == 12) k_pack_gauge<S, 12><<<grid, LAYOUT_BLOCK, 0, s>>>(g, e, o, gs.dir_bytes, U); \
    else k_pack_gauge<S, 18><<<grid, LAYOUT_BLOCK, 0, s>>>(g, e, o, gs.dir_bytes, U)
    switch (gs.prec) {
    case WD_F64: WD_G(double); break;
    case WD_F32: WD_G(float); break;
    case WD_F16: WD_G(__half); break;
    case WD_BF16: WD_G(__nv_bfloat16); break;
    case WD_DF64: WD_G(df64); break;
    default: return cudaErrorInvalidValue;
    }
#undef WD_G
    return cudaGetLastError();
}

}  // namespace wd
