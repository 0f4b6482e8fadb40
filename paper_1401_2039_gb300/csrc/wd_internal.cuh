// Internal declarations of libwd: storage-precision traits, the
// structure-of-arrays field layout, vectorised loads/stores and lattice
// geometry shared by the kernels.
//
// Field layout (one parity, Vh sites, site index h = lex / 2):
//   a record of N reals of storage type S occupies N*sizeof(S) bytes split
//   into NF = bytes / 16 planes of 16-byte vectors followed by one tail plane
//   of (bytes % 16) bytes per site; plane j of site h lives at
//   base + j * stride * 16 + h * 16 and the tail at base + NF * stride * 16 +
//   h * tail.  Consecutive threads (consecutive h) therefore read consecutive
//   16-byte words: every load of a warp is one fully-used 512-byte request.
//   stride = Vh rounded up to a multiple of 64 sites; padding stays zero.
//   Spinor records are 24 reals ([colour][spin][re,im]); link records are 18
//   reals (3x3, row-major) or 12 (rows 0 and 1).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/wd.h"
#include "df64.cuh"

namespace wd {

// ---------------------------------------------------------------- precision
template <int P> struct Prec;
template <> struct Prec<WD_F64> { using S = double;        using R = double; };
template <> struct Prec<WD_F32> { using S = float;         using R = float;  };
template <> struct Prec<WD_F16> { using S = __half;        using R = float;  };
template <> struct Prec<WD_BF16> { using S = __nv_bfloat16; using R = float; };

// Internal precision code of double-float fields (FP64-sized, FP32 pipes).
constexpr int WD_DF64 = 4;
// hop launches only: double-float fields and links read in FP32 arithmetic
constexpr int WD_DF64_F32 = 5;
template <> struct Prec<WD_DF64> { using S = df64; using R = df64; };

inline size_t prec_bytes(int p) {
    return (p == WD_F64 || p == WD_DF64) ? 8 : p == WD_F32 ? 4 : 2;
}

// Bytes of one field of Vh records of nreal reals in precision p.
inline size_t field_bytes(int p, long stride, int nreal) {
    size_t rec = (size_t)nreal * prec_bytes(p);
    size_t nf = rec / 16, tail = rec % 16;
    return nf * stride * 16 + tail * stride;
}

inline long pad_stride(long vh) { return (vh + 63) / 64 * 64; }

// ---------------------------------------------------------------- loads
__device__ __forceinline__ uint4 ld_nc_v4(const void *p) {
    uint4 v;
    asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}
// Streaming load that is not kept in L1 (links: each is read once per launch).
__device__ __forceinline__ uint4 ld_stream_v4(const void *p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ uint2 ld_stream_v2(const void *p) {
    uint2 v;
    asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];"
                 : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_stream_u32(const void *p) {
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint4 ld_v4(const void *p) {
    return *reinterpret_cast<const uint4 *>(p);
}
__device__ __forceinline__ void st_v4(void *p, uint4 v) { *reinterpret_cast<uint4 *>(p) = v; }
__device__ __forceinline__ void st_v2(void *p, uint2 v) { *reinterpret_cast<uint2 *>(p) = v; }
__device__ __forceinline__ void st_u32(void *p, uint32_t v) { *reinterpret_cast<uint32_t *>(p) = v; }

// ---------------------------------------------------------------- word <-> real
template <typename S, typename R> struct Words;
template <> struct Words<double, double> {
    static constexpr int per_word = 0;  // two words per real
    __device__ static void unpack(const uint32_t *w, double *r, int n) {
#pragma unroll
        for (int i = 0; i < n; ++i) r[i] = __hiloint2double((int)w[2 * i + 1], (int)w[2 * i]);
    }
    __device__ static void pack(const double *r, uint32_t *w, int n) {
#pragma unroll
        for (int i = 0; i < n; ++i) {
            w[2 * i] = (uint32_t)__double2loint(r[i]);
            w[2 * i + 1] = (uint32_t)__double2hiint(r[i]);
        }
    }
};
template <> struct Words<float, float> {
    __device__ static void unpack(const uint32_t *w, float *r, int n) {
#pragma unroll
        for (int i = 0; i < n; ++i) r[i] = __uint_as_float(w[i]);
    }
    __device__ static void pack(const float *r, uint32_t *w, int n) {
#pragma unroll
        for (int i = 0; i < n; ++i) w[i] = __float_as_uint(r[i]);
    }
};
template <> struct Words<__half, float> {
    __device__ static void unpack(const uint32_t *w, float *r, int n) {
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            __half2 h = *reinterpret_cast<const __half2 *>(&w[i]);
            float2 f = __half22float2(h);
            r[2 * i] = f.x;
            r[2 * i + 1] = f.y;
        }
    }
    __device__ static void pack(const float *r, uint32_t *w, int n) {
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            __half2 h = __floats2half2_rn(r[2 * i], r[2 * i + 1]);
            w[i] = *reinterpret_cast<uint32_t *>(&h);
        }
    }
};
template <> struct Words<__nv_bfloat16, float> {
    __device__ static void unpack(const uint32_t *w, float *r, int n) {
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(&w[i]);
            float2 f = __bfloat1622float2(h);
            r[2 * i] = f.x;
            r[2 * i + 1] = f.y;
        }
    }
    __device__ static void pack(const float *r, uint32_t *w, int n) {
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            __nv_bfloat162 h = __floats2bfloat162_rn(r[2 * i], r[2 * i + 1]);
            w[i] = *reinterpret_cast<uint32_t *>(&h);
        }
    }
};

// Low-precision storage read into / written from FP64 registers (layout
// conversions and the reliable-update kernels): go through the FP32 form;
// FP32 -> FP64 is exact and FP64 -> FP16/BF16 rounds once via FP32.
template <typename S> struct WordsViaFloat {
    __device__ static void unpack(const uint32_t *w, double *r, int n) {
        float f[24];
        Words<S, float>::unpack(w, f, n);
#pragma unroll
        for (int i = 0; i < n; ++i) r[i] = (double)f[i];
    }
    __device__ static void pack(const double *r, uint32_t *w, int n) {
        float f[24];
#pragma unroll
        for (int i = 0; i < n; ++i) f[i] = (float)r[i];
        Words<S, float>::pack(f, w, n);
    }
};
template <> struct Words<float, double> : WordsViaFloat<float> {};
template <> struct Words<__half, double> : WordsViaFloat<__half> {};
template <> struct Words<__nv_bfloat16, double> : WordsViaFloat<__nv_bfloat16> {};

// Double-float storage: word pairs (hi, lo).
template <> struct Words<df64, df64> {
    __device__ static void unpack(const uint32_t *w, df64 *r, int n) {
#pragma unroll
        for (int i = 0; i < n; ++i) r[i] = df64(__uint_as_float(w[2 * i]), __uint_as_float(w[2 * i + 1]));
    }
    __device__ static void pack(const df64 *r, uint32_t *w, int n) {
#pragma unroll
        for (int i = 0; i < n; ++i) {
            w[2 * i] = __float_as_uint(r[i].hi);
            w[2 * i + 1] = __float_as_uint(r[i].lo);
        }
    }
};
// ... from / to FP64 registers (layout conversions at the boundary)
template <> struct Words<df64, double> {
    __device__ static void unpack(const uint32_t *w, double *r, int n) {
#pragma unroll
        for (int i = 0; i < n; ++i)
            r[i] = (double)__uint_as_float(w[2 * i]) + (double)__uint_as_float(w[2 * i + 1]);
    }
    __device__ static void pack(const double *r, uint32_t *w, int n) {
#pragma unroll
        for (int i = 0; i < n; ++i) {
            const df64 v = split_double(r[i]);
            w[2 * i] = __float_as_uint(v.hi);
            w[2 * i + 1] = __float_as_uint(v.lo);
        }
    }
};
// ... to FP32 registers (the low-precision copy of a residual)
template <> struct Words<df64, float> {
    __device__ static void unpack(const uint32_t *w, float *r, int n) {
#pragma unroll
        for (int i = 0; i < n; ++i) r[i] = __uint_as_float(w[2 * i]) + __uint_as_float(w[2 * i + 1]);
    }
    __device__ static void pack(const float *r, uint32_t *w, int n) {
#pragma unroll
        for (int i = 0; i < n; ++i) {
            w[2 * i] = __float_as_uint(r[i]);
            w[2 * i + 1] = 0u;
        }
    }
};

// A record of N reals of storage type S in the SoA layout described above.
template <typename S, int N> struct Rec {
    static constexpr int BYTES = N * (int)sizeof(S);
    static constexpr int NF = BYTES / 16;
    static constexpr int TAIL = BYTES % 16;
    static constexpr int WORDS = BYTES / 4;
    static_assert(TAIL == 0 || TAIL == 4 || TAIL == 8, "unsupported record");

    // LoadKind: 0 = read-only cached (spinors), 1 = streaming (links).
    template <int KIND>
    __device__ __forceinline__ static void load_words(const char *base, long stride, long h,
                                                      uint32_t *w) {
#pragma unroll
        for (int j = 0; j < NF; ++j) {
            const char *p = base + ((long)j * stride + h) * 16;
            uint4 v = KIND ? ld_stream_v4(p) : ld_nc_v4(p);
            w[4 * j] = v.x; w[4 * j + 1] = v.y; w[4 * j + 2] = v.z; w[4 * j + 3] = v.w;
        }
        if (TAIL == 8) {
            uint2 v = ld_stream_v2(base + (long)NF * stride * 16 + h * 8);
            w[4 * NF] = v.x; w[4 * NF + 1] = v.y;
        } else if (TAIL == 4) {
            w[4 * NF] = ld_stream_u32(base + (long)NF * stride * 16 + h * 4);
        }
    }
    template <typename R, int KIND = 0>
    __device__ __forceinline__ static void load(const void *base, long stride, long h, R *r) {
        uint32_t w[WORDS];
        load_words<KIND>((const char *)base, stride, h, w);
        Words<S, R>::unpack(w, r, N);
    }
    // Plain (coherent) load, for fields the same kernel may have written.
    template <typename R>
    __device__ __forceinline__ static void load_coherent(const void *base, long stride, long h,
                                                         R *r) {
        static_assert(TAIL == 0, "coherent loads only for whole 16-byte records");
        uint32_t w[WORDS];
#pragma unroll
        for (int j = 0; j < NF; ++j) {
            uint4 v = ld_v4((const char *)base + ((long)j * stride + h) * 16);
            w[4 * j] = v.x; w[4 * j + 1] = v.y; w[4 * j + 2] = v.z; w[4 * j + 3] = v.w;
        }
        Words<S, R>::unpack(w, r, N);
    }
    template <typename R>
    __device__ __forceinline__ static void store(void *base, long stride, long h, const R *r) {
        uint32_t w[WORDS];
        Words<S, R>::pack(r, w, N);
        char *b = (char *)base;
#pragma unroll
        for (int j = 0; j < NF; ++j)
            st_v4(b + ((long)j * stride + h) * 16,
                  make_uint4(w[4 * j], w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]));
        if (TAIL == 8) st_v2(b + (long)NF * stride * 16 + h * 8, make_uint2(w[4 * NF], w[4 * NF + 1]));
        else if (TAIL == 4) st_u32(b + (long)NF * stride * 16 + h * 4, w[4 * NF]);
    }
};

// One 16-byte chunk of a spinor field as 16 / sizeof(S) reals of type R.
template <typename S, typename R> struct Chunk16 {
    static constexpr int K = 16 / (int)sizeof(S);
    __device__ __forceinline__ static void load(const void *base, long i, R *r) {
        uint4 v = ld_v4((const char *)base + i * 16);
        uint32_t w[4] = {v.x, v.y, v.z, v.w};
        Words<S, R>::unpack(w, r, K);
    }
    __device__ __forceinline__ static void store(void *base, long i, const R *r) {
        uint32_t w[4];
        Words<S, R>::pack(r, w, K);
        st_v4((char *)base + i * 16, make_uint4(w[0], w[1], w[2], w[3]));
    }
};

// ---------------------------------------------------------------- geometry
// Division of an index n < 2^31 by an invariant d >= 1 as one widening
// multiply and a shift (Granlund and Montgomery, "Division by invariant
// integers using multiplication", PLDI 1994, Thm. 4.2 with N = 31 bits):
// with l = ceil(log2 d) and m = floor(2^(31 + l) / d) + 1, 2^(31+l) < m d <=
// 2^(31+l) + 2^l, so floor(n / d) = floor(m n / 2^(31+l)); m < 2^32.
struct Divisor {
    unsigned m;     // multiplier
    unsigned s;     // shift, 31 + l
};

inline Divisor make_divisor(unsigned d) {
    unsigned l = 0;
    while (l < 32 && (1ull << l) < d) ++l;
    const unsigned s = 31 + l;
    return Divisor{(unsigned)((1ull << s) / d + 1), s};
}

__host__ __device__ __forceinline__ unsigned udiv(unsigned n, Divisor d) {
    return (unsigned)(((unsigned long long)n * d.m) >> d.s);
}

struct Geom {
    int L[4];       // Lx, Ly, Lz, Lt
    int hx;         // Lx / 2
    long vh;        // V / 2
    long stride;    // padded plane stride (sites)
    // half-lattice index step of a hop in direction mu = 1, 2, 3 (entry 0
    // unused: x hops depend on the site's parity) and the step back across
    // the periodic boundary, (L_mu - 1) * step
    unsigned step[4];
    unsigned back[4];
    Divisor div_hx, div_y, div_z;   // by hx, L[1], L[2] (site_coords)
};

// Geometry of a dims[0] x ... x dims[3] lattice (dims[0] even) whose fields
// have plane stride stride.
inline Geom make_geom(const int dims[4], long stride) {
    Geom g{};
    for (int m = 0; m < 4; ++m) g.L[m] = dims[m];
    g.hx = dims[0] / 2;
    g.vh = (long)dims[0] * dims[1] * dims[2] * dims[3] / 2;
    g.stride = stride;
    unsigned st = (unsigned)g.hx;
    for (int m = 1; m < 4; ++m) {
        g.step[m] = st;
        g.back[m] = (unsigned)(dims[m] - 1) * st;
        st *= (unsigned)dims[m];
    }
    g.div_hx = make_divisor((unsigned)g.hx);
    g.div_y = make_divisor((unsigned)dims[1]);
    g.div_z = make_divisor((unsigned)dims[2]);
    return g;
}

// Coordinates of half-lattice site h of parity p (32-bit arithmetic: the
// volume is limited to 2^31 sites).
__device__ __forceinline__ void site_coords(const Geom &g, long h, int p, int c[4]) {
    const unsigned hu = (unsigned)h;
    unsigned r = udiv(hu, g.div_hx);
    const int xh = (int)(hu - r * (unsigned)g.hx);
    const unsigned r1 = udiv(r, g.div_y);
    c[1] = (int)(r - r1 * (unsigned)g.L[1]);
    const unsigned r2 = udiv(r1, g.div_z);
    c[2] = (int)(r1 - r2 * (unsigned)g.L[2]);
    c[3] = (int)r2;
    c[0] = 2 * xh + ((c[1] + c[2] + c[3] + p) & 1);
}

__device__ __forceinline__ long half_index(const Geom &g, const int c[4]) {
    return ((((long)c[3] * g.L[2] + c[2]) * g.L[1] + c[1]) * g.L[0] + c[0]) >> 1;
}

// ---------------------------------------------------------------- reductions
// Scalars of the Krylov solver, resident in device memory so that kernels
// chain without host round trips.
struct SolverScalars {
    double nz;          // ||z||^2 of the current z = A^dag r
    double pAp;         // ||A p||^2
    double alpha, beta;
    double alpha_x;     // step still owed to x: the x += alpha p of the last
                        // iteration runs in the next p update (or the fold)
    double nr;          // ||r||^2 of the iterated residual
    double scratch[4];  // results of plain reductions
    int iter;           // iterations completed
    int flags;          // bit 0: breakdown (zero or non-finite denominator)
    int frozen;         // converged system of a batch: alpha = beta = 0 from now on
    double hist[64];    // ||r||^2 after iteration k at hist[k % 64]
};
static_assert(sizeof(SolverScalars) % 8 == 0, "copied in 8-byte words (launch_copy_small)");

enum FinalOp {
    FIN_NONE = 0,
    FIN_STORE0 = 1,   // scratch[0] = sum
    FIN_STORE1 = 2,   // scratch[1] = sum
    FIN_ALPHA = 3,    // pAp = sum; alpha = nz / pAp
    FIN_BETA = 4,     // beta = sum / nz; nz = sum
    FIN_NR = 5,       // nr = sum; hist[iter % 64] = sum; ++iter
    FIN_STORE2 = 6,   // scratch[2] = sum
    FIN_STORE3 = 7,   // scratch[3] = sum
};

// Partial sums of one reduction: one double per block, plus the arrival
// counter of the last-block-done pattern (reset by the last block).
struct Reduction {
    df64 *partials;          // per-block or per-warp partial sums
    unsigned int *counter;
    SolverScalars *scalars;
    int op;
};

__device__ __forceinline__ void apply_final(SolverScalars *s, int op, double sum) {
    switch (op) {
    case FIN_STORE0: s->scratch[0] = sum; break;
    case FIN_STORE1: s->scratch[1] = sum; break;
    case FIN_STORE2: s->scratch[2] = sum; break;
    case FIN_STORE3: s->scratch[3] = sum; break;
    case FIN_ALPHA: {
        s->pAp = sum;
        double a = 0.0;                   // z = 0: the residual vanished exactly
        if (s->nz != 0.0 && !s->frozen) {
            a = s->nz / sum;
            if (!(sum > 0.0) || !isfinite(a)) { s->flags |= 1; a = 0.0; }
        }
        s->alpha = a;
        s->alpha_x = a;
        break;
    }
    case FIN_BETA: {
        // nz = +inf before the first iteration gives beta = 0; so does z = 0
        if (s->frozen) { s->beta = 0.0; break; }
        double b = sum == 0.0 ? 0.0 : sum / s->nz;
        if (!isfinite(sum) || isnan(b)) { s->flags |= 1; b = 0.0; }
        s->beta = b;
        s->nz = sum;
        break;
    }
    case FIN_NR:
        if (s->frozen) break;
        s->nr = sum;
        s->hist[s->iter & 63] = sum;
        s->iter += 1;
        if (!isfinite(sum)) s->flags |= 1;
        break;
    default: break;
    }
}

// Reductions add in double-float arithmetic (df64.cuh) on the FP32 pipes.
// GB300 runs FP64 at a small fraction of its FP32 rate; a final pass over
// tens of thousands of partials in FP64 inside one block took 10-15 us, and
// FP64 shuffle trees in every warp of a hopping-term kernel added more.
// Double-float keeps about 48 significand bits, ample for the scalars of
// the iteration, and every sum below has a fixed tree, so results are
// reproducible bit for bit.
__device__ __forceinline__ double ldcg(const double *p) { return __ldcg(p); }
__device__ __forceinline__ df64 ldcg(const df64 *p) {
    const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    return df64(v.x, v.y);
}
__device__ __forceinline__ df64 to_df(float v) { return df64(v, 0.0f); }
__device__ __forceinline__ df64 to_df(double v) { return df64(v); }
__device__ __forceinline__ df64 to_df(df64 v) { return v; }

__device__ __forceinline__ df64 warp_sum(df64 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = v + df64(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
    return v;
}

// Arrival counting for "the last block to finish adds the partials".  One
// counter for thousands of blocks serialises their atomics in one L2 slice,
// so the count runs in two levels: block b bumps group counter b mod
// ARRIVE_GROUPS, each on its own 128-byte line; the block that completes a
// group bumps the top counter; the block that completes the top counter is
// the last one.  Counters are reset by the blocks that complete them, so
// they read zero again when the kernel ends.  Call from one thread after a
// __threadfence() that publishes the block's partials; the caller fences
// again before reading the other blocks' partials.
constexpr int ARRIVE_GROUPS = 64;
constexpr int ARRIVE_STRIDE = 32;   // unsigned ints per 128-byte line
constexpr int ARRIVE_WORDS = ARRIVE_STRIDE * (ARRIVE_GROUPS + 1);

__device__ __forceinline__ bool arrive_last(unsigned int *counters, unsigned int nblocks,
                                            unsigned int b) {
    const unsigned int g = b % ARRIVE_GROUPS;
    const unsigned int group_size = (nblocks - g + ARRIVE_GROUPS - 1) / ARRIVE_GROUPS;
    unsigned int *gc = counters + ARRIVE_STRIDE * (g + 1);
    if (atomicAdd(gc, 1u) != group_size - 1) return false;
    *gc = 0u;
    __threadfence();
    const unsigned int groups = nblocks < ARRIVE_GROUPS ? nblocks : ARRIVE_GROUPS;
    if (atomicAdd(counters, 1u) != groups - 1) return false;
    *counters = 0u;
    return true;
}

// sum_k p[(lane + k * LANES) * es] for k = 0, 1, ... while the index is
// below n, in that order.  The loads go out sixteen at a time so that a
// pass over thousands of partials is not a chain of dependent L2 round
// trips; the additions keep their order (out-of-range terms are zeros).
template <int LANES, typename T>
__device__ __forceinline__ T strided_sum(const T *p, long n, long lane, long es = 1) {
    constexpr int DEPTH = 16;
    T s = T(0);
    for (long base = lane; base < n; base += (long)LANES * DEPTH) {
        T t[DEPTH];
#pragma unroll
        for (int j = 0; j < DEPTH; ++j) {
            const long i = base + (long)j * LANES;
            t[j] = i < n ? ldcg(&p[i * es]) : T(0);
        }
#pragma unroll
        for (int j = 0; j < DEPTH; ++j) s = s + t[j];
    }
    return s;
}

// Block-wide sum of v (every thread of the block calls it), then the
// deterministic grid-wide finish: the last block to arrive adds the
// per-block partials in block order and applies the final operation.
template <int BLOCK, typename T>
__device__ __forceinline__ void block_reduce_finish(T v_in, const Reduction &red) {
    __shared__ df64 warp_sums[BLOCK / 32];
    __shared__ bool is_last;
    df64 v = warp_sum(to_df(v_in));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_sums[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        df64 s = 0;
#pragma unroll
        for (int i = 0; i < BLOCK / 32; ++i) s = s + warp_sums[i];
        red.partials[blockIdx.x] = s;
        __threadfence();
        is_last = arrive_last(red.counter, gridDim.x, blockIdx.x);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    df64 s = warp_sum(strided_sum<BLOCK>(red.partials, gridDim.x, threadIdx.x));
    __syncthreads();   // every thread has read warp_sums above
    if (lane == 0) warp_sums[wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        df64 t = 0;
#pragma unroll
        for (int i = 0; i < BLOCK / 32; ++i) t = t + warp_sums[i];
        apply_final(red.scalars, red.op, (double)t);
    }
}

// Sum of one value per output site whose rounding does not depend on the
// launch configuration, in two kernels.  The producing kernel writes one
// partial per 32-site warp -- site h = base + i * BLOCK + threadIdx.x, so
// warp w of step i covers sites [32 k, 32 k + 32) with k = (base + i * BLOCK)
// / 32 + w -- with no barrier, fence or atomic: a block's threads retire as
// soon as their sites are stored.  The one-block kernel behind
// launch_finish_partials then adds the ceil(n_sites / 32) partials in a
// fixed order and applies the final operation.  Sites past the end
// contribute zeros.
template <int BLOCK, int SPT>
__device__ __forceinline__ void warp_partials(const df64 (&v)[SPT], long n_sites,
                                              df64 *partials) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long n_warps = (n_sites + 31) / 32;
#pragma unroll
    for (int i = 0; i < SPT; ++i) {
        const df64 s = warp_sum(v[i]);
        const long k = ((long)blockIdx.x * BLOCK * SPT + (long)i * BLOCK) / 32 + wid;
        if (lane == 0 && k < n_warps) partials[k] = s;
    }
}

// ---------------------------------------------------------------- host side
struct Field {          // one parity spinor field in the internal layout
    void *ptr = nullptr;
    int prec = WD_F64;
};

struct GaugeSet {       // links of both parities, one precision/reconstruction
    void *ptr[2] = {nullptr, nullptr};  // [parity] -> 4 direction blocks
    size_t dir_bytes = 0;               // bytes of one direction block
    int prec = WD_F64;
    int recon = 18;
};

enum Epilogue { EPI_PLAIN = 0, EPI_XPAY = 1 };

struct DslashLaunch {
    Geom g;
    const GaugeSet *gauge;
    int out_parity;
    int dagger;
    double phase[8];
    void *out;
    const void *in;
    const void *x;       // EPI_XPAY: out = x + scale * H in
    double scale;
    int epi;
    const Reduction *red;  // optional ||out||^2
    int cfg = 0;           // launch configuration (tuned per operator)
    // twisted mass: t != 0 makes the xpay epilogue out = (1 + i t gamma5) x +
    // scale H in, and the plain one out = scale (1 - i t gamma5) H in
    double twist = 0.0;
    // output sites [h_begin, h_end) only (h_end < 0: to the end); a launch
    // with a fused norm covers every site
    long h_begin = 0, h_end = -1;
};

// bit mu set unless direction mu's boundary phase (re, im) is exactly (1, 0):
// the hop kernels skip the multiplication by a phase of 1
inline unsigned phase_mask(const double phase[8]) {
    unsigned m = 0;
    for (int mu = 0; mu < 4; ++mu)
        if (phase[2 * mu] != 1.0 || phase[2 * mu + 1] != 0.0) m |= 1u << mu;
    return m;
}

// dslash.cu
cudaError_t launch_dslash(const DslashLaunch &L, int prec, cudaStream_t s);

// blas.cu
// r -= alpha Ap and ||r||^2; then, next iteration, x += alpha_x p and
// p = z + beta p (the x step deferred into the pass over p)
cudaError_t launch_cg_update_r(int prec, const Geom &g, void *r, const void *Ap,
                               const Reduction &red, cudaStream_t s);
cudaError_t launch_cg_update_px(int prec, const Geom &g, void *x, void *p, const void *z,
                                const SolverScalars *sc, cudaStream_t s);
cudaError_t launch_norm2(int prec, const Geom &g, const void *v, const Reduction &red,
                         cudaStream_t s);
cudaError_t launch_xmy_norm(int prec, const Geom &g, void *out, const void *x, const void *y,
                            const Reduction &red, cudaStream_t s);
// out = c (1 + i t gamma5) in on a residual-precision (FP64 or double-float)
// half-lattice field, site by site (in place allowed).
cudaError_t launch_twist_hi(int prec, const Geom &g, void *out, const void *in, double t, double c,
                            cudaStream_t s);
// Adds the n partials warp_partials wrote (fixed order) and applies red.op.
cudaError_t launch_finish_partials(const Reduction &red, long n, cudaStream_t s);
// copies by the SMs (not the copy engines): small (bytes, addresses multiples
// of 8; either side may be mapped host memory) and whole fields (multiples of 16)
cudaError_t launch_copy_small(void *dst, const void *src, size_t bytes, cudaStream_t s);
cudaError_t launch_copy_field(void *dst, const void *src, size_t bytes, cudaStream_t s);
cudaError_t launch_xpay_hi(int prec, const Geom &g, void *out, const void *y, double a,
                           const void *x, cudaStream_t s);
cudaError_t launch_f64_df64(void *buf, long n_reals, int to_df, cudaStream_t s);
cudaError_t launch_convert_scaled(int prec_out, void *out, int prec_in, const void *in,
                                  const Geom &g, const double *scale_dev, double scale_host,
                                  cudaStream_t s);
// x_lo += alpha_x p (the owed step, then alpha_x = 0); x_hi += x_lo / scale;
// x_lo = 0
cudaError_t launch_fold_x(int prec_lo, int prec_hi, const Geom &g, void *x_hi, void *x_lo,
                          const void *p, SolverScalars *sc, const double *inv_scale_dev,
                          cudaStream_t s);
cudaError_t launch_rescale_lo(int prec_lo, const Geom &g, void *p, SolverScalars *sc,
                              const double *ratio_dev, cudaStream_t s);
int reduction_blocks(const Geom &g);

// layout.cu
cudaError_t launch_pack_half(int prec, const Geom &g, void *dst, const double *src,
                             cudaStream_t s);
cudaError_t launch_unpack_half(int prec, const Geom &g, double *dst, const void *src,
                               cudaStream_t s);
// canonical sites [lex0, lex1) (lex1 < 0: to the end)
cudaError_t launch_pack_full(int prec, const Geom &g, void *dst_even, void *dst_odd,
                             const double *src, cudaStream_t s, long lex0 = 0, long lex1 = -1);
cudaError_t launch_unpack_full(int prec, const Geom &g, double *dst, const void *src_even,
                               const void *src_odd, cudaStream_t s);
cudaError_t launch_pack_gauge(const GaugeSet &gs, const Geom &g, const double *U,
                              cudaStream_t s);

}  // namespace wd
