// Vector kernels of the Krylov solver (Alg. "CGNR" lines on x, r, p and
// the norms), fused so that each touches every vector once, plus the
// precision conversions of the reliable updates.
//
// Spinor fields are whole 16-byte planes (no tail), so the element-wise
// kernels walk the flat array of 16-byte chunks (NF * stride of them;
// the zero padding of each plane stays zero under every update).  Norms
// accumulate in FP64 and finish with the deterministic last-block sum.
#include <algorithm>
#include <cstdint>

#include "wd_internal.cuh"

namespace wd {

constexpr int BLAS_BLOCK = 256;
constexpr int BLAS_MAX_GRID = 152 * 8;

template <typename S, typename R> using Chunk = Chunk16<S, R>;

inline long spinor_chunks(int prec, const Geom &g) {
    return (long)(24 * prec_bytes(prec) / 16) * g.stride;
}

inline unsigned blas_grid(long n) {
    long b = (n + BLAS_BLOCK - 1) / BLAS_BLOCK;
    if (b > BLAS_MAX_GRID) b = BLAS_MAX_GRID;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// partials: one per 32 output sites (warp_partials), or one per BLAS block
int reduction_blocks(const Geom &g) {
    long d = (g.vh + 31) / 32;
    return (int)(d > BLAS_MAX_GRID ? d : BLAS_MAX_GRID);
}

constexpr int FINISH_BLOCK = 1024;

__global__ void __launch_bounds__(FINISH_BLOCK) k_finish_partials(Reduction red, long n) {
    __shared__ df64 warp_sums[FINISH_BLOCK / 32];
    const df64 s = warp_sum(strided_sum<FINISH_BLOCK>(red.partials, n, threadIdx.x));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_sums[wid] = s;
    __syncthreads();
    if (wid == 0) {
        const df64 t = warp_sum(warp_sums[lane]);
        if (lane == 0) apply_final(red.scalars, red.op, (double)t);
    }
}

// Copies done by the SMs instead of the copy engines: a solve's small host
// transfers (its scalars, per-refresh constants) then never queue behind a
// large upload or download another stream has on the copy engines.  src and
// dst may be host memory the device can address (mapped pinned buffers).
__global__ void k_copy_u64(unsigned long long *dst, const unsigned long long *src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
    __threadfence_system();
}
__global__ void k_copy_u4(uint4 *dst, const uint4 *src, long n) {
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

cudaError_t launch_copy_small(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (bytes % 8 || (uintptr_t)dst % 8 || (uintptr_t)src % 8) return cudaErrorInvalidValue;
    k_copy_u64<<<1, 128, 0, s>>>((unsigned long long *)dst, (const unsigned long long *)src,
                                 (int)(bytes / 8));
    return cudaGetLastError();
}

cudaError_t launch_copy_field(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (bytes % 16 || (uintptr_t)dst % 16 || (uintptr_t)src % 16) return cudaErrorInvalidValue;
    const long n = (long)(bytes / 16);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long grid = std::min<long>((n + 255) / 256, (long)sms * 8);
    k_copy_u4<<<(unsigned)std::max<long>(grid, 1), 256, 0, s>>>((uint4 *)dst, (const uint4 *)src, n);
    return cudaGetLastError();
}

cudaError_t launch_finish_partials(const Reduction &red, long n, cudaStream_t s) {
    k_finish_partials<<<1, FINISH_BLOCK, 0, s>>>(red, n);
    return cudaGetLastError();
}

// Per-thread accumulator of a norm: FP64 kernels keep FP64; FP32 arithmetic
// accumulates its per-chunk sums in double-float (the FP64 adder of GB300 is
// slow enough that one DADD per 16-byte chunk showed in the update kernel).
template <typename R> struct ThreadAccOf { using T = df64; };
template <> struct ThreadAccOf<double> { using T = double; };
template <typename R> using ThreadAcc = typename ThreadAccOf<R>::T;
template <typename R> __device__ __forceinline__ ThreadAcc<R> thread_term(R s) { return to_df(s); }
template <> __device__ __forceinline__ double thread_term<double>(double s) { return s; }

// r -= alpha Ap;  ||r||^2  (alpha from the device scalars).  The matching
// x += alpha p is deferred to the next p update (k_cg_update_px), which reads
// the same p anyway: one field pass fewer per iteration.
template <typename S, typename R>
__global__ void __launch_bounds__(BLAS_BLOCK)
k_cg_update_r(long n, void *r, const void *Ap, Reduction red) {
    using C = Chunk<S, R>;
    const R alpha = (R)red.scalars->alpha;
    ThreadAcc<R> acc = 0;
    for (long i = (long)blockIdx.x * BLAS_BLOCK + threadIdx.x; i < n;
         i += (long)gridDim.x * BLAS_BLOCK) {
        R rv[C::K], av[C::K];
        C::load(r, i, rv);
        C::load(Ap, i, av);
        R s = 0;
#pragma unroll
        for (int k = 0; k < C::K; ++k) {
            rv[k] -= alpha * av[k];
            s += rv[k] * rv[k];
        }
        C::store(r, i, rv);
        acc = acc + thread_term<R>(s);
    }
    block_reduce_finish<BLAS_BLOCK>(acc, red);
}

// x += alpha_x p (the previous iteration's step);  p = z + beta p
template <typename S, typename R>
__global__ void __launch_bounds__(BLAS_BLOCK)
k_cg_update_px(long n, void *x, void *p, const void *z, const SolverScalars *sc) {
    using C = Chunk<S, R>;
    const R alpha = (R)sc->alpha_x, beta = (R)sc->beta;
    for (long i = (long)blockIdx.x * BLAS_BLOCK + threadIdx.x; i < n;
         i += (long)gridDim.x * BLAS_BLOCK) {
        R xv[C::K], pv[C::K], zv[C::K];
        C::load(x, i, xv);
        C::load(p, i, pv);
        C::load(z, i, zv);
#pragma unroll
        for (int k = 0; k < C::K; ++k) {
            xv[k] = fma(alpha, pv[k], xv[k]);
            pv[k] = zv[k] + beta * pv[k];
        }
        C::store(x, i, xv);
        C::store(p, i, pv);
    }
}

// |v|^2 of a double-float field, accumulated in double-float per thread.
__global__ void __launch_bounds__(BLAS_BLOCK) k_norm2_df(long n, const void *v, Reduction red) {
    using C = Chunk16<df64, df64>;
    df64 acc = 0;
    for (long i = (long)blockIdx.x * BLAS_BLOCK + threadIdx.x; i < n;
         i += (long)gridDim.x * BLAS_BLOCK) {
        df64 a[C::K];
        C::load(v, i, a);
#pragma unroll
        for (int k = 0; k < C::K; ++k) acc += a[k] * a[k];
    }
    block_reduce_finish<BLAS_BLOCK>((double)acc, red);
}

// out = x - y and |out|^2 in double-float
__global__ void __launch_bounds__(BLAS_BLOCK)
k_xmy_norm_df(long n, void *out, const void *x, const void *y, Reduction red) {
    using C = Chunk16<df64, df64>;
    df64 acc = 0;
    for (long i = (long)blockIdx.x * BLAS_BLOCK + threadIdx.x; i < n;
         i += (long)gridDim.x * BLAS_BLOCK) {
        df64 a[C::K], b[C::K];
        C::load(x, i, a);
        C::load(y, i, b);
#pragma unroll
        for (int k = 0; k < C::K; ++k) {
            a[k] = a[k] - b[k];
            acc += a[k] * a[k];
        }
        C::store(out, i, a);
    }
    block_reduce_finish<BLAS_BLOCK>((double)acc, red);
}

// out = y + a x in double-float
__global__ void __launch_bounds__(BLAS_BLOCK)
k_xpay_df(long n, void *out, const void *y, df64 a, const void *x) {
    using C = Chunk16<df64, df64>;
    for (long i = (long)blockIdx.x * BLAS_BLOCK + threadIdx.x; i < n;
         i += (long)gridDim.x * BLAS_BLOCK) {
        df64 yv[C::K], xv[C::K];
        C::load(y, i, yv);
        C::load(x, i, xv);
#pragma unroll
        for (int k = 0; k < C::K; ++k) yv[k] += a * xv[k];
        C::store(out, i, yv);
    }
}

// x_lo + alpha p rounded to storage precision S, as k_cg_update_px would
// have stored it (the same FMA in the same arithmetic, then one rounding)
template <typename S, typename R> __device__ __forceinline__ R owed_step(R lo, R a, R p) {
    const R v = fma(a, p, lo);
    if constexpr (std::is_same<S, __half>::value) return __half2float(__float2half_rn(v));
    else if constexpr (std::is_same<S, __nv_bfloat16>::value)
        return __bfloat162float(__float2bfloat16_rn(v));
    else return v;
}

// x_lo += alpha_x p (the step the last iteration still owes x), then
// x_hi (double-float) += inv_scale * x_lo;  x_lo = 0
template <typename S>
__global__ void __launch_bounds__(BLAS_BLOCK)
k_fold_x_df(long vh, long stride, void *x_hi, void *x_lo, const void *p,
            const SolverScalars *sc, const double *inv_scale) {
    const df64 is = df64(*inv_scale);
    const float a = (float)sc->alpha_x;
    for (long h = (long)blockIdx.x * BLAS_BLOCK + threadIdx.x; h < vh;
         h += (long)gridDim.x * BLAS_BLOCK) {
        float lo[24], pv[24];
        df64 hi[24];
        Rec<S, 24>::template load_coherent<float>(x_lo, stride, h, lo);
        Rec<S, 24>::template load_coherent<float>(p, stride, h, pv);
        Rec<df64, 24>::template load_coherent<df64>(x_hi, stride, h, hi);
#pragma unroll
        for (int i = 0; i < 24; ++i) {
            hi[i] += is * df64(owed_step<S>(lo[i], a, pv[i]), 0.0f);
            lo[i] = 0.0f;
        }
        Rec<df64, 24>::store(x_hi, stride, h, hi);
        Rec<S, 24>::store(x_lo, stride, h, lo);
    }
}

// out (precision SO) = scale * in (double-float), in FP32: the low-precision
// copy needs only the leading part.
template <typename SO>
__global__ void __launch_bounds__(BLAS_BLOCK)
k_convert_from_df(long vh, long stride, void *out, const void *in, const double *scale_dev,
                  double scale_host) {
    const float sc = (float)(scale_dev ? *scale_dev : scale_host);
    for (long h = (long)blockIdx.x * BLAS_BLOCK + threadIdx.x; h < vh;
         h += (long)gridDim.x * BLAS_BLOCK) {
        float v[24];
        Rec<df64, 24>::template load_coherent<float>(in, stride, h, v);
#pragma unroll
        for (int i = 0; i < 24; ++i) v[i] *= sc;
        Rec<SO, 24>::store(out, stride, h, v);
    }
}

// FP64 <-> double-float, element-wise over n eight-byte reals
__global__ void k_f64_df64(long n, void *buf, int to_df) {
    for (long i = (long)blockIdx.x * BLAS_BLOCK + threadIdx.x; i < n;
         i += (long)gridDim.x * BLAS_BLOCK) {
        if (to_df) {
            const double d = reinterpret_cast<double *>(buf)[i];
            const df64 v = split_double(d);
            reinterpret_cast<float2 *>(buf)[i] = make_float2(v.hi, v.lo);
        } else {
            const float2 f = reinterpret_cast<float2 *>(buf)[i];
            reinterpret_cast<double *>(buf)[i] = (double)f.x + (double)f.y;
        }
    }
}

template <typename S, typename R>
__global__ void __launch_bounds__(BLAS_BLOCK) k_norm2(long n, const void *v, Reduction red) {
    using C = Chunk<S, R>;
    ThreadAcc<R> acc = 0;
    for (long i = (long)blockIdx.x * BLAS_BLOCK + threadIdx.x; i < n;
         i += (long)gridDim.x * BLAS_BLOCK) {
        R a[C::K];
        C::load(v, i, a);
        R s = 0;
#pragma unroll
        for (int k = 0; k < C::K; ++k) s += a[k] * a[k];
        acc = acc + thread_term<R>(s);
    }
    block_reduce_finish<BLAS_BLOCK>(acc, red);
}

// out = x - y and ||out||^2, FP64
__global__ void __launch_bounds__(BLAS_BLOCK)
k_xmy_norm(long n, double *out, const double *x, const double *y, Reduction red) {
    double acc = 0.0;
    for (long i = (long)blockIdx.x * BLAS_BLOCK + threadIdx.x; i < n;
         i += (long)gridDim.x * BLAS_BLOCK) {
        double2 a = reinterpret_cast<const double2 *>(x)[i];
        double2 b = reinterpret_cast<const double2 *>(y)[i];
        double2 d = {a.x - b.x, a.y - b.y};
        reinterpret_cast<double2 *>(out)[i] = d;
        acc += d.x * d.x + d.y * d.y;
    }
    block_reduce_finish<BLAS_BLOCK>(acc, red);
}

// out = y + a x, FP64
__global__ void __launch_bounds__(BLAS_BLOCK)
k_xpay_f64(long n, double *out, const double *y, double a, const double *x) {
    for (long i = (long)blockIdx.x * BLAS_BLOCK + threadIdx.x; i < n;
         i += (long)gridDim.x * BLAS_BLOCK) {
        const double2 yv = reinterpret_cast<const double2 *>(y)[i];
        const double2 xv = reinterpret_cast<const double2 *>(x)[i];
        reinterpret_cast<double2 *>(out)[i] = make_double2(yv.x + a * xv.x, yv.y + a * xv.y);
    }
}

// out (precision SO) = scale * in (precision SI), one site per thread.
template <typename SO, typename SI>
__global__ void __launch_bounds__(BLAS_BLOCK)
k_convert_scaled(long vh, long stride, void *out, const void *in, const double *scale_dev,
                 double scale_host) {
    const double sc = scale_dev ? *scale_dev : scale_host;
    for (long h = (long)blockIdx.x * BLAS_BLOCK + threadIdx.x; h < vh;
         h += (long)gridDim.x * BLAS_BLOCK) {
        double v[24];
        Rec<SI, 24>::template load_coherent<double>(in, stride, h, v);
#pragma unroll
        for (int i = 0; i < 24; ++i) v[i] *= sc;
        Rec<SO, 24>::store(out, stride, h, v);
    }
}

// x_hi += inv_scale * x_lo;  x_lo = 0
template <typename S>
__global__ void __launch_bounds__(BLAS_BLOCK)
k_fold_x(long vh, long stride, double *x_hi, void *x_lo, const void *p, const SolverScalars *sc,
         const double *inv_scale) {
    using R = typename std::conditional<std::is_same<S, double>::value, double, float>::type;
    const double is = *inv_scale;
    const R a = (R)sc->alpha_x;
    for (long h = (long)blockIdx.x * BLAS_BLOCK + threadIdx.x; h < vh;
         h += (long)gridDim.x * BLAS_BLOCK) {
        R lo[24], pv[24];
        double hi[24];
        Rec<S, 24>::template load_coherent<R>(x_lo, stride, h, lo);
        Rec<S, 24>::template load_coherent<R>(p, stride, h, pv);
        Rec<double, 24>::template load_coherent<double>(x_hi, stride, h, hi);
#pragma unroll
        for (int i = 0; i < 24; ++i) {
            hi[i] += is * (double)owed_step<S>(lo[i], a, pv[i]);
            lo[i] = 0;
        }
        Rec<double, 24>::store(x_hi, stride, h, hi);
        Rec<S, 24>::store(x_lo, stride, h, lo);
    }
}

// p *= ratio and nz *= ratio^2: the Krylov direction follows a change of
// the residual's scale.
template <typename S, typename R>
__global__ void __launch_bounds__(BLAS_BLOCK)
k_rescale(long n, void *p, SolverScalars *sc, const double *ratio_dev) {
    using C = Chunk<S, R>;
    const double ratio = *ratio_dev;
    for (long i = (long)blockIdx.x * BLAS_BLOCK + threadIdx.x; i < n;
         i += (long)gridDim.x * BLAS_BLOCK) {
        R v[C::K];
        C::load(p, i, v);
#pragma unroll
        for (int k = 0; k < C::K; ++k) v[k] *= (R)ratio;
        C::store(p, i, v);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->nz *= ratio * ratio;
}

// ------------------------------------------------------------------ launchers
#define WD_PREC_DISPATCH(prec, CALL)                                                    \
    switch (prec) {                                                                     \
    case WD_F64: { using S = double; using R = double; CALL; break; }                   \
    case WD_F32: { using S = float; using R = float; CALL; break; }                     \
    case WD_F16: { using S = __half; using R = float; CALL; break; }                    \
    case WD_BF16: { using S = __nv_bfloat16; using R = float; CALL; break; }            \
    default: return cudaErrorInvalidValue;                                              \
    }

cudaError_t launch_cg_update_r(int prec, const Geom &g, void *r, const void *Ap,
                               const Reduction &red, cudaStream_t s) {
    const long n = spinor_chunks(prec, g);
    WD_PREC_DISPATCH(prec, (k_cg_update_r<S, R><<<blas_grid(n), BLAS_BLOCK, 0, s>>>(
                               n, r, Ap, red)));
    return cudaGetLastError();
}

cudaError_t launch_cg_update_px(int prec, const Geom &g, void *x, void *p, const void *z,
                                const SolverScalars *sc, cudaStream_t s) {
    const long n = spinor_chunks(prec, g);
    WD_PREC_DISPATCH(prec, (k_cg_update_px<S, R><<<blas_grid(n), BLAS_BLOCK, 0, s>>>(
                               n, x, p, z, sc)));
    return cudaGetLastError();
}

cudaError_t launch_norm2(int prec, const Geom &g, const void *v, const Reduction &red,
                         cudaStream_t s) {
    const long n = spinor_chunks(prec, g);
    if (prec == WD_DF64) {
        k_norm2_df<<<blas_grid(n), BLAS_BLOCK, 0, s>>>(n, v, red);
        return cudaGetLastError();
    }
    WD_PREC_DISPATCH(prec, (k_norm2<S, R><<<blas_grid(n), BLAS_BLOCK, 0, s>>>(n, v, red)));
    return cudaGetLastError();
}

cudaError_t launch_xmy_norm(int prec, const Geom &g, void *out, const void *x, const void *y,
                            const Reduction &red, cudaStream_t s) {
    const long n = spinor_chunks(WD_F64, g);
    if (prec == WD_DF64)
        k_xmy_norm_df<<<blas_grid(n), BLAS_BLOCK, 0, s>>>(n, out, x, y, red);
    else
        k_xmy_norm<<<blas_grid(n), BLAS_BLOCK, 0, s>>>(n, (double *)out, (const double *)x,
                                                       (const double *)y, red);
    return cudaGetLastError();
}

cudaError_t launch_xpay_hi(int prec, const Geom &g, void *out, const void *y, double a,
                           const void *x, cudaStream_t s) {
    const long n = spinor_chunks(WD_F64, g);
    if (prec == WD_DF64)
        k_xpay_df<<<blas_grid(n), BLAS_BLOCK, 0, s>>>(n, out, y, df64(a), x);
    else
        k_xpay_f64<<<blas_grid(n), BLAS_BLOCK, 0, s>>>(n, (double *)out, (const double *)y, a,
                                                       (const double *)x);
    return cudaGetLastError();
}

// out = c (1 + i t gamma5) in over 16-byte chunks of an FP64 or double-float
// field: chunk i holds the complex component j = i / stride of its site, j =
// 4 colour + spin, and gamma5 = diag(1, 1, -1, -1) on the spin.
template <typename H>
__global__ void __launch_bounds__(BLAS_BLOCK)
k_twist_hi(long n, long stride, void *out, const void *in, H t, H c) {
    using C = Chunk16<H, H>;
    for (long i = (long)blockIdx.x * BLAS_BLOCK + threadIdx.x; i < n;
         i += (long)gridDim.x * BLAS_BLOCK) {
        H v[C::K];
        C::load(in, i, v);
        const int spin = (int)((i / stride) & 3);
        const H ts = spin < 2 ? t : -t;
        const H re = v[0], im = v[1];
        v[0] = c * (re - ts * im);
        v[1] = c * (im + ts * re);
        C::store(out, i, v);
    }
}

cudaError_t launch_twist_hi(int prec, const Geom &g, void *out, const void *in, double t, double c,
                            cudaStream_t s) {
    const long n = spinor_chunks(WD_F64, g);
    if (prec == WD_DF64)
        k_twist_hi<df64><<<blas_grid(n), BLAS_BLOCK, 0, s>>>(n, g.stride, out, in, df64(t), df64(c));
    else
        k_twist_hi<double><<<blas_grid(n), BLAS_BLOCK, 0, s>>>(n, g.stride, out, in, t, c);
    return cudaGetLastError();
}

cudaError_t launch_f64_df64(void *buf, long n_reals, int to_df, cudaStream_t s) {
    k_f64_df64<<<blas_grid(n_reals), BLAS_BLOCK, 0, s>>>(n_reals, buf, to_df);
    return cudaGetLastError();
}

template <typename SO>
static cudaError_t convert_from(int prec_in, void *out, const void *in, const Geom &g,
                                const double *sd, double sh, cudaStream_t s) {
    const unsigned grid = blas_grid(g.vh);
    switch (prec_in) {
    case WD_F64: k_convert_scaled<SO, double><<<grid, BLAS_BLOCK, 0, s>>>(g.vh, g.stride, out, in, sd, sh); break;
    case WD_F32: k_convert_scaled<SO, float><<<grid, BLAS_BLOCK, 0, s>>>(g.vh, g.stride, out, in, sd, sh); break;
    case WD_F16: k_convert_scaled<SO, __half><<<grid, BLAS_BLOCK, 0, s>>>(g.vh, g.stride, out, in, sd, sh); break;
    case WD_BF16: k_convert_scaled<SO, __nv_bfloat16><<<grid, BLAS_BLOCK, 0, s>>>(g.vh, g.stride, out, in, sd, sh); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_convert_scaled(int prec_out, void *out, int prec_in, const void *in,
                                  const Geom &g, const double *scale_dev, double scale_host,
                                  cudaStream_t s) {
    if (prec_in == WD_DF64 && prec_out != WD_F64) {
        const unsigned grid = blas_grid(g.vh);
        switch (prec_out) {
        case WD_F32: k_convert_from_df<float><<<grid, BLAS_BLOCK, 0, s>>>(g.vh, g.stride, out, in, scale_dev, scale_host); break;
        case WD_F16: k_convert_from_df<__half><<<grid, BLAS_BLOCK, 0, s>>>(g.vh, g.stride, out, in, scale_dev, scale_host); break;
        case WD_BF16: k_convert_from_df<__nv_bfloat16><<<grid, BLAS_BLOCK, 0, s>>>(g.vh, g.stride, out, in, scale_dev, scale_host); break;
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    switch (prec_out) {
    case WD_F64: return convert_from<double>(prec_in, out, in, g, scale_dev, scale_host, s);
    case WD_F32: return convert_from<float>(prec_in, out, in, g, scale_dev, scale_host, s);
    case WD_F16: return convert_from<__half>(prec_in, out, in, g, scale_dev, scale_host, s);
    case WD_BF16: return convert_from<__nv_bfloat16>(prec_in, out, in, g, scale_dev, scale_host, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fold_x(int prec_lo, int prec_hi, const Geom &g, void *x_hi, void *x_lo,
                          const void *p, SolverScalars *sc, const double *inv_scale_dev,
                          cudaStream_t s) {
    const unsigned grid = blas_grid(g.vh);
    if (prec_hi == WD_DF64) {
        switch (prec_lo) {
        case WD_F32: k_fold_x_df<float><<<grid, BLAS_BLOCK, 0, s>>>(g.vh, g.stride, x_hi, x_lo, p, sc, inv_scale_dev); break;
        case WD_F16: k_fold_x_df<__half><<<grid, BLAS_BLOCK, 0, s>>>(g.vh, g.stride, x_hi, x_lo, p, sc, inv_scale_dev); break;
        case WD_BF16: k_fold_x_df<__nv_bfloat16><<<grid, BLAS_BLOCK, 0, s>>>(g.vh, g.stride, x_hi, x_lo, p, sc, inv_scale_dev); break;
        default: return cudaErrorInvalidValue;
        }
    } else {
        WD_PREC_DISPATCH(prec_lo, (k_fold_x<S><<<grid, BLAS_BLOCK, 0, s>>>(
                                      g.vh, g.stride, (double *)x_hi, x_lo, p, sc,
                                      inv_scale_dev)));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the owed step is settled: the next p update must not add it again
    return cudaMemsetAsync(&sc->alpha_x, 0, sizeof(double), s);
}

cudaError_t launch_rescale_lo(int prec_lo, const Geom &g, void *p, SolverScalars *sc,
                              const double *ratio_dev, cudaStream_t s) {
    const long n = spinor_chunks(prec_lo, g);
    WD_PREC_DISPATCH(prec_lo, (k_rescale<S, R><<<blas_grid(n), BLAS_BLOCK, 0, s>>>(n, p, sc,
                                                                                     ratio_dev)));
    return cudaGetLastError();
}

}  // namespace wd
