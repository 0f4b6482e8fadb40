// Flexible GCR on the full Wilson-Dirac system D x = b, with an optional
// right preconditioner (the learned PTC network).  Not in the paper; the
// plain even-odd CGNR of wd_solve_cg stays the fallback and the reference
// for its error.
//
// Restarted FGCR(m): from the residual r,
//   z_j = N(r)  (or z_j = r without a network),  w_j = D z_j,
//   w_j, z_j orthogonalised against w_0..w_{j-1} (modified Gram-Schmidt,
//   complex coefficients <w_i, w_j> / <w_i, w_i>),
//   alpha = <w_j, r> / <w_j, w_j>,  x += alpha z_j,  r -= alpha w_j,
// and after m directions (or when the recursive residual meets the target)
// the residual is recomputed as b - D x with the FP64 operator.  w = D z uses
// the storage-precision operator; x, r and the basis are FP64 canonical
// fields [V][3][4].
//
// The vector work is written for GB300, whose FP64 units run at a small
// fraction of the FP32 rate (one FP64 dot product or axpy per basis vector
// and per direction made the orthogonalisation cost more than the operator):
// classical Gram-Schmidt, so that all the coefficients of a direction come
// from one multi-dot pass and one host read; inner products from FP32
// products accumulated in double-float; linear combinations accumulated in
// FP32 and added to the FP64 fields with one FP64 add per real.  These
// roundings (2^-24 of each correction) only perturb the basis and the
// recursive residual: every restart recomputes the residual with the FP64
// operator, and the solve stops on that residual alone.
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <string>
#include <vector>

#include "wd_internal.cuh"

namespace wd {

constexpr int FG_BLOCK = 256;
constexpr int FG_GRID = 1024;

// partial sums of conj(a) . b (complex) per block
__global__ void __launch_bounds__(FG_BLOCK)
k_cdot(long n, const double2 *__restrict__ a, const double2 *__restrict__ b, double2 *partials) {
    __shared__ double2 ws[FG_BLOCK / 32];
    double re = 0.0, im = 0.0;
    for (long i = (long)blockIdx.x * FG_BLOCK + threadIdx.x; i < n; i += (long)gridDim.x * FG_BLOCK) {
        const double2 x = a[i], y = b[i];
        re += x.x * y.x + x.y * y.y;
        im += x.x * y.y - x.y * y.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = make_double2(re, im);
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 t = make_double2(0.0, 0.0);
        for (int w = 0; w < FG_BLOCK / 32; ++w) { t.x += ws[w].x; t.y += ws[w].y; }
        partials[blockIdx.x] = t;
    }
}

// y = x - y
__global__ void __launch_bounds__(FG_BLOCK)
k_xmy_c(long n, const double2 *__restrict__ x, double2 *__restrict__ y) {
    for (long i = (long)blockIdx.x * FG_BLOCK + threadIdx.x; i < n; i += (long)gridDim.x * FG_BLOCK) {
        const double2 a = x[i], b = y[i];
        y[i] = make_double2(a.x - b.x, a.y - b.y);
    }
}

constexpr int FG_MV = 8;   // vectors per multi-vector pass

// FP64 -> FP32 on the bit pattern, rounding half away from zero: GB300 runs
// the hardware conversion at its FP64 rate, which made the multi-vector
// passes below four times slower than their memory traffic.  Magnitudes under
// 2^-126 flush to zero; from 2^128 (and NaN) they give infinity.
__device__ __forceinline__ float fg_narrow(double d) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const unsigned long long a = (u & 0x7FFFFFFFFFFFFFFFull) + (1ull << 28);
    const int e = (int)(a >> 52) - (1023 - 127);
    unsigned int bits = 0u;
    if (e >= 255) bits = 0x7F800000u;
    else if (e > 0) bits = ((unsigned int)e << 23) | (unsigned int)((a >> 29) & 0x7FFFFFu);
    return __uint_as_float(bits | ((unsigned int)(u >> 32) & 0x80000000u));
}

// FP32 -> FP64 on the bit pattern (exact); FP32 subnormals flush to zero,
// infinities and NaNs keep their class
__device__ __forceinline__ double fg_widen(float f) {
    const unsigned int b = __float_as_uint(f);
    const unsigned int e = (b >> 23) & 0xFFu;
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    if (e == 0) return __longlong_as_double((long long)sign);
    const unsigned long long de = e == 255 ? 0x7FFull : (unsigned long long)(e + (1023 - 127));
    return __longlong_as_double(
        (long long)(sign | (de << 52) | ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}

struct FgVecs {
    const double2 *v[FG_MV];
    float2 coef[FG_MV];
    int nv;
};

// per block and vector k: sum_i conj(a_i) b_k,i as FP32 products summed in
// double-float; partials[k * gridDim + block] = (re.hi, re.lo, im.hi, im.lo)
__global__ void __launch_bounds__(FG_BLOCK)
k_mdot(long n, const double2 *__restrict__ a, const FgVecs b, float4 *partials) {
    __shared__ df64 ws[FG_BLOCK / 32][2 * FG_MV];
    df64 re[FG_MV], im[FG_MV];
#pragma unroll
    for (int k = 0; k < FG_MV; ++k) re[k] = im[k] = df64(0.0f, 0.0f);
    for (long i = (long)blockIdx.x * FG_BLOCK + threadIdx.x; i < n; i += (long)gridDim.x * FG_BLOCK) {
        const double2 av = a[i];
        const float ar = fg_narrow(av.x), ai = fg_narrow(av.y);
#pragma unroll
        for (int k = 0; k < FG_MV; ++k)
            if (k < b.nv) {
                const double2 bv = b.v[k][i];
                const float br = fg_narrow(bv.x), bi = fg_narrow(bv.y);
                re[k] = re[k] + to_df(fmaf(ar, br, ai * bi));
                im[k] = im[k] + to_df(fmaf(ar, bi, -ai * br));
            }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < FG_MV; ++k) {
        const df64 r = warp_sum(re[k]), m = warp_sum(im[k]);
        if (lane == 0) { ws[w][2 * k] = r; ws[w][2 * k + 1] = m; }
    }
    __syncthreads();
    if (threadIdx.x < b.nv) {
        const int k = threadIdx.x;
        df64 r = ws[0][2 * k], m = ws[0][2 * k + 1];
        for (int j = 1; j < FG_BLOCK / 32; ++j) {
            r = r + ws[j][2 * k];
            m = m + ws[j][2 * k + 1];
        }
        partials[(long)k * gridDim.x + blockIdx.x] = make_float4(r.hi, r.lo, m.hi, m.lo);
    }
}

// y += sum_k coef_k v_k, the sum in FP32, one FP64 add per real of y
__global__ void __launch_bounds__(FG_BLOCK)
k_maxpy(long n, double2 *__restrict__ y, const FgVecs b) {
    for (long i = (long)blockIdx.x * FG_BLOCK + threadIdx.x; i < n; i += (long)gridDim.x * FG_BLOCK) {
        float sr = 0.0f, si = 0.0f;
#pragma unroll
        for (int k = 0; k < FG_MV; ++k)
            if (k < b.nv) {
                const double2 v = b.v[k][i];
                const float vr = fg_narrow(v.x), vi = fg_narrow(v.y);
                const float2 c = b.coef[k];
                sr = fmaf(c.x, vr, fmaf(-c.y, vi, sr));
                si = fmaf(c.x, vi, fmaf(c.y, vr, si));
            }
        double2 yv = y[i];
        yv.x += fg_widen(sr);
        yv.y += fg_widen(si);
        y[i] = yv;
    }
}

}  // namespace wd

using namespace wd;

static thread_local std::string g_fg_error;
static int fg_fail(int code, const std::string &m) {
    g_fg_error = m;
    return code;
}
#define FG_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fg_fail(e_ == cudaErrorMemoryAllocation ? WD_ERR_NOMEM : WD_ERR_CUDA,    \
                           std::string(#call) + ": " + cudaGetErrorString(e_));             \
    } while (0)
#define FG_TRY(call)                                                                        \
    do {                                                                                    \
        int rc_ = (call);                                                                   \
        if (rc_ != WD_OK) {                                                                 \
            if (g_fg_error.empty()) g_fg_error = wd_last_error();                           \
            return rc_;                                                                     \
        }                                                                                   \
    } while (0)

struct wd_fgcr {
    wd_op *op_lo = nullptr, *op_hi = nullptr;
    wd_ptc *net = nullptr;
    int m = 0;
    long n = 0;                       // complex entries per field (12 V)
    double2 *r = nullptr, *xv = nullptr, *t = nullptr;
    std::vector<double2 *> z, w;
    std::vector<double> wn;           // <w_i, w_i>
    double2 *partials = nullptr, *partials_host = nullptr;
    float4 *mpart = nullptr, *mpart_host = nullptr;   // multi-dot partials
    std::vector<void *> allocs;
};

static int fg_alloc(wd_fgcr *s, void **p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fg_fail(WD_ERR_NOMEM, "cudaMalloc failed");
    }
    s->allocs.push_back(*p);
    FG_CUDA(cudaMemset(*p, 0, bytes));
    return WD_OK;
}

static int fg_dot(wd_fgcr *s, const double2 *a, const double2 *b, std::complex<double> &out) {
    k_cdot<<<FG_GRID, FG_BLOCK>>>(s->n, a, b, s->partials);
    FG_CUDA(cudaGetLastError());
    FG_CUDA(cudaMemcpy(s->partials_host, s->partials, sizeof(double2) * FG_GRID,
                       cudaMemcpyDeviceToHost));
    double re = 0.0, im = 0.0;
    for (int i = 0; i < FG_GRID; ++i) { re += s->partials_host[i].x; im += s->partials_host[i].y; }
    out = std::complex<double>(re, im);
    return WD_OK;
}

// out[k] = <a, b_k> for k < nb (one pass over a per FG_MV vectors, one host read each)
static int fg_mdot(wd_fgcr *s, const double2 *a, const double2 *const *b, int nb,
                   std::complex<double> *out) {
    for (int k0 = 0; k0 < nb; k0 += FG_MV) {
        FgVecs v{};
        v.nv = std::min(FG_MV, nb - k0);
        for (int k = 0; k < v.nv; ++k) v.v[k] = b[k0 + k];
        k_mdot<<<FG_GRID, FG_BLOCK>>>(s->n, a, v, s->mpart);
        FG_CUDA(cudaGetLastError());
        FG_CUDA(cudaMemcpy(s->mpart_host, s->mpart, sizeof(float4) * FG_GRID * v.nv,
                           cudaMemcpyDeviceToHost));
        for (int k = 0; k < v.nv; ++k) {
            double re = 0.0, im = 0.0;
            for (int i = 0; i < FG_GRID; ++i) {
                const float4 p = s->mpart_host[(long)k * FG_GRID + i];
                re += (double)p.x + (double)p.y;
                im += (double)p.z + (double)p.w;
            }
            out[k0 + k] = std::complex<double>(re, im);
        }
    }
    return WD_OK;
}

// y += sum_k c_k b_k
static int fg_maxpy(wd_fgcr *s, double2 *y, const double2 *const *b,
                    const std::complex<double> *c, int nb) {
    for (int k0 = 0; k0 < nb; k0 += FG_MV) {
        FgVecs v{};
        v.nv = std::min(FG_MV, nb - k0);
        for (int k = 0; k < v.nv; ++k) {
            v.v[k] = b[k0 + k];
            v.coef[k] = make_float2((float)c[k0 + k].real(), (float)c[k0 + k].imag());
        }
        k_maxpy<<<FG_GRID, FG_BLOCK>>>(s->n, y, v);
        FG_CUDA(cudaGetLastError());
    }
    return WD_OK;
}

extern "C" {

const char *wd_fgcr_last_error(void) { return g_fg_error.c_str(); }

void wd_fgcr_destroy(wd_fgcr *s) {
    if (!s) return;
    cudaDeviceSynchronize();
    for (void *p : s->allocs) cudaFree(p);
    if (s->partials_host) cudaFreeHost(s->partials_host);
    if (s->mpart_host) cudaFreeHost(s->mpart_host);
    delete s;
}

int wd_fgcr_create(wd_fgcr **out, wd_op *op_lo, wd_op *op_hi, wd_ptc *net, int nkrylov) {
    if (!out || !op_lo || !op_hi) return fg_fail(WD_ERR_ARG, "null argument to wd_fgcr_create");
    *out = nullptr;
    if (nkrylov < 1 || nkrylov > 128) return fg_fail(WD_ERR_ARG, "nkrylov must be 1..128");
    wd_fgcr *s = new wd_fgcr();
    s->op_lo = op_lo;
    s->op_hi = op_hi;
    s->net = net;
    s->m = nkrylov;
    const long vh = wd_op_half_volume(op_lo);
    if (vh != wd_op_half_volume(op_hi)) {
        delete s;
        return fg_fail(WD_ERR_ARG, "the two operators must share the lattice");
    }
    s->n = 2 * vh * 12;
    const size_t bytes = sizeof(double2) * s->n;
    int rc = fg_alloc(s, (void **)&s->r, bytes);
    if (rc == WD_OK) rc = fg_alloc(s, (void **)&s->xv, bytes);
    if (rc == WD_OK) rc = fg_alloc(s, (void **)&s->t, bytes);
    s->z.assign(s->m, nullptr);
    s->w.assign(s->m, nullptr);
    s->wn.assign(s->m, 0.0);
    for (int j = 0; j < s->m && rc == WD_OK; ++j) {
        rc = fg_alloc(s, (void **)&s->z[j], bytes);
        if (rc == WD_OK) rc = fg_alloc(s, (void **)&s->w[j], bytes);
    }
    if (rc == WD_OK) rc = fg_alloc(s, (void **)&s->partials, sizeof(double2) * FG_GRID);
    if (rc == WD_OK) rc = fg_alloc(s, (void **)&s->mpart, sizeof(float4) * FG_GRID * FG_MV);
    if (rc == WD_OK &&
        cudaMallocHost((void **)&s->mpart_host, sizeof(float4) * FG_GRID * FG_MV) != cudaSuccess)
        rc = fg_fail(WD_ERR_NOMEM, "pinned host buffer");
    if (rc == WD_OK && cudaMallocHost((void **)&s->partials_host, sizeof(double2) * FG_GRID) != cudaSuccess)
        rc = fg_fail(WD_ERR_NOMEM, "pinned host buffer");
    if (rc != WD_OK) {
        std::string m = g_fg_error;
        wd_fgcr_destroy(s);
        g_fg_error = m;
        return rc;
    }
    *out = s;
    return WD_OK;
}

int wd_fgcr_solve(wd_fgcr *s, double *x, const double *b, double tol, int maxiter,
                  wd_solve_info *info) {
    auto t0 = std::chrono::steady_clock::now();
    g_fg_error.clear();
    if (!s || !x || !b) return fg_fail(WD_ERR_ARG, "null argument to wd_fgcr_solve");
    if (!(tol > 0) || maxiter < 0) return fg_fail(WD_ERR_ARG, "tol must be > 0, maxiter >= 0");
    if (info) memset(info, 0, sizeof(*info));
    const double2 *bb = (const double2 *)b;
    std::complex<double> c;
    FG_CUDA(cudaDeviceSynchronize());
    FG_TRY(fg_dot(s, bb, bb, c));
    const double nb = std::sqrt(c.real());
    const double target = tol * nb;
    // x = 0, r = b
    FG_CUDA(cudaMemset(s->xv, 0, sizeof(double2) * s->n));
    FG_CUDA(cudaMemcpy(s->r, bb, sizeof(double2) * s->n, cudaMemcpyDeviceToDevice));
    double rn = nb;
    int iters = 0, restarts = 0, status = WD_ERR_NOT_CONVERGED;
    double applies = 0.0, nets = 0.0;
    std::vector<std::complex<double>> cf(s->m);
    while (rn > target && iters < maxiter) {
        int j = 0;
        for (; j < s->m && iters < maxiter; ++j, ++iters) {
            double2 *zj = s->z[j], *wj = s->w[j];
            if (s->net) {
                FG_CUDA(cudaDeviceSynchronize());
                FG_TRY(wd_ptc_apply(s->net, (double *)zj, (const double *)s->r));
                nets += 1;
            } else {
                FG_CUDA(cudaMemcpy(zj, s->r, sizeof(double2) * s->n, cudaMemcpyDeviceToDevice));
            }
            FG_TRY(wd_apply(s->op_lo, (double *)wj, (const double *)zj, 0));
            applies += 1;
            FG_CUDA(cudaDeviceSynchronize());
            if (j > 0) {   // classical Gram-Schmidt against w_0..w_{j-1}
                FG_TRY(fg_mdot(s, wj, s->w.data(), j, cf.data()));   // <w_j, w_i>
                for (int i = 0; i < j; ++i) cf[i] = -std::conj(cf[i]) / s->wn[i];
                FG_TRY(fg_maxpy(s, wj, s->w.data(), cf.data(), j));
                FG_TRY(fg_maxpy(s, zj, s->z.data(), cf.data(), j));
            }
            const double2 *pair[2] = {wj, s->r};
            std::complex<double> d2[2];
            FG_TRY(fg_mdot(s, wj, pair, 2, d2));   // <w_j, w_j>, <w_j, r>
            s->wn[j] = d2[0].real();
            if (!(s->wn[j] > 0.0)) { status = WD_ERR_BREAKDOWN; break; }
            const std::complex<double> alpha = d2[1] / s->wn[j];
            const double2 *zs[1] = {zj}, *wsv[1] = {wj};
            const std::complex<double> pa[1] = {alpha}, ma[1] = {-alpha};
            FG_TRY(fg_maxpy(s, s->xv, zs, pa, 1));
            FG_TRY(fg_maxpy(s, s->r, wsv, ma, 1));
            // |r - alpha w_j|^2 = |r|^2 - |<w_j, r>|^2 / |w_j|^2 (the minimising alpha);
            // where that difference cancels to under 1e-4 of |r|^2 it is summed
            // afresh.  The restart below replaces this recursive value by the
            // true residual.
            const double r2 = rn * rn - std::norm(d2[1]) / s->wn[j];
            if (r2 > 1e-4 * rn * rn) {
                rn = std::sqrt(r2);
            } else {
                const double2 *rr[1] = {s->r};
                FG_TRY(fg_mdot(s, s->r, rr, 1, d2));
                rn = std::sqrt(d2[0].real());
            }
            if (rn <= target) { ++iters; ++j; break; }
        }
        if (status == WD_ERR_BREAKDOWN) break;
        // true residual with the FP64 operator
        FG_TRY(wd_apply(s->op_hi, (double *)s->t, (const double *)s->xv, 0));
        FG_CUDA(cudaDeviceSynchronize());
        k_xmy_c<<<FG_GRID, FG_BLOCK>>>(s->n, bb, s->t);
        FG_CUDA(cudaGetLastError());
        FG_CUDA(cudaMemcpy(s->r, s->t, sizeof(double2) * s->n, cudaMemcpyDeviceToDevice));
        FG_TRY(fg_dot(s, s->r, s->r, c));
        rn = std::sqrt(c.real());
        restarts += 1;
        if (rn <= target) status = WD_OK;
    }
    if (rn <= target) status = WD_OK;
    FG_CUDA(cudaMemcpy(x, s->xv, sizeof(double2) * s->n, cudaMemcpyDeviceToDevice));
    FG_CUDA(cudaDeviceSynchronize());
    if (info) {
        info->iters = iters;
        info->reliable_updates = restarts;
        info->true_rel_resid = nb > 0 ? rn / nb : 0.0;
        info->dslash_lo = 2 * applies;
        info->dslash_hi = 2 * restarts;
        info->launches = nets;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (status != WD_OK) fg_fail(status, wd_status_string(status));
    return status;
}

}  // extern "C"
