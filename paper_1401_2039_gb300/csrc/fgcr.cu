// Flexible GCR on the full Wilson-Dirac system D x = b, with an optional
// right preconditioner (the learned PTC network).  Not in the paper; the
// plain even-odd CGNR of wd_solve_cg stays the fallback and the judge of its
// error.
//
// Restarted FGCR(m): from the residual r,
//   z_j = N(r)  (or z_j = r without a network),  w_j = D z_j,
//   w_j, z_j orthogonalised against w_0..w_{j-1} (modified Gram-Schmidt,
//   complex coefficients <w_i, w_j> / <w_i, w_i>),
//   alpha = <w_j, r> / <w_j, w_j>,  x += alpha z_j,  r -= alpha w_j,
// and after m directions (or when the recursive residual meets the target)
// the residual is recomputed as b - D x with the FP64 operator.  w = D z uses
// the storage-precision operator; x, r and the basis are FP64 canonical
// fields [V][3][4] and every inner product accumulates in FP64.
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

// y += alpha x  (complex alpha)
__global__ void __launch_bounds__(FG_BLOCK)
k_caxpy(long n, double ar, double ai, const double2 *__restrict__ x, double2 *__restrict__ y) {
    for (long i = (long)blockIdx.x * FG_BLOCK + threadIdx.x; i < n; i += (long)gridDim.x * FG_BLOCK) {
        const double2 v = x[i];
        double2 w = y[i];
        w.x += ar * v.x - ai * v.y;
        w.y += ar * v.y + ai * v.x;
        y[i] = w;
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

static int fg_axpy(wd_fgcr *s, std::complex<double> a, const double2 *x, double2 *y) {
    k_caxpy<<<FG_GRID, FG_BLOCK>>>(s->n, a.real(), a.imag(), x, y);
    FG_CUDA(cudaGetLastError());
    return WD_OK;
}

extern "C" {

const char *wd_fgcr_last_error(void) { return g_fg_error.c_str(); }

void wd_fgcr_destroy(wd_fgcr *s) {
    if (!s) return;
    cudaDeviceSynchronize();
    for (void *p : s->allocs) cudaFree(p);
    if (s->partials_host) cudaFreeHost(s->partials_host);
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
            for (int i = 0; i < j; ++i) {
                FG_TRY(fg_dot(s, s->w[i], wj, c));
                const std::complex<double> beta = c / s->wn[i];
                FG_TRY(fg_axpy(s, -beta, s->w[i], wj));
                FG_TRY(fg_axpy(s, -beta, s->z[i], zj));
            }
            FG_TRY(fg_dot(s, wj, wj, c));
            s->wn[j] = c.real();
            if (!(s->wn[j] > 0.0)) { status = WD_ERR_BREAKDOWN; break; }
            FG_TRY(fg_dot(s, wj, s->r, c));
            const std::complex<double> alpha = c / s->wn[j];
            FG_TRY(fg_axpy(s, alpha, zj, s->xv));
            FG_TRY(fg_axpy(s, -alpha, wj, s->r));
            FG_TRY(fg_dot(s, s->r, s->r, c));
            rn = std::sqrt(c.real());
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
