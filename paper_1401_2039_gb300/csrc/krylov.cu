// The other Krylov solvers of the paper's solver comparison (Sec. 5, Fig.
// "algosxp": CGNR, CRNE, MCR1 and MCR2, all on the Schur-reduced system),
// which the paper names but does not define.  Textbook readings:
//
//   CR (Saad, "Iterative Methods for Sparse Linear Systems", 2nd ed., Alg.
//   6.20) on a Hermitian B y = c minimises ||c - B y|| over K_k(B, c):
//     alpha = (r|B r) / (Bp|Bp),  y += alpha p,  r -= alpha Bp,
//     beta = (r'|B r') / (r|B r), p = r' + beta p, Bp = B r' + beta Bp.
//   CRNE: B = A A^dag, x = A^dag y.  Tracked here through x itself:
//     s = A^dag r, t = A s = B r, q = A^dag p, w = A q = B p, (r|B r) = |s|^2,
//     so x += alpha q and q = s + beta q replace the updates of y and p.
//   MCR1/MCR2: B = gamma5 A, c = gamma5 b.  gamma5 A is Hermitian because
//     A^dag = gamma5 A gamma5 (Fig. "id"); with a twisted mass that identity
//     fails (gamma5 A(mu) gamma5 = A(-mu)^dag), so MCR needs mu = 0.  MCR1
//     forms B p with the operator each iteration (two applications of A),
//     MCR2 by the recurrence (one).
//   CGNR: Alg. "CGNR", in the same host-driven form, so that the four
//     methods are compared with the same vector kernels.
// A = Mhat_p, the Schur operator of the op (Alg. "schur"), applied in FP64
// through wd_apply_eo; x, r and every direction are FP64 canonical
// half-lattice fields [Vh][3][4]; every inner product sums in FP64 and is
// read by the host once per iteration.  The solve wraps the method in the
// Schur preparation and reconstruction and accepts x only on the FP64 true
// residual of the full system; if the recursive residual met the target but
// the true one does not, the method restarts from the current x with an
// explicitly computed residual.
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "op.cuh"

namespace wd {

constexpr int KR_BLOCK = 256;
constexpr int KR_GRID = 4 * 152;   // four blocks per SM of a GB300

// gamma5 of the DeGrand-Rossi basis is diag(1, 1, -1, -1); spin is the
// fastest index of the canonical [colour][spin] layout
__device__ __forceinline__ double kr_g5(long i) { return (i & 3) < 2 ? 1.0 : -1.0; }

// two complex sums (re, im, re, im)
struct __align__(16) KrSum4 {
    double x, y, z, w;
};

// per block: <a0, b0> and, when a1 != nullptr, <a1, b1> (complex, FP64)
__global__ void __launch_bounds__(KR_BLOCK)
k_kr_dot2(long n, const double2 *__restrict__ a0, const double2 *__restrict__ b0,
          const double2 *__restrict__ a1, const double2 *__restrict__ b1, KrSum4 *partials) {
    __shared__ KrSum4 ws[KR_BLOCK / 32];
    KrSum4 s = {0.0, 0.0, 0.0, 0.0};
    for (long i = (long)blockIdx.x * KR_BLOCK + threadIdx.x; i < n; i += (long)gridDim.x * KR_BLOCK) {
        const double2 x = a0[i], y = b0[i];
        s.x += x.x * y.x + x.y * y.y;
        s.y += x.x * y.y - x.y * y.x;
        if (a1) {
            const double2 u = a1[i], v = b1[i];
            s.z += u.x * v.x + u.y * v.y;
            s.w += u.x * v.y - u.y * v.x;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
        s.z += __shfl_xor_sync(0xffffffffu, s.z, o);
        s.w += __shfl_xor_sync(0xffffffffu, s.w, o);
    }
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        KrSum4 t = ws[0];
        for (int w = 1; w < KR_BLOCK / 32; ++w) {
            t.x += ws[w].x; t.y += ws[w].y; t.z += ws[w].z; t.w += ws[w].w;
        }
        partials[blockIdx.x] = t;
    }
}

// x += alpha p;  r -= alpha w
__global__ void __launch_bounds__(KR_BLOCK)
k_kr_step(long n, double alpha, double2 *__restrict__ x, const double2 *__restrict__ p,
          double2 *__restrict__ r, const double2 *__restrict__ w) {
    for (long i = (long)blockIdx.x * KR_BLOCK + threadIdx.x; i < n; i += (long)gridDim.x * KR_BLOCK) {
        const double2 pv = p[i], wv = w[i];
        double2 xv = x[i], rv = r[i];
        xv.x += alpha * pv.x; xv.y += alpha * pv.y;
        rv.x -= alpha * wv.x; rv.y -= alpha * wv.y;
        x[i] = xv;
        r[i] = rv;
    }
}

// q = s + beta q  and, when w != nullptr, w = t + beta w
__global__ void __launch_bounds__(KR_BLOCK)
k_kr_dir(long n, double beta, double2 *__restrict__ q, const double2 *__restrict__ s,
         double2 *__restrict__ w, const double2 *__restrict__ t) {
    for (long i = (long)blockIdx.x * KR_BLOCK + threadIdx.x; i < n; i += (long)gridDim.x * KR_BLOCK) {
        const double2 sv = s[i];
        double2 qv = q[i];
        qv.x = sv.x + beta * qv.x; qv.y = sv.y + beta * qv.y;
        q[i] = qv;
        if (w) {
            const double2 tv = t[i];
            double2 wv = w[i];
            wv.x = tv.x + beta * wv.x; wv.y = tv.y + beta * wv.y;
            w[i] = wv;
        }
    }
}

// out = g (a + c b), g = gamma5 when g5 != 0, else 1 (out may alias a or b)
__global__ void __launch_bounds__(KR_BLOCK)
k_kr_comb(long n, double2 *out, const double2 *a, double c, const double2 *b, int g5) {
    for (long i = (long)blockIdx.x * KR_BLOCK + threadIdx.x; i < n; i += (long)gridDim.x * KR_BLOCK) {
        const double2 av = a[i];
        double2 v = av;
        if (b) {
            const double2 bv = b[i];
            v.x += c * bv.x; v.y += c * bv.y;
        }
        if (g5 && kr_g5(i) < 0.0) { v.x = -v.x; v.y = -v.y; }
        out[i] = v;
    }
}

// v = c (1 + i s gamma5) v per canonical element (the twisted-mass block
// A = 1 + i t gamma5 and its inverse (1 - i t gamma5) / (1 + t^2))
__global__ void __launch_bounds__(KR_BLOCK)
k_kr_twist(long n, double2 *v, double s, double c) {
    for (long i = (long)blockIdx.x * KR_BLOCK + threadIdx.x; i < n; i += (long)gridDim.x * KR_BLOCK) {
        const double2 a = v[i];
        const double sg = s * kr_g5(i);
        v[i] = make_double2(c * (a.x - sg * a.y), c * (a.y + sg * a.x));
    }
}

// Parity p of full-lattice site lex (Lx even: the pair (2h, 2h+1) shares y, z, t).
__device__ __forceinline__ int kr_parity(long lex, int Lx, int Ly, int Lz) {
    const long row = lex / Lx;
    const int x = (int)(lex - row * Lx);
    const int y = (int)(row % Ly);
    const long r1 = row / Ly;
    const int z = (int)(r1 % Lz);
    const int t = (int)(r1 / Lz);
    return (x + y + z + t) & 1;
}

// split (to_half != 0): half[par][lex/2] = full[lex];  merge: the reverse
__global__ void __launch_bounds__(KR_BLOCK)
k_kr_parity(long n_full, double2 *full, double2 *even, double2 *odd, int Lx, int Ly, int Lz,
            int to_half) {
    for (long i = (long)blockIdx.x * KR_BLOCK + threadIdx.x; i < n_full;
         i += (long)gridDim.x * KR_BLOCK) {
        const long lex = i / 12;
        const int c = (int)(i - lex * 12);
        double2 *half = kr_parity(lex, Lx, Ly, Lz) ? odd : even;
        const long j = (lex >> 1) * 12 + c;
        if (to_half)
            half[j] = full[i];
        else
            full[i] = half[j];
    }
}

}  // namespace wd

using namespace wd;

static thread_local std::string g_kr_error;
static int kr_fail(int code, const std::string &m) {
    g_kr_error = m;
    return code;
}
#define KR_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return kr_fail(e_ == cudaErrorMemoryAllocation ? WD_ERR_NOMEM : WD_ERR_CUDA,    \
                           std::string(#call) + ": " + cudaGetErrorString(e_));             \
    } while (0)
#define KR_TRY(call)                                                                        \
    do {                                                                                    \
        int rc_ = (call);                                                                   \
        if (rc_ != WD_OK) {                                                                 \
            if (g_kr_error.empty()) g_kr_error = wd_last_error();                           \
            return rc_;                                                                     \
        }                                                                                   \
    } while (0)

struct wd_krylov {
    wd_op *op = nullptr;
    int method = 0;
    long n = 0;                      // complex entries of a half-lattice field (12 Vh)
    double2 *x = nullptr, *r = nullptr, *f[4] = {}, *bh = nullptr, *bq = nullptr;
    double2 *full = nullptr;         // full-lattice work field (24 Vh entries)
    KrSum4 *partials = nullptr, *partials_host = nullptr;
    std::vector<void *> allocs;
    long launches = 0;               // kernels queued by the current solve
    long applies = 0;                // Schur-operator applications of the current solve
};

static int kr_alloc(wd_krylov *s, void **p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return kr_fail(WD_ERR_NOMEM, "cudaMalloc failed");
    }
    s->allocs.push_back(*p);
    KR_CUDA(cudaMemset(*p, 0, bytes));
    return WD_OK;
}

static cudaStream_t kr_stream(const wd_krylov *s) { return s->op->user; }

static int kr_check(wd_krylov *s) {
    s->launches += 1;
    KR_CUDA(cudaGetLastError());
    return WD_OK;
}

// out[0] = <a0, b0>, out[1] = <a1, b1> (a1 may be null), summed on the host in
// a fixed order
static int kr_dot2(wd_krylov *s, long n, const double2 *a0, const double2 *b0,
                   const double2 *a1, const double2 *b1, double out[4]) {
    k_kr_dot2<<<KR_GRID, KR_BLOCK, 0, kr_stream(s)>>>(n, a0, b0, a1, b1, s->partials);
    KR_TRY(kr_check(s));
    KR_CUDA(cudaMemcpyAsync(s->partials_host, s->partials, sizeof(KrSum4) * KR_GRID,
                            cudaMemcpyDeviceToHost, kr_stream(s)));
    KR_CUDA(cudaStreamSynchronize(kr_stream(s)));
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < KR_GRID; ++i) {
        t[0] += s->partials_host[i].x; t[1] += s->partials_host[i].y;
        t[2] += s->partials_host[i].z; t[3] += s->partials_host[i].w;
    }
    memcpy(out, t, sizeof(t));
    return WD_OK;
}

static int kr_comb(wd_krylov *s, long n, double2 *out, const double2 *a, double c,
                   const double2 *b, int g5) {
    k_kr_comb<<<KR_GRID, KR_BLOCK, 0, kr_stream(s)>>>(n, out, a, c, b, g5);
    return kr_check(s);
}

// out = Mhat_p in (dagger: Mhat_p^dag in)
static int kr_apply(wd_krylov *s, double2 *out, const double2 *in, int parity, int dagger) {
    s->applies += 1;
    s->launches += 4;   // pack, two hopping terms, unpack
    KR_TRY(wd_apply_eo(s->op, (double *)out, (const double *)in, parity, dagger));
    return WD_OK;
}

// v = A^-1 v on one parity (nothing for mu = 0)
static int kr_twist_inverse(wd_krylov *s, double2 *v) {
    const double t = s->op->twist(0);
    if (t == 0.0) return WD_OK;
    k_kr_twist<<<KR_GRID, KR_BLOCK, 0, kr_stream(s)>>>(s->n, v, -t, 1.0 / (1.0 + t * t));
    return kr_check(s);
}

static int kr_parity(wd_krylov *s, double2 *full, double2 *even, double2 *odd, int to_half) {
    const int *L = s->op->g.L;
    k_kr_parity<<<KR_GRID, KR_BLOCK, 0, kr_stream(s)>>>(2 * s->n, full, even, odd, L[0], L[1],
                                                         L[2], to_half);
    return kr_check(s);
}

// The method's state after the residual r is known: directions and (r|B r).
struct KrState {
    double rho = 0.0;   // CGNR: |A^dag r|^2; CRNE: |A^dag r|^2; MCR: Re (r|B r)
    double rr = 0.0;    // |r|^2
};

// Fields per method (f[0..3]):
//   CGNR  z = f0, p = f1, Ap = f2
//   CRNE  s = f0, t = f1, q = f2, w = f3
//   MCR   Br = f0, p = f1, Bp = f2
static int kr_start(wd_krylov *s, int p, KrState &st) {
    double d[4];
    double2 **f = s->f;
    switch (s->method) {
    case WD_KRYLOV_CGNR:
        KR_TRY(kr_apply(s, f[0], s->r, p, 1));                        // z = A^dag r
        KR_CUDA(cudaMemcpyAsync(f[1], f[0], sizeof(double2) * s->n, cudaMemcpyDeviceToDevice,
                                kr_stream(s)));                       // p = z
        KR_TRY(kr_dot2(s, s->n, f[0], f[0], s->r, s->r, d));
        break;
    case WD_KRYLOV_CRNE:
        KR_TRY(kr_apply(s, f[0], s->r, p, 1));                        // s = A^dag r
        KR_TRY(kr_apply(s, f[1], f[0], p, 0));                        // t = A s
        KR_CUDA(cudaMemcpyAsync(f[2], f[0], sizeof(double2) * s->n, cudaMemcpyDeviceToDevice,
                                kr_stream(s)));                       // q = s
        KR_CUDA(cudaMemcpyAsync(f[3], f[1], sizeof(double2) * s->n, cudaMemcpyDeviceToDevice,
                                kr_stream(s)));                       // w = t
        KR_TRY(kr_dot2(s, s->n, f[0], f[0], s->r, s->r, d));
        break;
    default:                                                          // MCR1, MCR2
        KR_TRY(kr_apply(s, f[0], s->r, p, 0));
        KR_TRY(kr_comb(s, s->n, f[0], f[0], 0.0, nullptr, 1));       // Br = gamma5 A r
        KR_CUDA(cudaMemcpyAsync(f[1], s->r, sizeof(double2) * s->n, cudaMemcpyDeviceToDevice,
                                kr_stream(s)));                       // p = r
        KR_CUDA(cudaMemcpyAsync(f[2], f[0], sizeof(double2) * s->n, cudaMemcpyDeviceToDevice,
                                kr_stream(s)));                       // Bp = Br
        KR_TRY(kr_dot2(s, s->n, s->r, f[0], s->r, s->r, d));
        break;
    }
    st.rho = d[0];
    st.rr = d[2];
    return WD_OK;
}

// One iteration; WD_ERR_BREAKDOWN on a zero or non-finite denominator.
static int kr_iterate(wd_krylov *s, int p, KrState &st) {
    double d[4];
    double2 **f = s->f;
    const long n = s->n;
    const cudaStream_t cs = kr_stream(s);
    if (s->method == WD_KRYLOV_CGNR) {
        KR_TRY(kr_apply(s, f[2], f[1], p, 0));                        // Ap = A p
        KR_TRY(kr_dot2(s, n, f[2], f[2], nullptr, nullptr, d));
        if (!(d[0] > 0.0) || !std::isfinite(st.rho)) return kr_fail(WD_ERR_BREAKDOWN, "CGNR: |Ap| = 0");
        const double alpha = st.rho / d[0];
        k_kr_step<<<KR_GRID, KR_BLOCK, 0, cs>>>(n, alpha, s->x, f[1], s->r, f[2]);
        KR_TRY(kr_check(s));
        KR_TRY(kr_apply(s, f[0], s->r, p, 1));                        // z = A^dag r
        KR_TRY(kr_dot2(s, n, f[0], f[0], s->r, s->r, d));
        const double beta = d[0] / st.rho;
        k_kr_dir<<<KR_GRID, KR_BLOCK, 0, cs>>>(n, beta, f[1], f[0], nullptr, nullptr);
        KR_TRY(kr_check(s));
        st.rho = d[0];
        st.rr = d[2];
        return WD_OK;
    }
    // CR: alpha = (r|B r) / |Bp|^2
    double2 *Bp = s->method == WD_KRYLOV_CRNE ? f[3] : f[2];
    double2 *dir = s->method == WD_KRYLOV_CRNE ? f[2] : f[1];
    KR_TRY(kr_dot2(s, n, Bp, Bp, nullptr, nullptr, d));
    if (!(d[0] > 0.0) || st.rho == 0.0 || !std::isfinite(st.rho))
        return kr_fail(WD_ERR_BREAKDOWN, "CR: (r|B r) or |B p| is zero");
    const double alpha = st.rho / d[0];
    k_kr_step<<<KR_GRID, KR_BLOCK, 0, cs>>>(n, alpha, s->x, dir, s->r, Bp);
    KR_TRY(kr_check(s));
    if (s->method == WD_KRYLOV_CRNE) {
        KR_TRY(kr_apply(s, f[0], s->r, p, 1));                        // s = A^dag r
        KR_TRY(kr_apply(s, f[1], f[0], p, 0));                        // t = A s = B r
        KR_TRY(kr_dot2(s, n, f[0], f[0], s->r, s->r, d));
        const double beta = d[0] / st.rho;
        k_kr_dir<<<KR_GRID, KR_BLOCK, 0, cs>>>(n, beta, f[2], f[0], f[3], f[1]);
        KR_TRY(kr_check(s));
    } else {
        KR_TRY(kr_apply(s, f[0], s->r, p, 0));
        KR_TRY(kr_comb(s, n, f[0], f[0], 0.0, nullptr, 1));          // Br = gamma5 A r
        KR_TRY(kr_dot2(s, n, s->r, f[0], s->r, s->r, d));
        const double beta = d[0] / st.rho;
        if (s->method == WD_KRYLOV_MCR2) {                            // Bp = Br + beta Bp
            k_kr_dir<<<KR_GRID, KR_BLOCK, 0, cs>>>(n, beta, f[1], s->r, f[2], f[0]);
            KR_TRY(kr_check(s));
        } else {                                                      // Bp = gamma5 A p
            k_kr_dir<<<KR_GRID, KR_BLOCK, 0, cs>>>(n, beta, f[1], s->r, nullptr, nullptr);
            KR_TRY(kr_check(s));
            KR_TRY(kr_apply(s, f[2], f[1], p, 0));
            KR_TRY(kr_comb(s, n, f[2], f[2], 0.0, nullptr, 1));
        }
    }
    st.rho = d[0];
    st.rr = d[2];
    return WD_OK;
}

extern "C" {

const char *wd_krylov_last_error(void) { return g_kr_error.c_str(); }

void wd_krylov_destroy(wd_krylov *s) {
    if (!s) return;
    for (void *p : s->allocs) cudaFree(p);
    if (s->partials_host) cudaFreeHost(s->partials_host);
    delete s;
}

int wd_krylov_create(wd_krylov **out, wd_op *op, int method) {
    g_kr_error.clear();
    if (!out || !op) return kr_fail(WD_ERR_ARG, "null argument to wd_krylov_create");
    *out = nullptr;
    if (method < WD_KRYLOV_CGNR || method > WD_KRYLOV_MCR2)
        return kr_fail(WD_ERR_ARG, "method must be WD_KRYLOV_CGNR, _CRNE, _MCR1 or _MCR2");
    if (op->prec != WD_F64)
        return kr_fail(WD_ERR_ARG, "the Krylov solvers need a WD_F64 operator");
    wd_krylov *s = new wd_krylov();
    s->op = op;
    s->method = method;
    s->n = 12 * op->g.vh;
    const size_t bytes = sizeof(double2) * s->n;
    int rc = kr_alloc(s, (void **)&s->x, bytes);
    if (rc == WD_OK) rc = kr_alloc(s, (void **)&s->r, bytes);
    for (int i = 0; i < 4 && rc == WD_OK; ++i) rc = kr_alloc(s, (void **)&s->f[i], bytes);
    if (rc == WD_OK) rc = kr_alloc(s, (void **)&s->bh, bytes);
    if (rc == WD_OK) rc = kr_alloc(s, (void **)&s->bq, bytes);
    if (rc == WD_OK) rc = kr_alloc(s, (void **)&s->full, 2 * bytes);
    if (rc == WD_OK) rc = kr_alloc(s, (void **)&s->partials, sizeof(KrSum4) * KR_GRID);
    if (rc == WD_OK &&
        cudaMallocHost((void **)&s->partials_host, sizeof(KrSum4) * KR_GRID) != cudaSuccess)
        rc = kr_fail(WD_ERR_NOMEM, "pinned host buffer");
    if (rc != WD_OK) {
        std::string m = g_kr_error;
        wd_krylov_destroy(s);
        g_kr_error = m;
        return rc;
    }
    *out = s;
    return WD_OK;
}

int wd_krylov_solve(wd_krylov *s, double *x_, const double *b_, double tol, int maxiter,
                    int parity, wd_solve_info *info) {
    auto t0 = std::chrono::steady_clock::now();
    g_kr_error.clear();
    if (!s || !x_ || !b_) return kr_fail(WD_ERR_ARG, "null argument to wd_krylov_solve");
    if (!(tol > 0) || maxiter < 0) return kr_fail(WD_ERR_ARG, "tol must be > 0, maxiter >= 0");
    if (parity != 0 && parity != 1) return kr_fail(WD_ERR_ARG, "parity must be 0 or 1");
    if (s->method >= WD_KRYLOV_MCR1 && s->op->mu != 0.0)
        return kr_fail(WD_ERR_ARG, "MCR needs gamma5-hermiticity: twisted mass must be 0");
    if (!s->op->gauge_loaded) return kr_fail(WD_ERR_STATE, "no gauge field loaded");
    if (info) memset(info, 0, sizeof(*info));
    s->launches = 0;
    s->applies = 0;
    double2 *x = (double2 *)x_;
    double2 *b = (double2 *)b_;
    const int p = parity, q = 1 - parity;
    const double kappa = s->op->kappa;
    double2 *xp = s->x, *xq = s->f[3], *bp = s->r;
    double d[4];

    // Alg. "schur": bhat = b_p + kappa H_pq A^-1 b_q; x_p from the caller's x
    KR_TRY(kr_parity(s, b, p ? s->bq : bp, p ? bp : s->bq, 1));
    KR_TRY(kr_dot2(s, 2 * s->n, b, b, nullptr, nullptr, d));
    const double nb = std::sqrt(d[0]);
    const double target = tol * nb;
    KR_TRY(kr_twist_inverse(s, s->bq));
    s->launches += 3;
    KR_TRY(wd_dslash_eo(s->op, (double *)s->bh, (const double *)s->bq, p, 0));
    KR_TRY(kr_comb(s, s->n, s->bh, bp, kappa, s->bh, 0));
    KR_TRY(kr_parity(s, x, p ? xq : xp, p ? xp : xq, 1));

    const bool mcr = s->method >= WD_KRYLOV_MCR1;
    int iters = 0, restarts = 0, status = WD_ERR_NOT_CONVERGED;
    double true_rel = 0.0;
    while (true) {
        const int iters_at_start = iters;
        // r = bhat - A x_p (gamma5 of it for MCR), the method's start
        KR_TRY(kr_apply(s, s->r, xp, p, 0));
        KR_TRY(kr_comb(s, s->n, s->r, s->bh, -1.0, s->r, 0));
        if (mcr) KR_TRY(kr_comb(s, s->n, s->r, s->r, 0.0, nullptr, 1));
        KrState st;
        KR_TRY(kr_start(s, p, st));
        int rc = WD_OK;
        while (std::sqrt(st.rr) > target && iters < maxiter) {
            rc = kr_iterate(s, p, st);
            if (rc != WD_OK) break;
            ++iters;
        }
        if (rc == WD_ERR_BREAKDOWN) { status = rc; break; }
        KR_TRY(rc);
        // reconstruction x_q = A^-1 (b_q + kappa H_qp x_p) and the true residual
        KR_TRY(kr_parity(s, b, p ? s->bq : s->f[0], p ? s->f[0] : s->bq, 1));
        s->launches += 3;
        KR_TRY(wd_dslash_eo(s->op, (double *)xq, (const double *)xp, q, 0));
        KR_TRY(kr_comb(s, s->n, xq, s->bq, kappa, xq, 0));
        KR_TRY(kr_twist_inverse(s, xq));
        KR_TRY(kr_parity(s, x, p ? xq : xp, p ? xp : xq, 0));
        s->launches += 4;
        KR_TRY(wd_apply(s->op, (double *)s->full, (const double *)x, 0));
        KR_TRY(kr_comb(s, 2 * s->n, s->full, b, -1.0, s->full, 0));
        KR_TRY(kr_dot2(s, 2 * s->n, s->full, s->full, nullptr, nullptr, d));
        restarts += 1;
        const double rn = std::sqrt(d[0]);
        true_rel = nb > 0 ? rn / nb : 0.0;
        if (!std::isfinite(rn)) { status = WD_ERR_BREAKDOWN; break; }
        if (rn <= target) { status = WD_OK; break; }
        // a pass that could not iterate (maxiter, or a recomputed residual
        // already under the target while the true one is not) ends the solve
        if (iters >= maxiter || iters == iters_at_start) break;
    }
    KR_CUDA(cudaStreamSynchronize(kr_stream(s)));
    if (info) {
        info->iters = iters;
        info->reliable_updates = restarts;
        info->true_rel_resid = true_rel;
        // two hopping terms per Schur application, one in the preparation,
        // one per reconstruction and two per full-lattice residual
        info->dslash_hi = 2.0 * (double)s->applies + 1.0 + 3.0 * restarts;
        info->launches = (double)s->launches;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (status != WD_OK) kr_fail(status, status == WD_ERR_BREAKDOWN && !g_kr_error.empty()
                                             ? g_kr_error : wd_status_string(status));
    return status;
}

}  // extern "C"
