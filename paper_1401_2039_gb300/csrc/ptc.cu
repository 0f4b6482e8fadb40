// Learned preconditioner: a linear, gauge-equivariant parallel-transport
// convolution (PTC) network (Lehner & Wettig, arXiv:2302.05419).  Not in the
// paper; it serves as the right preconditioner of the flexible GCR solve.
//
// Layer l maps C_in channels of spinor fields to C_out channels:
//   out_c'(x) = sum_c sum_{k=0..8} W[c', c, k] (T_k in_c)(x)
// W[c', c, k] complex 4x4 (spin), T_0 = 1, T_{1+mu} psi(x) = U_mu(x) phi psi(x+mu),
// T_{5+mu} psi(x) = U_mu(x-mu)^dag phi^* psi(x-mu) (phases on wrapping hops).
//
// GB300 mapping.  Rows m = (site x, colour a), M = 3V.  A layer is
//   1. gather   A[m][(part, k, c, s)] = Re/Im (T_k in_c)(x)[a][s]  (BF16,
//      K = 2 * C_in * 36 columns, padded to a multiple of 64; the channel
//      index inside the transport index, so that the threads of a warp,
//      consecutive channels of a site, store consecutive 8-byte chunks),
//   2. GEMM     F_out[m][(part', c', s')] = sum A[m][.] B[(part', c', s')][.]
//      on the tensor cores (tcgen05, FP32 accumulation), with the complex
//      weights laid out as the real block matrix [[Wr, -Wi], [Wi, Wr]],
// and the FP32 output rows F[m] = (Re in_c'(x)[a][s'], then Im) are directly
// the input rows of the next layer's gather.  Training runs the same GEMM
// for the input gradient, dA = dF_out B, and its transposed form for the
// weight gradient, dB^T = A^T dF_out (a reduction over the 3V rows, split
// over CTAs and summed in a fixed order): every product of the network, in
// inference and training, is a tcgen05 kernel of this library.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "tc_gemm.cuh"
#include "wd_internal.cuh"

namespace wd {

constexpr int PTC_NK = 9;
constexpr int PTC_MAX_LAYERS = 8;
constexpr int PTC_BLOCK = 128;

inline long pad_to(long v, long m) { return (v + m - 1) / m * m; }

// canonical complex128 [V][3][4] -> F rows (x, a): [Re s0..3, Im s0..3], row stride ld
__global__ void k_ptc_in(long V, const double2 *__restrict__ r, float *__restrict__ F, int ld,
                         float scale) {
    const long i = (long)blockIdx.x * PTC_BLOCK + threadIdx.x;   // (x, a)
    if (i >= 3 * V) return;
    float *row = F + i * ld;
    for (int s = 0; s < 4; ++s) {
        const double2 v = r[i * 4 + s];
        row[s] = (float)v.x * scale;
        row[4 + s] = (float)v.y * scale;
    }
}

// F rows (x, a) [Re s0..3, Im s0..3] -> canonical complex128, times scale
__global__ void k_ptc_out(long V, const float *__restrict__ F, int ld, double2 *__restrict__ y,
                          double scale) {
    const long i = (long)blockIdx.x * PTC_BLOCK + threadIdx.x;
    if (i >= 3 * V) return;
    const float *row = F + i * ld;
    for (int s = 0; s < 4; ++s) y[i * 4 + s] = make_double2(row[s] * scale, row[4 + s] * scale);
}

struct PtcGeom {
    int L[4];
    long V;
    float ph[8];
};

__device__ __forceinline__ void lex_coords(const PtcGeom &g, long x, int c[4]) {
    unsigned r = (unsigned)x;
    for (int m = 0; m < 3; ++m) {
        const unsigned q = r / (unsigned)g.L[m];
        c[m] = (int)(r - q * (unsigned)g.L[m]);
        r = q;
    }
    c[3] = (int)r;
}

__device__ __forceinline__ long lex_of(const PtcGeom &g, const int c[4]) {
    return (((long)c[3] * g.L[2] + c[2]) * g.L[1] + c[1]) * g.L[0] + c[0];
}

// Neighbour x +- mu with its wrap flag.
__device__ __forceinline__ long ptc_neighbour(const PtcGeom &g, const int c[4], int mu, int dir,
                                              bool &wrap) {
    int n[4] = {c[0], c[1], c[2], c[3]};
    n[mu] += dir;
    wrap = false;
    if (n[mu] == g.L[mu]) { n[mu] = 0; wrap = true; }
    if (n[mu] < 0) { n[mu] = g.L[mu] - 1; wrap = true; }
    return lex_of(g, n);
}

// the four spins of channel c in an activation row: Re and Im as float4
__device__ __forceinline__ void load_spins(const float *row, int cin, int c, float2 v[4]) {
    const float4 re = *reinterpret_cast<const float4 *>(row + c * 4);
    const float4 im = *reinterpret_cast<const float4 *>(row + 4 * cin + c * 4);
    v[0] = make_float2(re.x, im.x);
    v[1] = make_float2(re.y, im.y);
    v[2] = make_float2(re.z, im.z);
    v[3] = make_float2(re.w, im.w);
}

// four BF16 values as one 8-byte store
__device__ __forceinline__ void store_bf16x4(__nv_bfloat16 *p, float a, float b, float c, float d) {
    const __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
    uint2 w;
    w.x = *reinterpret_cast<const uint32_t *>(&lo);
    w.y = *reinterpret_cast<const uint32_t *>(&hi);
    *reinterpret_cast<uint2 *>(p) = w;
}

}  // namespace wd

#include "ptc_fused.cuh"

namespace wd {

// Gather: one thread per (site x, input channel c).  F_in row stride ldf holds
// [Re (c, s)][Im (c, s)] blocks of 4*C_in values; A row stride lda.
__global__ void __launch_bounds__(PTC_BLOCK)
k_ptc_gather(PtcGeom g, int cin, const float *__restrict__ F, int ldf,
             const float2 *__restrict__ U, __nv_bfloat16 *__restrict__ A, int lda) {
    const long t = (long)blockIdx.x * PTC_BLOCK + threadIdx.x;
    if (t >= g.V * cin) return;
    const long x = t / cin;
    const int c = (int)(t - x * cin);
    int co[4];
    lex_coords(g, x, co);
    const int K = cin * 36;
    for (int k = 0; k < PTC_NK; ++k) {
        float2 v[3][4];
        if (k == 0) {
            for (int a = 0; a < 3; ++a) load_spins(F + (x * 3 + a) * (long)ldf, cin, c, v[a]);
        } else {
            const int mu = (k - 1) & 3;
            const bool fwd = k <= 4;
            bool wrap;
            const long xn = ptc_neighbour(g, co, mu, fwd ? 1 : -1, wrap);
            float2 p[3][4];
            for (int b = 0; b < 3; ++b) load_spins(F + (xn * 3 + b) * (long)ldf, cin, c, p[b]);
            const float2 *Ul = U + ((fwd ? x : xn) * 4 + mu) * 9;
            float pr = 1.f, pi = 0.f;
            if (wrap) { pr = g.ph[2 * mu]; pi = fwd ? g.ph[2 * mu + 1] : -g.ph[2 * mu + 1]; }
            for (int a = 0; a < 3; ++a)
                for (int s = 0; s < 4; ++s) {
                    float re = 0.f, im = 0.f;
                    for (int b = 0; b < 3; ++b) {
                        // forward: U[a][b]; backward: conj(U[b][a])
                        const float2 u = fwd ? Ul[3 * a + b] : Ul[3 * b + a];
                        const float ui = fwd ? u.y : -u.y;
                        re += u.x * p[b][s].x - ui * p[b][s].y;
                        im += u.x * p[b][s].y + ui * p[b][s].x;
                    }
                    v[a][s] = make_float2(re * pr - im * pi, re * pi + im * pr);
                }
        }
        for (int a = 0; a < 3; ++a) {
            __nv_bfloat16 *row = A + (x * 3 + a) * (long)lda + (k * cin + c) * 4;
            store_bf16x4(row, v[a][0].x, v[a][1].x, v[a][2].x, v[a][3].x);
            store_bf16x4(row + K, v[a][0].y, v[a][1].y, v[a][2].y, v[a][3].y);
        }
    }
}

// Real block form of the complex weights: B[(p', c', s')][(p, k, c, s)], row
// stride ldb, from W (complex64 as float2) [cout][cin][9][4][4].
__global__ void k_ptc_weights(int cout, int cin, const float2 *__restrict__ W,
                              __nv_bfloat16 *__restrict__ B, int ldb) {
    const int K = cin * 36, N = cout * 4;
    const long i = (long)blockIdx.x * PTC_BLOCK + threadIdx.x;
    if (i >= (long)N * K) return;
    const int n = (int)(i / K), kk = (int)(i - (long)n * K);
    const int cp = n >> 2, sp = n & 3;
    const int k = kk / (4 * cin), c = (kk >> 2) % cin, s = kk & 3;   // kk = (k cin + c) 4 + s
    const float2 w = W[((((long)cp * cin + c) * PTC_NK + k) * 4 + sp) * 4 + s];
    B[(long)n * ldb + kk] = __float2bfloat16_rn(w.x);              // Re out <- Re in:  Wr
    B[(long)n * ldb + K + kk] = __float2bfloat16_rn(-w.y);         // Re out <- Im in: -Wi
    B[(long)(N + n) * ldb + kk] = __float2bfloat16_rn(w.y);        // Im out <- Re in:  Wi
    B[(long)(N + n) * ldb + K + kk] = __float2bfloat16_rn(w.x);    // Im out <- Im in:  Wr
}

__global__ void k_c128_to_c64(long n, const double2 *in, float2 *out) {
    const long i = (long)blockIdx.x * PTC_BLOCK + threadIdx.x;
    if (i < n) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

__global__ void k_c64_to_c128(long n, const float2 *in, double2 *out) {
    const long i = (long)blockIdx.x * PTC_BLOCK + threadIdx.x;
    if (i < n) out[i] = make_double2(in[i].x, in[i].y);
}

// |v|^2 of a canonical complex128 field, one block-level partial per block
// (deterministic final sum on the host side of the launch helper).
// blockIdx.y selects the field (fields n entries apart), partials [y][x].
__global__ void k_norm2_c128(long n, const double2 *v, double *partials) {
    __shared__ double ws[PTC_BLOCK / 32];
    double s = 0.0;
    v += (long)blockIdx.y * n;
    partials += (long)blockIdx.y * gridDim.x;
    for (long i = (long)blockIdx.x * PTC_BLOCK + threadIdx.x; i < n; i += (long)gridDim.x * PTC_BLOCK)
        s += v[i].x * v[i].x + v[i].y * v[i].y;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < PTC_BLOCK / 32; ++w) t += ws[w];
        partials[blockIdx.x] = t;
    }
}


// ------------------------------------------------------------------ backward
// Loss gradient at the network output: G = 2 (y - e) / |e|^2 in the activation
// layout (FP32, and a BF16 copy with row stride ldb), |y - e|^2 per block.
__global__ void k_ptc_loss_grad(long V, const float *__restrict__ F, int ld,
                                const double2 *__restrict__ e, const double *__restrict__ inv_ne_p,
                                float *__restrict__ G, __nv_bfloat16 *__restrict__ Gb, int ldb,
                                double *partials) {
    __shared__ double ws[PTC_BLOCK / 32];
    const double inv_ne = *inv_ne_p;
    const long i = (long)blockIdx.x * PTC_BLOCK + threadIdx.x;   // (x, a)
    double d2 = 0.0;
    if (i < 3 * V) {
        const float *row = F + i * ld;
        for (int s = 0; s < 4; ++s) {
            const double2 ev = e[i * 4 + s];
            const double dr = row[s] - ev.x, di = row[4 + s] - ev.y;
            d2 += dr * dr + di * di;
            const float gr = (float)(2.0 * dr * inv_ne), gi = (float)(2.0 * di * inv_ne);
            G[i * ld + s] = gr;
            G[i * ld + 4 + s] = gi;
            Gb[i * ldb + s] = __float2bfloat16_rn(gr);
            Gb[i * ldb + 4 + s] = __float2bfloat16_rn(gi);
        }
    }
    for (int o = 16; o > 0; o >>= 1) d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = d2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < PTC_BLOCK / 32; ++w) t += ws[w];
        partials[blockIdx.x] = t * inv_ne;
    }
}

// Adjoint of the gather: dF_c(x) = sum_k (T_k^dag dA_{c,k})(x) with
// T_{1+mu}^dag = T_{5+mu} and T_{5+mu}^dag = T_{1+mu}; dA rows (y, a) hold
// [Re (k, c, s)][Im (k, c, s)].  One thread per (site x, channel c).
__global__ void __launch_bounds__(PTC_BLOCK)
k_ptc_scatter(PtcGeom g, int cin, const float *__restrict__ dA, int lda,
              const float2 *__restrict__ U, float *__restrict__ dF, int ldf,
              __nv_bfloat16 *__restrict__ dFb, int ldfb) {
    const long t = (long)blockIdx.x * PTC_BLOCK + threadIdx.x;
    if (t >= g.V * cin) return;
    const long x = t / cin;
    const int c = (int)(t - x * cin);
    int co[4];
    lex_coords(g, x, co);
    const int K = cin * 36;
    float2 acc[3][4];
    for (int a = 0; a < 3; ++a)
        for (int s = 0; s < 4; ++s) {
            const float *row = dA + (x * 3 + a) * (long)lda + c * 4;
            acc[a][s] = make_float2(row[s], row[K + s]);
        }
    for (int k = 1; k < PTC_NK; ++k) {
        const int mu = (k - 1) & 3;
        // dA_{c,k} is transported by T_k^dag: backward hop for k <= 4, forward otherwise
        const bool fwd = k > 4;
        bool wrap;
        const long xn = ptc_neighbour(g, co, mu, fwd ? 1 : -1, wrap);
        const float2 *Ul = U + ((fwd ? x : xn) * 4 + mu) * 9;
        float pr = 1.f, pi = 0.f;
        if (wrap) { pr = g.ph[2 * mu]; pi = fwd ? g.ph[2 * mu + 1] : -g.ph[2 * mu + 1]; }
        float2 p[3][4];
        for (int b = 0; b < 3; ++b)
            for (int s = 0; s < 4; ++s) {
                const float *row = dA + (xn * 3 + b) * (long)lda + (k * cin + c) * 4;
                p[b][s] = make_float2(row[s], row[K + s]);
            }
        for (int a = 0; a < 3; ++a)
            for (int s = 0; s < 4; ++s) {
                float re = 0.f, im = 0.f;
                for (int b = 0; b < 3; ++b) {
                    const float2 u = fwd ? Ul[3 * a + b] : Ul[3 * b + a];
                    const float ui = fwd ? u.y : -u.y;
                    re += u.x * p[b][s].x - ui * p[b][s].y;
                    im += u.x * p[b][s].y + ui * p[b][s].x;
                }
                acc[a][s].x += re * pr - im * pi;
                acc[a][s].y += re * pi + im * pr;
            }
    }
    for (int a = 0; a < 3; ++a) {
        float *row = dF + (x * 3 + a) * (long)ldf;
        __nv_bfloat16 *rb = dFb + (x * 3 + a) * (long)ldfb;
        for (int s = 0; s < 4; ++s) {
            row[c * 4 + s] = acc[a][s].x;
            row[4 * cin + c * 4 + s] = acc[a][s].y;
            rb[c * 4 + s] = __float2bfloat16_rn(acc[a][s].x);
            rb[4 * cin + c * 4 + s] = __float2bfloat16_rn(acc[a][s].y);
        }
    }
}

// Transposed real block weights Bt[(p, k, c, s)][(p', c', s')], row stride ldbt.
__global__ void k_ptc_weights_t(int cout, int cin, const float2 *__restrict__ W,
                                __nv_bfloat16 *__restrict__ Bt, int ldbt) {
    const int K = cin * 36, N = cout * 4;
    const long i = (long)blockIdx.x * PTC_BLOCK + threadIdx.x;
    if (i >= (long)N * K) return;
    const int n = (int)(i / K), kk = (int)(i - (long)n * K);
    const int cp = n >> 2, sp = n & 3;
    const int k = kk / (4 * cin), c = (kk >> 2) % cin, s = kk & 3;   // kk = (k cin + c) 4 + s
    const float2 w = W[((((long)cp * cin + c) * PTC_NK + k) * 4 + sp) * 4 + s];
    Bt[(long)kk * ldbt + n] = __float2bfloat16_rn(w.x);
    Bt[(long)(K + kk) * ldbt + n] = __float2bfloat16_rn(-w.y);
    Bt[(long)kk * ldbt + N + n] = __float2bfloat16_rn(w.y);
    Bt[(long)(K + kk) * ldbt + N + n] = __float2bfloat16_rn(w.x);
}

// Packed complex weight gradient from the transposed real block gradient
// dBt[k'][n'] (row stride ldbt): g = dL/dRe W + i dL/dIm W.
__global__ void k_ptc_wgrad(int cout, int cin, const float *__restrict__ dBt, int ldbt,
                            double2 *__restrict__ gW) {
    const int K = cin * 36, N = cout * 4;
    const long i = (long)blockIdx.x * PTC_BLOCK + threadIdx.x;
    if (i >= (long)N * K) return;
    const int n = (int)(i / K), kk = (int)(i - (long)n * K);
    const int cp = n >> 2, sp = n & 3;
    const int k = kk / (4 * cin), c = (kk >> 2) % cin, s = kk & 3;   // kk = (k cin + c) 4 + s
    const double gr = (double)dBt[(long)kk * ldbt + n] + dBt[(long)(K + kk) * ldbt + N + n];
    const double gi = -(double)dBt[(long)(K + kk) * ldbt + n] + dBt[(long)kk * ldbt + N + n];
    gW[((((long)cp * cin + c) * PTC_NK + k) * 4 + sp) * 4 + s] = make_double2(gr, gi);
}

// dBt += sum over the splits of the weight-gradient GEMM's partial products,
// in split order (the sum does not depend on how the splits were scheduled).
__global__ void k_ptc_sum_splits(long n, int splits, const float *__restrict__ part,
                                 float *__restrict__ dBt) {
    const long i = (long)blockIdx.x * PTC_BLOCK + threadIdx.x;
    if (i >= n) return;
    float t = dBt[i];
    for (int s = 0; s < splits; ++s) t += part[(long)s * n + i];
    dBt[i] = t;
}

// out = the sum of n partials in a fixed order (one block: strided per-thread
// sums, then a fixed tree).
__global__ void k_ptc_sum_loss(long n, const double *__restrict__ partials, double *out) {
    __shared__ double ws[PTC_BLOCK];
    double t = 0.0;
    for (long i = threadIdx.x; i < n; i += PTC_BLOCK) t += partials[i];
    ws[threadIdx.x] = t;
    __syncthreads();
    for (int o = PTC_BLOCK / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) ws[threadIdx.x] += ws[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = ws[0];
}

// inv_ne[i] = 1 / |e_i|^2 from per-block partials of the squared norms of
// nsamples fields (one block per (sample, chunk)), summed in block order.
__global__ void k_ptc_inv_norms(int nsamples, int chunks, const double *__restrict__ partials,
                                double *__restrict__ inv_ne) {
    const int i = blockIdx.x * PTC_BLOCK + threadIdx.x;
    if (i >= nsamples) return;
    double t = 0.0;
    for (int c = 0; c < chunks; ++c) t += partials[(long)i * chunks + c];
    inv_ne[i] = 1.0 / t;
}

// Adam on the real and imaginary parts of the weights.
__global__ void k_ptc_adam(long n, float2 *W, const double2 *g, float2 *m, float2 *v, float lr,
                           float b1, float b2, float eps, float c1, float c2) {
    const long i = (long)blockIdx.x * PTC_BLOCK + threadIdx.x;
    if (i >= n) return;
    const float gr = (float)g[i].x, gi = (float)g[i].y;
    float2 mm = m[i], vv = v[i], w = W[i];
    mm.x = b1 * mm.x + (1.f - b1) * gr;
    mm.y = b1 * mm.y + (1.f - b1) * gi;
    vv.x = b2 * vv.x + (1.f - b2) * gr * gr;
    vv.y = b2 * vv.y + (1.f - b2) * gi * gi;
    w.x -= lr * (mm.x / c1) / (sqrtf(vv.x / c2) + eps);
    w.y -= lr * (mm.y / c1) / (sqrtf(vv.y / c2) + eps);
    m[i] = mm;
    v[i] = vv;
    W[i] = w;
}

}  // namespace wd

// =================================================================== host side
using namespace wd;

static thread_local std::string g_ptc_error;
static int ptc_fail(int code, const std::string &m) {
    g_ptc_error = m;
    return code;
}
#define PTC_CUDA(call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return ptc_fail(e_ == cudaErrorMemoryAllocation ? WD_ERR_NOMEM : WD_ERR_CUDA,   \
                            std::string(#call) + ": " + cudaGetErrorString(e_));            \
    } while (0)
#define PTC_TRY(call)                                                                       \
    do {                                                                                    \
        int rc_ = (call);                                                                   \
        if (rc_ != WD_OK) return rc_;                                                       \
    } while (0)

struct wd_ptc {
    PtcGeom g{};
    int nl = 0;
    int ch[PTC_MAX_LAYERS + 1] = {};
    long M = 0, Mp = 0;                       // rows 3V, padded to 128
    int Kp[PTC_MAX_LAYERS] = {};              // gathered columns, padded to 64
    int Np[PTC_MAX_LAYERS] = {};              // output columns, padded to 16
    int ldF[PTC_MAX_LAYERS + 1] = {};         // activation row strides
    float *F[PTC_MAX_LAYERS + 1] = {};        // activations, FP32
    __nv_bfloat16 *A[PTC_MAX_LAYERS] = {};    // gathered operands, BF16
    __nv_bfloat16 *B[PTC_MAX_LAYERS] = {};    // weight matrices, BF16
    float2 *W[PTC_MAX_LAYERS] = {};           // complex weights (FP32 master copy)
    long wcount[PTC_MAX_LAYERS] = {};
    float2 *U = nullptr;                      // links, complex64 [V][4][3][3]
    double *partials = nullptr;
    double *partials_host = nullptr;
    int *err = nullptr;
    cudaStream_t stream = nullptr;            // work stream owned by the network
    cudaStream_t user = nullptr;              // caller's stream (nullptr = legacy)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // training
    bool train_ready = false;
    int Rp[PTC_MAX_LAYERS + 1] = {};          // BF16 gradient row strides (multiple of 64)
    float *dF[PTC_MAX_LAYERS + 1] = {};       // activation gradients, FP32
    __nv_bfloat16 *dFb[PTC_MAX_LAYERS + 1] = {};
    float *dA = nullptr;                      // gathered-operand gradient, FP32
    __nv_bfloat16 *Bt[PTC_MAX_LAYERS] = {};   // transposed weight matrices
    float *dBt[PTC_MAX_LAYERS] = {};          // real block weight gradients, [Kp][Np]
    float *wsplit = nullptr;                  // partial products of the weight-gradient splits
    long wsplit_elems = 0;
    double *inv_ne = nullptr;                 // 1 / |e_i|^2 of the samples of a call
    double *loss_dev = nullptr;               // per-sample losses of a call
    int inv_ne_cap = 0;
    double *norm_partials = nullptr;          // per-block partial norms, [sample][chunk]
    double2 *gW = nullptr;                    // packed complex gradient, all layers
    float2 *adam_m = nullptr, *adam_v = nullptr;
    long adam_t = 0;
    // bounded waits of the tensor-core GEMMs: polls per wait, and a test hook
    // that makes the GEMMs issue no MMA (their waits then run out)
    unsigned spin_limit = TC_SPIN_LIMIT;
    int withhold = 0;
    // layers with 16 input channels (16 or 1 output channels) of forward-only
    // applications run as one fused transport + tensor-core kernel
    // (wd_ptc_set_fused)
    int fused = 1;
    std::vector<void *> allocs;
};

// Work of a call is ordered after what the caller queued on its stream and
// before what it queues later.
static int ptc_fork(wd_ptc *n) {
    PTC_CUDA(cudaEventRecord(n->ev_fork, n->user));
    PTC_CUDA(cudaStreamWaitEvent(n->stream, n->ev_fork, 0));
    return WD_OK;
}
static int ptc_join(wd_ptc *n) {
    PTC_CUDA(cudaEventRecord(n->ev_join, n->stream));
    PTC_CUDA(cudaStreamWaitEvent(n->user, n->ev_join, 0));
    return WD_OK;
}

static int ptc_alloc(wd_ptc *n, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return ptc_fail(WD_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    n->allocs.push_back(*p);
    PTC_CUDA(cudaMemset(*p, 0, bytes));
    return WD_OK;
}

static unsigned grid_for(long n) { return (unsigned)std::max<long>(1, (n + PTC_BLOCK - 1) / PTC_BLOCK); }

// dynamic shared memory of the GEMM kernels: the ring of A and B tiles.  At
// BN = 128 it also keeps at most two CTAs per SM, within the SM's 512 TMEM
// columns.  Set once per process (and device ordinal 0..63).
static int ptc_gemm_attrs() {
    static bool done[64] = {};
    int dev = 0;
    PTC_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && done[dev]) return WD_OK;
    PTC_CUDA(cudaFuncSetAttribute(k_gemm_bf16_tc<128, TC_NT>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, tc_gemm_smem_bytes<128>()));
    PTC_CUDA(cudaFuncSetAttribute(k_gemm_bf16_tc<16, TC_NT>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, tc_gemm_smem_bytes<16>()));
    PTC_CUDA(cudaFuncSetAttribute(k_gemm_bf16_tc<128, TC_TN>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, TC_TN_SMEM_BYTES));
    PTC_CUDA(cudaFuncSetAttribute(k_gemm_bf16_tc<16, TC_TN>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, TC_TN_SMEM_BYTES));
    if (dev >= 0 && dev < 64) done[dev] = true;
    return WD_OK;
}

static TcArgs tc_args(wd_ptc *n, const __nv_bfloat16 *A, const __nv_bfloat16 *B, float *D,
                      int lda, int ldb, int ldd, long k_total) {
    TcArgs a{};
    a.A = A;
    a.B = B;
    a.D = D;
    a.lda = lda;
    a.ldb = ldb;
    a.ldd = ldd;
    a.k_total = k_total;
    a.k_split = k_total;
    a.d_split = 0;
    a.err = n->err;
    a.spin_limit = n->spin_limit;
    a.withhold = n->withhold;
    return a;
}

// D = A * B^T on the tensor cores; N must be a multiple of 16 (tiles of 128 when possible).
static int ptc_gemm(wd_ptc *n, const __nv_bfloat16 *A, const __nv_bfloat16 *B, float *D, long M,
                    int N, int K, int lda, int ldb, int ldd) {
    if (M % TC_BM || K % TC_BK || N % 16)
        return ptc_fail(WD_ERR_ARG, "GEMM shape not tile aligned");
    PTC_TRY(ptc_gemm_attrs());
    const TcArgs a = tc_args(n, A, B, D, lda, ldb, ldd, K);
    if (N % 128 == 0) {
        dim3 grid((unsigned)(M / TC_BM), (unsigned)(N / 128));
        k_gemm_bf16_tc<128, TC_NT><<<grid, TC_THREADS, tc_gemm_smem_bytes<128>(), n->stream>>>(a);
    } else {
        dim3 grid((unsigned)(M / TC_BM), (unsigned)(N / 16));
        k_gemm_bf16_tc<16, TC_NT><<<grid, TC_THREADS, tc_gemm_smem_bytes<16>(), n->stream>>>(a);
    }
    PTC_CUDA(cudaGetLastError());
    return WD_OK;
}

// Splits of the reduction of the transposed GEMM: enough CTAs to fill the
// GPU's SMs about once (at least one 64-row step per split).
static int tn_splits(long tiles, long R, int sms) {
    long s = std::max<long>(1, (sms + tiles - 1) / tiles);
    s = std::min<long>(s, std::max<long>(1, R / TC_BK));
    return (int)std::min<long>(s, 64);
}

// D += A^T B on the tensor cores: A [R][M], B [R][N] row-major (a reduction
// over the R rows), D [M][N] row stride ldd.  The rows are split over CTAs;
// each split writes a partial product into n->wsplit and k_ptc_sum_splits
// adds them to D in split order.  M % 128 == 0, N % 16 == 0, R % 64 == 0.
static int ptc_gemm_tn(wd_ptc *n, const __nv_bfloat16 *A, const __nv_bfloat16 *B, float *D,
                       long R, int M, int N, int lda, int ldb, int ldd) {
    if (M % TC_BM || R % TC_BK || N % 16 || ldd != N)
        return ptc_fail(WD_ERR_ARG, "transposed GEMM shape not tile aligned");
    PTC_TRY(ptc_gemm_attrs());
    int dev = 0, sms = 148;
    PTC_CUDA(cudaGetDevice(&dev));
    PTC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int bn = N % 128 == 0 ? 128 : 16;
    const long tiles = (long)(M / TC_BM) * (N / bn);
    const int splits = tn_splits(tiles, R, sms);
    const long elems = (long)M * N;
    if ((long)splits * elems > n->wsplit_elems) {   // grows (stream-ordered) to the largest product
        PTC_CUDA(cudaStreamSynchronize(n->stream));
        PTC_TRY(ptc_alloc(n, (void **)&n->wsplit, sizeof(float) * splits * elems));
        n->wsplit_elems = (long)splits * elems;
    }
    TcArgs a = tc_args(n, A, B, n->wsplit, lda, ldb, N, R);
    a.k_split = (R / splits + TC_BK - 1) / TC_BK * TC_BK;
    a.d_split = elems;
    const int used = (int)((R + a.k_split - 1) / a.k_split);   // splits with rows
    dim3 grid((unsigned)(M / TC_BM), (unsigned)(N / bn), (unsigned)used);
    if (bn == 128)
        k_gemm_bf16_tc<128, TC_TN><<<grid, TC_THREADS, TC_TN_SMEM_BYTES, n->stream>>>(a);
    else
        k_gemm_bf16_tc<16, TC_TN><<<grid, TC_THREADS, TC_TN_SMEM_BYTES, n->stream>>>(a);
    PTC_CUDA(cudaGetLastError());
    k_ptc_sum_splits<<<grid_for(elems), PTC_BLOCK, 0, n->stream>>>(elems, used, n->wsplit, D);
    PTC_CUDA(cudaGetLastError());
    return WD_OK;
}

static int ptc_check_err(wd_ptc *n) {
    int h = 0;
    PTC_CUDA(cudaMemcpyAsync(&h, n->err, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
    PTC_CUDA(cudaStreamSynchronize(n->stream));
    if (h) {
        PTC_CUDA(cudaMemsetAsync(n->err, 0, sizeof(int), n->stream));
        PTC_CUDA(cudaStreamSynchronize(n->stream));
        return ptc_fail(WD_ERR_TIMEOUT, h == 2 ? "tensor-core GEMM gave up waiting for its MMAs "
                                                 "and for their drain"
                                               : "tensor-core GEMM gave up waiting for its MMAs");
    }
    return WD_OK;
}

// One fused layer with 16 input channels (ptc_fused.cuh): F[l + 1] from
// F[l], no gathered operand.
template <int COUT>
static int ptc_layer_fused_t(wd_ptc *n, int l) {
    static bool attr_done[64] = {};
    int dev = 0;
    PTC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64 || !attr_done[dev]) {
        PTC_CUDA(cudaFuncSetAttribute(k_ptc_layer_fused<COUT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      pf_smem_bytes<COUT>()));
        if (dev >= 0 && dev < 64) attr_done[dev] = true;
    }
    if (n->Np[l] != pf_n<COUT>()) return ptc_fail(WD_ERR_ARG, "fused layer: output width");
    int sms = 1;
    PTC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PfArgs a;
    a.g = n->g;
    a.F = n->F[l];
    a.ldf = n->ldF[l];
    a.U = n->U;
    a.B = n->B[l];
    a.ldb = n->Kp[l];
    a.out = n->F[l + 1];
    a.ldo = n->ldF[l + 1];
    a.ntiles = (n->g.V + PF_SITES - 1) / PF_SITES;
    a.err = n->err;
    a.spin_limit = n->spin_limit;
    a.withhold = n->withhold;
    const unsigned grid = (unsigned)std::min<long>(a.ntiles, sms);
    k_ptc_layer_fused<COUT><<<grid, PF_ALL_THREADS, pf_smem_bytes<COUT>(), n->stream>>>(a);
    PTC_CUDA(cudaGetLastError());
    return WD_OK;
}

static int ptc_layer_fused(wd_ptc *n, int l) {
    return n->ch[l + 1] == 1 ? ptc_layer_fused_t<1>(n, l) : ptc_layer_fused_t<16>(n, l);
}

// forward through every layer, activations left in F[0..nl]; with
// keep_operands (training: the weight gradient needs them) every layer
// gathers its operand into A[l], otherwise layers with 16 input channels
// (and 16 or 1 output channels) run fused
static int ptc_forward(wd_ptc *n, const double *r, double in_scale, bool keep_operands = false) {
    const long V = n->g.V;
    k_ptc_in<<<grid_for(3 * V), PTC_BLOCK, 0, n->stream>>>(V, (const double2 *)r, n->F[0],
                                                            n->ldF[0], (float)in_scale);
    PTC_CUDA(cudaGetLastError());
    for (int l = 0; l < n->nl; ++l) {
        const int cin = n->ch[l];
        if (!keep_operands && n->fused && cin == PF_CIN &&
            (n->ch[l + 1] == 16 || n->ch[l + 1] == 1)) {
            PTC_TRY(ptc_layer_fused(n, l));
            continue;
        }
        k_ptc_gather<<<grid_for(V * cin), PTC_BLOCK, 0, n->stream>>>(n->g, cin, n->F[l], n->ldF[l],
                                                                      n->U, n->A[l], n->Kp[l]);
        PTC_CUDA(cudaGetLastError());
        PTC_TRY(ptc_gemm(n, n->A[l], n->B[l], n->F[l + 1], n->Mp, n->Np[l], n->Kp[l], n->Kp[l],
                         n->Kp[l], n->ldF[l + 1]));
    }
    return WD_OK;
}

extern "C" {

const char *wd_ptc_last_error(void) { return g_ptc_error.c_str(); }

void wd_ptc_destroy(wd_ptc *n) {
    if (!n) return;
    if (n->stream) cudaStreamSynchronize(n->stream);
    for (void *p : n->allocs) cudaFree(p);
    if (n->partials_host) cudaFreeHost(n->partials_host);
    if (n->ev_fork) cudaEventDestroy(n->ev_fork);
    if (n->ev_join) cudaEventDestroy(n->ev_join);
    if (n->stream) cudaStreamDestroy(n->stream);
    delete n;
}

int wd_ptc_create(wd_ptc **out, const int dims[4], const double phase[8], int nlayers,
                  const int *channels, void *stream) {
    if (!out || !dims || !phase || !channels) return ptc_fail(WD_ERR_ARG, "null argument");
    *out = nullptr;
    if (nlayers < 1 || nlayers > PTC_MAX_LAYERS) return ptc_fail(WD_ERR_ARG, "1..8 layers");
    long V = 1;
    for (int m = 0; m < 4; ++m) {
        if (dims[m] < 2 || dims[m] % 2) return ptc_fail(WD_ERR_DIMS, "extents must be even, >= 2");
        V *= dims[m];
    }
    if (channels[0] != 1 || channels[nlayers] != 1)
        return ptc_fail(WD_ERR_ARG, "the network maps one spinor field to one");
    for (int l = 0; l <= nlayers; ++l)
        if (channels[l] < 1 || channels[l] > 32) return ptc_fail(WD_ERR_ARG, "1..32 channels");
    wd_ptc *n = new wd_ptc();
    for (int m = 0; m < 4; ++m) n->g.L[m] = dims[m];
    n->g.V = V;
    for (int i = 0; i < 8; ++i) n->g.ph[i] = (float)phase[i];
    n->nl = nlayers;
    for (int l = 0; l <= nlayers; ++l) n->ch[l] = channels[l];
    n->M = 3 * V;
    n->Mp = pad_to(n->M, TC_BM);
    auto fail_free = [&](int rc) { std::string m = g_ptc_error; wd_ptc_destroy(n); g_ptc_error = m; return rc; };
    n->user = (cudaStream_t)stream;
    if (cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&n->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&n->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return fail_free(ptc_fail(WD_ERR_CUDA, "stream creation failed"));
    n->ldF[0] = 8;
    for (int l = 0; l < nlayers; ++l) {
        // a multiple of 128: the weight-gradient GEMM takes these columns as
        // its 128-row output tiles
        n->Kp[l] = (int)pad_to(2L * channels[l] * 36, TC_BM);
        n->Np[l] = (int)pad_to(2L * channels[l + 1] * 4, 16);
        n->ldF[l + 1] = n->Np[l];
        n->wcount[l] = (long)channels[l + 1] * channels[l] * PTC_NK * 16;
    }
    int rc = WD_OK;
    for (int l = 0; l <= nlayers && rc == WD_OK; ++l)
        rc = ptc_alloc(n, (void **)&n->F[l], sizeof(float) * n->Mp * n->ldF[l]);
    for (int l = 0; l < nlayers && rc == WD_OK; ++l) {
        rc = ptc_alloc(n, (void **)&n->A[l], sizeof(__nv_bfloat16) * n->Mp * n->Kp[l]);
        if (rc == WD_OK) rc = ptc_alloc(n, (void **)&n->B[l], sizeof(__nv_bfloat16) * (long)n->Np[l] * n->Kp[l]);
        if (rc == WD_OK) rc = ptc_alloc(n, (void **)&n->W[l], sizeof(float2) * n->wcount[l]);
    }
    if (rc == WD_OK) rc = ptc_alloc(n, (void **)&n->U, sizeof(float2) * V * 36);
    if (rc == WD_OK) rc = ptc_alloc(n, (void **)&n->partials, sizeof(double) * 4096);
    if (rc == WD_OK) rc = ptc_alloc(n, (void **)&n->err, sizeof(int) * 4);
    if (rc == WD_OK && cudaMallocHost((void **)&n->partials_host, sizeof(double) * 4096) != cudaSuccess)
        rc = ptc_fail(WD_ERR_NOMEM, "pinned host buffer");
    if (rc != WD_OK) return fail_free(rc);
    *out = n;
    return WD_OK;
}

int wd_ptc_set_gauge(wd_ptc *n, const double *U) {
    if (!n || !U) return ptc_fail(WD_ERR_ARG, "null argument");
    PTC_TRY(ptc_fork(n));
    const long cnt = n->g.V * 36;
    k_c128_to_c64<<<grid_for(cnt), PTC_BLOCK, 0, n->stream>>>(cnt, (const double2 *)U, n->U);
    PTC_CUDA(cudaGetLastError());
    PTC_CUDA(cudaStreamSynchronize(n->stream));
    return ptc_join(n);
}

static int ptc_rebuild_b(wd_ptc *n) {
    for (int l = 0; l < n->nl; ++l) {
        const long cnt = (long)n->ch[l + 1] * 4 * n->ch[l] * 36;
        k_ptc_weights<<<grid_for(cnt), PTC_BLOCK, 0, n->stream>>>(n->ch[l + 1], n->ch[l], n->W[l],
                                                                   n->B[l], n->Kp[l]);
        if (n->train_ready)
            k_ptc_weights_t<<<grid_for(cnt), PTC_BLOCK, 0, n->stream>>>(
                n->ch[l + 1], n->ch[l], n->W[l], n->Bt[l], n->Rp[l + 1]);
        PTC_CUDA(cudaGetLastError());
    }
    return WD_OK;
}

// Training buffers, allocated on the first gradient request.
static int ptc_train_setup(wd_ptc *n) {
    if (n->train_ready) return WD_OK;
    int kmax = 0;
    long wtot = 0;
    for (int l = 0; l <= n->nl; ++l) {
        n->Rp[l] = (int)pad_to(n->ldF[l], TC_BK);
        PTC_TRY(ptc_alloc(n, (void **)&n->dF[l], sizeof(float) * n->Mp * n->ldF[l]));
        PTC_TRY(ptc_alloc(n, (void **)&n->dFb[l], sizeof(__nv_bfloat16) * n->Mp * n->Rp[l]));
    }
    long wmax = 0;
    for (int l = 0; l < n->nl; ++l) {
        kmax = std::max(kmax, n->Kp[l]);
        wtot += n->wcount[l];
        wmax = std::max(wmax, (long)n->Kp[l] * n->Np[l]);
        PTC_TRY(ptc_alloc(n, (void **)&n->Bt[l], sizeof(__nv_bfloat16) * (long)n->Kp[l] * n->Rp[l + 1]));
        PTC_TRY(ptc_alloc(n, (void **)&n->dBt[l], sizeof(float) * (long)n->Kp[l] * n->Np[l]));
    }
    PTC_TRY(ptc_alloc(n, (void **)&n->dA, sizeof(float) * n->Mp * kmax));
    PTC_TRY(ptc_alloc(n, (void **)&n->gW, sizeof(double2) * wtot));
    PTC_TRY(ptc_alloc(n, (void **)&n->adam_m, sizeof(float2) * wtot));
    PTC_TRY(ptc_alloc(n, (void **)&n->adam_v, sizeof(float2) * wtot));
    n->wsplit_elems = 64 * wmax;   // at most 64 splits (tn_splits)
    PTC_TRY(ptc_alloc(n, (void **)&n->wsplit, sizeof(float) * n->wsplit_elems));
    (void)kmax;
    n->train_ready = true;
    return ptc_rebuild_b(n);
}

// 1 / |e_i|^2 of nsamples fields on the device (no host round trip).
static int ptc_inv_norms(wd_ptc *n, const double *e, int ns) {
    constexpr int CHUNKS = 256;
    if (ns > n->inv_ne_cap) {
        const int cap = std::max(ns, 64);
        PTC_TRY(ptc_alloc(n, (void **)&n->inv_ne, sizeof(double) * cap));
        PTC_TRY(ptc_alloc(n, (void **)&n->loss_dev, sizeof(double) * cap));
        PTC_TRY(ptc_alloc(n, (void **)&n->norm_partials, sizeof(double) * cap * CHUNKS));
        n->inv_ne_cap = cap;
    }
    const long fs = n->g.V * 12;
    k_norm2_c128<<<dim3(CHUNKS, (unsigned)ns), PTC_BLOCK, 0, n->stream>>>(fs, (const double2 *)e,
                                                                          n->norm_partials);
    k_ptc_inv_norms<<<grid_for(ns), PTC_BLOCK, 0, n->stream>>>(ns, CHUNKS, n->norm_partials,
                                                               n->inv_ne);
    PTC_CUDA(cudaGetLastError());
    return WD_OK;
}

// Loss of the samples and the gradient accumulated into dBt[] (not yet
// folded).  The samples run back to back on the work stream: the 1/|e_i|^2
// factors stay on the device, each sample's loss is summed on the device
// in a fixed order, and the host reads the per-sample losses and adds them,
// in order, after one synchronisation at the end.
static int ptc_accumulate(wd_ptc *n, const double *r, const double *e, int ns, double *loss) {
    const long V = n->g.V;
    const long fs = V * 12;    // complex entries per field
    const int L_ = n->nl;
    const unsigned nbl = grid_for(3 * V);
    if (nbl > 4096) return ptc_fail(WD_ERR_DIMS, "lattice too large for the loss reduction");
    if (ns > 4096) return ptc_fail(WD_ERR_ARG, "at most 4096 samples per call");
    for (int l = 0; l < n->nl; ++l)
        PTC_CUDA(cudaMemsetAsync(n->dBt[l], 0, sizeof(float) * (long)n->Np[l] * n->Kp[l], n->stream));
    PTC_TRY(ptc_inv_norms(n, e, ns));
    for (int i = 0; i < ns; ++i) {
        const double2 *ei = (const double2 *)e + i * fs;
        PTC_TRY(ptc_forward(n, r + i * fs * 2, 1.0, true));
        k_ptc_loss_grad<<<nbl, PTC_BLOCK, 0, n->stream>>>(V, n->F[L_], n->ldF[L_], ei, n->inv_ne + i,
                                                          n->dF[L_], n->dFb[L_], n->Rp[L_],
                                                          n->partials);
        k_ptc_sum_loss<<<1, PTC_BLOCK, 0, n->stream>>>(nbl, n->partials, n->loss_dev + i);
        PTC_CUDA(cudaGetLastError());
        for (int l = L_ - 1; l >= 0; --l) {
            // dB[l]^T += A[l]^T dF[l+1] on the tensor cores (split reduction over the rows)
            PTC_TRY(ptc_gemm_tn(n, n->A[l], n->dFb[l + 1], n->dBt[l], n->Mp, n->Kp[l], n->Np[l],
                                n->Kp[l], n->Rp[l + 1], n->Np[l]));
            if (l == 0) break;
            // dA = dF[l+1] B[l] on the tensor cores, then the adjoint transports
            PTC_TRY(ptc_gemm(n, n->dFb[l + 1], n->Bt[l], n->dA, n->Mp, n->Kp[l], n->Rp[l + 1],
                             n->Rp[l + 1], n->Rp[l + 1], n->Kp[l]));
            k_ptc_scatter<<<grid_for(V * n->ch[l]), PTC_BLOCK, 0, n->stream>>>(
                n->g, n->ch[l], n->dA, n->Kp[l], n->U, n->dF[l], n->ldF[l], n->dFb[l], n->Rp[l]);
            PTC_CUDA(cudaGetLastError());
        }
    }
    PTC_CUDA(cudaMemcpyAsync(n->partials_host, n->loss_dev, sizeof(double) * ns,
                             cudaMemcpyDeviceToHost, n->stream));
    PTC_CUDA(cudaStreamSynchronize(n->stream));
    double L = 0.0;
    for (int i = 0; i < ns; ++i) L += n->partials_host[i];
    if (loss) *loss = L;
    return ptc_check_err(n);
}

static int ptc_fold_grad(wd_ptc *n) {
    long off = 0;
    for (int l = 0; l < n->nl; ++l) {
        const long cnt = (long)n->ch[l + 1] * 4 * n->ch[l] * 36;
        k_ptc_wgrad<<<grid_for(cnt), PTC_BLOCK, 0, n->stream>>>(n->ch[l + 1], n->ch[l], n->dBt[l],
                                                                 n->Np[l], n->gW + off);
        off += n->wcount[l];
    }
    PTC_CUDA(cudaGetLastError());
    return WD_OK;
}

long wd_ptc_weight_count(const wd_ptc *n) {
    if (!n) return 0;
    long t = 0;
    for (int l = 0; l < n->nl; ++l) t += n->wcount[l];
    return t;
}

int wd_ptc_set_weights(wd_ptc *n, const double *W) {
    if (!n || !W) return ptc_fail(WD_ERR_ARG, "null argument");
    PTC_TRY(ptc_fork(n));
    long off = 0;
    for (int l = 0; l < n->nl; ++l) {
        k_c128_to_c64<<<grid_for(n->wcount[l]), PTC_BLOCK, 0, n->stream>>>(
            n->wcount[l], (const double2 *)W + off, n->W[l]);
        off += n->wcount[l];
    }
    PTC_CUDA(cudaGetLastError());
    PTC_TRY(ptc_rebuild_b(n));
    PTC_CUDA(cudaStreamSynchronize(n->stream));
    return ptc_join(n);
}

int wd_ptc_get_weights(wd_ptc *n, double *W) {
    if (!n || !W) return ptc_fail(WD_ERR_ARG, "null argument");
    PTC_TRY(ptc_fork(n));
    long off = 0;
    for (int l = 0; l < n->nl; ++l) {
        k_c64_to_c128<<<grid_for(n->wcount[l]), PTC_BLOCK, 0, n->stream>>>(
            n->wcount[l], n->W[l], (double2 *)W + off);
        off += n->wcount[l];
    }
    PTC_CUDA(cudaGetLastError());
    PTC_CUDA(cudaStreamSynchronize(n->stream));
    return ptc_join(n);
}

int wd_ptc_apply(wd_ptc *n, double *y, const double *r) {
    if (!n || !y || !r) return ptc_fail(WD_ERR_ARG, "null argument");
    PTC_TRY(ptc_fork(n));
    PTC_TRY(ptc_forward(n, r, 1.0));
    k_ptc_out<<<grid_for(3 * n->g.V), PTC_BLOCK, 0, n->stream>>>(
        n->g.V, n->F[n->nl], n->ldF[n->nl], (double2 *)y, 1.0);
    PTC_CUDA(cudaGetLastError());
    PTC_TRY(ptc_check_err(n));
    return ptc_join(n);
}

int wd_ptc_loss_grad(wd_ptc *n, const double *r, const double *e, int nsamples, double *loss,
                     double *grad) {
    if (!n || !r || !e || nsamples < 1) return ptc_fail(WD_ERR_ARG, "bad argument");
    PTC_TRY(ptc_fork(n));
    PTC_TRY(ptc_train_setup(n));
    PTC_TRY(ptc_accumulate(n, r, e, nsamples, loss));
    PTC_TRY(ptc_fold_grad(n));
    if (grad) {
        long tot = 0;
        for (int l = 0; l < n->nl; ++l) tot += n->wcount[l];
        PTC_CUDA(cudaMemcpyAsync(grad, n->gW, sizeof(double2) * tot, cudaMemcpyDeviceToDevice,
                                 n->stream));
    }
    PTC_CUDA(cudaStreamSynchronize(n->stream));
    return ptc_join(n);
}

int wd_ptc_train_step(wd_ptc *n, const double *r, const double *e, int nsamples, double lr,
                      double *loss) {
    if (!n || !r || !e || nsamples < 1 || !(lr > 0)) return ptc_fail(WD_ERR_ARG, "bad argument");
    PTC_TRY(ptc_fork(n));
    PTC_TRY(ptc_train_setup(n));
    PTC_TRY(ptc_accumulate(n, r, e, nsamples, loss));
    PTC_TRY(ptc_fold_grad(n));
    const float b1 = 0.9f, b2 = 0.999f;
    n->adam_t += 1;
    const float c1 = 1.f - powf(b1, (float)n->adam_t), c2 = 1.f - powf(b2, (float)n->adam_t);
    long off = 0;
    for (int l = 0; l < n->nl; ++l) {
        k_ptc_adam<<<grid_for(n->wcount[l]), PTC_BLOCK, 0, n->stream>>>(
            n->wcount[l], n->W[l], n->gW + off, n->adam_m + off, n->adam_v + off, (float)lr, b1, b2,
            1e-8f, c1, c2);
        off += n->wcount[l];
    }
    PTC_CUDA(cudaGetLastError());
    PTC_TRY(ptc_rebuild_b(n));
    PTC_CUDA(cudaStreamSynchronize(n->stream));
    return ptc_join(n);
}

// Bounded waits of the tensor-core GEMMs (see tc_gemm.cuh).
int wd_ptc_set_wait_limit(wd_ptc *n, unsigned polls, int withhold_mma) {
    if (!n || polls == 0 || (withhold_mma != 0 && withhold_mma != 1))
        return ptc_fail(WD_ERR_ARG, "bad argument");
    n->spin_limit = polls;
    n->withhold = withhold_mma;
    return WD_OK;
}

int wd_ptc_set_fused(wd_ptc *n, int on) {
    if (!n || (on != 0 && on != 1)) return ptc_fail(WD_ERR_ARG, "bad argument");
    n->fused = on;
    return WD_OK;
}

// D = A^T B through the transposed (weight-gradient) GEMM, for tests of
// the GEMM alone: A [R x M], B [R x N] BF16 row-major (device), D [M x N] FP32.
int wd_tc_gemm_bf16_tn(wd_ptc *n, const void *A, const void *B, float *D, long R, int M, int N) {
    if (!n || !A || !B || !D) return ptc_fail(WD_ERR_ARG, "null argument");
    if (R <= 0 || M <= 0 || N <= 0) return ptc_fail(WD_ERR_ARG, "empty product");
    PTC_TRY(ptc_fork(n));
    PTC_CUDA(cudaMemsetAsync(D, 0, sizeof(float) * M * (long)N, n->stream));
    PTC_TRY(ptc_gemm_tn(n, (const __nv_bfloat16 *)A, (const __nv_bfloat16 *)B, D, R, M, N, M, N, N));
    PTC_TRY(ptc_check_err(n));
    return ptc_join(n);
}

// D = A * B^T through the tensor-core GEMM, for tests of the GEMM alone:
// A [M x K], B [N x K] BF16 row-major (device), D [M x N] FP32.
int wd_tc_gemm_bf16(wd_ptc *n, const void *A, const void *B, float *D, long M, int N, int K) {
    if (!n || !A || !B || !D) return ptc_fail(WD_ERR_ARG, "null argument");
    PTC_TRY(ptc_fork(n));
    PTC_TRY(ptc_gemm(n, (const __nv_bfloat16 *)A, (const __nv_bfloat16 *)B, D, M, N, K, K, K, N));
    PTC_TRY(ptc_check_err(n));
    return ptc_join(n);
}

}  // extern "C"
