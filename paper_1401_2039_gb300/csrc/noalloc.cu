// Schur operator without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while a host
// framework is capturing its stream into a CUDA graph, plug-ins whose host
// application owns every device allocation through its own memory pool, and
// real-time or signal-handling paths that must not enter the driver's
// allocator.  wd_apply_eo_noalloc serves them: it needs no operator handle
// (wd_op_create allocates), reads the caller's canonical FP64 arrays
// directly, and keeps its one intermediate field, the hopping term on the
// other parity, in a fixed file-scope device array.
//
// That array, g_noalloc_tmp, holds WD_NOALLOC_MAX_VH half-lattice sites of
// 12 complex doubles (12,582,912 bytes).  It is placed on a GPU when this
// entry point is first called there and stays until the process exits.  In host code its name is only a host-side
// stand-in, so the host takes its device address with cudaGetSymbolAddress
// once per device (with that device current) and passes that address to the
// kernels.  All calls share the array and it keeps the last call's
// contents: the first kernel overwrites every entry the second one reads,
// so nothing needs clearing, but calls that overlap on the GPU (other
// streams, other host threads) race on it.
#include <mutex>
#include <string>

#include "dslash.cuh"

namespace wd {

static __device__ __align__(256) double2 g_noalloc_tmp[WD_NOALLOC_MAX_VH * 12];

constexpr int NOALLOC_BLOCK = 128;

struct Phase8 { double v[8]; };
constexpr int NOALLOC_MAX_DEVICES = 64;

// Hopping term onto parity p from canonical arrays: spinors are
// [Vh][3][4] complex128 (entry lex / 2), links [V][4][3][3] complex128.
// out = scale * H in  (XPAY = 0)  or  x + scale * H in  (XPAY = 1).
template <int DAG, int XPAY>
__global__ void __launch_bounds__(NOALLOC_BLOCK)
k_hop_canonical(Geom g, int parity, const double2 *__restrict__ in,
                const double2 *__restrict__ U, double2 *__restrict__ out,
                const double2 *__restrict__ x, double scale, Phase8 ph) {
    const long h = (long)blockIdx.x * NOALLOC_BLOCK + threadIdx.x;
    if (h >= g.vh) return;
    int c[4];
    site_coords(g, h, parity, c);
    const long lex = (((long)c[3] * g.L[2] + c[2]) * g.L[1] + c[1]) * g.L[0] + c[0];
    double acc[24];
#pragma unroll
    for (int i = 0; i < 24; ++i) acc[i] = 0.0;
    constexpr int SF = DAG ? +1 : -1;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        for (int dir = 0; dir < 2; ++dir) {
            int n[4] = {c[0], c[1], c[2], c[3]};
            n[mu] += dir == 0 ? 1 : -1;
            bool wrap = false;
            if (n[mu] == g.L[mu]) { n[mu] = 0; wrap = true; }
            if (n[mu] < 0) { n[mu] = g.L[mu] - 1; wrap = true; }
            const long nlex = (((long)n[3] * g.L[2] + n[2]) * g.L[1] + n[1]) * g.L[0] + n[0];
            double psi[24], L18[18];
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                double2 v = in[(nlex >> 1) * 12 + i];
                psi[2 * i] = v.x;
                psi[2 * i + 1] = v.y;
            }
            const double2 *link = U + ((dir == 0 ? lex : nlex) * 4 + mu) * 9;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                double2 v = link[i];
                L18[2 * i] = v.x;
                L18[2 * i + 1] = v.y;
            }
            cx<double> hs[2][3], u[2][3];
            // forward hops project with 1 + SF gamma, backward with 1 - SF gamma
#define WD_HOP(MU)                                                                         \
    if (dir == 0) {                                                                        \
        project<MU, SF>(psi, hs);                                                          \
        su3_mul(L18, hs, u);                                                               \
        if (wrap) phase_mul(u, ph.v[2 * MU], ph.v[2 * MU + 1]);                          \
        accumulate<MU, SF>(acc, u);                                                        \
    } else {                                                                               \
        project<MU, -SF>(psi, hs);                                                         \
        su3_adj_mul(L18, hs, u);                                                           \
        if (wrap) phase_mul(u, ph.v[2 * MU], -ph.v[2 * MU + 1]);                         \
        accumulate<MU, -SF>(acc, u);                                                       \
    }
            if (mu == 0) { WD_HOP(0) } else if (mu == 1) { WD_HOP(1) }
            else if (mu == 2) { WD_HOP(2) } else { WD_HOP(3) }
#undef WD_HOP
        }
    }
#pragma unroll
    for (int i = 0; i < 12; ++i) {
        double2 r = {scale * acc[2 * i], scale * acc[2 * i + 1]};
        if (XPAY) {
            const double2 xv = x[h * 12 + i];
            r.x += xv.x;
            r.y += xv.y;
        }
        out[h * 12 + i] = r;
    }
}

static std::mutex g_noalloc_mutex;
static void *g_noalloc_addr[NOALLOC_MAX_DEVICES];

}  // namespace wd

using namespace wd;

static thread_local std::string g_noalloc_error;

static int noalloc_fail(int code, const std::string &msg) {
    g_noalloc_error = msg;
    return code;
}

extern "C" const char *wd_noalloc_last_error(void) { return g_noalloc_error.c_str(); }

extern "C" int wd_apply_eo_noalloc(double *out, const double *in, const double *U,
                                   const int dims[4], double kappa, const double phase[8],
                                   int parity, int dagger, void *stream) {
    if (!out || !in || !U || !dims || !phase)
        return noalloc_fail(WD_ERR_ARG, "null argument to wd_apply_eo_noalloc");
    if (parity != 0 && parity != 1) return noalloc_fail(WD_ERR_ARG, "parity must be 0 or 1");
    if (dagger != 0 && dagger != 1) return noalloc_fail(WD_ERR_ARG, "dagger must be 0 or 1");
    // The volume is checked after every factor: each extent is at most
    // 2^31 and the running product at most 2 * WD_NOALLOC_MAX_VH before a
    // multiplication, so the product cannot wrap around.
    long V = 1;
    for (int m = 0; m < 4; ++m) {
        if (dims[m] < 2 || dims[m] % 2)
            return noalloc_fail(WD_ERR_DIMS, "every lattice extent must be even and >= 2");
        V *= dims[m];
        if (V / 2 > WD_NOALLOC_MAX_VH)
            return noalloc_fail(WD_ERR_DIMS,
                                "half-lattice volume exceeds the no-allocation maximum of " +
                                    std::to_string((long)WD_NOALLOC_MAX_VH) + " sites");
    }
    // device address of the scratch array, looked up once per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(WD_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return noalloc_fail(WD_ERR_ARG, "device ordinal above 63");
    void *tmp = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_addr[dev]) {
            // Load all four kernels on this device now, so that no later call
            // (with the other dagger flag) triggers a lazy module load.
            cudaFuncAttributes fa;
            const void *kernels[4] = {(const void *)k_hop_canonical<0, 0>,
                                      (const void *)k_hop_canonical<0, 1>,
                                      (const void *)k_hop_canonical<1, 0>,
                                      (const void *)k_hop_canonical<1, 1>};
            for (const void *k : kernels) {
                e = cudaFuncGetAttributes(&fa, k);
                if (e != cudaSuccess)
                    return noalloc_fail(WD_ERR_CUDA, std::string("cudaFuncGetAttributes: ") +
                                                         cudaGetErrorString(e));
            }
            e = cudaGetSymbolAddress(&g_noalloc_addr[dev], g_noalloc_tmp);
            if (e != cudaSuccess) {
                g_noalloc_addr[dev] = nullptr;
                return noalloc_fail(WD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") +
                                                     cudaGetErrorString(e));
            }
        }
        tmp = g_noalloc_addr[dev];
    }
    const Geom g = make_geom(dims, V / 2);
    Phase8 ph{};
    for (int i = 0; i < 8; ++i) ph.v[i] = phase[i];
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned grid = (unsigned)((g.vh + NOALLOC_BLOCK - 1) / NOALLOC_BLOCK);
    const int q = 1 - parity;
    const double2 *in2 = (const double2 *)in, *U2 = (const double2 *)U;
    double2 *t2 = (double2 *)tmp, *out2 = (double2 *)out;
    // tmp = H_qp in;  out = in - kappa^2 H_pq tmp
    if (dagger) {
        k_hop_canonical<1, 0><<<grid, NOALLOC_BLOCK, 0, s>>>(g, q, in2, U2, t2, nullptr, 1.0, ph);
        k_hop_canonical<1, 1><<<grid, NOALLOC_BLOCK, 0, s>>>(g, parity, t2, U2, out2, in2,
                                                             -kappa * kappa, ph);
    } else {
        k_hop_canonical<0, 0><<<grid, NOALLOC_BLOCK, 0, s>>>(g, q, in2, U2, t2, nullptr, 1.0, ph);
        k_hop_canonical<0, 1><<<grid, NOALLOC_BLOCK, 0, s>>>(g, parity, t2, U2, out2, in2,
                                                             -kappa * kappa, ph);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(WD_ERR_CUDA, cudaGetErrorString(e));
    return WD_OK;
}
