// Hopping term in double-float arithmetic with double-float storage and
// 18-real links: the residuals r = b - M x of the reliable updates.
//
// The arithmetic is that of dslash.cuh instantiated with df64 (lazily
// normalised compensated sums, rounded once per output real).  The eight
// hops, however, run as a loop instead of being unrolled: unrolled, one
// site's double-float hopping term is about 10^4 instructions of straight-line
// code, far more than the instruction cache holds, and warps then wait
// mostly on instruction fetch.  The loop body is one hop.  The direction's
// spin projector and reconstruction are chosen at run time from the pattern
// of the DeGrand-Rossi gamma matrices:
//   - which spin rows pair up: (0,3)(1,2) for x and y, (0,2)(1,3) for z and t;
//   - whether the coefficients are +-1 (y, t) or +-i (x, z);
//   - their signs.
// The backward hop's U^dag is formed in registers, so one SU(3) product
// serves both directions.
#include "dslash.cuh"

namespace wd {
namespace {

using cdf = cx<dfl>;

// f q for f = s (im false) or f = s i (im true), s = +-1 (exact)
__device__ __forceinline__ cdf times(cdf q, bool im, float s) {
    cdf r;
    r.re = im ? dfl(-s * q.im.s, -s * q.im.e) : dfl(s * q.re.s, s * q.re.e);
    r.im = im ? dfl(s * q.re.s, s * q.re.e) : dfl(s * q.im.s, s * q.im.e);
    return r;
}

__device__ __forceinline__ cdf sel(bool first, cdf a, cdf b) { return first ? a : b; }

template <int DAG, int EPI, int NORM, int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_dslash_df(const DslashArgs<df64> a) {
    df64 nrm[1] = {df64(0.0f, 0.0f)};
    const long h = (long)blockIdx.x * BLOCK + threadIdx.x;
    if (h < a.g.vh) {
        int c[4];
        site_coords(a.g, h, a.parity, c);
        const long s1 = a.g.hx, s2 = s1 * a.g.L[1], s3 = s2 * a.g.L[2];
        dfl acc[24];
#pragma unroll
        for (int k = 0; k < 24; ++k) acc[k] = 0;
#pragma unroll 1
        for (int hop = 0; hop < 8; ++hop) {
            const int mu = hop >> 1;
            const bool fwd = (hop & 1) == 0;
            // projector 1 + sgn gamma_mu: forward (1 - gamma) for H, (1 + gamma) for H^dag
            const float sgn = (fwd == (DAG != 0)) ? 1.0f : -1.0f;
            // neighbour x +- mu and whether the hop wraps
            long hn;
            bool wrap;
            if (mu == 0) {
                int xn = c[0] + (fwd ? 1 : -1);
                wrap = fwd ? (xn == a.g.L[0]) : (xn < 0);
                if (wrap) xn = fwd ? 0 : a.g.L[0] - 1;
                hn = h + ((xn >> 1) - (c[0] >> 1));
            } else {
                const long step = mu == 1 ? s1 : mu == 2 ? s2 : s3;
                const int cm = mu == 1 ? c[1] : mu == 2 ? c[2] : c[3];
                const int Lm = a.g.L[mu];
                wrap = fwd ? (cm == Lm - 1) : (cm == 0);
                const long jump = (long)(Lm - 1) * step;
                hn = fwd ? (wrap ? h - jump : h + step) : (wrap ? h + jump : h - step);
            }
            df64 psi[24];
            Rec<df64, 24>::template load<df64, 0>(a.in, a.g.stride, hn, psi);
            df64 U[18];
            Rec<df64, 18>::template load<df64, 1>(
                (fwd ? a.gauge_out : a.gauge_in) + mu * a.dir_bytes, a.g.stride, fwd ? h : hn, U);

            const bool swap = mu < 2;          // rows (0,3)(1,2), else (0,2)(1,3)
            const bool im = (mu & 1) == 0;     // coefficients +-i, else +-1
            const float f0 = (mu == 1 ? -1.0f : 1.0f) * sgn;
            const float f1 = (mu == 2 ? -1.0f : 1.0f) * sgn;
            const float g2 = (im ? -1.0f : 1.0f) * sgn;
            const float g3 = (swap ? -1.0f : 1.0f) * sgn;

            cdf hs[2][3];
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                const cdf p0 = {psi[8 * cc + 0], psi[8 * cc + 1]};
                const cdf p1 = {psi[8 * cc + 2], psi[8 * cc + 3]};
                const cdf p2 = {psi[8 * cc + 4], psi[8 * cc + 5]};
                const cdf p3 = {psi[8 * cc + 6], psi[8 * cc + 7]};
                hs[0][cc] = cadd(p0, times(sel(swap, p3, p2), im, f0));
                hs[1][cc] = cadd(p1, times(sel(swap, p2, p3), im, f1));
            }
            if (!fwd) {   // U <- U^dag
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = i + 1; j < 3; ++j) {
                        const df64 r = U[2 * (3 * i + j)], q = U[2 * (3 * i + j) + 1];
                        U[2 * (3 * i + j)] = U[2 * (3 * j + i)];
                        U[2 * (3 * i + j) + 1] = U[2 * (3 * j + i) + 1];
                        U[2 * (3 * j + i)] = r;
                        U[2 * (3 * j + i) + 1] = q;
                    }
#pragma unroll
                for (int k = 0; k < 9; ++k) U[2 * k + 1] = -U[2 * k + 1];
            }
            cdf u[2][3];
            su3_mul(U, hs, u);
            if (wrap) {
                const df64 pr = a.ph[2 * mu], pi = a.ph[2 * mu + 1];
                phase_mul(u, pr, fwd ? pi : -pi);
            }
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                const cdf r2 = times(sel(swap, u[1][cc], u[0][cc]), im, g2);
                const cdf r3 = times(sel(swap, u[0][cc], u[1][cc]), im, g3);
                acc[8 * cc + 0] += u[0][cc].re; acc[8 * cc + 1] += u[0][cc].im;
                acc[8 * cc + 2] += u[1][cc].re; acc[8 * cc + 3] += u[1][cc].im;
                acc[8 * cc + 4] += r2.re;       acc[8 * cc + 5] += r2.im;
                acc[8 * cc + 6] += r3.re;       acc[8 * cc + 7] += r3.im;
            }
        }
        df64 o[24];
        if (EPI == EPI_XPAY) {
            df64 xv[24];
            Rec<df64, 24>::template load<df64, 0>(a.x, a.g.stride, h, xv);
#pragma unroll
            for (int k = 0; k < 24; ++k) o[k] = settle(xv[k] + a.scale * acc[k]);
        } else {
#pragma unroll
            for (int k = 0; k < 24; ++k) o[k] = settle(a.scale * acc[k]);
        }
        Rec<df64, 24>::store(a.out, a.g.stride, h, o);
        if (NORM) {
            df64 sq = 0;
#pragma unroll
            for (int k = 0; k < 24; ++k) sq += o[k] * o[k];
            nrm[0] = sq;
        }
    }
    if (NORM) warp_partials<BLOCK, 1>(nrm, a.g.vh, a.red.partials);
}

template <int DAG, int EPI, int NORM, int CFG>
void launch_df(const DslashArgs<df64> &a, cudaStream_t s) {
    constexpr DslashCfg C = DSLASH_DF_CFGS[CFG];
    const unsigned grid = (unsigned)((a.g.vh + C.block - 1) / C.block);
    k_dslash_df<DAG, EPI, NORM, C.block, C.minb><<<grid, C.block, 0, s>>>(a);
}

template <int DAG, int EPI>
void launch_df_cfg(int cfg, const DslashArgs<df64> &a, cudaStream_t s) {
    switch (cfg) {
    case 1: launch_df<DAG, EPI, 0, 1>(a, s); break;
    case 2: launch_df<DAG, EPI, 0, 2>(a, s); break;
    case 3: launch_df<DAG, EPI, 0, 3>(a, s); break;
    case 4: launch_df<DAG, EPI, 0, 4>(a, s); break;
    default: launch_df<DAG, EPI, 0, 0>(a, s); break;
    }
}

}  // namespace

cudaError_t launch_dslash_df64_r18(const DslashLaunch &L, cudaStream_t s) {
    DslashArgs<df64> a;
    a.g = L.g;
    a.gauge_out = (const char *)L.gauge->ptr[L.out_parity];
    a.gauge_in = (const char *)L.gauge->ptr[1 - L.out_parity];
    a.dir_bytes = L.gauge->dir_bytes;
    a.out = L.out;
    a.in = L.in;
    a.x = L.x;
    a.scale = df64(L.scale);
    for (int i = 0; i < 8; ++i) a.ph[i] = df64(L.phase[i]);
    a.parity = L.out_parity;
    a.red = L.red ? *L.red : Reduction{nullptr, nullptr, nullptr, FIN_NONE};
    if (L.red) {   // fused norm; the residuals never use it: one configuration
        if (L.dagger) launch_df<1, EPI_XPAY, 1, 0>(a, s);
        else launch_df<0, EPI_XPAY, 1, 0>(a, s);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return launch_finish_partials(a.red, (L.g.vh + 31) / 32, s);
    } else if (L.epi == EPI_PLAIN) {
        if (L.dagger) launch_df_cfg<1, EPI_PLAIN>(L.cfg, a, s);
        else launch_df_cfg<0, EPI_PLAIN>(L.cfg, a, s);
    } else {
        if (L.dagger) launch_df_cfg<1, EPI_XPAY>(L.cfg, a, s);
        else launch_df_cfg<0, EPI_XPAY>(L.cfg, a, s);
    }
    return cudaGetLastError();
}

}  // namespace wd
