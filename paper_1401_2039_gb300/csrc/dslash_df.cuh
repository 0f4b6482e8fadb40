// Hopping term in double-float arithmetic as a loop over the eight hops
// (the residuals r = b - M x of the reliable updates), shared by the
// single-field kernel and the batched kernel.
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
#pragma once

#include "dslash.cuh"

namespace wd {

using cdf = cx<dfl>;

// f q for f = s (im false) or f = s i (im true), s = +-1 (exact)
__device__ __forceinline__ cdf times(cdf q, bool im, float s) {
    cdf r;
    r.re = im ? dfl(-s * q.im.s, -s * q.im.e) : dfl(s * q.re.s, s * q.re.e);
    r.im = im ? dfl(s * q.re.s, s * q.re.e) : dfl(s * q.im.s, s * q.im.e);
    return r;
}

__device__ __forceinline__ cdf sel(bool first, cdf a, cdf b) { return first ? a : b; }

// neighbour x +- mu of half-lattice site h (coordinates c) for hop
// 2 mu + (0 forward | 1 backward), and whether the hop wraps
__device__ __forceinline__ long df_neighbour(const Geom &g, long h, const int c[4], int hop,
                                             bool &wrap) {
    const int mu = hop >> 1;
    const bool fwd = (hop & 1) == 0;
    if (mu == 0) {
        int xn = c[0] + (fwd ? 1 : -1);
        wrap = fwd ? (xn == g.L[0]) : (xn < 0);
        if (wrap) xn = fwd ? 0 : g.L[0] - 1;
        return h + ((xn >> 1) - (c[0] >> 1));
    }
    const long step = g.step[mu], back = g.back[mu];
    const int cm = mu == 1 ? c[1] : mu == 2 ? c[2] : c[3];
    wrap = fwd ? (cm == g.L[mu] - 1) : (cm == 0);
    return fwd ? (wrap ? h - back : h + step) : (wrap ? h + back : h - step);
}

// Link staging of the single-field kernel: the next hop's link record (nine
// 16-byte planes) is copied into shared memory by cp.async while the
// current hop computes; two buffers, laid out [buffer][plane][thread].
constexpr int DF_LINK_PLANES = 9;
template <int BLOCK>
__device__ __forceinline__ void df_stage_link(const Geom &g, const char *gauge_out,
                                              const char *gauge_in, size_t dir_bytes, long h,
                                              const int c[4], int hop, uint4 *stage) {
    bool wrap;
    const bool fwd = (hop & 1) == 0;
    const long site = fwd ? h : df_neighbour(g, h, c, hop, wrap);
    const char *base = (fwd ? gauge_out : gauge_in) + (hop >> 1) * dir_bytes + site * 16;
    uint4 *dst = stage + (hop & 1) * DF_LINK_PLANES * BLOCK + threadIdx.x;
#pragma unroll
    for (int j = 0; j < DF_LINK_PLANES; ++j)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                     :: "r"((uint32_t)__cvta_generic_to_shared(dst + j * BLOCK)),
                        "l"(base + (long)j * g.stride * 16)
                     : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// acc += H in at output site h (coordinates c, 18-real double-float links).
// The input field holds nrhs right-hand sides with the rhs index innermost:
// site s, rhs r at record s * nrhs + r of plane stride in_stride.  ph: the
// boundary phases (re, im per direction), double or df64.  stage (BLOCK
// threads, 2 x 9 x BLOCK chunks of shared memory): links staged one hop ahead.
// phase_on: bit mu clear when direction mu's phase is exactly 1 (skipped).
template <int DAG, int BLOCK = 0, typename PH>
__device__ __forceinline__ void df_hops(const Geom &g, const char *gauge_out, const char *gauge_in,
                                        size_t dir_bytes, const PH *ph, const void *in,
                                        long in_stride, int nrhs, int r, long h, const int c[4],
                                        dfl acc[24], uint4 *stage = nullptr,
                                        unsigned phase_on = 0xFu) {
    if constexpr (BLOCK > 0) df_stage_link<BLOCK>(g, gauge_out, gauge_in, dir_bytes, h, c, 0, stage);
#pragma unroll 1
    for (int hop = 0; hop < 8; ++hop) {
        const int mu = hop >> 1;
        const bool fwd = (hop & 1) == 0;
        // projector 1 + sgn gamma_mu: forward (1 - gamma) for H, (1 + gamma) for H^dag
        const float sgn = (fwd == (DAG != 0)) ? 1.0f : -1.0f;
        bool wrap;
        const long hn = df_neighbour(g, h, c, hop, wrap);
        df64 psi[24];
        Rec<df64, 24>::template load<df64, 0>(in, in_stride, hn * nrhs + r, psi);
        df64 U[18];
        if constexpr (BLOCK > 0) {
            if (hop < 7) df_stage_link<BLOCK>(g, gauge_out, gauge_in, dir_bytes, h, c, hop + 1, stage);
            else asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group 1;" ::: "memory");   // this hop's link is in
            const uint4 *src = stage + (hop & 1) * DF_LINK_PLANES * BLOCK + threadIdx.x;
#pragma unroll
            for (int j = 0; j < DF_LINK_PLANES; ++j) {
                const uint4 v = src[j * BLOCK];
                U[2 * j] = df64(__uint_as_float(v.x), __uint_as_float(v.y));
                U[2 * j + 1] = df64(__uint_as_float(v.z), __uint_as_float(v.w));
            }
        } else {
            Rec<df64, 18>::template load<df64, 1>((fwd ? gauge_out : gauge_in) + mu * dir_bytes,
                                                 g.stride, fwd ? h : hn, U);
        }

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
                    const df64 re = U[2 * (3 * i + j)], q = U[2 * (3 * i + j) + 1];
                    U[2 * (3 * i + j)] = U[2 * (3 * j + i)];
                    U[2 * (3 * i + j) + 1] = U[2 * (3 * j + i) + 1];
                    U[2 * (3 * j + i)] = re;
                    U[2 * (3 * j + i) + 1] = q;
                }
#pragma unroll
            for (int k = 0; k < 9; ++k) U[2 * k + 1] = -U[2 * k + 1];
        }
        cdf u[2][3];
        su3_mul(U, hs, u);
        if (wrap && (phase_on >> mu & 1u)) {
            const df64 pr = df64(ph[2 * mu]), pi = df64(ph[2 * mu + 1]);
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
}

}  // namespace wd
