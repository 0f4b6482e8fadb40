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

// A complex double-float value with its real and imaginary parts in the two
// lanes of packed FP32 pairs: s = (re.s, im.s), e = (re.e, im.e).  Every
// operation below is the scalar double-float operation of df64.cuh done on
// both lanes at once, with the same FP32 roundings in the same order, so the
// hop gives bitwise the scalar loop's result in about half the FP32
// instructions.
struct dfc2 {
    f2 s, e;
};

__device__ __forceinline__ dfc2 dfc2_of(df64 re, df64 im) {
    return {f2_pack(re.hi, im.hi), f2_pack(re.lo, im.lo)};
}
__device__ __forceinline__ cdf cdf_of(dfc2 a) {
    cdf r;
    f2_unpack(a.s, r.re.s, r.im.s);
    f2_unpack(a.e, r.re.e, r.im.e);
    return r;
}
__device__ __forceinline__ dfc2 dfc2_of(cdf a) {
    return {f2_pack(a.re.s, a.im.s), f2_pack(a.re.e, a.im.e)};
}
__device__ __forceinline__ f2 f2_swap(f2 a) {
    float lo, hi;
    f2_unpack(a, lo, hi);
    return f2_pack(hi, lo);
}
__device__ __forceinline__ f2 f2_sel(bool first, f2 a, f2 b) { return first ? a : b; }
__device__ __forceinline__ dfc2 dfc2_sel(bool first, dfc2 a, dfc2 b) {
    return {f2_sel(first, a.s, b.s), f2_sel(first, a.e, b.e)};
}
// a + b: lazy_add<1> on each lane
__device__ __forceinline__ dfc2 dfc2_add(dfc2 a, dfc2 b) {
    const f2 s = f2_add(a.s, b.s);
    const f2 v = f2_sub(s, a.s);
    const f2 t = f2_add(f2_sub(a.s, f2_sub(s, v)), f2_sub(b.s, v));
    return {s, f2_add(a.e, f2_add(t, b.e))};
}
// a b for a real double-float a: operator*(df64, dfl) on each lane
__device__ __forceinline__ dfc2 dfc2_scale(df64 a, dfc2 b) {
    const f2 ah = f2_bcast(a.hi), al = f2_bcast(a.lo);
    const f2 p = f2_mul(ah, b.s);
    f2 c = f2_fma(ah, b.s, f2_neg(p));
    c = f2_fma(ah, b.e, c);
    c = f2_fma(al, b.s, c);
    return {p, c};
}
// times(q, im, s) on the pair: s q, or s i q = (-s q.im, s q.re)
__device__ __forceinline__ dfc2 dfc2_times(dfc2 q, bool im, float sg) {
    const f2 m = im ? f2_pack(-sg, sg) : f2_pack(sg, sg);
    return {f2_mul(im ? f2_swap(q.s) : q.s, m), f2_mul(im ? f2_swap(q.e) : q.e, m)};
}
// i a = (-a.im, a.re), exact
__device__ __forceinline__ dfc2 dfc2_muli(dfc2 a) {
    const f2 m = f2_pack(-1.0f, 1.0f);
    return {f2_mul(f2_swap(a.s), m), f2_mul(f2_swap(a.e), m)};
}

// u[k][a] = sum_b U[a][b] h[k][b] with ih = i h: the chains of su3_mul, the
// products U.im h.im entering as U.im (-h.im), i.e. through ih
__device__ __forceinline__ void su3_mul_dfc2(const df64 *U, const dfc2 h[2][3],
                                             const dfc2 ih[2][3], dfc2 u[2][3]) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            dfc2 acc = dfc2_scale(U[6 * a], h[k][0]);
            acc = dfc2_add(acc, dfc2_scale(U[6 * a + 1], ih[k][0]));
#pragma unroll
            for (int b = 1; b < 3; ++b) {
                acc = dfc2_add(acc, dfc2_scale(U[2 * (3 * a + b)], h[k][b]));
                acc = dfc2_add(acc, dfc2_scale(U[2 * (3 * a + b) + 1], ih[k][b]));
            }
            u[k][a] = acc;
        }
}

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
    dfc2 acc2[12];   // (spin, colour) 4 colour + spin: acc[2 k] + i acc[2 k + 1]
#pragma unroll
    for (int k = 0; k < 12; ++k) acc2[k] = dfc2_of(cdf{acc[2 * k], acc[2 * k + 1]});
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

        dfc2 hs[2][3], ihs[2][3];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            const dfc2 p0 = dfc2_of(psi[8 * cc + 0], psi[8 * cc + 1]);
            const dfc2 p1 = dfc2_of(psi[8 * cc + 2], psi[8 * cc + 3]);
            const dfc2 p2 = dfc2_of(psi[8 * cc + 4], psi[8 * cc + 5]);
            const dfc2 p3 = dfc2_of(psi[8 * cc + 6], psi[8 * cc + 7]);
            hs[0][cc] = dfc2_add(p0, dfc2_times(dfc2_sel(swap, p3, p2), im, f0));
            hs[1][cc] = dfc2_add(p1, dfc2_times(dfc2_sel(swap, p2, p3), im, f1));
            ihs[0][cc] = dfc2_muli(hs[0][cc]);
            ihs[1][cc] = dfc2_muli(hs[1][cc]);
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
        dfc2 u[2][3];
        su3_mul_dfc2(U, hs, ihs, u);
        if (wrap && (phase_on >> mu & 1u)) {   // rare: the scalar phase product
            const df64 pr = df64(ph[2 * mu]), pi = df64(ph[2 * mu + 1]);
            cdf us[2][3];
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int a = 0; a < 3; ++a) us[k][a] = cdf_of(u[k][a]);
            phase_mul(us, pr, fwd ? pi : -pi);
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int a = 0; a < 3; ++a) u[k][a] = dfc2_of(us[k][a]);
        }
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            const dfc2 r2 = dfc2_times(dfc2_sel(swap, u[1][cc], u[0][cc]), im, g2);
            const dfc2 r3 = dfc2_times(dfc2_sel(swap, u[0][cc], u[1][cc]), im, g3);
            acc2[4 * cc + 0] = dfc2_add(acc2[4 * cc + 0], u[0][cc]);
            acc2[4 * cc + 1] = dfc2_add(acc2[4 * cc + 1], u[1][cc]);
            acc2[4 * cc + 2] = dfc2_add(acc2[4 * cc + 2], r2);
            acc2[4 * cc + 3] = dfc2_add(acc2[4 * cc + 3], r3);
        }
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const cdf v = cdf_of(acc2[k]);
        acc[2 * k] = v.re;
        acc[2 * k + 1] = v.im;
    }
}

}  // namespace wd
