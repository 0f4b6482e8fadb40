// Hopping term (Dslash) of the Wilson-Dirac operator, one output parity.
//
//   out(x) = sum_mu [ (1 + s_f gamma_mu) U_mu(x)        phi_mu  in(x+mu)
//                   + (1 + s_b gamma_mu) U_mu(x-mu)^dag  phi_mu* in(x-mu) ]
//   s_f = -1, s_b = +1 for H (Fig. "dirac"); swapped for H^dag.
//
// One thread per output site.  Each of the eight hops
//   1. loads the neighbour's 24 reals (read-only path, L1/L2 reuse between
//      the eight sites that read it),
//   2. projects them onto the two independent spin rows of (1 +- gamma_mu)
//      (rank 2, two entries per row from {+-1, +-i}, Sec. 4.2),
//   3. multiplies the 3x2 half spinor by the link (streamed, not cached in
//      L1; 12-real links rebuild the third row as conj(row0 x row1)),
//   4. applies the boundary phase if the hop wrapped,
//   5. expands back to four spin rows and accumulates.
// Gamma matrices: DeGrand-Rossi basis (gamma_5 = diag(1, 1, -1, -1)).
// Arithmetic type R = double for FP64 storage, float otherwise, df64
// (double-float) for the residuals of the reliable updates.  Intermediates
// (half spinors, transported half spinors, the accumulator) use Acc<R>: R
// itself, except that df64 keeps them as lazily normalised pairs (dfl, the
// compensated dot product of df64.cuh) and rounds once, before the store.
#pragma once

#include <type_traits>

#include "wd_internal.cuh"

namespace wd {

template <typename R> struct cx { R re, im; };

template <typename R> struct AccOf { using T = R; };
template <> struct AccOf<df64> { using T = dfl; };
template <typename R> using Acc = typename AccOf<R>::T;

__device__ __forceinline__ float settle(float a) { return a; }
__device__ __forceinline__ double settle(double a) { return a; }
__device__ __forceinline__ df64 settle(dfl a) { return normalise(a); }

template <typename R>
__device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
// i * a
template <typename R>
__device__ __forceinline__ cx<R> cmuli(cx<R> a) { return {-a.im, a.re}; }

// Half spinor h[spin row k][colour] from the 24 reals of a site, projector
// 1 + SGN * gamma_MU.  psi real index = 2 * (4 * colour + spin) + (0 re | 1 im).
template <int MU, int SGN, typename R, typename A>
__device__ __forceinline__ void project(const R *psi, cx<A> h[2][3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cx<A> p0 = {psi[8 * c + 0], psi[8 * c + 1]};
        cx<A> p1 = {psi[8 * c + 2], psi[8 * c + 3]};
        cx<A> p2 = {psi[8 * c + 4], psi[8 * c + 5]};
        cx<A> p3 = {psi[8 * c + 6], psi[8 * c + 7]};
        if (MU == 0) {          // gamma_x: rows (3, i) (2, i) (1, -i) (0, -i)
            h[0][c] = SGN > 0 ? cadd(p0, cmuli(p3)) : csub(p0, cmuli(p3));
            h[1][c] = SGN > 0 ? cadd(p1, cmuli(p2)) : csub(p1, cmuli(p2));
        } else if (MU == 1) {   // gamma_y: rows (3, -1) (2, 1) (1, 1) (0, -1)
            h[0][c] = SGN > 0 ? csub(p0, p3) : cadd(p0, p3);
            h[1][c] = SGN > 0 ? cadd(p1, p2) : csub(p1, p2);
        } else if (MU == 2) {   // gamma_z: rows (2, i) (3, -i) (0, -i) (1, i)
            h[0][c] = SGN > 0 ? cadd(p0, cmuli(p2)) : csub(p0, cmuli(p2));
            h[1][c] = SGN > 0 ? csub(p1, cmuli(p3)) : cadd(p1, cmuli(p3));
        } else {                // gamma_t: rows (2, 1) (3, 1) (0, 1) (1, 1)
            h[0][c] = SGN > 0 ? cadd(p0, p2) : csub(p0, p2);
            h[1][c] = SGN > 0 ? cadd(p1, p3) : csub(p1, p3);
        }
    }
}

// acc += (1 + SGN gamma_MU) expanded from the transported half spinor u:
// rows 0, 1 are u itself, rows 2, 3 are fixed multiples of u rows.
template <int MU, int SGN, typename A>
__device__ __forceinline__ void accumulate(A *acc, const cx<A> u[2][3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cx<A> r2, r3;
        if (MU == 0) {          // r2 = -SGN i u1, r3 = -SGN i u0
            r2 = cmuli(u[1][c]); r3 = cmuli(u[0][c]);
            if (SGN > 0) { r2 = {-r2.re, -r2.im}; r3 = {-r3.re, -r3.im}; }
        } else if (MU == 1) {   // r2 = SGN u1, r3 = -SGN u0
            r2 = u[1][c]; r3 = u[0][c];
            if (SGN > 0) r3 = {-r3.re, -r3.im}; else r2 = {-r2.re, -r2.im};
        } else if (MU == 2) {   // r2 = -SGN i u0, r3 = SGN i u1
            r2 = cmuli(u[0][c]); r3 = cmuli(u[1][c]);
            if (SGN > 0) r2 = {-r2.re, -r2.im}; else r3 = {-r3.re, -r3.im};
        } else {                // r2 = SGN u0, r3 = SGN u1
            r2 = u[0][c]; r3 = u[1][c];
            if (SGN < 0) { r2 = {-r2.re, -r2.im}; r3 = {-r3.re, -r3.im}; }
        }
        acc[8 * c + 0] += u[0][c].re; acc[8 * c + 1] += u[0][c].im;
        acc[8 * c + 2] += u[1][c].re; acc[8 * c + 3] += u[1][c].im;
        acc[8 * c + 4] += r2.re;      acc[8 * c + 5] += r2.im;
        acc[8 * c + 6] += r3.re;      acc[8 * c + 7] += r3.im;
    }
}

// (a0, a1) +-= (b0, b1) as one packed FP32 pair operation (add.rn.f32x2 /
// sub.rn.f32x2, each lane rounded as the scalar add)
template <bool SUB>
__device__ __forceinline__ void acc_x2(float &a0, float &a1, float b0, float b1) {
    if constexpr (SUB)
        asm("{\n\t.reg .b64 a, b;\n\tmov.b64 a, {%0, %1};\n\tmov.b64 b, {%2, %3};\n\t"
            "sub.rn.f32x2 a, a, b;\n\tmov.b64 {%0, %1}, a;\n\t}"
            : "+f"(a0), "+f"(a1) : "f"(b0), "f"(b1));
    else
        asm("{\n\t.reg .b64 a, b;\n\tmov.b64 a, {%0, %1};\n\tmov.b64 b, {%2, %3};\n\t"
            "add.rn.f32x2 a, a, b;\n\tmov.b64 {%0, %1}, a;\n\t}"
            : "+f"(a0), "+f"(a1) : "f"(b0), "f"(b1));
}

// (d0, d1) = s (a0, a1) [+ (x0, x1)] as one packed FP32 pair operation
__device__ __forceinline__ void scale_x2(float &d0, float &d1, float a0, float a1, float s) {
    asm("{\n\t.reg .b64 a, s, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 s, {%4, %4};\n\t"
        "mul.rn.f32x2 d, s, a;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(d0), "=f"(d1) : "f"(a0), "f"(a1), "f"(s));
}
__device__ __forceinline__ void scale_add_x2(float &d0, float &d1, float a0, float a1, float s,
                                             float x0, float x1) {
    asm("{\n\t.reg .b64 a, s, x, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 s, {%4, %4};\n\t"
        "mov.b64 x, {%5, %6};\n\tfma.rn.f32x2 d, s, a, x;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(d0), "=f"(d1) : "f"(a0), "f"(a1), "f"(s), "f"(x0), "f"(x1));
}

// Two FP32 lanes in one 64-bit register pair, and the packed FP32 pair
// operations on them (add/sub/mul/fma .rn.f32x2: each lane rounded as the
// scalar operation).
typedef unsigned long long f2;   // two FP32 lanes in one 64-bit register pair

__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
    f2 d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ void f2_unpack(f2 a, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a));
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// a b + c, one rounding per lane
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 f2_neg(f2 a) { return f2_mul(a, f2_pack(-1.0f, -1.0f)); }
__device__ __forceinline__ f2 f2_bcast(float a) { return f2_pack(a, a); }

// (q0, q1) += (a0, a1)^2 elementwise, one packed FP32 pair FMA
__device__ __forceinline__ void sq_acc_x2(float &q0, float &q1, float a0, float a1) {
    asm("{\n\t.reg .b64 a, q;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 q, {%0, %1};\n\t"
        "fma.rn.f32x2 q, a, a, q;\n\tmov.b64 {%0, %1}, q;\n\t}"
        : "+f"(q0), "+f"(q1) : "f"(a0), "f"(a1));
}

// accumulate<MU, SGN> with the complex additions of real sign as packed pair
// operations; the +-i terms (directions 0 and 2) stay scalar.  Same sums,
// same roundings.
template <int MU, int SGN>
__device__ __forceinline__ void accumulate_x2(float *acc, const cx<float> u[2][3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float *a = acc + 8 * c;
        acc_x2<false>(a[0], a[1], u[0][c].re, u[0][c].im);
        acc_x2<false>(a[2], a[3], u[1][c].re, u[1][c].im);
        if (MU == 1) {          // spin 2 += SGN u1, spin 3 -= SGN u0
            acc_x2<(SGN < 0)>(a[4], a[5], u[1][c].re, u[1][c].im);
            acc_x2<(SGN > 0)>(a[6], a[7], u[0][c].re, u[0][c].im);
        } else if (MU == 3) {   // spin 2 += SGN u0, spin 3 += SGN u1
            acc_x2<(SGN < 0)>(a[4], a[5], u[0][c].re, u[0][c].im);
            acc_x2<(SGN < 0)>(a[6], a[7], u[1][c].re, u[1][c].im);
        } else {
            // MU 0: spin 2 += -SGN i u1, spin 3 += -SGN i u0;
            // MU 2: spin 2 += -SGN i u0, spin 3 += SGN i u1;  i v = (-v.im, v.re)
            const cx<float> v2 = MU == 0 ? u[1][c] : u[0][c];
            const cx<float> v3 = MU == 0 ? u[0][c] : u[1][c];
            constexpr bool n3 = MU == 0 ? SGN > 0 : SGN < 0;   // spin 3 coefficient is -i
            if (SGN > 0) { a[4] += v2.im; a[5] -= v2.re; }
            else         { a[4] -= v2.im; a[5] += v2.re; }
            if (n3) { a[6] += v3.im; a[7] -= v3.re; }
            else    { a[6] -= v3.im; a[7] += v3.re; }
        }
    }
}

// Link as 18 reals (row-major, re/im); 12-real records rebuild row 2.
template <typename S, typename R, int RECON>
__device__ __forceinline__ void load_link(const void *base, long stride, long h, R *U) {
    Rec<S, RECON>::template load<R, 1>(base, stride, h, U);
    if (RECON == 12) {
        // row2 = conj(row0 x row1): (a1 b2 - a2 b1)^*, (a2 b0 - a0 b2)^*, (a0 b1 - a1 b0)^*
        const R a0r = U[0], a0i = U[1], a1r = U[2], a1i = U[3], a2r = U[4], a2i = U[5];
        const R b0r = U[6], b0i = U[7], b1r = U[8], b1i = U[9], b2r = U[10], b2i = U[11];
        R t;
        t = a1r * b2r; t -= a1i * b2i; t -= a2r * b1r; t += a2i * b1i; U[12] = t;
        t = a2r * b1i; t += a2i * b1r; t -= a1r * b2i; t -= a1i * b2r; U[13] = t;
        t = a2r * b0r; t -= a2i * b0i; t -= a0r * b2r; t += a0i * b2i; U[14] = t;
        t = a0r * b2i; t += a0i * b2r; t -= a2r * b0i; t -= a2i * b0r; U[15] = t;
        t = a0r * b1r; t -= a0i * b1i; t -= a1r * b0r; t += a1i * b0i; U[16] = t;
        t = a1r * b0i; t += a1i * b0r; t -= a0r * b1i; t -= a0i * b1r; U[17] = t;
    }
}

// c + a b and c - a b with one rounding, and a b, spelled with the
// round-to-nearest intrinsics in FP32 and FP64 so that the compiler cannot
// pick which product of a chain to fuse: every kernel that forms these
// products (the batched hop's one- and two-rhs forms among them) then rounds
// them identically.  Other arithmetic types use their own operators.
template <typename A, typename R>
__device__ __forceinline__ A pmul(R a, A b) {
    if constexpr (std::is_same<A, float>::value) return __fmul_rn(a, b);
    else if constexpr (std::is_same<A, double>::value) return __dmul_rn(a, b);
    else return a * b;
}
template <typename A, typename R>
__device__ __forceinline__ A pmac(R a, A b, A c) {
    if constexpr (std::is_same<A, float>::value) return __fmaf_rn(a, b, c);
    else if constexpr (std::is_same<A, double>::value) return __fma_rn(a, b, c);
    else return c + a * b;
}
template <typename A, typename R>
__device__ __forceinline__ A pmsub(R a, A b, A c) {
    if constexpr (std::is_same<A, float>::value) return __fmaf_rn(-a, b, c);
    else if constexpr (std::is_same<A, double>::value) return __fma_rn(-a, b, c);
    else return c - a * b;
}

// u[k][a] = sum_b U[a][b] h[k][b], written as chains of single
// multiply-adds so that every real product becomes one FMA.
template <typename R, typename A>
__device__ __forceinline__ void su3_mul(const R *U, const cx<A> h[2][3], cx<A> u[2][3]) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            A re = pmul(U[6 * a], h[k][0].re);
            A im = pmul(U[6 * a], h[k][0].im);
            re = pmsub(U[6 * a + 1], h[k][0].im, re);
            im = pmac(U[6 * a + 1], h[k][0].re, im);
#pragma unroll
            for (int b = 1; b < 3; ++b) {
                const R ur = U[2 * (3 * a + b)], ui = U[2 * (3 * a + b) + 1];
                re = pmac(ur, h[k][b].re, re);
                re = pmsub(ui, h[k][b].im, re);
                im = pmac(ur, h[k][b].im, im);
                im = pmac(ui, h[k][b].re, im);
            }
            u[k][a] = {re, im};
        }
}

// u[k][a] = sum_b conj(U[b][a]) h[k][b]
template <typename R, typename A>
__device__ __forceinline__ void su3_adj_mul(const R *U, const cx<A> h[2][3], cx<A> u[2][3]) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            A re = pmul(U[2 * a], h[k][0].re);
            A im = pmul(U[2 * a], h[k][0].im);
            re = pmac(U[2 * a + 1], h[k][0].im, re);
            im = pmsub(U[2 * a + 1], h[k][0].re, im);
#pragma unroll
            for (int b = 1; b < 3; ++b) {
                const R ur = U[2 * (3 * b + a)], ui = U[2 * (3 * b + a) + 1];
                re = pmac(ur, h[k][b].re, re);
                re = pmac(ui, h[k][b].im, re);
                im = pmac(ur, h[k][b].im, im);
                im = pmsub(ui, h[k][b].re, im);
            }
            u[k][a] = {re, im};
        }
}

template <typename R, typename A>
__device__ __forceinline__ void phase_mul(cx<A> u[2][3], R pr, R pi) {
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const A re = u[k][a].re * pr - u[k][a].im * pi;
            const A im = u[k][a].re * pi + u[k][a].im * pr;
            u[k][a] = {re, im};
        }
}

template <typename R> struct DslashArgs {
    Geom g;
    const char *gauge_out;   // links of the output parity (4 direction blocks)
    const char *gauge_in;    // links of the input parity
    size_t dir_bytes;
    void *out;
    const void *in;
    const void *x;
    R scale;
    R ph[8];
    unsigned phase_on;       // bit mu set: the boundary phase of direction mu is not 1
    int parity;              // output parity
    Reduction red;
    R twist;                 // twisted mass factor t (twist_on != 0)
    int twist_on;
    long h0, h1;             // output sites [h0, h1)
};

// v <- (1 + i t gamma5) v on one site's 24 reals.  gamma5 = diag(1, 1, -1, -1)
// in the DeGrand-Rossi basis: spins 0 and 1 take 1 + i t, spins 2 and 3 1 - i t.
template <typename R>
__device__ __forceinline__ void twist_site(R *v, R t) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const R ts = s < 2 ? t : -t;
            const R re = v[8 * c + 2 * s], im = v[8 * c + 2 * s + 1];
            v[8 * c + 2 * s] = re - ts * im;
            v[8 * c + 2 * s + 1] = im + ts * re;
        }
}

// The same factor on K consecutive reals of a site record starting at real
// index base (base even): the pair at index k is spin (k % 8) / 2.
template <int K, typename R>
__device__ __forceinline__ void twist_reals(R *v, int base, R t) {
#pragma unroll
    for (int m = 0; m < K / 2; ++m) {
        const int s = ((base + 2 * m) & 7) >> 1;
        const R ts = s < 2 ? t : -t;
        const R re = v[2 * m], im = v[2 * m + 1];
        v[2 * m] = re - ts * im;
        v[2 * m + 1] = im + ts * re;
    }
}

// Half-lattice index of the neighbour x +- mu of site h (coordinates c),
// from offsets: h = ((t*Lz + z)*Ly + y)*(Lx/2) + x/2.
template <int MU, int DIR>
__device__ __forceinline__ long neighbour(const Geom &g, long h, const int c[4], bool &wrap) {
    if (MU == 0) {
        int xn = c[0] + DIR;
        wrap = DIR > 0 ? (xn == g.L[0]) : (xn < 0);
        if (wrap) xn = DIR > 0 ? 0 : g.L[0] - 1;
        return h + ((xn >> 1) - (c[0] >> 1));
    }
    const long step = g.step[MU], back = g.back[MU];
    wrap = DIR > 0 ? (c[MU] == g.L[MU] - 1) : (c[MU] == 0);
    if (DIR > 0) return wrap ? h - back : h + step;
    return wrap ? h + back : h - step;
}

template <typename S, typename R, int RECON, int MU, int DAG>
__device__ __forceinline__ void hop_pair(const DslashArgs<R> &a, const int c[4], long h,
                                         Acc<R> *acc) {
    constexpr int SF = DAG ? +1 : -1;   // forward projector 1 + SF gamma
    constexpr int SB = -SF;
    // forward hop: U_mu(x) in(x + mu)
    {
        bool wrap;
        const long hn = neighbour<MU, +1>(a.g, h, c, wrap);
        R psi[24];
        Rec<S, 24>::template load<R, 0>(a.in, a.g.stride, hn, psi);
        cx<Acc<R>> hs[2][3], u[2][3];
        project<MU, SF>(psi, hs);
        R U[18];
        load_link<S, R, RECON>(a.gauge_out + MU * a.dir_bytes, a.g.stride, h, U);
        su3_mul(U, hs, u);
        if (wrap && (a.phase_on >> MU & 1u)) phase_mul(u, a.ph[2 * MU], a.ph[2 * MU + 1]);
        if constexpr (std::is_same<Acc<R>, float>::value) accumulate_x2<MU, SF>(acc, u);
        else accumulate<MU, SF>(acc, u);
    }
    // backward hop: U_mu(x - mu)^dag in(x - mu)
    {
        bool wrap;
        const long hn = neighbour<MU, -1>(a.g, h, c, wrap);
        R psi[24];
        Rec<S, 24>::template load<R, 0>(a.in, a.g.stride, hn, psi);
        cx<Acc<R>> hs[2][3], u[2][3];
        project<MU, SB>(psi, hs);
        R U[18];
        load_link<S, R, RECON>(a.gauge_in + MU * a.dir_bytes, a.g.stride, hn, U);
        su3_adj_mul(U, hs, u);
        if (wrap && (a.phase_on >> MU & 1u)) phase_mul(u, a.ph[2 * MU], -a.ph[2 * MU + 1]);
        if constexpr (std::is_same<Acc<R>, float>::value) accumulate_x2<MU, SB>(acc, u);
        else accumulate<MU, SB>(acc, u);
    }
}

// ------------------------------------------------------ FP16 and BF16 storage
// With 16-bit storage the generic hop spends about a sixth of its
// instructions converting elements to FP32 (one conversion per stored
// element).  This variant keeps spinors and links in their packed 32-bit
// words (one complex number each, real part in the low half): the spin
// projection adds packed words in 16-bit arithmetic, and every product of the
// SU(3) multiply is a mixed-precision FMA, 16-bit x 16-bit -> f32 (PTX
// fma.rn.f32.f16 or fma.rn.f32.bf16), accumulating in FP32.  The product of
// two FP16 (or two BF16) numbers is exact in FP32, so the one new rounding is
// the projection sum (relative 2^-11 for FP16, 2^-8 for BF16: the size of the
// storage rounding).  The twelve-real links rebuild row 2 = conj(row0 x row1)
// with the same mixed FMAs and round it to the storage type, as an 18-real
// link would store it.
#define WD_MIXED_FMA(NAME, SA, SB)                                                           \
    template <typename HT>                                                                   \
    __device__ __forceinline__ float NAME(uint32_t a, uint32_t b, float c) {                 \
        float d;                                                                             \
        if constexpr (std::is_same<HT, __half>::value)                                       \
            asm("{\n\t.reg .b16 a0, a1, b0, b1;\n\t"                                         \
                "mov.b32 {a0, a1}, %1;\n\tmov.b32 {b0, b1}, %2;\n\t"                         \
                "fma.rn.f32.f16 %0, " SA ", " SB ", %3;\n\t}"                                \
                : "=f"(d) : "r"(a), "r"(b), "f"(c));                                         \
        else                                                                                 \
            asm("{\n\t.reg .b16 a0, a1, b0, b1;\n\t"                                         \
                "mov.b32 {a0, a1}, %1;\n\tmov.b32 {b0, b1}, %2;\n\t"                         \
                "fma.rn.f32.bf16 %0, " SA ", " SB ", %3;\n\t}"                               \
                : "=f"(d) : "r"(a), "r"(b), "f"(c));                                         \
        return d;                                                                            \
    }
// mf_XY<HT>(a, b, c) = a.X * b.Y + c with X, Y in {l = real, h = imaginary}, for
// packed words of HT = __half (fma.rn.f32.f16) or __nv_bfloat16 (fma.rn.f32.bf16)
WD_MIXED_FMA(mf_ll, "a0", "b0")
WD_MIXED_FMA(mf_lh, "a0", "b1")
WD_MIXED_FMA(mf_hl, "a1", "b0")
WD_MIXED_FMA(mf_hh, "a1", "b1")
#undef WD_MIXED_FMA


// the packed two-element type of HT, and its words
template <typename HT> struct Pair2;
template <> struct Pair2<__half> {
    using T = __half2;
    __device__ static T of(float a, float b) { return __floats2half2_rn(a, b); }
};
template <> struct Pair2<__nv_bfloat16> {
    using T = __nv_bfloat162;
    __device__ static T of(float a, float b) { return __floats2bfloat162_rn(a, b); }
};
template <typename HT>
__device__ __forceinline__ typename Pair2<HT>::T as_p2(uint32_t a) {
    return *reinterpret_cast<typename Pair2<HT>::T *>(&a);
}
template <typename P2> __device__ __forceinline__ uint32_t as_u32(P2 a) {
    return *reinterpret_cast<uint32_t *>(&a);
}

// -a on both halves of a packed word, written as the type's own negation so
// that the compiler can fold it into the consuming multiply-add
template <typename HT> __device__ __forceinline__ uint32_t h2_neg(uint32_t a) {
    uint32_t d;
    if constexpr (std::is_same<HT, __half>::value)
        asm("neg.f16x2 %0, %1;" : "=r"(d) : "r"(a));
    else
        asm("neg.bf16x2 %0, %1;" : "=r"(d) : "r"(a));
    return d;
}

// p + F q on packed complex words (HT pairs), F = +1, -1, +i, -i (codes 0..3)
template <typename HT, int F>
__device__ __forceinline__ uint32_t h2_comb(uint32_t p, uint32_t q) {
    if (F == 0) return as_u32(__hadd2(as_p2<HT>(p), as_p2<HT>(q)));
    if (F == 1) return as_u32(__hsub2(as_p2<HT>(p), as_p2<HT>(q)));
    // i q = (-q.im, q.re), -i q = (q.im, -q.re): swap the halves, then one FMA
    const auto sq = __lowhigh2highlow(as_p2<HT>(q));
    const auto sg = F == 2 ? Pair2<HT>::of(-1.0f, 1.0f) : Pair2<HT>::of(1.0f, -1.0f);
    return as_u32(__hfma2(sq, sg, as_p2<HT>(p)));
}

// half spinor h[k][colour] (half2 words) of the site's 12 words (word 4 c + s)
template <typename HT, int MU, int SGN>
__device__ __forceinline__ void project_h2(const uint32_t *p, uint32_t h[2][3]) {
    constexpr int PI = SGN > 0 ? 2 : 3, MI = SGN > 0 ? 3 : 2;   // SGN i, -SGN i
    constexpr int P1 = SGN > 0 ? 0 : 1, M1 = SGN > 0 ? 1 : 0;   // SGN, -SGN
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const uint32_t p0 = p[4 * c], p1 = p[4 * c + 1], p2 = p[4 * c + 2], p3 = p[4 * c + 3];
        if (MU == 0) {
            h[0][c] = h2_comb<HT, PI>(p0, p3);
            h[1][c] = h2_comb<HT, PI>(p1, p2);
        } else if (MU == 1) {
            h[0][c] = h2_comb<HT, M1>(p0, p3);
            h[1][c] = h2_comb<HT, P1>(p1, p2);
        } else if (MU == 2) {
            h[0][c] = h2_comb<HT, PI>(p0, p2);
            h[1][c] = h2_comb<HT, MI>(p1, p3);
        } else {
            h[0][c] = h2_comb<HT, P1>(p0, p2);
            h[1][c] = h2_comb<HT, P1>(p1, p3);
        }
    }
}

// link as 9 half2 words (row-major); 12-real records rebuild row 2
template <typename HT, int RECON>
__device__ __forceinline__ void load_link_h2(const char *base, long stride, long site,
                                             uint32_t U[9]) {
    Rec<HT, RECON>::template load_words<1>(base, stride, site, U);
    if (RECON == 12) {
        // row2_j = conj(row0_k row1_l - row0_l row1_k), (j, k, l) cyclic
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int k = (j + 1) % 3, l = (j + 2) % 3;
            const uint32_t x = U[k], y = U[3 + l], z = U[l], w = U[3 + k];
            const uint32_t yn = h2_neg<HT>(y), wn = h2_neg<HT>(w);
            float re = mf_ll<HT>(x, y, 0.0f);
            re = mf_hh<HT>(x, yn, re);
            re = mf_ll<HT>(z, wn, re);
            re = mf_hh<HT>(z, w, re);
            float im = mf_lh<HT>(x, yn, 0.0f);
            im = mf_hl<HT>(x, yn, im);
            im = mf_lh<HT>(z, w, im);
            im = mf_hl<HT>(z, w, im);
            U[6 + j] = as_u32(Pair2<HT>::of(re, im));
        }
    }
}

// u[k][a] = sum_b U[a][b] h[k][b]
template <typename HT>
__device__ __forceinline__ void su3_mul_h2(const uint32_t U[9], const uint32_t h[2][3],
                                           cx<float> u[2][3]) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        uint32_t hn[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) hn[b] = h2_neg<HT>(h[k][b]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float re = mf_ll<HT>(U[3 * a], h[k][0], 0.0f);
            float im = mf_lh<HT>(U[3 * a], h[k][0], 0.0f);
            re = mf_hh<HT>(U[3 * a], hn[0], re);
            im = mf_hl<HT>(U[3 * a], h[k][0], im);
#pragma unroll
            for (int b = 1; b < 3; ++b) {
                re = mf_ll<HT>(U[3 * a + b], h[k][b], re);
                re = mf_hh<HT>(U[3 * a + b], hn[b], re);
                im = mf_lh<HT>(U[3 * a + b], h[k][b], im);
                im = mf_hl<HT>(U[3 * a + b], h[k][b], im);
            }
            u[k][a] = {re, im};
        }
    }
}

// u[k][a] = sum_b conj(U[b][a]) h[k][b]
template <typename HT>
__device__ __forceinline__ void su3_adj_mul_h2(const uint32_t U[9], const uint32_t h[2][3],
                                               cx<float> u[2][3]) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        uint32_t hn[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) hn[b] = h2_neg<HT>(h[k][b]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float re = mf_ll<HT>(U[a], h[k][0], 0.0f);
            float im = mf_lh<HT>(U[a], h[k][0], 0.0f);
            re = mf_hh<HT>(U[a], h[k][0], re);
            im = mf_hl<HT>(U[a], hn[0], im);
#pragma unroll
            for (int b = 1; b < 3; ++b) {
                re = mf_ll<HT>(U[3 * b + a], h[k][b], re);
                re = mf_hh<HT>(U[3 * b + a], h[k][b], re);
                im = mf_lh<HT>(U[3 * b + a], h[k][b], im);
                im = mf_hl<HT>(U[3 * b + a], hn[b], im);
            }
            u[k][a] = {re, im};
        }
    }
}

// acc += the forward and backward hops in direction MU.  The input field
// holds nrhs right-hand sides with the rhs index innermost (site s, rhs r at
// record s * nrhs + r of plane stride in_stride); ph: the boundary phases,
// phase_on: bit mu clear when direction mu's phase is exactly 1 (skipped).
template <int RECON, int MU, int DAG, typename PH>
__device__ __forceinline__ void hop_pair_h2(const Geom &g, const char *gauge_out,
                                            const char *gauge_in, size_t dir_bytes, const PH *ph,
                                            const void *in, long in_stride, int nrhs, int r,
                                            const int c[4], long h, float *acc,
                                            unsigned phase_on) {
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    const float pr = (float)ph[2 * MU], pi = (float)ph[2 * MU + 1];
    {
        bool wrap;
        const long hn = neighbour<MU, +1>(g, h, c, wrap);
        uint32_t p[12];
        Rec<__half, 24>::template load_words<0>((const char *)in, in_stride, hn * nrhs + r, p);
        uint32_t hs[2][3];
        project_h2<__half, MU, SF>(p, hs);
        uint32_t U[9];
        load_link_h2<__half, RECON>(gauge_out + MU * dir_bytes, g.stride, h, U);
        cx<float> u[2][3];
        su3_mul_h2<__half>(U, hs, u);
        if (wrap && (phase_on >> MU & 1u)) phase_mul(u, pr, pi);
        accumulate_x2<MU, SF>(acc, u);
    }
    {
        bool wrap;
        const long hn = neighbour<MU, -1>(g, h, c, wrap);
        uint32_t p[12];
        Rec<__half, 24>::template load_words<0>((const char *)in, in_stride, hn * nrhs + r, p);
        uint32_t hs[2][3];
        project_h2<__half, MU, SB>(p, hs);
        uint32_t U[9];
        load_link_h2<__half, RECON>(gauge_in + MU * dir_bytes, g.stride, hn, U);
        cx<float> u[2][3];
        su3_adj_mul_h2<__half>(U, hs, u);
        if (wrap && (phase_on >> MU & 1u)) phase_mul(u, pr, -pi);
        accumulate_x2<MU, SB>(acc, u);
    }
}

// The single-system FP16/BF16 hop computes in 32-bit site indices and byte
// offsets from precomputed hop steps (Geom::step, Geom::back), and runs its
// eight hops in one of three ways, all measured and offered to the autotuner:
//  * pipelined: the neighbour spinor and link words of hop i + 1 are loaded
//    into registers before the arithmetic of hop i, so every hop's loads are
//    in flight while the previous hop computes;
//  * staged: at kernel start every thread copies the link records of all
//    eight hops into shared memory with cp.async (global -> shared, no
//    registers held), one commit group per hop, so the block's link bytes
//    are all requested at once and each hop waits for its own group only;
//    the neighbour spinors (read by eight sites, mostly from L1/L2) go
//    through registers, two hops ahead;
//  * staged, three ahead: as staged, with three spinor buffers in registers.
// Measured at 32^3 x 64 (plain hop / xpay hop with fused norm): pipelined
// 60.3 / 85.2 us, staged 59.1 / 76.2 us, staged three ahead 53.7-55.4 /
// 72.2 us; the kernel waits mostly on the latency of the neighbour reads,
// so more of them in flight pays.
template <int MU, int DIR>
__device__ __forceinline__ unsigned neighbour32(const Geom &g, unsigned h, const int c[4],
                                                bool &wrap) {
    if (MU == 0) {
        int xn = c[0] + DIR;
        wrap = DIR > 0 ? (xn == g.L[0]) : (xn < 0);
        if (wrap) xn = DIR > 0 ? 0 : g.L[0] - 1;
        return h + (unsigned)((xn >> 1) - (c[0] >> 1));
    }
    const unsigned step = g.step[MU], back = g.back[MU];
    wrap = DIR > 0 ? (c[MU] == g.L[MU] - 1) : (c[MU] == 0);
    if (DIR > 0) return wrap ? h - back : h + step;
    return wrap ? h + back : h - step;
}

// 16-bit link records: NF 16-byte planes and a TAIL-byte plane
template <int RECON> struct LinkPlanes {
    static constexpr int NF = RECON == 12 ? 1 : 2;
    static constexpr int TAIL = RECON == 12 ? 8 : 4;
};

struct SpinorH2 {
    uint32_t p[12];
    bool wrap;
};

template <int MU, int DIR>
__device__ __forceinline__ void load_spinor_h2(const DslashArgs<float> &a, const int c[4],
                                               unsigned h, SpinorH2 &d) {
    const unsigned hn = neighbour32<MU, DIR>(a.g, h, c, d.wrap);
    const size_t plane = (size_t)a.g.stride * 16;
    const char *p0 = (const char *)a.in + (size_t)hn * 16;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const uint4 v = ld_nc_v4(p0 + j * plane);
        d.p[4 * j] = v.x; d.p[4 * j + 1] = v.y; d.p[4 * j + 2] = v.z; d.p[4 * j + 3] = v.w;
    }
}

// the link record of hop (MU, DIR): U_mu(x) forward, U_mu(x - mu) backward
template <int MU, int DIR>
__device__ __forceinline__ const char *link_base(const DslashArgs<float> &a) {
    return (DIR > 0 ? a.gauge_out : a.gauge_in) + MU * a.dir_bytes;
}

template <int RECON, int MU, int DIR>
__device__ __forceinline__ void load_link_words(const DslashArgs<float> &a, unsigned site,
                                                uint32_t U[9]) {
    constexpr int NF = LinkPlanes<RECON>::NF;
    const char *base = link_base<MU, DIR>(a);
    const size_t plane = (size_t)a.g.stride * 16;
#pragma unroll
    for (int j = 0; j < NF; ++j) {
        const uint4 v = ld_stream_v4(base + (size_t)site * 16 + j * plane);
        U[4 * j] = v.x; U[4 * j + 1] = v.y; U[4 * j + 2] = v.z; U[4 * j + 3] = v.w;
    }
    if (RECON == 12) {
        const uint2 v = ld_stream_v2(base + NF * plane + (size_t)site * 8);
        U[4] = v.x; U[5] = v.y;
    } else {
        U[8] = ld_stream_u32(base + NF * plane + (size_t)site * 4);
    }
}

// acc += hop (MU, DIR) of the neighbour words p with the link words U
// (12-real records: words 0..5, row 2 rebuilt here)
template <typename HT, int RECON, int MU, int DIR, int DAG>
__device__ __forceinline__ void compute_hop_h2(const DslashArgs<float> &a, const uint32_t p[12],
                                               bool wrap, uint32_t U[9], float *acc) {
    constexpr int SF = DAG ? +1 : -1;
    constexpr int S = DIR > 0 ? SF : -SF;
    if (RECON == 12) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int k = (j + 1) % 3, l = (j + 2) % 3;
            const uint32_t x = U[k], y = U[3 + l], z = U[l], w = U[3 + k];
            const uint32_t yn = h2_neg<HT>(y), wn = h2_neg<HT>(w);
            float re = mf_ll<HT>(x, y, 0.0f);
            re = mf_hh<HT>(x, yn, re);
            re = mf_ll<HT>(z, wn, re);
            re = mf_hh<HT>(z, w, re);
            float im = mf_lh<HT>(x, yn, 0.0f);
            im = mf_hl<HT>(x, yn, im);
            im = mf_lh<HT>(z, w, im);
            im = mf_hl<HT>(z, w, im);
            U[6 + j] = as_u32(Pair2<HT>::of(re, im));
        }
    }
    uint32_t hs[2][3];
    project_h2<HT, MU, S>(p, hs);
    cx<float> u[2][3];
    if (DIR > 0) su3_mul_h2<HT>(U, hs, u);
    else su3_adj_mul_h2<HT>(U, hs, u);
    if (wrap && (a.phase_on >> MU & 1u)) {   // a phase of exactly 1 is skipped
        const float pr = (float)a.ph[2 * MU], pi = (float)a.ph[2 * MU + 1];
        phase_mul(u, pr, DIR > 0 ? pi : -pi);
    }
    accumulate_x2<MU, S>(acc, u);
}

// ---- pipelined: spinor and link words of the next hop in registers
struct HopH2 {
    SpinorH2 s;
    uint32_t U[9];
};

template <int RECON, int I>
__device__ __forceinline__ void load_hop_h2(const DslashArgs<float> &a, const int c[4], unsigned h,
                                            HopH2 &d) {
    constexpr int MU = I / 2, DIR = (I & 1) ? -1 : +1;
    load_spinor_h2<MU, DIR>(a, c, h, d.s);
    bool wrap;
    const unsigned site = DIR > 0 ? h : neighbour32<MU, DIR>(a.g, h, c, wrap);
    load_link_words<RECON, MU, DIR>(a, site, d.U);
}

template <typename HT, int RECON, int DAG>
__device__ __forceinline__ void hops_h2_pipelined(const DslashArgs<float> &a, const int c[4],
                                                  unsigned h, float *acc) {
    HopH2 d0, d1;
    load_hop_h2<RECON, 0>(a, c, h, d0);
    load_hop_h2<RECON, 1>(a, c, h, d1);
    compute_hop_h2<HT, RECON, 0, +1, DAG>(a, d0.s.p, d0.s.wrap, d0.U, acc);
    load_hop_h2<RECON, 2>(a, c, h, d0);
    compute_hop_h2<HT, RECON, 0, -1, DAG>(a, d1.s.p, d1.s.wrap, d1.U, acc);
    load_hop_h2<RECON, 3>(a, c, h, d1);
    compute_hop_h2<HT, RECON, 1, +1, DAG>(a, d0.s.p, d0.s.wrap, d0.U, acc);
    load_hop_h2<RECON, 4>(a, c, h, d0);
    compute_hop_h2<HT, RECON, 1, -1, DAG>(a, d1.s.p, d1.s.wrap, d1.U, acc);
    load_hop_h2<RECON, 5>(a, c, h, d1);
    compute_hop_h2<HT, RECON, 2, +1, DAG>(a, d0.s.p, d0.s.wrap, d0.U, acc);
    load_hop_h2<RECON, 6>(a, c, h, d0);
    compute_hop_h2<HT, RECON, 2, -1, DAG>(a, d1.s.p, d1.s.wrap, d1.U, acc);
    load_hop_h2<RECON, 7>(a, c, h, d1);
    compute_hop_h2<HT, RECON, 3, +1, DAG>(a, d0.s.p, d0.s.wrap, d0.U, acc);
    compute_hop_h2<HT, RECON, 3, -1, DAG>(a, d1.s.p, d1.s.wrap, d1.U, acc);
}

// ---- staged: the eight link records in shared memory, [hop][plane][thread]
template <int RECON, int BLOCK> struct LinkStage {
    uint4 w[8][LinkPlanes<RECON>::NF][BLOCK];
    typename std::conditional<RECON == 12, uint2, uint32_t>::type tail[8][BLOCK];
};

__device__ __forceinline__ void cp_async_16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                 :: "r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;"
                 :: "r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src), "n"(BYTES)
                 : "memory");
}

// copy the link record of hop I into the stage as commit group I
template <int RECON, int I, int BLOCK>
__device__ __forceinline__ void stage_link_h2(const DslashArgs<float> &a, const int c[4],
                                              unsigned h, LinkStage<RECON, BLOCK> &st) {
    constexpr int MU = I / 2, DIR = (I & 1) ? -1 : +1;
    constexpr int NF = LinkPlanes<RECON>::NF, TAIL = LinkPlanes<RECON>::TAIL;
    bool wrap;
    const unsigned site = DIR > 0 ? h : neighbour32<MU, DIR>(a.g, h, c, wrap);
    const char *base = link_base<MU, DIR>(a);
    const size_t plane = (size_t)a.g.stride * 16;
#pragma unroll
    for (int j = 0; j < NF; ++j)
        cp_async_16(&st.w[I][j][threadIdx.x], base + (size_t)site * 16 + j * plane);
    cp_async_small<TAIL>(&st.tail[I][threadIdx.x], base + NF * plane + (size_t)site * TAIL);
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// wait for group I (groups I + 1 .. 7 may still be in flight), then compute
template <typename HT, int RECON, int I, int DAG, int BLOCK>
__device__ __forceinline__ void compute_staged_h2(const DslashArgs<float> &a, const SpinorH2 &d,
                                                  const LinkStage<RECON, BLOCK> &st, float *acc) {
    asm volatile("cp.async.wait_group %0;" :: "n"(7 - I) : "memory");
    uint32_t U[9];
#pragma unroll
    for (int j = 0; j < LinkPlanes<RECON>::NF; ++j) {
        const uint4 v = st.w[I][j][threadIdx.x];
        U[4 * j] = v.x; U[4 * j + 1] = v.y; U[4 * j + 2] = v.z; U[4 * j + 3] = v.w;
    }
    if constexpr (RECON == 12) {
        const uint2 t = st.tail[I][threadIdx.x];
        U[4] = t.x; U[5] = t.y;
    } else {
        U[8] = st.tail[I][threadIdx.x];
    }
    compute_hop_h2<HT, RECON, I / 2, (I & 1) ? -1 : +1, DAG>(a, d.p, d.wrap, U, acc);
}

template <typename HT, int RECON, int DAG, int BLOCK>
__device__ __forceinline__ void hops_h2_staged(const DslashArgs<float> &a, const int c[4],
                                               unsigned h, LinkStage<RECON, BLOCK> &st,
                                               float *acc) {
    stage_link_h2<RECON, 0>(a, c, h, st);
    stage_link_h2<RECON, 1>(a, c, h, st);
    stage_link_h2<RECON, 2>(a, c, h, st);
    stage_link_h2<RECON, 3>(a, c, h, st);
    stage_link_h2<RECON, 4>(a, c, h, st);
    stage_link_h2<RECON, 5>(a, c, h, st);
    stage_link_h2<RECON, 6>(a, c, h, st);
    stage_link_h2<RECON, 7>(a, c, h, st);
    SpinorH2 d0, d1;
    load_spinor_h2<0, +1>(a, c, h, d0);
    load_spinor_h2<0, -1>(a, c, h, d1);
    compute_staged_h2<HT, RECON, 0, DAG>(a, d0, st, acc);
    load_spinor_h2<1, +1>(a, c, h, d0);
    compute_staged_h2<HT, RECON, 1, DAG>(a, d1, st, acc);
    load_spinor_h2<1, -1>(a, c, h, d1);
    compute_staged_h2<HT, RECON, 2, DAG>(a, d0, st, acc);
    load_spinor_h2<2, +1>(a, c, h, d0);
    compute_staged_h2<HT, RECON, 3, DAG>(a, d1, st, acc);
    load_spinor_h2<2, -1>(a, c, h, d1);
    compute_staged_h2<HT, RECON, 4, DAG>(a, d0, st, acc);
    load_spinor_h2<3, +1>(a, c, h, d0);
    compute_staged_h2<HT, RECON, 5, DAG>(a, d1, st, acc);
    load_spinor_h2<3, -1>(a, c, h, d1);
    compute_staged_h2<HT, RECON, 6, DAG>(a, d0, st, acc);
    compute_staged_h2<HT, RECON, 7, DAG>(a, d1, st, acc);
}

// staged links, and the neighbour spinors three hops in flight: three
// register buffers, each refilled (three hops ahead) as soon as its hop has
// computed
template <typename HT, int RECON, int DAG, int BLOCK>
__device__ __forceinline__ void hops_h2_staged3(const DslashArgs<float> &a, const int c[4],
                                                unsigned h, LinkStage<RECON, BLOCK> &st,
                                                float *acc) {
    stage_link_h2<RECON, 0>(a, c, h, st);
    stage_link_h2<RECON, 1>(a, c, h, st);
    stage_link_h2<RECON, 2>(a, c, h, st);
    stage_link_h2<RECON, 3>(a, c, h, st);
    stage_link_h2<RECON, 4>(a, c, h, st);
    stage_link_h2<RECON, 5>(a, c, h, st);
    stage_link_h2<RECON, 6>(a, c, h, st);
    stage_link_h2<RECON, 7>(a, c, h, st);
    SpinorH2 d0, d1, d2;
    load_spinor_h2<0, +1>(a, c, h, d0);
    load_spinor_h2<0, -1>(a, c, h, d1);
    load_spinor_h2<1, +1>(a, c, h, d2);
    compute_staged_h2<HT, RECON, 0, DAG>(a, d0, st, acc);
    load_spinor_h2<1, -1>(a, c, h, d0);
    compute_staged_h2<HT, RECON, 1, DAG>(a, d1, st, acc);
    load_spinor_h2<2, +1>(a, c, h, d1);
    compute_staged_h2<HT, RECON, 2, DAG>(a, d2, st, acc);
    load_spinor_h2<2, -1>(a, c, h, d2);
    compute_staged_h2<HT, RECON, 3, DAG>(a, d0, st, acc);
    load_spinor_h2<3, +1>(a, c, h, d0);
    compute_staged_h2<HT, RECON, 4, DAG>(a, d1, st, acc);
    load_spinor_h2<3, -1>(a, c, h, d1);
    compute_staged_h2<HT, RECON, 5, DAG>(a, d2, st, acc);
    compute_staged_h2<HT, RECON, 6, DAG>(a, d0, st, acc);
    compute_staged_h2<HT, RECON, 7, DAG>(a, d1, st, acc);
}

template <typename S> constexpr bool packed16() {
    return std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value;
}

// One output site per (thread, i < SPT): site h = block base + i * BLOCK +
// thread, so each of a warp's loads stays one contiguous request.  STAGE
// (16-bit storage, one site per thread): links staged in shared memory, with
// the neighbour spinors two (STAGE 1) or three (STAGE 2) hops in flight.
template <typename S, typename R, int RECON, int DAG, int EPI, int NORM, int BLOCK, int MINB,
          int SPT, int STAGE>
__global__ void __launch_bounds__(BLOCK, MINB) k_dslash(const DslashArgs<R> a) {
    static_assert(!STAGE || (packed16<S>() && SPT == 1), "staging: 16-bit storage, one site");
    df64 nrm[SPT];
#pragma unroll
    for (int i = 0; i < SPT; ++i) nrm[i] = df64(0.0f, 0.0f);
#pragma unroll
    for (int i = 0; i < SPT; ++i) {
        const long h = a.h0 + (long)blockIdx.x * (BLOCK * SPT) + i * BLOCK + threadIdx.x;
        if (h < a.h1) {
            int c[4];
            site_coords(a.g, h, a.parity, c);
            Acc<R> acc[24];
#pragma unroll
            for (int k = 0; k < 24; ++k) acc[k] = 0;
            if constexpr (STAGE == 2) {
                __shared__ LinkStage<RECON, BLOCK> stage;
                hops_h2_staged3<S, RECON, DAG>(a, c, (unsigned)h, stage, acc);
            } else if constexpr (STAGE) {
                __shared__ LinkStage<RECON, BLOCK> stage;
                hops_h2_staged<S, RECON, DAG>(a, c, (unsigned)h, stage, acc);
            } else if constexpr (packed16<S>()) {
                hops_h2_pipelined<S, RECON, DAG>(a, c, (unsigned)h, acc);
            } else {
                hop_pair<S, R, RECON, 0, DAG>(a, c, h, acc);
                hop_pair<S, R, RECON, 1, DAG>(a, c, h, acc);
                hop_pair<S, R, RECON, 2, DAG>(a, c, h, acc);
                hop_pair<S, R, RECON, 3, DAG>(a, c, h, acc);
            }
            // epilogue one 16-byte plane (K reals) of the output record at a
            // time: only one plane's inputs and outputs are live, which keeps
            // the xpay and norm variants within the register cap
            constexpr int K = 16 / (int)sizeof(S);
            R sq = 0, sq1 = 0;   // FP32: even and odd reals in a packed pair
#pragma unroll
            for (int j = 0; j < 24 / K; ++j) {
                R ov[K];
                if (EPI == EPI_XPAY) {
                    R xv[K];
                    const uint4 w = ld_nc_v4((const char *)a.x + ((long)j * a.g.stride + h) * 16);
                    const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
                    Words<S, R>::unpack(ww, xv, K);
                    if (a.twist_on) twist_reals<K>(xv, j * K, a.twist);
                    if constexpr (std::is_same<R, float>::value) {
#pragma unroll
                        for (int t = 0; t < K; t += 2)
                            scale_add_x2(ov[t], ov[t + 1], acc[j * K + t], acc[j * K + t + 1],
                                         a.scale, xv[t], xv[t + 1]);
                    } else {
#pragma unroll
                        for (int t = 0; t < K; ++t) ov[t] = settle(xv[t] + a.scale * acc[j * K + t]);
                    }
                } else {
                    if constexpr (std::is_same<R, float>::value) {
#pragma unroll
                        for (int t = 0; t < K; t += 2)
                            scale_x2(ov[t], ov[t + 1], acc[j * K + t], acc[j * K + t + 1], a.scale);
                    } else {
#pragma unroll
                        for (int t = 0; t < K; ++t) ov[t] = settle(a.scale * acc[j * K + t]);
                    }
                    if (a.twist_on) twist_reals<K>(ov, j * K, -a.twist);
                }
                uint32_t ow[4];
                Words<S, R>::pack(ov, ow, K);
                st_v4((char *)a.out + ((long)j * a.g.stride + h) * 16,
                      make_uint4(ow[0], ow[1], ow[2], ow[3]));
                if (NORM) {
                    if constexpr (std::is_same<R, float>::value) {
#pragma unroll
                        for (int t = 0; t < K; t += 2) sq_acc_x2(sq, sq1, ov[t], ov[t + 1]);
                    } else {
#pragma unroll
                        for (int t = 0; t < K; ++t) sq += ov[t] * ov[t];
                    }
                }
            }
            if (NORM) {
                if constexpr (std::is_same<R, float>::value) nrm[i] = to_df(sq + sq1);
                else nrm[i] = to_df(sq);
            }
        }
    }
    if (NORM) warp_partials<BLOCK, SPT>(nrm, a.g.vh, a.red.partials);
}

// Launch configurations the tuner chooses from: threads per block, the
// minimum resident blocks per SM handed to the register allocator, output
// sites per thread, and (16-bit storage only) links staged in shared memory
// with the neighbour spinors two (stage 1) or three (stage 2) hops ahead.
// A fused norm adds in the same order under every configuration
// (warp_partials), so every variant can take its own tuned one.
struct DslashCfg { int block, minb, spt, stage; };
constexpr int N_DSLASH_CFG = 8;
constexpr DslashCfg DSLASH_CFGS[N_DSLASH_CFG] = {
    {128, 1, 1, 0}, {128, 8, 1, 0}, {128, 6, 1, 0}, {256, 4, 1, 0},
    {128, 1, 2, 0}, {128, 5, 1, 2}, {128, 6, 1, 1}, {128, 6, 1, 2}};
// whether candidate k is distinct for storage precision prec (staging
// applies to 16-bit storage only; elsewhere it repeats an unstaged entry)
inline bool dslash_cfg_applies(int k, int prec) {
    return !DSLASH_CFGS[k].stage || prec == WD_F16 || prec == WD_BF16;
}
// The double-float hopping term (one site per thread, a loop over the hops)
// has its own table: its register appetite makes the minimum resident blocks,
// i.e. the register cap, the parameter that matters; stage = 1 copies each
// hop's link into shared memory one hop ahead (36 KB per 128-thread block).
constexpr int N_DSLASH_DF_CFG = 8;
constexpr DslashCfg DSLASH_DF_CFGS[N_DSLASH_DF_CFG] = {
    {128, 3, 1, 0}, {128, 1, 1, 0}, {128, 2, 1, 0}, {128, 4, 1, 0},
    {256, 2, 1, 0}, {128, 3, 1, 1}, {128, 4, 1, 1}, {128, 2, 1, 1}};

template <typename S, typename R, int RECON, int DAG, int EPI, int NORM, int CFG>
void launch_cfg(const DslashArgs<R> &a, cudaStream_t s) {
    constexpr DslashCfg C = DSLASH_CFGS[CFG];
    constexpr int STAGE = packed16<S>() ? C.stage : 0;
    const long per_block = (long)C.block * C.spt;
    const unsigned grid = (unsigned)((a.h1 - a.h0 + per_block - 1) / per_block);
    k_dslash<S, R, RECON, DAG, EPI, NORM, C.block, C.minb, C.spt, STAGE><<<grid, C.block, 0, s>>>(a);
}

template <typename S, typename R, int RECON, int DAG, int EPI, int NORM>
void launch_any_cfg(int cfg, const DslashArgs<R> &a, cudaStream_t s) {
    switch (cfg) {
    case 1: launch_cfg<S, R, RECON, DAG, EPI, NORM, 1>(a, s); break;
    case 2: launch_cfg<S, R, RECON, DAG, EPI, NORM, 2>(a, s); break;
    case 3: launch_cfg<S, R, RECON, DAG, EPI, NORM, 3>(a, s); break;
    case 4: launch_cfg<S, R, RECON, DAG, EPI, NORM, 4>(a, s); break;
    case 5: launch_cfg<S, R, RECON, DAG, EPI, NORM, 5>(a, s); break;
    case 6: launch_cfg<S, R, RECON, DAG, EPI, NORM, 6>(a, s); break;
    case 7: launch_cfg<S, R, RECON, DAG, EPI, NORM, 7>(a, s); break;
    default: launch_cfg<S, R, RECON, DAG, EPI, NORM, 0>(a, s); break;
    }
}

template <typename S, typename R, int RECON>
cudaError_t launch_dslash_t(const DslashLaunch &L, cudaStream_t s) {
    DslashArgs<R> a;
    a.g = L.g;
    const int q = 1 - L.out_parity;
    a.gauge_out = (const char *)L.gauge->ptr[L.out_parity];
    a.gauge_in = (const char *)L.gauge->ptr[q];
    a.dir_bytes = L.gauge->dir_bytes;
    a.out = L.out;
    a.in = L.in;
    a.x = L.x;
    a.scale = (R)L.scale;
    for (int i = 0; i < 8; ++i) a.ph[i] = (R)L.phase[i];
    a.phase_on = phase_mask(L.phase);
    a.parity = L.out_parity;
    if (L.red) a.red = *L.red;
    else a.red = Reduction{nullptr, nullptr, nullptr, FIN_NONE};
    a.twist = (R)L.twist;
    a.twist_on = L.twist != 0.0;
    a.h0 = L.h_begin;
    a.h1 = L.h_end < 0 ? L.g.vh : L.h_end;
    if (a.h0 < 0 || a.h1 > L.g.vh || a.h0 > a.h1) return cudaErrorInvalidValue;
    if (a.h1 == a.h0) return cudaSuccess;
    const int cfg = L.cfg;
    if (L.red) {   // the per-warp partials assume a launch over every site
        if (a.h0 != 0 || a.h1 != L.g.vh) return cudaErrorInvalidValue;
    }
    if (L.red) {   // fused norm (after an xpay epilogue), then the fixed-order finish
        if (L.dagger) launch_any_cfg<S, R, RECON, 1, EPI_XPAY, 1>(cfg, a, s);
        else launch_any_cfg<S, R, RECON, 0, EPI_XPAY, 1>(cfg, a, s);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return launch_finish_partials(*L.red, (L.g.vh + 31) / 32, s);
    } else if (L.epi == EPI_PLAIN) {
        if (L.dagger) launch_any_cfg<S, R, RECON, 1, EPI_PLAIN, 0>(cfg, a, s);
        else launch_any_cfg<S, R, RECON, 0, EPI_PLAIN, 0>(cfg, a, s);
    } else {
        if (L.dagger) launch_any_cfg<S, R, RECON, 1, EPI_XPAY, 0>(cfg, a, s);
        else launch_any_cfg<S, R, RECON, 0, EPI_XPAY, 0>(cfg, a, s);
    }
    return cudaGetLastError();
}

}  // namespace wd
