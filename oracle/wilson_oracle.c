/*
 * Wilson-Dirac oracle: plain, slow, FP64 CPU implementation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or helper with the
 * CUDA library: its own gamma tables, its own site indexing, its own solver.
 *
 * What it computes (Barthou et al., "Automated Code Generation for Lattice
 * QCD and beyond", arXiv:1401.2039):
 *
 *   D = I - kappa * H                         (Fig. "dirac", with mu = 0;
 *                                              the twisted mass mu != 0 is
 *                                              in the *_tm functions below)
 *   (H psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x)       phi_mu(x)  psi(x+mu)
 *                        + (1 + gamma_mu) U_mu(x-mu)^dag phi_mu*(x) psi(x-mu) ]
 *
 *   phi_mu is a complex boundary phase that multiplies a hop that wraps
 *   around the lattice in direction mu (conjugated on the backward hop);
 *   Fig. "id" states isPeriodic(L) = true, the phases generalise it.
 *   The hop orientation is the gauge-covariant reading of Fig. "dirac":
 *   U[s x d]^dag = U[(s+d) x -d] (Fig. "id") makes U_mu(x-mu)^dag the link
 *   of the backward hop.
 *
 *   The spin-colour action of one hop uses the identity of Sec. 4.2,
 *   (M1 (x) M2) V = M1 V M2^t with V the 3x4 colour-by-spin matrix of a site.
 *
 *   Even-odd Schur complement (Alg. "schur"): with P_e, P_o the parity
 *   projections, D11 = P_e D P_e^t = I (mu = 0), D22 = P_o D P_o^t = I,
 *   D21 = P_o D P_e^t = -kappa P_o H P_e^t, D12 = P_e D P_o^t = -kappa P_e H P_o^t,
 *   the Schur operator on parity p is
 *   Mhat_p = D_pp - D_pq D_qq^-1 D_qp = I - kappa^2 P_p H P_q^t P_q H P_p^t.
 *
 *   CGNR (Alg. "CGNR") solves A x = b through A^dag A x = A^dag b keeping the
 *   residual r = b - A x of the original system.
 *
 * Layout of every array (the canonical layout of the library boundary):
 *   site index  lex = ((t*Lz + z)*Ly + y)*Lx + x
 *   spinor      psi[lex][colour 3][spin 4]  complex double (re, im)
 *   gauge links U[lex][mu 4][row 3][col 3]    complex double, mu = x,y,z,t
 *   half-lattice vectors of parity p: entry lex/2 for every site with
 *   (x+y+z+t) % 2 == p (Lx even).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* ---------------------------------------------------------------------- */
/* Gamma matrices, DeGrand-Rossi basis (the paper only fixes their algebra
 * in Fig. "id": hermitian, gamma5^2 = 1, gamma5 anticommutes with gamma_d,
 * gamma5 diagonal).                                                        */
static void gamma_matrix(int mu, cplx g[4][4]) {
    memset(g, 0, 16 * sizeof(cplx));
    switch (mu) {
    case 0: /* gamma_x */
        g[0][3] = I;  g[1][2] = I;  g[2][1] = -I; g[3][0] = -I; break;
    case 1: /* gamma_y */
        g[0][3] = -1; g[1][2] = 1;  g[2][1] = 1;  g[3][0] = -1; break;
    case 2: /* gamma_z */
        g[0][2] = I;  g[1][3] = -I; g[2][0] = -I; g[3][1] = I;  break;
    case 3: /* gamma_t */
        g[0][2] = 1;  g[1][3] = 1;  g[2][0] = 1;  g[3][1] = 1;  break;
    default: { /* gamma_5 = gamma_x gamma_y gamma_z gamma_t */
        cplx a[4][4], b[4][4], c[4][4];
        gamma_matrix(0, a);
        for (int k = 1; k < 4; ++k) {
            gamma_matrix(k, b);
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) {
                    cplx s = 0;
                    for (int l = 0; l < 4; ++l) s += a[i][l] * b[l][j];
                    c[i][j] = s;
                }
            memcpy(a, c, sizeof(a));
        }
        memcpy(g, a, 16 * sizeof(cplx));
    }
    }
}

/* Exported so the tests can check the basis against the Clifford algebra. */
void oracle_gamma(int mu, double *out /* 4x4 complex, row-major, re/im */) {
    cplx g[4][4];
    gamma_matrix(mu, g);
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            out[2 * (4 * i + j)] = creal(g[i][j]);
            out[2 * (4 * i + j) + 1] = cimag(g[i][j]);
        }
}

/* ---------------------------------------------------------------------- */
/* Lattice geometry                                                        */
typedef struct { int L[4]; long vol; } geom;

static geom make_geom(const int *dims) {
    geom g;
    g.vol = 1;
    for (int m = 0; m < 4; ++m) { g.L[m] = dims[m]; g.vol *= dims[m]; }
    return g;
}

static void lex_to_coord(const geom *g, long lex, int c[4]) {
    for (int m = 0; m < 4; ++m) { c[m] = (int)(lex % g->L[m]); lex /= g->L[m]; }
}

static long coord_to_lex(const geom *g, const int c[4]) {
    return ((long)(c[3] * g->L[2] + c[2]) * g->L[1] + c[1]) * g->L[0] + c[0];
}

static int parity_of(const int c[4]) { return (c[0] + c[1] + c[2] + c[3]) & 1; }

/* ---------------------------------------------------------------------- */
/* Hopping term at one site: acc = (H in)(site) (or (H^dag in)(site)).     */
/* H^dag swaps the projectors: (1 - gamma) <-> (1 + gamma) (gamma hermitian,
 * the adjoint of a forward hop is a backward hop with the adjoint link).   */
static void hop_site(const geom *g, long site, cplx acc[3][4], const cplx *in, const cplx *U,
                     const double *phase, int dagger) {
    cplx proj_fwd[4][4][4], proj_bwd[4][4][4]; /* [mu][s][s'] */
    for (int mu = 0; mu < 4; ++mu) {
        cplx gm[4][4];
        gamma_matrix(mu, gm);
        double sf = dagger ? +1.0 : -1.0; /* forward hop: 1 - gamma (1 + gamma if dagger) */
        for (int s = 0; s < 4; ++s)
            for (int t = 0; t < 4; ++t) {
                cplx id = (s == t) ? 1.0 : 0.0;
                proj_fwd[mu][s][t] = id + sf * gm[s][t];
                proj_bwd[mu][s][t] = id - sf * gm[s][t];
            }
    }
    int c[4];
    lex_to_coord(g, site, c);
    memset(acc, 0, 12 * sizeof(cplx));
    for (int mu = 0; mu < 4; ++mu) {
        cplx ph = phase[2 * mu] + I * phase[2 * mu + 1];
        /* forward neighbour x + mu */
        int cf[4] = {c[0], c[1], c[2], c[3]};
        cplx wf = 1.0;
        cf[mu] += 1;
        if (cf[mu] == g->L[mu]) { cf[mu] = 0; wf = ph; }
        /* backward neighbour x - mu */
        int cb[4] = {c[0], c[1], c[2], c[3]};
        cplx wb = 1.0;
        cb[mu] -= 1;
        if (cb[mu] < 0) { cb[mu] = g->L[mu] - 1; wb = conj(ph); }
        long lf = coord_to_lex(g, cf), lb = coord_to_lex(g, cb);
        const cplx *Uf = U + (site * 4 + mu) * 9; /* U_mu(x)      */
        const cplx *Ub = U + (lb * 4 + mu) * 9;   /* U_mu(x - mu) */
        const cplx *pf = in + lf * 12, *pb = in + lb * 12;
        /* (U (x) P) V = U . V . P^t, V = 3x4 colour-by-spin matrix */
        for (int a = 0; a < 3; ++a)
            for (int s = 0; s < 4; ++s) {
                cplx sum = 0;
                for (int b = 0; b < 3; ++b)
                    for (int t = 0; t < 4; ++t) {
                        sum += wf * Uf[3 * a + b] * proj_fwd[mu][s][t] * pf[4 * b + t];
                        sum += wb * conj(Ub[3 * b + a]) * proj_bwd[mu][s][t] * pb[4 * b + t];
                    }
                acc[a][s] += sum;
            }
    }
}

/* Hopping term, full lattice: out = H in (dagger = 0) or H^dag in.        */
void oracle_hop(double *out_, const double *in_, const double *U_,
                const int *dims, const double *phase, int dagger) {
    geom g = make_geom(dims);
#pragma omp parallel for schedule(static)
    for (long site = 0; site < g.vol; ++site) {
        cplx acc[3][4];
        hop_site(&g, site, acc, (const cplx *)in_, (const cplx *)U_, phase, dagger);
        memcpy((cplx *)out_ + site * 12, acc, sizeof(acc));
    }
}

/* The same at the n listed lex sites only: out[k] = (H in)(sites[k]).      */
void oracle_hop_sites(double *out_, const double *in_, const double *U_, const int *dims,
                      const double *phase, int dagger, const long *sites, long n) {
    geom g = make_geom(dims);
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; ++k) {
        cplx acc[3][4];
        hop_site(&g, sites[k], acc, (const cplx *)in_, (const cplx *)U_, phase, dagger);
        memcpy((cplx *)out_ + k * 12, acc, sizeof(acc));
    }
}

/* D in = in - kappa * H in (dagger: in - kappa * H^dag in). */
void oracle_apply(double *out_, const double *in_, const double *U,
                  const int *dims, double kappa, const double *phase, int dagger) {
    geom g = make_geom(dims);
    cplx *out = (cplx *)out_;
    const cplx *in = (const cplx *)in_;
    cplx *h = (cplx *)malloc(sizeof(cplx) * 12 * g.vol);
    oracle_hop((double *)h, in_, U, dims, phase, dagger);
    for (long i = 0; i < 12 * g.vol; ++i) out[i] = in[i] - kappa * h[i];
    free(h);
}

/* ---------------------------------------------------------------------- */
/* Parity projections P_p (half -> full embedding is P_p^t).               */
static void embed_half(const geom *g, cplx *full, const cplx *half, int p) {
    memset(full, 0, sizeof(cplx) * 12 * g->vol);
    for (long site = 0; site < g->vol; ++site) {
        int c[4];
        lex_to_coord(g, site, c);
        if (parity_of(c) == p) memcpy(full + site * 12, half + (site / 2) * 12, 12 * sizeof(cplx));
    }
}

static void project_half(const geom *g, cplx *half, const cplx *full, int p) {
    for (long site = 0; site < g->vol; ++site) {
        int c[4];
        lex_to_coord(g, site, c);
        if (parity_of(c) == p) memcpy(half + (site / 2) * 12, full + site * 12, 12 * sizeof(cplx));
    }
}

/* Schur operator on parity p:
 *   Mhat_p = I - kappa^2 P_p H P_q^t P_q H P_p^t,   q = 1 - p
 * (D11 = D22 = I for mu = 0).  dagger applies Mhat_p^dag, which is the same
 * expression with H^dag.                                                  */
void oracle_apply_eo(double *out_, const double *in_, const double *U,
                     const int *dims, double kappa, const double *phase,
                     int parity, int dagger) {
    geom g = make_geom(dims);
    long vh = g.vol / 2;
    int q = 1 - parity;
    cplx *a = (cplx *)malloc(sizeof(cplx) * 12 * g.vol);
    cplx *b = (cplx *)malloc(sizeof(cplx) * 12 * g.vol);
    cplx *t = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    embed_half(&g, a, (const cplx *)in_, parity);          /* P_p^t x        */
    oracle_hop((double *)b, (double *)a, U, dims, phase, dagger);
    project_half(&g, t, b, q);                              /* P_q H P_p^t x  */
    embed_half(&g, a, t, q);
    oracle_hop((double *)b, (double *)a, U, dims, phase, dagger);
    project_half(&g, t, b, parity);                         /* P_p H P_q^t .. */
    const cplx *in = (const cplx *)in_;
    cplx *out = (cplx *)out_;
    for (long i = 0; i < 12 * vh; ++i) out[i] = in[i] - kappa * kappa * t[i];
    free(a); free(b); free(t);
}

/* Hopping term restricted to one output parity: out_half = P_p H P_q^t in_half. */
void oracle_hop_eo(double *out_, const double *in_, const double *U,
                   const int *dims, const double *phase, int out_parity, int dagger) {
    geom g = make_geom(dims);
    cplx *a = (cplx *)malloc(sizeof(cplx) * 12 * g.vol);
    cplx *b = (cplx *)malloc(sizeof(cplx) * 12 * g.vol);
    embed_half(&g, a, (const cplx *)in_, 1 - out_parity);
    oracle_hop((double *)b, (double *)a, U, dims, phase, dagger);
    project_half(&g, (cplx *)out_, b, out_parity);
    free(a); free(b);
}

/* ---------------------------------------------------------------------- */
/* Alg. "schur", right-hand side on the solved parity p (q the other):
 *   bhat_p = b_p - D_pq D_qq^-1 b_q = b_p + kappa P_p H P_q^t b_q
 * and reconstruction of the other parity:
 *   x_q = D_qq^-1 (b_q - D_qp x_p) = b_q + kappa P_q H P_p^t x_p.
 * The algorithm's later re-assignment v1 = P_e(2 kappa b) is read as
 * v1 = P_e b: with D11 = I the factor 2 kappa would not give D x = b.     */
void oracle_schur_prepare(double *bhat_, const double *b_full, const double *U,
                          const int *dims, double kappa, const double *phase, int parity) {
    geom g = make_geom(dims);
    long vh = g.vol / 2;
    int q = 1 - parity;
    cplx *bq = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    cplx *bp = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    cplx *hb = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    project_half(&g, bq, (const cplx *)b_full, q);
    project_half(&g, bp, (const cplx *)b_full, parity);
    oracle_hop_eo((double *)hb, (double *)bq, U, dims, phase, parity, 0);
    cplx *bhat = (cplx *)bhat_;
    for (long i = 0; i < 12 * vh; ++i) bhat[i] = bp[i] + kappa * hb[i];
    free(bq); free(bp); free(hb);
}

void oracle_schur_reconstruct(double *x_full, const double *x_p, const double *b_full,
                              const double *U, const int *dims, double kappa,
                              const double *phase, int parity) {
    geom g = make_geom(dims);
    long vh = g.vol / 2;
    int q = 1 - parity;
    cplx *bq = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    cplx *hx = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    cplx *xq = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    project_half(&g, bq, (const cplx *)b_full, q);
    oracle_hop_eo((double *)hx, x_p, U, dims, phase, q, 0);
    for (long i = 0; i < 12 * vh; ++i) xq[i] = bq[i] + kappa * hx[i];
    cplx *x = (cplx *)x_full;
    cplx *a = (cplx *)malloc(sizeof(cplx) * 12 * g.vol);
    embed_half(&g, x, (const cplx *)x_p, parity);   /* P_p^t x_p */
    embed_half(&g, a, xq, q);                        /* P_q^t x_q */
    for (long i = 0; i < 12 * g.vol; ++i) x[i] += a[i];
    free(bq); free(hx); free(xq); free(a);
}

/* ---------------------------------------------------------------------- */
/* Inner product (a|b) = sum conj(a) b; the norms the solver needs are real. */
static double norm2(const cplx *a, long n) {
    double s = 0;
    for (long i = 0; i < n; ++i) s += creal(conj(a[i]) * a[i]);
    return s;
}

/* Alg. "CGNR" with A = Mhat_p on half-lattice vectors.
 * Stops when ||r|| <= tol * ||b|| (the algorithm's n_r > epsilon test with
 * epsilon = tol^2 ||b||^2) or after maxiter iterations.
 * resid (optional, length maxiter + 1) receives ||r_k|| for k = 0..iters.
 * Returns 0 when converged, 1 when maxiter was reached.                   */
int oracle_cgnr(double *x_, const double *b_, const double *U, const int *dims,
                double kappa, const double *phase, int parity, double tol,
                int maxiter, int *iters_out, double *resid) {
    geom g = make_geom(dims);
    long n = 12 * (g.vol / 2);
    cplx *x = (cplx *)x_;
    const cplx *b = (const cplx *)b_;
    cplx *r = (cplx *)malloc(sizeof(cplx) * n);
    cplx *z = (cplx *)malloc(sizeof(cplx) * n);
    cplx *p = (cplx *)malloc(sizeof(cplx) * n);
    cplx *Ap = (cplx *)malloc(sizeof(cplx) * n);

    memcpy(r, b, sizeof(cplx) * n);                                         /* r = b       */
    oracle_apply_eo((double *)z, (double *)r, U, dims, kappa, phase, parity, 1); /* z = A^dag r */
    memcpy(p, z, sizeof(cplx) * n);                                         /* p = z       */
    memset(x, 0, sizeof(cplx) * n);                                         /* x = 0       */
    double nz = norm2(z, n);
    double nr = norm2(r, n);
    double eps = tol * tol * norm2(b, n);
    int k = 0;
    if (resid) resid[0] = sqrt(nr);
    while (nr > eps && k < maxiter) {
        oracle_apply_eo((double *)Ap, (double *)p, U, dims, kappa, phase, parity, 0);
        double alpha = nz / norm2(Ap, n);
        for (long i = 0; i < n; ++i) x[i] += alpha * p[i];
        for (long i = 0; i < n; ++i) r[i] -= alpha * Ap[i];
        oracle_apply_eo((double *)z, (double *)r, U, dims, kappa, phase, parity, 1);
        double nz1 = norm2(z, n);
        double beta = nz1 / nz;
        for (long i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        nz = nz1;
        nr = norm2(r, n);
        ++k;
        if (resid) resid[k] = sqrt(nr);
    }
    if (iters_out) *iters_out = k;
    free(r); free(z); free(p); free(Ap);
    return nr > eps ? 1 : 0;
}

/* The goal xx = Dirac^-1 bb with templates "CGNR schur": Schur reduction to
 * parity p, CGNR on Mhat_p, reconstruction of the other parity.
 * tol is relative to ||b|| of the full right-hand side; because the
 * reconstructed parity has zero residual, the full residual equals the
 * Schur residual.                                                          */
int oracle_solve(double *x_full, const double *b_full, const double *U, const int *dims,
                 double kappa, const double *phase, int parity, double tol,
                 int maxiter, int *iters_out) {
    geom g = make_geom(dims);
    long vh = g.vol / 2;
    cplx *bhat = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    cplx *xp = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    oracle_schur_prepare((double *)bhat, b_full, U, dims, kappa, phase, parity);
    double nb = sqrt(norm2((const cplx *)b_full, 12 * g.vol));
    double nbh = sqrt(norm2(bhat, 12 * vh));
    double rel = nbh > 0 ? tol * nb / nbh : tol;
    int rc = oracle_cgnr((double *)xp, (double *)bhat, U, dims, kappa, phase, parity,
                         rel, maxiter, iters_out, NULL);
    oracle_schur_reconstruct(x_full, (double *)xp, b_full, U, dims, kappa, phase, parity);
    free(bhat); free(xp);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Twisted mass (Fig. "dirac" with mu != 0):
 *   D = I + 2 i kappa mu (I_L (x) I_C (x) gamma_5) - kappa H.
 * The diagonal blocks D_ee = D_oo = A := I + 2 i kappa mu gamma_5 act on the
 * spin index of each site alone.  Fig. "id" states that gamma_5 is diagonal,
 * so A is diagonal and A^-1 has the reciprocal diagonal entries; this code
 * checks the diagonality of its own gamma_5 (the product of the four gamma
 * matrices) instead of assuming a basis.  Because gamma_5 is hermitian,
 * D^dag = I - 2 i kappa mu gamma_5 - kappa H^dag: the adjoint flips mu.
 *
 * out = A in (inverse = 0) or A^-1 in (inverse = 1) on n sites.
 * Returns 0, or -1 if gamma_5 is not diagonal.                            */
int oracle_twist(double *out_, const double *in_, long n, double kappa, double mu, int inverse) {
    cplx g5[4][4];
    gamma_matrix(4, g5);
    cplx d[4];
    for (int s = 0; s < 4; ++s) {
        for (int t = 0; t < 4; ++t)
            if (t != s && cabs(g5[s][t]) != 0.0) return -1;
        const cplx a = 1.0 + 2.0 * I * kappa * mu * g5[s][s];   /* A_ss */
        d[s] = inverse ? 1.0 / a : a;
    }
    cplx *out = (cplx *)out_;
    const cplx *in = (const cplx *)in_;
    for (long site = 0; site < n; ++site)
        for (int c = 0; c < 3; ++c)
            for (int s = 0; s < 4; ++s)
                out[site * 12 + 4 * c + s] = d[s] * in[site * 12 + 4 * c + s];
    return 0;
}

/* out = D in with the twisted mass (dagger: D^dag in = A(-mu) in - kappa H^dag in). */
void oracle_apply_tm(double *out_, const double *in_, const double *U, const int *dims,
                     double kappa, double mu, const double *phase, int dagger) {
    geom g = make_geom(dims);
    cplx *out = (cplx *)out_;
    cplx *h = (cplx *)malloc(sizeof(cplx) * 12 * g.vol);
    cplx *a = (cplx *)malloc(sizeof(cplx) * 12 * g.vol);
    oracle_hop((double *)h, in_, U, dims, phase, dagger);
    oracle_twist((double *)a, in_, g.vol, kappa, dagger ? -mu : mu, 0);
    for (long i = 0; i < 12 * g.vol; ++i) out[i] = a[i] - kappa * h[i];
    free(h); free(a);
}

/* Schur operator with the twisted mass on parity p (q = 1 - p):
 *   Mhat_p = D_pp - D_pq D_qq^-1 D_qp = A - kappa^2 P_p H P_q^t A^-1 P_q H P_p^t
 * dagger: the same with H^dag and -mu.                                    */
void oracle_apply_eo_tm(double *out_, const double *in_, const double *U, const int *dims,
                        double kappa, double mu, const double *phase, int parity, int dagger) {
    geom g = make_geom(dims);
    long vh = g.vol / 2;
    int q = 1 - parity;
    double m = dagger ? -mu : mu;
    cplx *t = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    cplx *ti = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    cplx *u = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    cplx *ax = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    oracle_hop_eo((double *)t, in_, U, dims, phase, q, dagger);       /* D_qp-part: H_qp x */
    oracle_twist((double *)ti, (double *)t, vh, kappa, m, 1);         /* A^-1 H_qp x       */
    oracle_hop_eo((double *)u, (double *)ti, U, dims, phase, parity, dagger);
    oracle_twist((double *)ax, in_, vh, kappa, m, 0);                 /* A x               */
    cplx *out = (cplx *)out_;
    for (long i = 0; i < 12 * vh; ++i) out[i] = ax[i] - kappa * kappa * u[i];
    free(t); free(ti); free(u); free(ax);
}

/* Alg. "schur" with the twisted mass:
 *   bhat_p = b_p - D_pq D_qq^-1 b_q = b_p + kappa P_p H P_q^t A^-1 b_q
 *   x_q = D_qq^-1 (b_q - D_qp x_p) = A^-1 (b_q + kappa P_q H P_p^t x_p).    */
void oracle_schur_prepare_tm(double *bhat_, const double *b_full, const double *U,
                             const int *dims, double kappa, double mu, const double *phase,
                             int parity) {
    geom g = make_geom(dims);
    long vh = g.vol / 2;
    int q = 1 - parity;
    cplx *bq = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    cplx *bqi = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    cplx *bp = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    cplx *hb = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    project_half(&g, bq, (const cplx *)b_full, q);
    project_half(&g, bp, (const cplx *)b_full, parity);
    oracle_twist((double *)bqi, (double *)bq, vh, kappa, mu, 1);
    oracle_hop_eo((double *)hb, (double *)bqi, U, dims, phase, parity, 0);
    cplx *bhat = (cplx *)bhat_;
    for (long i = 0; i < 12 * vh; ++i) bhat[i] = bp[i] + kappa * hb[i];
    free(bq); free(bqi); free(bp); free(hb);
}

void oracle_schur_reconstruct_tm(double *x_full, const double *x_p, const double *b_full,
                                 const double *U, const int *dims, double kappa, double mu,
                                 const double *phase, int parity) {
    geom g = make_geom(dims);
    long vh = g.vol / 2;
    int q = 1 - parity;
    cplx *bq = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    cplx *hx = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    cplx *v = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    cplx *xq = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    project_half(&g, bq, (const cplx *)b_full, q);
    oracle_hop_eo((double *)hx, x_p, U, dims, phase, q, 0);
    for (long i = 0; i < 12 * vh; ++i) v[i] = bq[i] + kappa * hx[i];
    oracle_twist((double *)xq, (double *)v, vh, kappa, mu, 1);
    cplx *x = (cplx *)x_full;
    cplx *a = (cplx *)malloc(sizeof(cplx) * 12 * g.vol);
    embed_half(&g, x, (const cplx *)x_p, parity);
    embed_half(&g, a, xq, q);
    for (long i = 0; i < 12 * g.vol; ++i) x[i] += a[i];
    free(bq); free(hx); free(v); free(xq); free(a);
}

/* Alg. "CGNR" on the twisted-mass Schur operator (the same loop as
 * oracle_cgnr, with Mhat_p of oracle_apply_eo_tm).                          */
int oracle_cgnr_tm(double *x_, const double *b_, const double *U, const int *dims,
                   double kappa, double mu, const double *phase, int parity, double tol,
                   int maxiter, int *iters_out, double *resid) {
    geom g = make_geom(dims);
    long n = 12 * (g.vol / 2);
    cplx *x = (cplx *)x_;
    const cplx *b = (const cplx *)b_;
    cplx *r = (cplx *)malloc(sizeof(cplx) * n);
    cplx *z = (cplx *)malloc(sizeof(cplx) * n);
    cplx *p = (cplx *)malloc(sizeof(cplx) * n);
    cplx *Ap = (cplx *)malloc(sizeof(cplx) * n);
    memcpy(r, b, sizeof(cplx) * n);
    oracle_apply_eo_tm((double *)z, (double *)r, U, dims, kappa, mu, phase, parity, 1);
    memcpy(p, z, sizeof(cplx) * n);
    memset(x, 0, sizeof(cplx) * n);
    double nz = norm2(z, n);
    double nr = norm2(r, n);
    double eps = tol * tol * norm2(b, n);
    int k = 0;
    if (resid) resid[0] = sqrt(nr);
    while (nr > eps && k < maxiter) {
        oracle_apply_eo_tm((double *)Ap, (double *)p, U, dims, kappa, mu, phase, parity, 0);
        double alpha = nz / norm2(Ap, n);
        for (long i = 0; i < n; ++i) x[i] += alpha * p[i];
        for (long i = 0; i < n; ++i) r[i] -= alpha * Ap[i];
        oracle_apply_eo_tm((double *)z, (double *)r, U, dims, kappa, mu, phase, parity, 1);
        double nz1 = norm2(z, n);
        for (long i = 0; i < n; ++i) p[i] = z[i] + (nz1 / nz) * p[i];
        nz = nz1;
        nr = norm2(r, n);
        ++k;
        if (resid) resid[k] = sqrt(nr);
    }
    if (iters_out) *iters_out = k;
    free(r); free(z); free(p); free(Ap);
    return nr > eps ? 1 : 0;
}

int oracle_solve_tm(double *x_full, const double *b_full, const double *U, const int *dims,
                    double kappa, double mu, const double *phase, int parity, double tol,
                    int maxiter, int *iters_out) {
    geom g = make_geom(dims);
    long vh = g.vol / 2;
    cplx *bhat = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    cplx *xp = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    oracle_schur_prepare_tm((double *)bhat, b_full, U, dims, kappa, mu, phase, parity);
    double nb = sqrt(norm2((const cplx *)b_full, 12 * g.vol));
    double nbh = sqrt(norm2(bhat, 12 * vh));
    double rel = nbh > 0 ? tol * nb / nbh : tol;
    int rc = oracle_cgnr_tm((double *)xp, (double *)bhat, U, dims, kappa, mu, phase, parity,
                            rel, maxiter, iters_out, NULL);
    oracle_schur_reconstruct_tm(x_full, (double *)xp, b_full, U, dims, kappa, mu, phase, parity);
    free(bhat); free(xp);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* Conjugate-residual solvers on the Schur system.  Sec. 5 (Fig. "algosxp")
 * compares CRNE, MCR1 and MCR2 with CGNR, all on the Schur-reduced system,
 * without defining them; these are the textbook readings.
 *
 * CR (Saad, "Iterative Methods for Sparse Linear Systems", 2nd ed., Alg.
 * 6.20) solves B y = c for a Hermitian B and minimises ||c - B y|| over the
 * Krylov space K_k(B, c):
 *   r = c, p = r, Bp = B p
 *   alpha = (r|B r) / (Bp|Bp),  y += alpha p,  r -= alpha Bp
 *   beta = (r'|B r') / (r|B r),  p = r' + beta p,  Bp = B r' + beta Bp
 *
 *   CRNE (method 1): B = A A^dag (Hermitian positive definite), c = b, and
 *                    x = A^dag y at the end.
 *   MCR1 (method 2): B = gamma_5 A, c = gamma_5 b.  gamma_5 A is Hermitian
 *                    because A^dag = gamma_5 A gamma_5 (Fig. "id"), and
 *                    indefinite.  Bp is formed by an application of B every
 *                    iteration.  With a twisted mass gamma_5 A(mu) gamma_5 =
 *                    A(-mu)^dag, so MCR is defined for mu = 0 only.
 *   MCR2 (method 3): as MCR1, with Bp from the recurrence above: one
 *                    application of A per iteration instead of two.
 * A = Mhat_p with the twisted mass (mu = 0: the Wilson operator).  The CR
 * residual r = c - B y has the norm of the Schur residual b - A x in every
 * case (gamma_5 is unitary).  (r|B r) is real for a Hermitian B; its
 * rounding-level imaginary part is dropped.
 */
typedef struct {
    const double *U, *phase;
    const int *dims;
    double kappa, mu;
    int parity, method;
    long n;
    cplx *tmp;
    double g5[4];
} cr_ctx;

static void cr_gamma5(const cr_ctx *c, cplx *v) {
    for (long i = 0; i < c->n; ++i) v[i] *= c->g5[i % 4];
}

/* out = B in */
static void cr_apply_B(const cr_ctx *c, cplx *out, const cplx *in) {
    if (c->method == 1) {
        oracle_apply_eo_tm((double *)c->tmp, (const double *)in, c->U, c->dims, c->kappa, c->mu,
                           c->phase, c->parity, 1);
        oracle_apply_eo_tm((double *)out, (const double *)c->tmp, c->U, c->dims, c->kappa, c->mu,
                           c->phase, c->parity, 0);
    } else {
        oracle_apply_eo_tm((double *)out, (const double *)in, c->U, c->dims, c->kappa, c->mu,
                           c->phase, c->parity, 0);
        cr_gamma5(c, out);
    }
}

static cplx dot(const cplx *a, const cplx *b, long n) {
    cplx s = 0;
    for (long i = 0; i < n; ++i) s += conj(a[i]) * b[i];
    return s;
}

/* The CR loop above with A = Mhat_p, on half-lattice vectors.
 * Stops when ||r|| <= tol * ||b|| or after maxiter iterations; resid
 * (optional, length maxiter + 1) receives ||r_k||.  Returns 0 when
 * converged, 1 at maxiter, 2 on a breakdown ((r|B r) or (Bp|Bp) zero),
 * -1 for an unknown method, MCR with mu != 0 or a non-diagonal gamma_5.   */
int oracle_cr(double *x_, const double *b_, const double *U, const int *dims, double kappa,
              double mu, const double *phase, int parity, int method, double tol, int maxiter,
              int *iters_out, double *resid) {
    if (method < 1 || method > 3 || (method != 1 && mu != 0.0)) return -1;
    geom g = make_geom(dims);
    cr_ctx c = {U, phase, dims, kappa, mu, parity, method, 12 * (g.vol / 2), NULL, {0}};
    cplx g5m[4][4];
    gamma_matrix(4, g5m);
    for (int s = 0; s < 4; ++s) {
        for (int t = 0; t < 4; ++t)
            if (t != s && cabs(g5m[s][t]) != 0.0) return -1;
        c.g5[s] = creal(g5m[s][s]);
    }
    const long n = c.n;
    const cplx *b = (const cplx *)b_;
    cplx *y = (cplx *)malloc(sizeof(cplx) * n);
    cplx *r = (cplx *)malloc(sizeof(cplx) * n);
    cplx *p = (cplx *)malloc(sizeof(cplx) * n);
    cplx *Br = (cplx *)malloc(sizeof(cplx) * n);
    cplx *Bp = (cplx *)malloc(sizeof(cplx) * n);
    c.tmp = (cplx *)malloc(sizeof(cplx) * n);

    memset(y, 0, sizeof(cplx) * n);                      /* y = 0           */
    memcpy(r, b, sizeof(cplx) * n);                      /* r = c           */
    if (method != 1) cr_gamma5(&c, r);
    memcpy(p, r, sizeof(cplx) * n);                      /* p = r           */
    cr_apply_B(&c, Br, r);                               /* B r             */
    memcpy(Bp, Br, sizeof(cplx) * n);                    /* B p = B r       */
    double rBr = creal(dot(r, Br, n));
    double nr = norm2(r, n);
    const double eps = tol * tol * norm2(b, n);
    int k = 0, rc = 1;
    if (resid) resid[0] = sqrt(nr);
    while (nr > eps && k < maxiter) {
        const double nBp = norm2(Bp, n);
        if (rBr == 0.0 || nBp == 0.0) { rc = 2; break; }
        const double alpha = rBr / nBp;
        for (long i = 0; i < n; ++i) y[i] += alpha * p[i];
        for (long i = 0; i < n; ++i) r[i] -= alpha * Bp[i];
        cr_apply_B(&c, Br, r);
        const double rBr1 = creal(dot(r, Br, n));
        const double beta = rBr1 / rBr;
        for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        if (method == 2)
            cr_apply_B(&c, Bp, p);
        else
            for (long i = 0; i < n; ++i) Bp[i] = Br[i] + beta * Bp[i];
        rBr = rBr1;
        nr = norm2(r, n);
        ++k;
        if (resid) resid[k] = sqrt(nr);
    }
    if (nr <= eps) rc = 0;
    if (method == 1)                                     /* x = A^dag y     */
        oracle_apply_eo_tm(x_, (const double *)y, U, dims, kappa, mu, phase, parity, 1);
    else
        memcpy(x_, y, sizeof(cplx) * n);
    if (iters_out) *iters_out = k;
    free(y); free(r); free(p); free(Br); free(Bp); free(c.tmp);
    return rc;
}

/* x = D^-1 b with Alg. "schur" around oracle_cr (tol relative to ||b||, as
 * in oracle_solve).                                                        */
int oracle_solve_cr(double *x_full, const double *b_full, const double *U, const int *dims,
                    double kappa, double mu, const double *phase, int parity, int method,
                    double tol, int maxiter, int *iters_out) {
    geom g = make_geom(dims);
    long vh = g.vol / 2;
    cplx *bhat = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    cplx *xp = (cplx *)malloc(sizeof(cplx) * 12 * vh);
    oracle_schur_prepare_tm((double *)bhat, b_full, U, dims, kappa, mu, phase, parity);
    double nb = sqrt(norm2((const cplx *)b_full, 12 * g.vol));
    double nbh = sqrt(norm2(bhat, 12 * vh));
    double rel = nbh > 0 ? tol * nb / nbh : tol;
    int rc = oracle_cr((double *)xp, (double *)bhat, U, dims, kappa, mu, phase, parity, method,
                       rel, maxiter, iters_out, NULL);
    if (rc >= 0)
        oracle_schur_reconstruct_tm(x_full, (double *)xp, b_full, U, dims, kappa, mu, phase,
                                    parity);
    free(bhat); free(xp);
    return rc;
}

/* Number of OpenMP threads the oracle uses (1 without OpenMP), and a setter
 * for timing it on fewer cores. */
#ifdef _OPENMP
#include <omp.h>
int oracle_num_threads(void) { return omp_get_max_threads(); }
void oracle_set_num_threads(int n) { if (n > 0) omp_set_num_threads(n); }
#else
int oracle_num_threads(void) { return 1; }
void oracle_set_num_threads(int n) { (void)n; }
#endif
