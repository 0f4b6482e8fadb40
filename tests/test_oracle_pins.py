"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test ties the oracle to mathematics the paper states or implies:

* Clifford algebra of the gamma basis (Fig. id: hermitian gammas, gamma5^2 = 1,
  gamma5 anticommuting and diagonal);
* free-field closed form: with unit links, plane waves are eigenvectors of
  D with the spin matrix 1 - 2 kappa sum_mu [cos p_mu - i gamma_mu sin p_mu]
  (Fig. dirac with U = 1), boundary phases entering through the allowed
  momenta;
* gamma5-hermiticity D^dag = gamma5 D gamma5 (Fig. id identities);
* gauge covariance under a random SU(3) transform (U[s x d]^dag = U[(s+d) x -d]);
* the Schur blocks of Alg. schur from the dense matrix of D;
* dense LU solves against Alg. CGNR + schur;
* kappa = 0 special case and the monotone CGNR residual.

A plausible slip in the oracle (a swapped projector sign, the wrong link on
the backward hop, a missing conjugate on a phase, a dropped kappa^2, the
2 kappa factor of the schur reconstruction) fails at least one of them.
"""
import numpy as np
import pytest

import synthetic as syn

# DeGrand-Rossi basis written out independently of the oracle's table.
_I = 1j
GAMMA_DR = [
    np.array([[0, 0, 0, _I], [0, 0, _I, 0], [0, -_I, 0, 0], [-_I, 0, 0, 0]]),
    np.array([[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]], dtype=complex),
    np.array([[0, 0, _I, 0], [0, 0, 0, -_I], [-_I, 0, 0, 0], [0, _I, 0, 0]]),
    np.array([[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]], dtype=complex),
]
G5 = np.diag([1, 1, -1, -1]).astype(complex)


def relerr(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def inner(a, b):
    return np.vdot(a.ravel(), b.ravel())


def g5(psi):
    return np.einsum("st,...ct->...cs", G5, psi)


def shift_plus(field, dims, mu):
    """field(x + mu) for a [V, ...] array, periodic, independent of the oracle."""
    Lx, Ly, Lz, Lt = dims
    f = field.reshape((Lt, Lz, Ly, Lx) + field.shape[1:])
    axis = 3 - mu
    return np.roll(f, -1, axis=axis).reshape(field.shape)


# ---------------------------------------------------------------------------
def test_gamma_basis_clifford(oracle_lib):
    g = [oracle_lib.gamma(m) for m in range(5)]
    I4 = np.eye(4)
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T, atol=0)
        for n in range(4):
            anti = g[m] @ g[n] + g[n] @ g[m]
            assert np.allclose(anti, 2 * I4 * (m == n), atol=0)
        assert np.allclose(g[4] @ g[m] + g[m] @ g[4], 0, atol=0)
    assert np.allclose(g[4] @ g[4], I4, atol=0)
    assert np.allclose(g[4], G5, atol=0)                     # diagonal gamma5
    assert np.allclose(g[4], g[0] @ g[1] @ g[2] @ g[3], atol=0)
    for m in range(4):                                       # the chosen basis
        assert np.allclose(g[m], GAMMA_DR[m], atol=0)


def test_independent_gamma_table_is_clifford():
    for m in range(4):
        for n in range(4):
            anti = GAMMA_DR[m] @ GAMMA_DR[n] + GAMMA_DR[n] @ GAMMA_DR[m]
            assert np.allclose(anti, 2 * np.eye(4) * (m == n))
    assert np.allclose(GAMMA_DR[0] @ GAMMA_DR[1] @ GAMMA_DR[2] @ GAMMA_DR[3], G5)


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims,theta,kappa", [
    ((4, 6, 4, 8), (0, 0, 0, np.pi), 0.12),            # periodic space, antiperiodic time
    ((6, 4, 2, 4), (0.3, -1.1, 0, np.pi), 0.124),       # twisted complex phases
    ((2, 2, 2, 2), (0, 0, 0, 0), 0.2),                  # 2^4: x+mu and x-mu coincide
])
def test_free_field_plane_waves(oracle_lib, dims, theta, kappa):
    U = syn.unit_links(dims)
    phase = np.exp(1j * np.asarray(theta))
    X = syn.coords(dims)
    rng = np.random.default_rng(7)
    for _ in range(4):
        n = [rng.integers(0, L) for L in dims]
        p = np.array([(2 * np.pi * n[m] + theta[m]) / dims[m] for m in range(4)])
        wave = np.exp(1j * (X @ p))
        # closed form spin matrix
        M_exact = (1 - 2 * kappa * np.cos(p).sum()) * np.eye(4) + 2j * kappa * sum(
            GAMMA_DR[m] * np.sin(p[m]) for m in range(4))
        for c0 in range(3):
            M = np.zeros((4, 4), dtype=complex)
            for s0 in range(4):
                psi = np.zeros((len(wave), 3, 4), dtype=complex)
                psi[:, c0, s0] = wave
                out = oracle_lib.apply(psi, U, dims, kappa, phase)
                # colour is untouched, and the result is wave * M[:, s0]
                others = [c for c in range(3) if c != c0]
                assert np.abs(out[:, others, :]).max() < 1e-14
                col = out[:, c0, :] / wave[:, None]
                assert np.abs(col - col[0]).max() < 1e-13
                M[:, s0] = col[0]
            assert np.abs(M - M_exact).max() < 1e-13
            # basis-independent form of the same fact
            ev = np.linalg.eigvals(M)
            ev = ev[np.argsort(ev.imag)]
            s = np.sqrt((np.sin(p) ** 2).sum())
            a = 1 - 2 * kappa * np.cos(p).sum()
            ref = np.array([a - 2j * kappa * s] * 2 + [a + 2j * kappa * s] * 2)
            assert np.abs(ev - ref).max() < 1e-7   # doubly degenerate roots


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 4)])
def test_gamma5_hermiticity(oracle_lib, dims):
    kappa = 0.13
    phase = np.exp(1j * np.array([0.4, 0.0, -0.7, np.pi]))
    U = syn.su3_links(dims, eps=0.3, seed=5)
    V = syn.volume(dims)
    phi = syn.gaussian_spinor(V, 8)
    psi = syn.gaussian_spinor(V, 9)
    Dpsi = oracle_lib.apply(psi, U, dims, kappa, phase)
    Ddag_phi = oracle_lib.apply(phi, U, dims, kappa, phase, dagger=True)
    # <phi, D psi> = <D^dag phi, psi>
    assert abs(inner(phi, Dpsi) - inner(Ddag_phi, psi)) < 1e-12 * abs(inner(phi, Dpsi))
    # D^dag = gamma5 D gamma5
    assert relerr(Ddag_phi, g5(oracle_lib.apply(g5(phi), U, dims, kappa, phase))) < 1e-14
    # the Schur operator inherits it, for both parities
    for par in (0, 1):
        ph = syn.to_half(phi, dims, par)
        ps = syn.to_half(psi, dims, par)
        Mps = oracle_lib.apply_eo(ps, U, dims, kappa, phase, par)
        Mdph = oracle_lib.apply_eo(ph, U, dims, kappa, phase, par, dagger=True)
        assert abs(inner(ph, Mps) - inner(Mdph, ps)) < 1e-12 * abs(inner(ph, Mps))
        assert relerr(Mdph, g5(oracle_lib.apply_eo(g5(ph), U, dims, kappa, phase, par))) < 1e-14


def test_dagger_is_not_trivial(oracle_lib):
    """Guards the hermiticity pin: D itself is not hermitian."""
    dims = (4, 4, 4, 4)
    U = syn.su3_links(dims, seed=5)
    psi = syn.gaussian_spinor(256, 3)
    a = oracle_lib.apply(psi, U, dims, 0.12, syn.workloads.APBC_T)
    b = oracle_lib.apply(psi, U, dims, 0.12, syn.workloads.APBC_T, dagger=True)
    assert relerr(a, b) > 1e-2


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 2, 6, 4)])
def test_gauge_covariance(oracle_lib, dims):
    kappa = 0.12
    phase = np.exp(1j * np.array([0.0, 0.2, 0.0, np.pi]))
    V = syn.volume(dims)
    U = syn.su3_links(dims, eps=0.3, seed=11)
    G = syn.random_su3(V, seed=12)
    UG = np.empty_like(U)
    for mu in range(4):
        Gp = shift_plus(G, dims, mu)
        UG[:, mu] = G @ U[:, mu] @ np.conj(np.swapaxes(Gp, -1, -2))
    psi = syn.gaussian_spinor(V, 13)
    Gpsi = G @ psi                                  # colour rotation, spin untouched
    lhs = oracle_lib.apply(Gpsi, UG, dims, kappa, phase)
    rhs = G @ oracle_lib.apply(psi, U, dims, kappa, phase)
    assert relerr(lhs, rhs) < 1e-14
    # and the test is not vacuous: the untransformed links give a different answer
    assert relerr(oracle_lib.apply(Gpsi, U, dims, kappa, phase), rhs) > 1e-2


# ---------------------------------------------------------------------------
def _parity_perm(dims):
    """Index maps of the dense matrix (lex*12 + c*4 + s) onto parity blocks."""
    ev = syn.parity_sites(dims, 0)
    od = syn.parity_sites(dims, 1)
    ie = (ev[:, None] * 12 + np.arange(12)).ravel()
    io = (od[:, None] * 12 + np.arange(12)).ravel()
    return ie, io


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
def test_schur_blocks_dense(oracle_lib, dims):
    kappa = 0.12
    phase = syn.workloads.APBC_T
    U = syn.su3_links(dims, eps=0.3, seed=21)
    D = oracle_lib.dense_matrix(U, dims, kappa, phase)
    ie, io = _parity_perm(dims)
    Dee, Deo = D[np.ix_(ie, ie)], D[np.ix_(ie, io)]
    Doe, Doo = D[np.ix_(io, ie)], D[np.ix_(io, io)]
    n = len(ie)
    # mu = 0: the diagonal blocks are the identity (D11 diagonal, Alg. schur)
    assert np.array_equal(Dee, np.eye(n)) and np.array_equal(Doo, np.eye(n))
    blocks = {0: Dee - Deo @ np.linalg.solve(Doo, Doe), 1: Doo - Doe @ np.linalg.solve(Dee, Deo)}
    for par in (0, 1):
        Mhat = np.empty((n, n), dtype=complex)
        e = np.zeros(n, dtype=complex)
        for j in range(n):
            e[:] = 0
            e[j] = 1
            Mhat[:, j] = oracle_lib.apply_eo(e.reshape(-1, 3, 4), U, dims, kappa, phase,
                                             par).ravel()
        assert np.abs(Mhat - blocks[par]).max() < 1e-14
    # D^dag from the dagger flag equals the conjugate transpose
    Dd = oracle_lib.dense_matrix(U, dims, kappa, phase, dagger=True)
    assert np.abs(Dd - D.conj().T).max() < 1e-15


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dims,kappa,parity", [
    ((2, 2, 2, 2), 0.12, 1),
    ((4, 4, 4, 4), 0.12, 1),
    ((4, 4, 4, 4), 0.124, 0),
])
def test_cgnr_schur_solve_matches_lu(oracle_lib, dims, kappa, parity):
    phase = syn.workloads.APBC_T
    U = syn.su3_links(dims, eps=0.3, seed=1)
    V = syn.volume(dims)
    b = syn.gaussian_spinor(V, 2)
    D = oracle_lib.dense_matrix(U, dims, kappa, phase)
    x_lu = np.linalg.solve(D, b.ravel())
    x, iters, ok = oracle_lib.solve(b, U, dims, kappa, phase, parity=parity, tol=1e-13)
    assert ok and iters > 0
    r = b.ravel() - D @ x.ravel()
    assert np.linalg.norm(r) <= 1.01e-13 * np.linalg.norm(b)
    cond = np.linalg.cond(D)
    assert relerr(x.ravel(), x_lu) < 10 * cond * 1e-13


def test_cgnr_on_schur_system_matches_lu(oracle_lib):
    dims, kappa, par = (4, 4, 4, 4), 0.12, 1
    phase = syn.workloads.APBC_T
    U = syn.su3_links(dims, seed=4)
    b = syn.gaussian_spinor(256, 6)
    bh = oracle_lib.schur_prepare(b, U, dims, kappa, phase, par)
    D = oracle_lib.dense_matrix(U, dims, kappa, phase)
    ie, io = _parity_perm(dims)
    # bhat_o = b_o - D_oe D_ee^-1 b_e
    bh_ref = b.ravel()[io] - D[np.ix_(io, ie)] @ np.linalg.solve(D[np.ix_(ie, ie)], b.ravel()[ie])
    assert relerr(bh.ravel(), bh_ref) < 1e-14
    x, iters, ok, hist = oracle_lib.cgnr(bh, U, dims, kappa, phase, par, tol=1e-13)
    assert ok
    Mhat = D[np.ix_(io, io)] - D[np.ix_(io, ie)] @ D[np.ix_(ie, io)]
    assert relerr(x.ravel(), np.linalg.solve(Mhat, bh_ref)) < 1e-11
    # CGNR minimises ||r|| over the Krylov space: the residual never grows
    assert np.all(np.diff(hist) <= 1e-12 * hist[0])
    # reconstruction gives the full solution
    xf = oracle_lib.schur_reconstruct(x, b, U, dims, kappa, phase, par)
    assert relerr(xf.ravel(), np.linalg.solve(D, b.ravel())) < 1e-11


def test_kappa_zero_is_identity(oracle_lib):
    dims = (4, 2, 2, 4)
    U = syn.su3_links(dims, seed=3)
    psi = syn.gaussian_spinor(64, 4)
    out = oracle_lib.apply(psi, U, dims, 0.0, syn.workloads.APBC_T)
    assert np.array_equal(out, psi)
    bh = syn.to_half(psi, dims, 1)
    assert np.array_equal(oracle_lib.apply_eo(bh, U, dims, 0.0, syn.workloads.APBC_T, 1), bh)
    x, iters, ok, _ = oracle_lib.cgnr(bh, U, dims, 0.0, syn.workloads.APBC_T, 1, tol=1e-14)
    assert ok and iters == 1 and relerr(x, bh) < 1e-15


def test_recursive_residual_tracks_true_residual(oracle_lib):
    dims, kappa, par = (4, 4, 4, 4), 0.124, 1
    phase = syn.workloads.APBC_T
    U = syn.su3_links(dims, seed=1)
    bh = syn.to_half(syn.gaussian_spinor(256, 2), dims, par)
    for it in (5, 20):
        x, iters, ok, hist = oracle_lib.cgnr(bh, U, dims, kappa, phase, par, tol=1e-30,
                                             maxiter=it)
        assert iters == it and not ok
        r_true = bh - oracle_lib.apply_eo(x, U, dims, kappa, phase, par)
        assert abs(np.linalg.norm(r_true) - hist[-1]) < 1e-12 * hist[0]


# ---------------------------------------------------------------------------
# Twisted mass (Fig. dirac with mu != 0): D = 1 + 2 i kappa mu gamma5 - kappa H.
@pytest.mark.parametrize("mu", [0.05, -0.3])
def test_twisted_free_field(oracle_lib, mu):
    """Unit links, plane waves: D acts on the spin index as
    (1 - 2 kappa sum cos p) + 2 i kappa mu gamma5 + 2 i kappa sum gamma_mu sin p_mu,
    whose eigenvalues are m +- i sqrt((2 kappa mu)^2 + sum (2 kappa sin p)^2)
    (gamma5 anticommutes with every gamma_mu and all square to one)."""
    dims, kappa = (4, 2, 4, 6), 0.11
    theta = (0.0, 0.0, 0.0, np.pi)
    U = syn.unit_links(dims)
    phase = np.exp(1j * np.asarray(theta))
    X = syn.coords(dims)
    rng = np.random.default_rng(11)
    for _ in range(3):
        n = [rng.integers(0, L) for L in dims]
        p = np.array([(2 * np.pi * n[m] + theta[m]) / dims[m] for m in range(4)])
        wave = np.exp(1j * (X @ p))
        m0 = 1 - 2 * kappa * np.cos(p).sum()
        M_exact = m0 * np.eye(4) + 2j * kappa * mu * G5 + 2j * kappa * sum(
            GAMMA_DR[k] * np.sin(p[k]) for k in range(4))
        M = np.zeros((4, 4), dtype=complex)
        for s0 in range(4):
            psi = np.zeros((len(wave), 3, 4), dtype=complex)
            psi[:, 1, s0] = wave
            out = oracle_lib.apply_tm(psi, U, dims, kappa, mu, phase)
            col = out[:, 1, :] / wave[:, None]
            assert np.abs(col - col[0]).max() < 1e-13
            M[:, s0] = col[0]
        assert np.abs(M - M_exact).max() < 1e-13
        ev = np.linalg.eigvals(M)
        ev = ev[np.argsort(ev.imag)]
        w = np.sqrt((2 * kappa * mu) ** 2 + ((2 * kappa * np.sin(p)) ** 2).sum())
        ref = np.array([m0 - 1j * w] * 2 + [m0 + 1j * w] * 2)
        assert np.abs(ev - ref).max() < 1e-7


def test_twisted_adjoint_flips_mu(oracle_lib):
    """D(mu)^dag = gamma5 D(-mu) gamma5 (gamma5 hermitian and diagonal,
    gamma5 H gamma5 = H^dag), for D and for the Schur operator."""
    dims, kappa, mu = (4, 4, 2, 4), 0.12, 0.2
    phase = np.exp(1j * np.array([0.4, 0.0, -0.7, np.pi]))
    U = syn.su3_links(dims, eps=0.3, seed=5)
    V = syn.volume(dims)
    phi, psi = syn.gaussian_spinor(V, 8), syn.gaussian_spinor(V, 9)
    Dpsi = oracle_lib.apply_tm(psi, U, dims, kappa, mu, phase)
    Ddphi = oracle_lib.apply_tm(phi, U, dims, kappa, mu, phase, dagger=True)
    assert abs(inner(phi, Dpsi) - inner(Ddphi, psi)) < 1e-12 * abs(inner(phi, Dpsi))
    assert relerr(Ddphi, g5(oracle_lib.apply_tm(g5(phi), U, dims, kappa, -mu, phase))) < 1e-14
    # the twist is not invisible to the adjoint: D(mu)^dag != gamma5 D(mu) gamma5
    assert relerr(Ddphi, g5(oracle_lib.apply_tm(g5(phi), U, dims, kappa, mu, phase))) > 1e-2
    for par in (0, 1):
        ph, ps = syn.to_half(phi, dims, par), syn.to_half(psi, dims, par)
        Mps = oracle_lib.apply_eo_tm(ps, U, dims, kappa, mu, phase, par)
        Mdph = oracle_lib.apply_eo_tm(ph, U, dims, kappa, mu, phase, par, dagger=True)
        assert abs(inner(ph, Mps) - inner(Mdph, ps)) < 1e-12 * abs(inner(ph, Mps))


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 2, 2)])
def test_twisted_schur_blocks_dense(oracle_lib, dims):
    """Dense D(mu): the diagonal parity blocks are 1 + 2 i kappa mu gamma5 on
    every site, and Mhat_p = D_pp - D_pq D_qq^-1 D_qp (Alg. schur)."""
    kappa, mu = 0.12, 0.15
    phase = syn.workloads.APBC_T
    U = syn.su3_links(dims, eps=0.3, seed=21)
    D = oracle_lib.dense_matrix(U, dims, kappa, phase, mu=mu)
    ie, io = _parity_perm(dims)
    n = len(ie)
    A = np.kron(np.eye(n // 12), np.kron(np.eye(3), np.eye(4) + 2j * kappa * mu * G5))
    assert np.abs(D[np.ix_(ie, ie)] - A).max() < 1e-15
    assert np.abs(D[np.ix_(io, io)] - A).max() < 1e-15
    for par, (ip, iq) in ((0, (ie, io)), (1, (io, ie))):
        ref = D[np.ix_(ip, ip)] - D[np.ix_(ip, iq)] @ np.linalg.solve(D[np.ix_(iq, iq)],
                                                                         D[np.ix_(iq, ip)])
        Mhat = np.empty((n, n), dtype=complex)
        e = np.zeros(n, dtype=complex)
        for j in range(n):
            e[:] = 0
            e[j] = 1
            Mhat[:, j] = oracle_lib.apply_eo_tm(e.reshape(-1, 3, 4), U, dims, kappa, mu, phase,
                                                par).ravel()
        assert np.abs(Mhat - ref).max() < 1e-14
    Dd = oracle_lib.dense_matrix(U, dims, kappa, phase, dagger=True, mu=mu)
    assert np.abs(Dd - D.conj().T).max() < 1e-15


@pytest.mark.parametrize("dims,parity", [((2, 2, 2, 2), 1), ((4, 4, 4, 4), 0)])
def test_twisted_solve_matches_lu(oracle_lib, dims, parity):
    """Schur prepare, CGNR and reconstruction with the twisted mass give the
    dense LU solution of D(mu) x = b."""
    kappa, mu = 0.124, 0.1
    phase = syn.workloads.APBC_T
    U = syn.su3_links(dims, eps=0.3, seed=1)
    b = syn.gaussian_spinor(syn.volume(dims), 2)
    D = oracle_lib.dense_matrix(U, dims, kappa, phase, mu=mu)
    x, iters, ok = oracle_lib.solve_tm(b, U, dims, kappa, mu, phase, parity=parity, tol=1e-13)
    assert ok and iters > 0
    assert np.linalg.norm(b.ravel() - D @ x.ravel()) <= 1.01e-13 * np.linalg.norm(b)
    x_lu = np.linalg.solve(D, b.ravel())
    assert relerr(x.ravel(), x_lu) < 10 * np.linalg.cond(D) * 1e-13


def test_twisted_mass_zero_is_the_wilson_operator(oracle_lib):
    dims, kappa = (4, 4, 2, 4), 0.12
    phase = syn.workloads.APBC_T
    U = syn.su3_links(dims, seed=3)
    psi = syn.gaussian_spinor(syn.volume(dims), 1)
    assert relerr(oracle_lib.apply_tm(psi, U, dims, kappa, 0.0, phase),
                  oracle_lib.apply(psi, U, dims, kappa, phase)) < 1e-15
    h = syn.to_half(psi, dims, 1)
    assert relerr(oracle_lib.apply_eo_tm(h, U, dims, kappa, 0.0, phase, 1),
                  oracle_lib.apply_eo(h, U, dims, kappa, phase, 1)) < 1e-15


# ---------------------------------------------------------------------------
# Conjugate-residual solvers.  Sec. 5 compares CRNE, MCR1 and MCR2 with CGNR
# on the Schur system without defining them; the oracle takes the textbook
# readings (CR on A A^dag, and CR on the Hermitian gamma5 A with B p formed by
# the operator or by recurrence).  CR minimises the residual over its Krylov
# space, so its k-th iterate is fixed by dense linear algebra alone.
def _dense_schur(oracle_lib, U, dims, kappa, phase, mu, parity):
    D = oracle_lib.dense_matrix(U, dims, kappa, phase, mu=mu)
    ie, io = _parity_perm(dims)
    ip, iq = (ie, io) if parity == 0 else (io, ie)
    return D[np.ix_(ip, ip)] - D[np.ix_(ip, iq)] @ np.linalg.solve(D[np.ix_(iq, iq)],
                                                                     D[np.ix_(iq, ip)])


def _krylov_minimiser(A, B, c, b, k):
    """argmin ||b - A x|| over x in K_k(B, c): an orthonormal basis of the
    Krylov space (Gram-Schmidt, applied twice) and a dense least-squares solve."""
    Q = np.zeros((len(c), k), dtype=complex)
    v = c / np.linalg.norm(c)
    for j in range(k):
        for _ in range(2):
            v = v - Q[:, :j] @ (Q[:, :j].conj().T @ v)
        Q[:, j] = v / np.linalg.norm(v)
        v = B @ Q[:, j]
    coef = np.linalg.lstsq(A @ Q, b, rcond=None)[0]
    return Q @ coef


@pytest.mark.parametrize("mu", [0.0, 0.1])
def test_cr_iterates_minimise_over_krylov_space(oracle_lib, mu):
    """CRNE's k-th iterate minimises ||b - A x|| over K_k(A^dag A, A^dag b);
    MCR1's and MCR2's over K_k(gamma5 A, gamma5 b) (mu = 0 only: gamma5 A is
    Hermitian for the Wilson operator alone)."""
    dims, kappa, parity = (4, 4, 2, 4), 0.124, 1
    phase = syn.workloads.APBC_T
    U = syn.su3_links(dims, eps=0.3, seed=4)
    b = syn.to_half(syn.gaussian_spinor(syn.volume(dims), 6), dims, parity)
    A = _dense_schur(oracle_lib, U, dims, kappa, phase, mu, parity)
    bv = b.ravel()
    G = np.kron(np.eye(len(bv) // 4), G5)
    spaces = {"crne": (A.conj().T @ A, A.conj().T @ bv), "mcr1": (G @ A, G @ bv),
              "mcr2": (G @ A, G @ bv)}
    for method, (B, c) in spaces.items():
        if method != "crne" and mu != 0.0:
            assert np.abs(G @ A - (G @ A).conj().T).max() > 1e-3   # not Hermitian
            with pytest.raises(ValueError):
                oracle_lib.cr(b, U, dims, kappa, phase, method, mu=mu, parity=parity)
            continue
        assert method == "crne" or np.abs(B - B.conj().T).max() < 1e-14
        for k in (1, 2, 4, 7):
            x, iters, status, _ = oracle_lib.cr(b, U, dims, kappa, phase, method, mu=mu,
                                                parity=parity, tol=1e-30, maxiter=k)
            assert iters == k and status == 1
            ref = _krylov_minimiser(A, B, c, bv, k)
            assert relerr(x.ravel(), ref) < 1e-9, (method, k, relerr(x.ravel(), ref))


@pytest.mark.parametrize("dims,parity", [((2, 2, 2, 2), 1), ((4, 4, 2, 4), 0)])
def test_cr_solves_match_lu(oracle_lib, dims, parity):
    """Schur prepare, CRNE / MCR1 / MCR2 and reconstruction give the dense LU
    solution of D x = b, with and without the twisted mass."""
    kappa = 0.124
    phase = syn.workloads.APBC_T
    U = syn.su3_links(dims, eps=0.3, seed=1)
    b = syn.gaussian_spinor(syn.volume(dims), 2)
    for mu in (0.0, 0.1):
        D = oracle_lib.dense_matrix(U, dims, kappa, phase, mu=mu)
        x_lu = np.linalg.solve(D, b.ravel())
        for method in ("crne", "mcr1", "mcr2") if mu == 0.0 else ("crne",):
            x, iters, status = oracle_lib.solve_cr(b, U, dims, kappa, phase, method, mu=mu,
                                                   parity=parity, tol=1e-13, maxiter=2000)
            assert status == 0 and iters > 0, (method, mu, status)
            assert np.linalg.norm(b.ravel() - D @ x.ravel()) <= 1.01e-13 * np.linalg.norm(b)
            assert relerr(x.ravel(), x_lu) < 10 * np.linalg.cond(D) * 1e-13


def test_cr_special_cases(oracle_lib):
    """kappa = 0 (A = 1): CRNE takes one iteration; MCR (B = gamma5, eigenvalues
    +-1) exactly two; both end at x = b.  The CR residual never grows
    (residual minimisation over nested spaces).  CRNE and CGNR minimise the
    same residual over the same space, so their iterates agree; MCR1 and MCR2
    differ only in how B p is formed."""
    dims, parity = (4, 4, 2, 4), 1
    phase = syn.workloads.APBC_T
    U = syn.su3_links(dims, eps=0.3, seed=2)
    b = syn.to_half(syn.gaussian_spinor(syn.volume(dims), 3), dims, parity)
    for method in ("crne", "mcr1", "mcr2"):
        # MCR's second step divides by its first coefficient (gamma5 b | b) / ||b||^2,
        # of order 1/sqrt(n): the exact two-step answer carries ~1e-14 rounding
        x, iters, status, _ = oracle_lib.cr(b, U, dims, 0.0, phase, method, parity=parity,
                                            tol=1e-12, maxiter=10)
        assert status == 0 and iters == (1 if method == "crne" else 2) and relerr(x, b) < 1e-12
        _, _, status, hist = oracle_lib.cr(b, U, dims, 0.124, phase, method, parity=parity,
                                           tol=1e-12, maxiter=500)
        assert status == 0 and np.all(np.diff(hist) <= 1e-14 * hist[0])
    for k in (3, 10, 25):
        xc, _, _, _ = oracle_lib.cgnr(b, U, dims, 0.124, phase, parity=parity, tol=1e-30,
                                      maxiter=k)
        xr, _, _, _ = oracle_lib.cr(b, U, dims, 0.124, phase, "crne", parity=parity, tol=1e-30,
                                    maxiter=k)
        assert relerr(xr, xc) < 1e-11
        x1, _, _, _ = oracle_lib.cr(b, U, dims, 0.124, phase, "mcr1", parity=parity, tol=1e-30,
                                    maxiter=k)
        x2, _, _, _ = oracle_lib.cr(b, U, dims, 0.124, phase, "mcr2", parity=parity, tol=1e-30,
                                    maxiter=k)
        assert relerr(x2, x1) < 1e-11


def test_cr_operators_hermitian_forms(oracle_lib):
    """The two Hermitian forms the CR readings rely on, from the dense D: gamma5
    Mhat is Hermitian and indefinite (eigenvalues of both signs: MCR is CR on
    an indefinite matrix), Mhat Mhat^dag is Hermitian positive definite (CRNE)."""
    dims, kappa = (4, 4, 2, 2), 0.124
    U = syn.su3_links(dims, eps=0.3, seed=9)
    A = _dense_schur(oracle_lib, U, dims, kappa, syn.workloads.APBC_T, 0.0, 1)
    G = np.kron(np.eye(A.shape[0] // 4), G5)
    B = G @ A
    assert np.abs(B - B.conj().T).max() < 1e-14
    ev = np.linalg.eigvalsh(B)
    assert ev.min() < -0.1 and ev.max() > 0.1
    N = A @ A.conj().T
    assert np.linalg.eigvalsh(N).min() > 0.0
