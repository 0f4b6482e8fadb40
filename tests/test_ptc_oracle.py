"""Pins of the parallel-transport-convolution oracle (oracle/ptc.py)."""
import numpy as np
import pytest

import oracle
import oracle.ptc as ptc
import synthetic as syn

DIMS = (4, 4, 2, 4)
PHASE = tuple(np.exp(1j * np.array([0.3, 0.0, -0.6, np.pi])))


def inner(a, b):
    return np.vdot(a.ravel(), b.ravel())


@pytest.fixture(scope="module")
def U():
    return syn.su3_links(DIMS, eps=0.3, seed=31)


def test_transports_are_adjoint_pairs(U):
    V = syn.volume(DIMS)
    phi = syn.gaussian_spinor(V, 1)
    psi = syn.gaussian_spinor(V, 2)
    for k in range(ptc.NK):
        lhs = inner(phi, ptc.transport(psi, U, DIMS, PHASE, k))
        rhs = inner(ptc.transport(phi, U, DIMS, PHASE, ptc.adjoint_index(k)), psi)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_wilson_weights_reproduce_the_dirac_operator(U):
    """One layer with W_0 = 1, W_{1+mu} = -kappa (1 - gamma_mu),
    W_{5+mu} = -kappa (1 + gamma_mu) is D = 1 - kappa H of the C oracle."""
    kappa = 0.13
    W = np.zeros((1, 1, ptc.NK, 4, 4), dtype=complex)
    W[0, 0, 0] = np.eye(4)
    for mu in range(4):
        g = oracle.gamma(mu)
        W[0, 0, 1 + mu] = -kappa * (np.eye(4) - g)
        W[0, 0, 5 + mu] = -kappa * (np.eye(4) + g)
    psi = syn.gaussian_spinor(syn.volume(DIMS), 3)
    got = ptc.layer_forward(psi[None], W, U, DIMS, PHASE)[0]
    ref = oracle.apply(psi, U, DIMS, kappa, PHASE)
    assert np.linalg.norm(got - ref) < 1e-13 * np.linalg.norm(ref)


def test_net_is_gauge_equivariant(U):
    layers = (1, 3, 3, 1)
    Ws = ptc.identity_init(5, scale=0.5, layers=layers)
    V = syn.volume(DIMS)
    G = syn.random_su3(V, seed=9)
    UG = np.empty_like(U)
    shp = (DIMS[3], DIMS[2], DIMS[1], DIMS[0])
    for mu in range(4):
        Gp = np.roll(G.reshape(shp + (3, 3)), -1, axis=3 - mu).reshape(V, 3, 3)
        UG[:, mu] = G @ U[:, mu] @ np.conj(np.swapaxes(Gp, -1, -2))
    r = syn.gaussian_spinor(V, 4)
    lhs = ptc.net_forward(G @ r, Ws, UG, DIMS, PHASE)
    rhs = G @ ptc.net_forward(r, Ws, U, DIMS, PHASE)
    assert np.linalg.norm(lhs - rhs) < 1e-12 * np.linalg.norm(rhs)


def test_gradients_match_central_differences(U):
    layers = (1, 2, 2, 1)
    Ws = ptc.identity_init(6, scale=0.8, layers=layers)
    V = syn.volume(DIMS)
    rs = [syn.gaussian_spinor(V, 10 + i) for i in range(2)]
    es = [syn.gaussian_spinor(V, 20 + i) for i in range(2)]
    L, grads = ptc.loss_and_grad(rs, es, Ws, U, DIMS, PHASE)
    rng = np.random.default_rng(3)
    for li in range(len(Ws)):
        d = rng.standard_normal(Ws[li].shape) + 1j * rng.standard_normal(Ws[li].shape)
        h = 1e-5
        Wp = [W.copy() for W in Ws]
        Wm = [W.copy() for W in Ws]
        Wp[li] = Wp[li] + h * d
        Wm[li] = Wm[li] - h * d
        Lp, _ = ptc.loss_and_grad(rs, es, Wp, U, DIMS, PHASE)
        Lm, _ = ptc.loss_and_grad(rs, es, Wm, U, DIMS, PHASE)
        fd = (Lp - Lm) / (2 * h)
        an = np.sum(np.real(np.conj(grads[li]) * d))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (li, fd, an)


def test_input_gradient_matches_central_differences(U):
    layers = (1, 2, 1)
    Ws = ptc.identity_init(8, scale=0.8, layers=layers)
    V = syn.volume(DIMS)
    r = syn.gaussian_spinor(V, 1)
    e = syn.gaussian_spinor(V, 2)
    y, acts = ptc.net_forward(r, Ws, U, DIMS, PHASE, keep=True)
    ne = np.vdot(e.ravel(), e.ravel()).real
    g = (2.0 / ne * (y - e))[None]
    for li in range(len(Ws) - 1, -1, -1):
        g, _ = ptc.layer_backward(acts[li], Ws[li], g, U, DIMS, PHASE)
    d = syn.gaussian_spinor(V, 5)
    h = 1e-5

    def loss(rr):
        yy = ptc.net_forward(rr, Ws, U, DIMS, PHASE)
        return np.vdot((yy - e).ravel(), (yy - e).ravel()).real / ne

    fd = (loss(r + h * d) - loss(r - h * d)) / (2 * h)
    an = np.sum(np.real(np.conj(g[0]) * d))
    assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


def test_identity_init_is_identity_at_zero_scale(U):
    Ws = ptc.identity_init(1, scale=0.0)
    r = syn.gaussian_spinor(syn.volume(DIMS), 7)
    assert np.allclose(ptc.net_forward(r, Ws, U, DIMS, PHASE), r, atol=1e-15)


def test_neumann_initialisation_is_the_degree_four_neumann_series(U):
    """The training driver's starting weights make the 1-16-16-16-1 network
    equal sum_{k<=4} (kappa H)^k (Horner's rule on two channels)."""
    from paper_1401_2039_gb300.train_preconditioner import neumann_weights
    kappa, ch = 0.12, (1, 16, 16, 16, 1)
    flat = neumann_weights(ch, kappa, 7, scale=0.0)
    Ws, off = [], 0
    for cin, cout in zip(ch[:-1], ch[1:]):
        n = cout * cin * 9 * 16
        Ws.append(flat[off:off + n].reshape(cout, cin, 9, 4, 4))
        off += n
    r = syn.gaussian_spinor(syn.volume(DIMS), 1)
    ref, t = r.copy(), r.copy()
    for _ in range(4):
        t = kappa * oracle.hop(t, U, DIMS, PHASE)
        ref = ref + t
    y = ptc.net_forward(r, Ws, U, DIMS, PHASE)
    assert np.linalg.norm(y - ref) < 1e-13 * np.linalg.norm(ref)


@pytest.mark.parametrize("dims", [(4, 4, 2, 4), (2, 2, 2, 2), (6, 4, 2, 4)])
def test_sampled_site_forward_equals_the_full_field_forward(dims):
    """net_forward_sites (receptive field of the samples only) against the
    pinned full-field forward, at every site and at a scattered subset that
    includes wrapping boundaries; Wilson-weight layers tie it to the C
    oracle's D through test_wilson_weights_reproduce_the_dirac_operator."""
    U = syn.su3_links(dims, eps=0.3, seed=32)
    Ws = ptc.identity_init(5, scale=0.7)
    V = syn.volume(dims)
    r = syn.gaussian_spinor(V, 9)
    full = ptc.net_forward(r, Ws, U, dims, PHASE)
    every = ptc.net_forward_sites(r, Ws, U, dims, PHASE, np.arange(V))
    assert np.abs(every - full).max() < 1e-12 * np.abs(full).max()
    some = np.array([V - 1, 0, 7, V // 2 + 1, 3])        # unsorted, with boundaries
    got = ptc.net_forward_sites(r, Ws, U, dims, PHASE, some)
    assert np.abs(got - full[some]).max() < 1e-12 * np.abs(full).max()


def test_sampled_site_layer_uses_the_backward_link_of_the_neighbour():
    """A single backward-transport layer at one site is U_mu(x - mu)^dag
    phi^* psi(x - mu), written out here for t = 0 (wraps, phase -1)."""
    dims = (4, 4, 4, 4)
    U = syn.su3_links(dims, eps=0.3, seed=33)
    V = syn.volume(dims)
    r = syn.gaussian_spinor(V, 10)
    W = np.zeros((1, 1, ptc.NK, 4, 4), dtype=complex)
    W[0, 0, 8] = np.eye(4)                                 # T_{5+3}: backward in t
    x = 5                                                  # t = 0
    nbr = x + 3 * 64                                       # t = 3, same x, y, z
    want = -np.einsum("ba,bs->as", np.conj(U[nbr, 3]), r[nbr])
    got = ptc.net_forward_sites(r, [W], U, dims, syn.workloads.APBC_T, np.array([x]))[0]
    assert np.abs(got - want).max() < 1e-13
