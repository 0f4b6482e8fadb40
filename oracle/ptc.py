"""FP64 numpy oracle of the learned preconditioner: a linear, gauge-equivariant
parallel-transport convolution (PTC) network (Lehner & Wettig,
arXiv:2302.05419) used as the right preconditioner of a flexible solver.
The paper (arXiv:1401.2039) has no learned component; this follows the
network the workload specifies: four layers, channels 1 -> 16 -> 16 -> 16 -> 1.

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the CUDA path.

One layer maps C_in spinor fields to C_out spinor fields:

    out_{c'}(x) = sum_{c < C_in} sum_{k = 0..8} W[c', c, k] (T_k in_c)(x)

* W[c', c, k] is a complex 4x4 matrix acting on spin;
* T_0 is the identity, T_{1+mu} the forward transport
  (T_{1+mu} psi)(x) = U_mu(x) phi_mu psi(x + mu) and T_{5+mu} the backward one
  (T_{5+mu} psi)(x) = U_mu(x - mu)^dag phi_mu^* psi(x - mu), with the boundary
  phase phi_mu on hops that wrap (the same links and phases as the
  Wilson-Dirac operator); T_{1+mu}^dag = T_{5+mu}.

Gradients are those of the real loss with respect to the real and imaginary
parts of the weights, packed as g = dL/dRe(W) + i dL/dIm(W).  For the loss
L = sum ||N(r) - e||^2 / ||e||^2 the gradient with respect to a layer output y
is 2 (y - e) / ||e||^2 in the same packing, and a layer propagates
g_in,c = sum_k T_k^dag (sum_c' W[c', c, k]^dag g_out,c'),
g_W[c', c, k] = sum_x g_out,c'(x) (T_k in_c)(x)^dag  (summed over colour).

Parity pins (tests/test_ptc_oracle.py): adjointness of the transports, a layer
with Wilson weights equals the C oracle's D, gauge equivariance of the whole
net, central finite differences of the gradients; the sampled-site forward
(net_forward_sites, for full-size checks) equals the full-field one at every
site and reproduces a backward transport written out by hand.
"""
from __future__ import annotations

import numpy as np

NK = 9          # transports per layer: identity, 4 forward, 4 backward
LAYERS = (1, 16, 16, 16, 1)


def _shape4(dims):
    Lx, Ly, Lz, Lt = (int(d) for d in dims)
    return (Lt, Lz, Ly, Lx)


def _wrap_mask(dims, mu, forward):
    """Sites whose hop in direction mu wraps around the lattice, [V] bool."""
    Lx, Ly, Lz, Lt = (int(d) for d in dims)
    L = (Lx, Ly, Lz, Lt)[mu]
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx),
                             indexing="ij")
    coord = (x, y, z, t)[mu].ravel()
    return coord == (L - 1 if forward else 0)


def transport(psi, U, dims, phase, k):
    """(T_k psi) for a field psi [V, 3, 4] (or [..., V, 3, 4] with leading batch dims)."""
    if k == 0:
        return psi.copy()
    shp = _shape4(dims)
    V = int(np.prod(shp))
    lead = psi.shape[:-3]
    f = psi.reshape(lead + shp + (3, 4))
    mu = (k - 1) % 4
    axis = len(lead) + 3 - mu
    ph = complex(phase[mu])
    if k <= 4:      # forward: U_mu(x) phi psi(x + mu)
        nb = np.roll(f, -1, axis=axis).reshape(lead + (V, 3, 4))
        w = np.where(_wrap_mask(dims, mu, True), ph, 1.0)
        return np.einsum("vab,...vbs->...vas", U[:, mu], nb) * w[:, None, None]
    # backward: U_mu(x - mu)^dag phi^* psi(x - mu)
    nb = np.roll(f, 1, axis=axis).reshape(lead + (V, 3, 4))
    Ub = np.roll(U[:, mu].reshape(shp + (3, 3)), 1, axis=3 - mu).reshape(V, 3, 3)
    w = np.where(_wrap_mask(dims, mu, False), np.conj(ph), 1.0)
    return np.einsum("vba,...vbs->...vas", np.conj(Ub), nb) * w[:, None, None]


def adjoint_index(k):
    """T_k^dag = T_{adjoint_index(k)}."""
    if k == 0:
        return 0
    return k + 4 if k <= 4 else k - 4


def layer_forward(inp, W, U, dims, phase):
    """inp [C_in, V, 3, 4], W [C_out, C_in, 9, 4, 4] -> out [C_out, V, 3, 4]."""
    out = np.zeros((W.shape[0],) + inp.shape[1:], dtype=np.complex128)
    for k in range(NK):
        Tk = transport(inp, U, dims, phase, k)                 # [C_in, V, 3, 4]
        out += np.einsum("dcst,cvat->dvas", W[:, :, k], Tk)
    return out


def layer_backward(inp, W, g_out, U, dims, phase):
    """Gradients (packed complex) of a layer: returns (g_in, g_W)."""
    g_in = np.zeros_like(inp)
    g_W = np.zeros_like(W)
    for k in range(NK):
        Tk = transport(inp, U, dims, phase, k)
        g_W[:, :, k] = np.einsum("dvas,cvat->dcst", g_out, np.conj(Tk))
        gk = np.einsum("dcst,dvas->cvat", np.conj(W[:, :, k]), g_out)   # W^dag g
        g_in += transport(gk, U, dims, phase, adjoint_index(k))
    return g_in, g_W


def net_forward(r, Ws, U, dims, phase, keep=False):
    """N(r) for r [V, 3, 4]; with keep=True also the layer inputs."""
    x = r[None]
    acts = []
    for W in Ws:
        acts.append(x)
        x = layer_forward(x, W, U, dims, phase)
    return (x[0], acts) if keep else x[0]


def loss_and_grad(rs, es, Ws, U, dims, phase):
    """L = sum_i ||N(r_i) - e_i||^2 / ||e_i||^2 and its packed weight gradients."""
    L = 0.0
    grads = [np.zeros_like(W) for W in Ws]
    for r, e in zip(rs, es):
        y, acts = net_forward(r, Ws, U, dims, phase, keep=True)
        ne = np.vdot(e.ravel(), e.ravel()).real
        d = y - e
        L += np.vdot(d.ravel(), d.ravel()).real / ne
        g = (2.0 / ne * d)[None]
        for li in range(len(Ws) - 1, -1, -1):
            g, gW = layer_backward(acts[li], Ws[li], g, U, dims, phase)
            grads[li] += gW
    return L, grads


def identity_init(seed: int, scale: float = 0.01, layers=LAYERS):
    """Weights that start as the identity map (channel 0 carried through by
    T_0 = 1) plus small complex Gaussian entries."""
    rng = np.random.default_rng(seed)
    Ws = []
    for cin, cout in zip(layers[:-1], layers[1:]):
        W = scale * (rng.standard_normal((cout, cin, NK, 4, 4))
                     + 1j * rng.standard_normal((cout, cin, NK, 4, 4))) / np.sqrt(2 * cin * NK)
        W[0, 0, 0] += np.eye(4)
        Ws.append(W)
    return Ws


# ----------------------------------------------------------------- sampled sites
def _coords_of(lex, dims):
    """Coordinates (x, y, z, t) of lexicographic site indices, [n, 4]."""
    L = [int(d) for d in dims]
    lex = np.asarray(lex, dtype=np.int64)
    x = lex % L[0]
    r = lex // L[0]
    y = r % L[1]
    r //= L[1]
    z = r % L[2]
    t = r // L[2]
    return np.stack([x, y, z, t], axis=1)


def _lex_of(c, dims):
    L = [int(d) for d in dims]
    return ((c[:, 3] * L[2] + c[:, 2]) * L[1] + c[:, 1]) * L[0] + c[:, 0]


def _stencil(sites, dims):
    """For each site: its 9 stencil sites (itself, x + mu, x - mu) and the
    wrap flags of the 8 hops, as [n, 9] indices and [n, 9] bools."""
    c = _coords_of(sites, dims)
    nb = [np.asarray(sites, dtype=np.int64)]
    wr = [np.zeros(len(sites), dtype=bool)]
    for fwd in (True, False):
        for mu in range(4):
            L = int(dims[mu])
            d = c.copy()
            d[:, mu] += 1 if fwd else -1
            wrap = (d[:, mu] == L) | (d[:, mu] < 0)
            d[:, mu] %= L
            nb.append(_lex_of(d, dims))
            wr.append(wrap)
    return np.stack(nb, axis=1), np.stack(wr, axis=1)


def layer_forward_sites(inp, in_sites, W, U, dims, phase, out_sites):
    """One layer at out_sites only.  inp [C_in, len(in_sites), 3, 4] holds the
    layer input on in_sites (sorted), which must contain every stencil site
    of out_sites.  Transport k = 1 + mu (forward) and 5 + mu (backward) as
    in transport(); returns [C_out, len(out_sites), 3, 4]."""
    nb, wr = _stencil(out_sites, dims)
    pos = np.searchsorted(in_sites, nb)
    assert np.all(in_sites[pos] == nb), "input does not cover the stencil"
    out = np.zeros((W.shape[0], len(out_sites), 3, 4), dtype=np.complex128)
    for k in range(NK):
        v = inp[:, pos[:, k]]                                   # [C_in, n, 3, 4]
        if k > 0:
            mu = (k - 1) % 4
            if k <= 4:      # U_mu(x) phi psi(x + mu)
                link = U[out_sites, mu]
                ph = complex(phase[mu])
            else:           # U_mu(x - mu)^dag phi^* psi(x - mu)
                link = np.conj(np.swapaxes(U[nb[:, k], mu], 1, 2))
                ph = np.conj(complex(phase[mu]))
            w = np.where(wr[:, k], ph, 1.0)
            v = np.einsum("nab,cnbs->cnas", link, v) * w[None, :, None, None]
        out += np.einsum("dcst,cnat->dnas", W[:, :, k], v)
    return out


def net_forward_sites(r, Ws, U, dims, phase, sites):
    """N(r) at the given sites only, for checks of full-size fields: the
    layers are evaluated backwards-expanded on the receptive field of the
    sites (each layer widens it by one stencil), so the cost grows with the
    number of sites, not with the volume.  Same result as
    net_forward(r, ...)[sites]."""
    need = [np.unique(np.asarray(sites, dtype=np.int64))]
    for _ in Ws:
        need.append(np.unique(_stencil(need[-1], dims)[0].ravel()))
    need = need[::-1]                      # need[l]: sites of the layer-l input
    x = np.asarray(r)[need[0]][None]
    for l, W in enumerate(Ws):
        x = layer_forward_sites(x, need[l], W, U, dims, phase, need[l + 1])
    out = x[0]
    order = np.searchsorted(need[-1], np.asarray(sites, dtype=np.int64))
    return out[order]
