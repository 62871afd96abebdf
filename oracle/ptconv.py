"""Gauge-equivariant parallel-transport convolution (the learned preconditioner).

Not in the paper (its learned-preconditioner form is an extension of the
solver's preconditioner slot, Sec. 3 steps (1)-(2)); reading C15:

  psi_out^a(x) = sum_b sum_{d in {0, +mu, -mu}} W_d^{ab} (T_d psi^b)(x)

  T_0 = 1,
  (T_{+mu} psi)(x) = U_mu(x) psi(x + mu),
  (T_{-mu} psi)(x) = U_mu(x - mu)^dag psi(x - mu),

with the fermion boundary phase of Eq. 1 on the t wrap, W_d^{ab} a complex
4x4 matrix on spin (identity on colour).  Direction index d: 0 self, 1+mu
forward, 5+mu backward.  The network N is two linear layers, 1 -> 4 -> 1
channels.  Loss over pairs (r, e): sum ||N(r) - e||^2 / ||e||^2.

Gradients are Wirtinger derivatives G = dL/d conj(W); the derivatives with
respect to the real and imaginary parts of W are 2 Re G and 2 Im G.
Fields: (C, Lt, Lz, Ly, Lx, 4, 3) complex128.  Weights: (C_out, C_in, 9, 4, 4).
"""
import numpy as np

from .lattice import shift


def transport(U, psi, d, antiperiodic_t=True):
    """(T_d psi)(x) for one field psi of shape (Lt, Lz, Ly, Lx, 4, 3)."""
    if d == 0:
        return psi
    mu = (d - 1) % 4
    if d <= 4:
        return np.einsum("...ab,...sb->...sa", U[..., mu, :, :], shift(psi, mu, +1, antiperiodic_t))
    ub = shift(U[..., mu, :, :], mu, -1, False)
    return np.einsum("...ba,...sb->...sa", np.conj(ub), shift(psi, mu, -1, antiperiodic_t))


REVERSE = [0, 5, 6, 7, 8, 1, 2, 3, 4]   # T_d^dag = T_{REVERSE[d]}


def layer(U, W, psi, antiperiodic_t=True):
    """One PT-conv layer: W (C_out, C_in, 9, 4, 4), psi (C_in, ...) -> (C_out, ...)."""
    cout, cin = W.shape[:2]
    out = np.zeros((cout,) + psi.shape[1:], dtype=np.complex128)
    for b in range(cin):
        for d in range(9):
            phi = transport(U, psi[b], d, antiperiodic_t)
            for a in range(cout):
                out[a] += np.einsum("st,...tc->...sc", W[a, b, d], phi)
    return out


def layer_adjoint(U, W, g, antiperiodic_t=True):
    """L^dag g: sum_a sum_d T_d^dag W_d^{ab dag} g^a, shape (C_in, ...)."""
    cout, cin = W.shape[:2]
    out = np.zeros((cin,) + g.shape[1:], dtype=np.complex128)
    for a in range(cout):
        for d in range(9):
            phi = transport(U, g[a], REVERSE[d], antiperiodic_t)
            for b in range(cin):
                out[b] += np.einsum("ts,...tc->...sc", np.conj(W[a, b, d]), phi)
    return out


def weight_grad(U, psi, g, antiperiodic_t=True):
    """G[a, b, d] = sum_{x, c} g^a(x)[s, c] conj((T_d psi^b)(x)[t, c])."""
    cout, cin = g.shape[0], psi.shape[0]
    G = np.zeros((cout, cin, 9, 4, 4), dtype=np.complex128)
    for b in range(cin):
        for d in range(9):
            phi = transport(U, psi[b], d, antiperiodic_t)
            for a in range(cout):
                G[a, b, d] = np.einsum("xsc,xtc->st", g[a].reshape(-1, 4, 3), np.conj(phi).reshape(-1, 4, 3))
    return G


def network(U, Ws, r, antiperiodic_t=True):
    """N(r) for a list of layer weights; r (Lt,..,4,3) -> same shape."""
    h = r[None]
    for W in Ws:
        h = layer(U, W, h, antiperiodic_t)
    return h[0]


def loss_and_grads(U, Ws, pairs, antiperiodic_t=True):
    """L = sum ||N(r) - e||^2 / ||e||^2 and the Wirtinger gradients per layer."""
    L = 0.0
    grads = [np.zeros_like(W) for W in Ws]
    for r, e in pairs:
        acts = [r[None]]
        for W in Ws:
            acts.append(layer(U, W, acts[-1], antiperiodic_t))
        y = acts[-1][0]
        ne = np.vdot(e, e).real
        L += np.vdot(y - e, y - e).real / ne
        g = ((y - e) / ne)[None]
        for li in range(len(Ws) - 1, -1, -1):
            grads[li] += weight_grad(U, acts[li], g, antiperiodic_t)
            if li > 0:
                g = layer_adjoint(U, Ws[li], g, antiperiodic_t)
    return L, grads


def wilson_weights(kappa):
    """Weights that make one layer the Wilson operator with c_sw = 0:
    W_0 = 1, W_{+mu} = -kappa (1 - gamma_mu), W_{-mu} = -kappa (1 + gamma_mu)."""
    from .gamma import GAMMA, ID4
    W = np.zeros((1, 1, 9, 4, 4), dtype=np.complex128)
    W[0, 0, 0] = ID4
    for mu in range(4):
        W[0, 0, 1 + mu] = -kappa * (ID4 - GAMMA[mu])
        W[0, 0, 5 + mu] = -kappa * (ID4 + GAMMA[mu])
    return W
