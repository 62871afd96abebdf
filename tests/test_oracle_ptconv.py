"""Pins of the oracle's parallel-transport convolution (reading C15)."""
import numpy as np
import pytest

import lqcd_inputs as li
from oracle import dirac, ptconv
from oracle.lattice import shift

DIMS = (4, 4, 2, 4)


def _w(shape, seed):
    return li.complex_normal(seed, li.STREAM_NN, shape) * 0.3


def _field(seed, idx=0):
    return li.rhs(DIMS, seed, idx)


def test_wilson_weights_reproduce_wilson_operator():
    U = li.gauge_field(DIMS, 0.6, 3)
    kappa = 0.13
    psi = _field(1)
    y = ptconv.network(U, [ptconv.wilson_weights(kappa)], psi)
    ref = dirac.WilsonClover(U, kappa, 0.0, True).apply(psi.reshape(psi.shape[:4] + (12,)))
    assert np.abs(y.reshape(ref.shape) - ref).max() < 1e-14


def test_gauge_equivariance():
    U = li.gauge_field(DIMS, 0.6, 4)
    om = li.gauge_transform(DIMS, 9)
    Up = np.empty_like(U)
    for mu in range(4):
        Up[..., mu, :, :] = om @ U[..., mu, :, :] @ np.conj(np.swapaxes(shift(om, mu, +1), -1, -2))
    Ws = [_w((4, 1, 9, 4, 4), 1), _w((1, 4, 9, 4, 4), 2)]
    psi = _field(2)
    rot = lambda f: np.einsum("...ab,...sb->...sa", om, f)
    assert np.abs(ptconv.network(Up, Ws, rot(psi)) - rot(ptconv.network(U, Ws, psi))).max() < 1e-12


def test_adjoint_identity():
    U = li.gauge_field(DIMS, 0.6, 5)
    W = _w((3, 2, 9, 4, 4), 3)
    psi = np.stack([_field(3, i) for i in range(2)])
    chi = np.stack([_field(4, i) for i in range(3)])
    lhs = np.vdot(chi, ptconv.layer(U, W, psi))
    rhs = np.vdot(ptconv.layer_adjoint(U, W, chi), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_gradients_match_finite_differences():
    U = li.gauge_field(DIMS, 0.6, 6)
    Ws = [_w((2, 1, 9, 4, 4), 5), _w((1, 2, 9, 4, 4), 6)]
    pairs = [(_field(7, k), _field(8, k)) for k in range(2)]
    L0, grads = ptconv.loss_and_grads(U, Ws, pairs)
    h = 1e-6
    rng = np.random.default_rng(0)
    for li_ in range(2):
        for _ in range(6):
            idx = tuple(rng.integers(0, n) for n in Ws[li_].shape)
            for part, unit in (("re", 1.0), ("im", 1j)):
                Wp = [w.copy() for w in Ws]
                Wm = [w.copy() for w in Ws]
                Wp[li_][idx] += unit * h
                Wm[li_][idx] -= unit * h
                fd = (ptconv.loss_and_grads(U, Wp, pairs)[0] - ptconv.loss_and_grads(U, Wm, pairs)[0]) / (2 * h)
                G = grads[li_][idx]
                an = 2 * (G.real if part == "re" else G.imag)
                assert abs(fd - an) <= 1e-7 * max(1.0, abs(an))


def test_identity_network_has_zero_loss_on_identity_pairs():
    U = li.gauge_field(DIMS, 0.6, 7)
    W1 = np.zeros((4, 1, 9, 4, 4), dtype=np.complex128)
    W1[0, 0, 0] = np.eye(4)
    W2 = np.zeros((1, 4, 9, 4, 4), dtype=np.complex128)
    W2[0, 0, 0] = np.eye(4)
    e = _field(9)
    L, grads = ptconv.loss_and_grads(U, [W1, W2], [(e, e)])
    assert L < 1e-28 and max(np.abs(g).max() for g in grads) < 1e-14
