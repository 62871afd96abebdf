"""Pins of the oracle's Wilson-clover operator (Eq. 1, Eq. 2, reading C1-C4)."""
import numpy as np
import pytest

import lqcd_inputs as li
from oracle import dirac
from oracle.gamma import GAMMA, GAMMA5
from oracle.lattice import face_mask


def _field(dims, seed, idx=0):
    return li.rhs(dims, seed, idx).reshape(li.lattice_shape(dims) + (12,))


def test_gamma_algebra():
    for mu in range(4):
        assert np.allclose(GAMMA[mu] @ GAMMA[mu], np.eye(4))
        assert np.allclose(GAMMA[mu], GAMMA[mu].conj().T)
        for nu in range(mu + 1, 4):
            assert np.allclose(GAMMA[mu] @ GAMMA[nu] + GAMMA[nu] @ GAMMA[mu], 0)
    # Eq. 2 and reading C2: gamma5 = -g1 g2 g3 g4 is diag(1, 1, -1, -1)
    assert np.allclose(GAMMA5, np.diag([1, 1, -1, -1]))


@pytest.mark.parametrize("dims,ap", [((4, 4, 4, 4), True), ((2, 4, 6, 4), False), ((4, 2, 2, 6), True)])
def test_apply_matches_entrywise_assembly(dims, ap):
    U = li.gauge_field(dims, 0.5, 9)
    op = dirac.WilsonClover(U, 0.13, 1.3, ap)
    S = dirac.sparse_matrix(U, 0.13, 1.3, ap)
    psi = _field(dims, 3)
    assert np.abs(S @ psi.reshape(-1) - op.apply(psi).reshape(-1)).max() < 1e-13


def test_gamma5_hermiticity_random_vectors():
    dims = (4, 4, 4, 4)
    op = dirac.WilsonClover(li.gauge_field(dims, 0.6, 2), 0.13, 1.0)
    psi, chi = _field(dims, 1), _field(dims, 2)
    lhs = np.vdot(chi, op.gamma5(op.apply(op.gamma5(psi))))
    rhs = np.vdot(op.apply(chi), psi)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_gamma5_hermiticity_dense_and_conjugate_pairs():
    dims = (2, 2, 2, 2)
    D = dirac.dense_matrix(li.gauge_field(dims, 0.6, 5), 0.13, 1.0)
    g5 = np.kron(np.eye(16), np.kron(np.diag([1, 1, -1, -1]), np.eye(3)))
    assert np.abs(g5 @ D @ g5 - D.conj().T).max() < 1e-14
    ev = np.linalg.eigvals(D)
    # eigenvalues of a gamma5-hermitian matrix come in complex-conjugate pairs
    d = np.abs(ev.conj()[:, None] - ev[None, :]).min(axis=1)
    assert d.max() < 1e-10


def test_gauge_covariance():
    dims = (4, 4, 2, 4)
    U = li.gauge_field(dims, 0.6, 4)
    om = li.gauge_transform(dims, 8)
    # U'_mu(x) = Om(x) U_mu(x) Om(x+mu)^dag
    from oracle.lattice import shift
    Up = np.empty_like(U)
    for mu in range(4):
        Up[..., mu, :, :] = om @ U[..., mu, :, :] @ np.conj(np.swapaxes(shift(om, mu, +1), -1, -2))
    psi = _field(dims, 6)
    rot = lambda f: np.einsum("...ab,...sb->...sa", om, f.reshape(f.shape[:4] + (4, 3))).reshape(f.shape)
    a = dirac.WilsonClover(Up, 0.125, 1.7).apply(rot(psi))
    b = rot(dirac.WilsonClover(U, 0.125, 1.7).apply(psi))
    assert np.abs(a - b).max() < 1e-13


@pytest.mark.parametrize("ap", [True, False])
def test_free_field_spectrum(ap):
    dims = (2, 2, 2, 2)
    kappa = 0.124
    ev = np.linalg.eigvals(dirac.dense_matrix(li.unit_gauge(dims), kappa, 1.0, ap))
    ref = dirac.free_spectrum(dims, kappa, ap)
    key = lambda z: np.sort_complex(np.round(z, 9))
    assert np.abs(key(ev) - key(ref)).max() < 1e-9


def test_free_field_plane_wave():
    dims = (4, 4, 4, 6)
    kappa = 0.13
    op = dirac.WilsonClover(li.unit_gauge(dims), kappa, 1.0, True)
    n = (1, 3, 2, 4)
    p = [2 * np.pi * n[0] / 4, 2 * np.pi * n[1] / 4, 2 * np.pi * n[2] / 4, (2 * n[3] + 1) * np.pi / 6]
    lt, lz, ly, lx = li.lattice_shape(dims)
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    u = np.arange(12) + 1j * np.arange(12)[::-1]
    psi = phase[..., None] * u
    Dp = (1 - 2 * kappa * sum(np.cos(q) for q in p)) * np.eye(12)
    for mu in range(4):
        Dp = Dp + 2j * kappa * np.sin(p[mu]) * np.kron(GAMMA[mu], np.eye(3))
    assert np.abs(op.apply(psi) - phase[..., None] * (Dp @ u)).max() < 1e-13


def test_clover_structure_and_limits():
    dims = (4, 4, 4, 4)
    U = li.gauge_field(dims, 0.6, 2)
    op = dirac.WilsonClover(U, 0.13, 1.0)
    F = op.F
    assert np.abs(F - np.conj(np.swapaxes(F, -1, -2))).max() < 1e-15        # Hermitian
    assert np.abs(F[..., :6, 6:]).max() == 0 and np.abs(F[..., 6:, :6]).max() == 0  # chiral blocks
    assert np.abs(np.trace(F, axis1=-2, axis2=-1)).max() < 1e-14
    psi = _field(dims, 1)
    # kappa = 0: D = 1 + F = 1 exactly (F is proportional to kappa)
    assert np.allclose(dirac.WilsonClover(U, 0.0, 1.0).apply(psi), psi, atol=0)
    # c_sw = 0: pure Wilson, D = 1 - kappa * hops
    w = dirac.WilsonClover(U, 0.13, 0.0)
    assert np.abs(w.F).max() == 0
    hops = sum(w.hop(psi, mu, s) for mu in range(4) for s in (1, -1))
    assert np.abs(w.apply(psi) - psi - hops).max() < 1e-14


def test_clover_constant_abelian_field():
    # colour-diagonal constant field strength in the x-y plane:
    # U_x(x) = diag(exp(i th_a y)), U_y = U_z = U_t = 1, th_a Ly in 2 pi Z, sum th_a = 0.
    # Every leaf of the x-y clover equals diag(exp(-i th_a)), so
    # F_xy = -diag(sin th_a) (traceless part), all other planes vanish.
    dims = (4, 6, 2, 2)
    ly = 6
    th = np.array([2, -1, -1]) * 2 * np.pi / ly
    U = li.unit_gauge(dims)
    lt, lz, lyy, lx = li.lattice_shape(dims)
    y = np.arange(ly)[None, None, :, None]
    for a in range(3):
        U[..., 0, a, a] = np.exp(1j * th[a] * y)
    fxy = dirac.field_strength(U, 0, 1)
    expect = -np.sin(th)
    expect = expect - expect.mean()
    assert np.abs(fxy - np.diag(expect)).max() < 1e-14
    for (mu, nu) in [(0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]:
        assert np.abs(dirac.field_strength(U, mu, nu)).max() < 1e-14
    kappa, csw = 0.12, 1.5
    from oracle.gamma import sigma_munu
    F = dirac.clover_field(U, kappa, csw)
    ref = -kappa * csw * np.kron(sigma_munu(0, 1), np.diag(expect))
    assert np.abs(F - ref).max() < 1e-14


def test_dsap_equals_d_with_cut_links():
    dims = (4, 4, 4, 4)
    block = (2, 2, 2, 2)
    U = li.gauge_field(dims, 0.6, 2)
    op = dirac.WilsonClover(U, 0.13, 1.0)
    Ucut = U.copy()
    for mu in range(4):
        m = face_mask(U.shape[:4], block, mu, +1)
        Ucut[..., mu, :, :] *= (~m)[..., None, None]
    cut = dirac.WilsonClover(Ucut, 0.13, 1.0)
    cut.F, cut.A = op.F, op.A     # clover built from the original links
    psi = _field(dims, 4)
    assert np.abs(op.apply_sap(psi, block) - cut.apply(psi)).max() < 1e-14
    # D = D_SAP + the face hops
    full = op.apply_sap(psi, block) + sum(op.block_hop(psi, mu, s, block) for mu in range(4) for s in (1, -1))
    assert np.abs(full - op.apply(psi)).max() < 1e-14


@pytest.mark.parametrize("dims, eps, seed, kappa, ap", [((4, 4, 4, 4), 0.3, 1, 0.124, True),
                                                        ((4, 6, 4, 8), 0.6, 7, 0.130, True),
                                                        ((6, 4, 4, 4), 0.6, 2, 0.130, False)])
def test_apply_at_matches_whole_lattice(dims, eps, seed, kappa, ap):
    # the per-site evaluation (used to sample large lattices) against the whole-lattice
    # operator at every site, including the t-wrap sites and periodic t
    U = li.gauge_field(dims, eps, seed)
    op = dirac.WilsonClover(U, kappa, 1.0, ap)
    psi = _field(dims, 4)
    ref = op.apply(psi).reshape(-1, 12)
    sites = [tuple(s) for s in np.ndindex(op.shape4)]
    got = dirac.apply_at(U, kappa, 1.0, psi, sites, ap)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
