"""Dirac matrices in the chiral basis (reading C2).

The paper fixes only gamma5 = -gamma1 gamma2 gamma3 gamma4 (Eq. 2).  We take
gamma_k = [[0, i sigma_k], [-i sigma_k, 0]] (k = 1, 2, 3) and
gamma_4 = [[0, 1], [1, 0]], for which gamma5 = diag(1, 1, -1, -1): the chiral
projectors P+- = (1 +- gamma5)/2 of the footnote in Sec. 3 select spins {0, 1}
and {2, 3}.
"""
import numpy as np

SIGMA = [
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
]
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)


def _block(a, b, c, d):
    return np.block([[a, b], [c, d]])


# GAMMA[mu] for mu = 0..3 <-> the paper's gamma_1..gamma_4 (x, y, z, t)
GAMMA = [_block(_Z2, 1j * s, -1j * s, _Z2) for s in SIGMA] + [_block(_Z2, _I2, _I2, _Z2)]
GAMMA5 = -GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ID4 = np.eye(4, dtype=np.complex128)


def sigma_munu(mu: int, nu: int) -> np.ndarray:
    """sigma_{mu nu} = (1/2i)[gamma_mu, gamma_nu] (reading C1); Hermitian."""
    g = GAMMA
    return (g[mu] @ g[nu] - g[nu] @ g[mu]) / 2j
