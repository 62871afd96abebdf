"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This module draws random numbers and turns them into input fields; it holds
none of the solver's arithmetic (no Dirac operator, no multigrid step).  It is
the single place both sides of a parity test take their inputs from.

Random numbers
--------------
SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) used in counter mode: the n-th 64-bit word of a
stream with key ``k`` is ``mix64(k + (n + 1) * 0x9E3779B97F4A7C15)``, where
``mix64`` is the published SplitMix64 finaliser.  The key of a stream is
``mix64(seed * 0x9E3779B97F4A7C15 + stream)``.  A word becomes a double in
(0, 1] as ``((w >> 11) + 1) * 2**-53``.  Normal deviates come from the
Box-Muller transform, one pair per two consecutive words: normal 2j is
``sqrt(-2 ln u_{2j}) cos(2 pi u_{2j+1})`` and normal 2j+1 the same with sin.

Draw order (fixes every value): canonical site index (x fastest, then y, z,
t) -> direction mu (x, y, z, t) -> matrix entry (row-major) -> (re, im).

Gauge links (the synthetic stand-in for the paper's JLDG ensembles A-C):
``U_mu(x) = exp(i eps H)``, ``H = (A + A^dag)/2 - tr(.)/3``, with A a 3x3
complex matrix whose real and imaginary parts are iid N(0, 1).  The
exponential is evaluated through the Hermitian eigendecomposition of H, so U
is unitary with det U = 1 to rounding.

Array shapes (all complex128, canonical order):
  gauge   (Lt, Lz, Ly, Lx, 4, 3, 3)   [site][mu][row][col]
  spinor  (Lt, Lz, Ly, Lx, 4, 3)      [site][spin][colour]
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream identifiers (one stream per kind of input, per seed)
STREAM_GAUGE = 1
STREAM_RHS = 2
STREAM_TESTVEC = 3
STREAM_GAUGE_XFORM = 4
STREAM_MISC = 5
STREAM_NN = 6


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        k = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GOLDEN + np.uint64(stream)
    return _mix64(np.array([k], dtype=np.uint64))[0]


def words(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """64-bit words ``start .. start+count-1`` of the (seed, stream) stream."""
    key = stream_key(seed, stream)
    n = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = key + n * _GOLDEN
    return _mix64(z)


def uniform(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Doubles in (0, 1]."""
    w = words(seed, stream, start, count)
    return ((w >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def normal(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """``count`` N(0,1) deviates, normals ``start .. start+count-1`` of the stream."""
    first_pair = start // 2
    last_pair = (start + count + 1) // 2
    npairs = last_pair - first_pair
    u = uniform(seed, stream, 2 * first_pair, 2 * npairs).reshape(npairs, 2)
    rad = np.sqrt(-2.0 * np.log(u[:, 0]))
    ang = 2.0 * np.pi * u[:, 1]
    out = np.empty((npairs, 2))
    out[:, 0] = rad * np.cos(ang)
    out[:, 1] = rad * np.sin(ang)
    out = out.reshape(-1)
    off = start - 2 * first_pair
    return out[off:off + count]


def complex_normal(seed: int, stream: int, shape, start: int = 0) -> np.ndarray:
    """Complex array with iid N(0,1) real and imaginary parts (re drawn before im)."""
    n = int(np.prod(shape))
    r = normal(seed, stream, 2 * n, 2 * start).reshape(n, 2)
    return (r[:, 0] + 1j * r[:, 1]).reshape(shape)


def lattice_shape(dims):
    """dims = (Lx, Ly, Lz, Lt) -> numpy shape (Lt, Lz, Ly, Lx)."""
    lx, ly, lz, lt = (int(d) for d in dims)
    return (lt, lz, ly, lx)


def _expi_hermitian(h: np.ndarray, eps: float, chunk: int = 1 << 20) -> np.ndarray:
    """exp(i eps h) for a stack of Hermitian 3x3 matrices via eigendecomposition."""
    out = np.empty_like(h)
    for s in range(0, h.shape[0], chunk):
        w, q = np.linalg.eigh(h[s:s + chunk])
        out[s:s + chunk] = np.einsum("nab,nb,ncb->nac", q, np.exp(1j * eps * w), q.conj())
    return out


def su3_from_normals(a: np.ndarray, eps: float) -> np.ndarray:
    """A stack (n,3,3) of complex Gaussian matrices -> exp(i eps H), H traceless Hermitian."""
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1).real / 3.0
    h = h - tr[:, None, None] * np.eye(3)
    return _expi_hermitian(h, eps)


def gauge_field(dims, eps: float, seed: int, chunk_sites: int = 1 << 18) -> np.ndarray:
    """Synthetic SU(3) gauge field, shape (Lt, Lz, Ly, Lx, 4, 3, 3)."""
    shp = lattice_shape(dims)
    vol = int(np.prod(shp))
    out = np.empty((vol, 4, 3, 3), dtype=np.complex128)
    for s in range(0, vol, chunk_sites):
        e = min(vol, s + chunk_sites)
        nmat = (e - s) * 4
        a = complex_normal(seed, STREAM_GAUGE, (nmat, 3, 3), start=s * 4 * 9)
        out[s:e] = su3_from_normals(a, eps).reshape(e - s, 4, 3, 3)
    return out.reshape(shp + (4, 3, 3))


def unit_gauge(dims) -> np.ndarray:
    shp = lattice_shape(dims)
    u = np.zeros(shp + (4, 3, 3), dtype=np.complex128)
    u[...] = np.eye(3)
    return u


def gaussian_spinor(dims, seed: int, stream: int = STREAM_RHS, index: int = 0) -> np.ndarray:
    """Complex Gaussian spinor field; ``index`` selects the index-th field of the stream."""
    shp = lattice_shape(dims)
    n = int(np.prod(shp)) * 12
    return complex_normal(seed, stream, shp + (4, 3), start=index * n)


def rhs(dims, seed: int, index: int = 0) -> np.ndarray:
    """Right-hand side: complex Gaussian, stream of seed + 1000."""
    return gaussian_spinor(dims, seed + 1000, STREAM_RHS, index)


def test_vectors(dims, seed: int, nvec: int) -> np.ndarray:
    """Initial random test vectors for the multigrid setup: (nvec, Lt, Lz, Ly, Lx, 4, 3)."""
    return np.stack([gaussian_spinor(dims, seed + 2000, STREAM_TESTVEC, i) for i in range(nvec)])


def coarse_test_vectors(cdims, seed: int, nvec: int, ndof: int, level: int = 1) -> np.ndarray:
    """Initial random test vectors of coarse level ``level`` (three or more
    grids): complex Gaussian, stream of seed + 2000 + 1000 * level,
    shape (nvec, Lt, Lz, Ly, Lx, ndof)."""
    shp = lattice_shape(cdims)
    return complex_normal(seed + 2000 + 1000 * level, STREAM_TESTVEC, (nvec,) + shp + (ndof,))


def point_source(dims, spin: int, colour: int, site=(0, 0, 0, 0)) -> np.ndarray:
    """Point source delta_{x,site} delta_{s,spin} delta_{c,colour}; site = (x, y, z, t)."""
    shp = lattice_shape(dims)
    b = np.zeros(shp + (4, 3), dtype=np.complex128)
    x, y, z, t = site
    b[t, z, y, x, spin, colour] = 1.0
    return b


def gauge_transform(dims, seed: int) -> np.ndarray:
    """Random SU(3) matrix per site, shape (Lt, Lz, Ly, Lx, 3, 3)."""
    shp = lattice_shape(dims)
    vol = int(np.prod(shp))
    a = complex_normal(seed, STREAM_GAUGE_XFORM, (vol, 3, 3))
    return su3_from_normals(a, 1.0).reshape(shp + (3, 3))


# --- flattening helpers (layout only) -------------------------------------

def to_interleaved(a: np.ndarray) -> np.ndarray:
    """complex128 array -> float64 array with a trailing (re, im) axis, C-contiguous."""
    return np.ascontiguousarray(np.stack([a.real, a.imag], axis=-1))


def from_interleaved(a: np.ndarray) -> np.ndarray:
    a = np.asarray(a, dtype=np.float64)
    return a[..., 0] + 1j * a[..., 1]
