"""Lattice geometry for the oracle (readings C3, C4, C10).

Arrays are indexed (t, z, y, x, ...); direction mu = 0, 1, 2, 3 is x, y, z, t.
Periodic boundary in x, y, z; the fermion hop across the t boundary carries a
factor -1 when ``antiperiodic_t`` is set (C3).  Gauge links are periodic.
"""
import numpy as np

AXIS = (3, 2, 1, 0)  # numpy axis of direction mu


def shift(f: np.ndarray, mu: int, sign: int, antiperiodic_t: bool = False) -> np.ndarray:
    """g(x) = f(x + sign * mu_hat), with the boundary phase on the t wrap."""
    ax = AXIS[mu]
    g = np.roll(f, -sign, axis=ax)
    if mu == 3 and antiperiodic_t:
        idx = f.shape[0] - 1 if sign > 0 else 0
        g[idx] = -g[idx]
    return g


def coords(shape4):
    """Coordinate arrays (x, y, z, t) broadcast over a (Lt, Lz, Ly, Lx) lattice."""
    lt, lz, ly, lx = shape4
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return (x, y, z, t)


def dims_of(shape4):
    lt, lz, ly, lx = shape4
    return (lx, ly, lz, lt)


def check_blocking(dims, block):
    """Blocks must tile the lattice with at least two blocks per direction."""
    for L, b in zip(dims, block):
        if L % b != 0 or L // b < 2:
            raise ValueError(f"block {block} does not tile lattice {dims} with >= 2 blocks per direction")


def face_mask(shape4, block, mu: int, sign: int) -> np.ndarray:
    """True at sites x whose neighbour x + sign*mu_hat lies in another block."""
    c = coords(shape4)[mu]
    b = block[mu]
    return (c % b == b - 1) if sign > 0 else (c % b == 0)


def block_colour(shape4, block) -> np.ndarray:
    """Domain colour (sum_mu X_mu) mod 2 of the block holding each site (C10)."""
    c = coords(shape4)
    s = sum(c[mu] // block[mu] for mu in range(4))
    return s % 2


def to_blocks(f: np.ndarray, block) -> np.ndarray:
    """(Lt,Lz,Ly,Lx,...) -> (Ct,Cz,Cy,Cx, bt,bz,by,bx, ...)."""
    lt, lz, ly, lx = f.shape[:4]
    bx, by, bz, bt = block
    rest = f.shape[4:]
    g = f.reshape((lt // bt, bt, lz // bz, bz, ly // by, by, lx // bx, bx) + rest)
    nr = len(rest)
    return g.transpose((0, 2, 4, 6, 1, 3, 5, 7) + tuple(range(8, 8 + nr)))


def from_blocks(g: np.ndarray) -> np.ndarray:
    """Inverse of to_blocks."""
    ct, cz, cy, cx, bt, bz, by, bx = g.shape[:8]
    rest = g.shape[8:]
    nr = len(rest)
    f = g.transpose((0, 4, 1, 5, 2, 6, 3, 7) + tuple(range(8, 8 + nr)))
    return f.reshape((ct * bt, cz * bz, cy * by, cx * bx) + rest)


def block_sum(f: np.ndarray, block) -> np.ndarray:
    """Sum of a per-site quantity (Lt,Lz,Ly,Lx) over each block -> (Ct,Cz,Cy,Cx)."""
    return to_blocks(f, block).sum(axis=(4, 5, 6, 7))


def block_broadcast(c: np.ndarray, block) -> np.ndarray:
    """Per-block value (Ct,Cz,Cy,Cx) -> per-site (Lt,Lz,Ly,Lx)."""
    bx, by, bz, bt = block
    return np.repeat(np.repeat(np.repeat(np.repeat(c, bt, 0), bz, 1), by, 2), bx, 3)
