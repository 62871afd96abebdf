"""Helpers for the GPU parity tests: build the library, move canonical fields
between numpy and the device, relative errors."""
import numpy as np

import lqcd_inputs as li


def capi():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2111_05012_gb300 import capi as c
    return c


def to_dev(a, dtype="float64"):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(li.to_interleaved(a)).reshape(-1))
    return t.to(dtype=getattr(torch, dtype)).cuda()


def from_dev(t, shape):
    return li.from_interleaved(t.double().cpu().numpy().reshape(shape + (2,)))


def rel(a, b):
    return float(np.linalg.norm((a - b).reshape(-1)) / np.linalg.norm(b.reshape(-1)))


class Field:
    """Lattice + gauge + Dirac handles for one synthetic configuration."""

    def __init__(self, dims, eps, seed, kappa, csw, antiperiodic=True):
        self.c = capi()
        self.dims = dims
        self.shape4 = li.lattice_shape(dims)
        self.V = int(np.prod(self.shape4))
        self.U = li.gauge_field(dims, eps, seed)
        self.kappa, self.csw = kappa, csw
        self.lat = self.c.amg_lattice_create(dims, antiperiodic)
        self.gauge = self.c.amg_gauge_create(self.lat, li.to_interleaved(self.U))
        self.d = self.c.amg_dirac_create(self.gauge, kappa, csw)

    def close(self):
        self.c.amg_dirac_destroy(self.d)
        self.c.amg_gauge_destroy(self.gauge)
        self.c.amg_lattice_destroy(self.lat)


def bf16_round(a):
    """Round FP32 values to the nearest bfloat16 (ties to even), kept as float64:
    keep the top 16 bits of the FP32 word after adding half an ulp of the
    16-bit truncation (plus one when the kept part is odd)."""
    x = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (x + 0x7FFF + ((x >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
