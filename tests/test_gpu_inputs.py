"""The device-side input generator (amg_gauge_random, amg_random_normal)
against the host definition in lqcd_inputs.

Both sides implement the same counter-based SplitMix64 stream, Box-Muller
transform and exp(i eps H) link construction.  The integer part is exact; the
doubles differ only by the rounding of ln, sqrt, cos and sin (CUDA's and
numpy's each within a few ulp) and of the 3x3 exponential (eigenvalue
interpolation on the device, LAPACK eigendecomposition on the host), so
values agree to a few 1e-15 in absolute terms: the tolerance is 1e-13."""
import numpy as np
import pytest

import lqcd_inputs as li
from gpu_util import capi, to_dev, from_dev, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims,eps,seed", [((4, 4, 4, 4), 0.3, 1), ((6, 4, 8, 10), 0.6, 7), ((8, 8, 8, 16), 0.5, 4)])
def test_gauge_random_matches_host_definition(dims, eps, seed):
    c = capi()
    lat = c.amg_lattice_create(dims, True)
    g = c.amg_gauge_random(lat, eps, seed)
    V = int(np.prod(dims))
    got = c.amg_gauge_get(g, V)
    U = got[..., 0] + 1j * got[..., 1]
    ref = li.gauge_field(dims, eps, seed).reshape(V, 4, 3, 3)
    assert np.abs(U - ref).max() < 1e-13
    # unitary with unit determinant
    assert np.abs(np.einsum("nmji,nmjk->nmik", U.conj(), U) - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-13
    c.amg_gauge_destroy(g)
    c.amg_lattice_destroy(lat)


def test_gauge_random_gives_the_same_operator():
    import torch
    c = capi()
    dims = (8, 8, 8, 8)
    lat = c.amg_lattice_create(dims, True)
    g1 = c.amg_gauge_random(lat, 0.6, 2)
    g2 = c.amg_gauge_create(lat, li.to_interleaved(li.gauge_field(dims, 0.6, 2)))
    d1, d2 = c.amg_dirac_create(g1, 0.13, 1.0), c.amg_dirac_create(g2, 0.13, 1.0)
    x = to_dev(li.rhs(dims, 2))
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    c.amg_apply_D(d1, x, y1, 1, c.AMG_F64)
    c.amg_apply_D(d2, x, y2, 1, c.AMG_F64)
    shape = li.lattice_shape(dims) + (12,)
    assert rel(from_dev(y1, shape), from_dev(y2, shape)) < 1e-13
    for d in (d1, d2):
        c.amg_dirac_destroy(d)
    for g in (g1, g2):
        c.amg_gauge_destroy(g)
    c.amg_lattice_destroy(lat)


@pytest.mark.parametrize("seed,stream,start,count", [(1002, 2, 0, 3072), (2004, 3, 12 * 4096 * 5, 12 * 4096),
                                                     (7, 5, 1, 1001), (2 ** 40 + 3, 3, 2 ** 33 + 17, 256)])
def test_random_normal_matches_host_definition(seed, stream, start, count):
    import torch
    c = capi()
    out = torch.full((2 * count,), float("nan"), dtype=torch.float64, device="cuda")
    c.amg_random_normal(seed, stream, start, count, out)
    got = out.cpu().numpy().reshape(count, 2)
    ref = li.complex_normal(seed, stream, (count,), start=start)
    assert np.abs(got[:, 0] - ref.real).max() < 1e-13
    assert np.abs(got[:, 1] - ref.imag).max() < 1e-13


def test_setup_from_device_vectors_matches_host_vectors():
    # amg_setup copies its initial vectors with cudaMemcpyDefault: device vectors drawn
    # by amg_random_normal give the hierarchy that the host-drawn vectors give
    import torch
    from gpu_util import Field
    c = capi()
    dims, nvec = (8, 8, 8, 8), 8
    f = Field(dims, 0.6, 2, 0.130, 1.0)
    p = c.amg_params_default()
    p.nvec[0] = nvec
    p.n_init, p.n_adapt = 1, 1
    p.prec_smoother = p.prec_coarsest = c.AMG_F64   # FP64: input differences of 1e-16 stay small
    V = f.V
    dev = torch.empty(nvec * V * 24, dtype=torch.float64, device="cuda")
    c.amg_random_normal(2 + 2000, li.STREAM_TESTVEC, 0, nvec * V * 12, dev)
    h1 = c.amg_setup(f.d, p, [dev])
    h2 = c.amg_setup(f.d, p, [li.to_interleaved(li.test_vectors(dims, 2, nvec))])
    v1, v2 = c.amg_get_vectors(h1, 0, nvec, V), c.amg_get_vectors(h2, 0, nvec, V)
    assert rel(v1, v2) < 1e-8
    c.amg_hierarchy_destroy(h1)
    c.amg_hierarchy_destroy(h2)
    f.close()
