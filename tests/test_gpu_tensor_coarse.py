"""Tensor-core (tcgen05) multi-right-hand-side coarse stencil: bfloat16
operands, FP32 accumulation.  Against the oracle's stencil applied to the
same bfloat16-rounded operator entries and vectors the difference is FP32
accumulation only (relative L2 <= 1e-5); against the exact FP64 operator and
vectors it is bfloat16 rounding (<= 1e-2)."""
import numpy as np
import pytest

import lqcd_inputs as li
from oracle import dirac as odirac, multigrid as omg
from oracle.multigrid import CoarseStencil
from gpu_util import Field, to_dev, from_dev, rel, bf16_round

pytestmark = pytest.mark.gpu

CASES = [
    # dims, eps, seed, kappa, block, nvec  (Nc = 2 nvec = 16, 48, 64)
    ((4, 4, 4, 4), 0.3, 1, 0.124, (2, 2, 2, 2), 8),
    ((8, 8, 8, 8), 0.6, 5, 0.130, (4, 4, 4, 4), 24),
    ((8, 8, 8, 8), 0.6, 6, 0.130, (4, 4, 4, 4), 32),
]


@pytest.fixture(scope="module", params=range(len(CASES)))
def tc(request):
    dims, eps, seed, kappa, block, nvec = CASES[request.param]
    f = Field(dims, eps, seed, kappa, 1.0)
    c = f.c
    p = c.amg_params_default()
    for mu in range(4):
        p.block[0][mu] = block[mu]
    p.nvec[0] = nvec
    p.prec_coarsest = c.AMG_BF16
    v0 = li.test_vectors(dims, seed, nvec)
    f.h = c.amg_setup_from_vectors(f.d, p, [li.to_interleaved(v0)])
    op = odirac.WilsonClover(f.U, kappa, 1.0, True)
    vo = omg.orthonormalise(v0.reshape((nvec,) + f.shape4 + (12,)), block)
    f.exact = omg.coarse_operator(op, vo, block)
    B = c.amg_get_coarse_op(f.h, 1)
    Bq = bf16_round(B).reshape(f.exact.B.shape + (2,))
    f.stored = CoarseStencil(Bq[..., 0] + 1j * Bq[..., 1], nvec)
    f.cdims, f.nc = c.amg_level_info(f.h, 1)
    f.cshape = li.lattice_shape(f.cdims)
    yield f
    c.amg_hierarchy_destroy(f.h)
    f.close()


@pytest.mark.parametrize("nrhs", [1, 5, 12, 16, 21])
def test_tensor_core_stencil(tc, nrhs):
    import torch
    f = tc
    c = f.c
    x = li.complex_normal(90 + nrhs, li.STREAM_MISC, (nrhs,) + f.cshape + (f.nc,))
    xd = to_dev(x, "float32")
    y = torch.zeros_like(xd)
    c.amg_apply_coarse(f.h, 1, xd, y, nrhs, c.AMG_BF16)
    got = from_dev(y, (nrhs,) + f.cshape + (f.nc,))
    xq = bf16_round(li.to_interleaved(from_dev(xd, (nrhs,) + f.cshape + (f.nc,))))
    xq = xq[..., 0] + 1j * xq[..., 1]
    for r in range(nrhs):
        assert rel(got[r], f.stored.apply(xq[r])) < 1e-5
        assert rel(got[r], f.exact.apply(x[r])) < 1e-2


def test_tensor_core_path_needs_a_bfloat16_stencil():
    import torch
    dims = (4, 4, 4, 4)
    f = Field(dims, 0.3, 1, 0.124, 1.0)
    c = f.c
    p = c.amg_params_default()
    for mu in range(4):
        p.block[0][mu] = 2
    p.nvec[0] = 8
    h = c.amg_setup_from_vectors(f.d, p, [li.to_interleaved(li.test_vectors(dims, 1, 8))])   # FP32 stencil
    x = torch.zeros(16 * 16 * 2, dtype=torch.float32, device="cuda")
    with pytest.raises(c.AMGError) as e:
        c.amg_apply_coarse(h, 1, x, torch.zeros_like(x), 1, c.AMG_BF16)
    assert e.value.status == c.AMG_EINVAL
    c.amg_hierarchy_destroy(h)
    f.close()
