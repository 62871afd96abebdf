"""amg_apply_D_noalloc, the allocation-free variant of amg_apply_D for callers
that cannot allocate device memory (its work fields live in a static device
array), must give the same result as amg_apply_D, call after call.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

import lqcd_inputs as li
from gpu_util import Field, to_dev, from_dev, rel

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-6, 2: 3e-3}


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_noalloc_matches_apply_D_two_calls(prec):
    import torch
    dims = (8, 8, 8, 8)
    f = Field(dims, 0.6, 2, 0.130, 1.0)
    c = f.c
    dt = "float64" if prec == 0 else "float32"
    for call in range(2):   # the shared array keeps the previous call's contents
        psi = np.stack([li.rhs(dims, 20 + call, i) for i in range(2)])
        x = to_dev(psi, dt)
        ref = torch.empty_like(x)
        got = torch.full_like(x, float("nan"))
        c.amg_apply_D(f.d, x, ref, 2, prec)
        c.amg_apply_D_noalloc(f.d, x, got, 2, prec)
        torch.cuda.synchronize()
        shape = (2,) + f.shape4 + (12,)
        assert rel(from_dev(got, shape), from_dev(ref, shape)) < TOL[prec]
    f.close()


def test_noalloc_rejects_sizes_beyond_its_array():
    dims = (16, 16, 16, 32)   # 131072 sites: one FP64 field = 24 MiB > 12 MiB
    f = Field(dims, 0.6, 2, 0.130, 1.0)
    c = f.c
    import torch
    x = torch.zeros(f.V * 24, dtype=torch.float64, device="cuda")
    with pytest.raises(c.AMGError) as e:
        c.amg_apply_D_noalloc(f.d, x, x.clone(), 1, c.AMG_F64)
    assert e.value.status == c.AMG_EINVAL
    assert "limit" in c.amg_last_error()
    f.close()
