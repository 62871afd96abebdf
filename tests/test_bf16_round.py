"""The bfloat16 rounding helper of the GPU tests (used to form the operator the
BF16 coarse stencil applies) on values whose rounding is fixed by hand, and
against PyTorch's CPU float32 -> bfloat16 conversion."""
import numpy as np

from gpu_util import bf16_round


def test_hand_values():
    ulp = 2.0 ** -7            # spacing of bfloat16 in [1, 2)
    cases = {
        1.0: 1.0,
        1.0 + ulp / 2: 1.0,               # tie, 1.0 is even
        1.0 + 3 * ulp / 2: 1.0 + 2 * ulp,  # tie, rounds up to the even neighbour
        1.0 + ulp / 2 + 2.0 ** -20: 1.0 + ulp,
        -(1.0 + ulp * 0.49): -1.0,
        3.0e-3: 197 * 2.0 ** -16,          # 1.536 * 2^-9: mantissa 196.6 rounds to 197
        0.0: 0.0,
    }
    for x, want in cases.items():
        assert bf16_round(np.array([x]))[0] == want, x


def test_matches_torch_cpu():
    import torch
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(100000) * np.exp(rng.uniform(-20, 20, 100000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(bf16_round(x), ref)
