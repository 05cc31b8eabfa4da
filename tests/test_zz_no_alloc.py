"""The allocation-free inner product (tt_dot_noalloc) through the C-ABI,
against the library's own tt_vec_dot and the oracle's TT contraction.

tt_dot_noalloc serves callers that cannot allocate device memory where they
need the result (a fixed memory budget, or a loop where cudaMalloc/cudaFree
would stall the device); its scratch is one fixed device array shared by all
calls.  This file is collected last so that a run stopping at the first
failure has run every other test first; it also passes alone in a fresh
process.
"""
import numpy as np
import pytest

import keig_inputs as ki
from oracle import ttref as R

pytestmark = pytest.mark.gpu

K = pytest.importorskip("paper_2309_03347_gb300")


def _dev_flat(cores):
    import torch
    return torch.from_numpy(np.concatenate([c.ravel() for c in cores])).to("cuda", torch.float64).contiguous()


def _scale(xc, yc):
    return np.sqrt(R.dot(xc, xc) * R.dot(yc, yc))


CASES = [
    ([4, 8, 10, 2, 2, 2, 2, 2, 2], [1, 3, 8, 12, 16, 16, 8, 4, 2, 1], [1, 2, 9, 20, 24, 12, 6, 5, 2, 1], 101),
    ([4, 8, 10, 2, 2, 2, 2, 2, 2], [1, 4, 16, 40, 64, 64, 32, 16, 4, 1], [1, 4, 32, 80, 96, 48, 24, 8, 2, 1], 202),
    # at the limits that size the scratch: bond ranks 128 around a mode of 64
    ([2, 64, 64, 2], [1, 2, 128, 128, 1], [1, 2, 128, 128, 1], 303),
]


def test_noalloc_dot_matches_tt_vec_dot_and_oracle_twice(ctx):
    import torch
    for modes, rx, ry, seed in CASES:  # calls in a row; the scratch keeps the previous call's contents
        xc = ki.random_cores(modes, rx, seed)
        yc = ki.random_cores(modes, ry, seed + 1)
        ref_lib = K.tt_vec_create(ctx, xc).dot(K.tt_vec_create(ctx, yc))
        ref_oracle = R.dot(xc, yc)
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        K.tt_dot_noalloc(_dev_flat(xc), rx, _dev_flat(yc), ry, modes, out)
        got = float(out.item())
        scale = _scale(xc, yc)
        assert abs(got - ref_oracle) <= 1e-12 * scale, (got, ref_oracle)
        assert abs(got - ref_lib) <= 1e-12 * scale, (got, ref_lib)


def test_noalloc_dot_rejects_sizes_above_limits(ctx):
    import torch
    modes = [2, 2]
    x = torch.zeros(2 * 129 * 2, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(K.KeigError) as e:
        K.tt_dot_noalloc(x, [1, 129, 1], x, [1, 129, 1], modes, out)
    assert e.value.code == K.TT_EINVAL and "128" in str(e.value)
    y = torch.zeros(65, dtype=torch.float64, device="cuda")
    with pytest.raises(K.KeigError) as e:
        K.tt_dot_noalloc(y, [1, 1], y, [1, 1], [65], out)
    assert e.value.code == K.TT_EINVAL and "64" in str(e.value)


def test_noalloc_dot_rejects_inconsistent_sizes_before_launch(ctx):
    import torch
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    x = torch.zeros(2 * 3 * 2, dtype=torch.float64, device="cuda")
    with pytest.raises(K.KeigError) as e:  # one rank too few for two cores
        K.tt_dot_noalloc(x, [1, 3], x, [1, 3, 1], [2, 2], out)
    assert e.value.code == K.TT_EINVAL and "len(n) + 1" in str(e.value)
    with pytest.raises(K.KeigError) as e:  # the tensor is shorter than the ranks and modes say
        K.tt_dot_noalloc(x[:-1].contiguous(), [1, 3, 1], x, [1, 3, 1], [2, 2], out)
    assert e.value.code == K.TT_EINVAL and "need" in str(e.value)
