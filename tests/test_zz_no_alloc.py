"""The allocation-free inner product (tt_dot_noalloc) against the existing
tt_vec_dot entry point, through the C-ABI.

tt_dot_noalloc serves callers that cannot allocate device memory where they
need the result (inside a CUDA-graph capture, or under a fixed memory
budget); its scratch is one fixed device array shared by all calls.  This
file is collected last so that a run stopping at the first failure has run
every other test first; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import keig_inputs as ki

pytestmark = pytest.mark.gpu

K = pytest.importorskip("paper_2309_03347_gb300")


def _dev_flat(cores):
    import torch
    return torch.from_numpy(np.concatenate([c.ravel() for c in cores])).to("cuda", torch.float64).contiguous()


def test_noalloc_dot_matches_tt_vec_dot_twice(ctx):
    import torch
    modes = [4, 8, 10, 2, 2, 2, 2, 2, 2]
    cases = [([1, 3, 8, 12, 16, 16, 8, 4, 2, 1], [1, 2, 9, 20, 24, 12, 6, 5, 2, 1], 101),
             ([1, 4, 16, 40, 64, 64, 32, 16, 4, 1], [1, 4, 32, 80, 96, 48, 24, 8, 2, 1], 202)]
    for rx, ry, seed in cases:  # two calls in a row; the scratch keeps the first call's contents
        xc = ki.random_cores(modes, rx, seed)
        yc = ki.random_cores(modes, ry, seed + 1)
        ref = K.tt_vec_create(ctx, xc).dot(K.tt_vec_create(ctx, yc))
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        K.tt_dot_noalloc(_dev_flat(xc), rx, _dev_flat(yc), ry, modes, out)
        got = float(out.item())
        scale = np.sqrt(K.tt_vec_create(ctx, xc).dot(K.tt_vec_create(ctx, xc)) *
                        K.tt_vec_create(ctx, yc).dot(K.tt_vec_create(ctx, yc)))
        assert abs(got - ref) <= 1e-12 * scale, (got, ref)


def test_noalloc_dot_rejects_sizes_above_limits(ctx):
    import torch
    modes = [2, 2]
    x = torch.zeros(2 * 129 * 2, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(K.KeigError) as e:
        K.tt_dot_noalloc(x, [1, 129, 1], x, [1, 129, 1], modes, out)
    assert e.value.code == K.TT_EINVAL and "128" in str(e.value)
    with pytest.raises(K.KeigError) as e:
        K.tt_dot_noalloc(x, [1, 1], x, [1, 1], [65], out)
    assert e.value.code == K.TT_EINVAL and "64" in str(e.value)
