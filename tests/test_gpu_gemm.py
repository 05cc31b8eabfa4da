"""Direct check of the FP32 contraction GEMMs of the mixed-precision local
solves (keig.h tt_gemm_f32) against an FP64 numpy product, element by
element: the SIMT GEMM, the tcgen05 TF32 three-term split and the tcgen05
BF16 three-term split, on ragged shapes (partial 128 x 64 tiles, K not a
multiple of the stage depth), all four transpose combinations, K long enough
to be split across CTAs, and batches.

Bound per element: |C - C_ref| <= tol * (|op(A)| |op(B)|)_ij, the
rounding-error scale of a dot product; tol is 1e-5 for FP32 SIMT and the
TF32 split (about 21 significant bits per product term) and 1e-4 for the
BF16 split (about 16)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

K = pytest.importorskip("paper_2309_03347_gb300")

SHAPES = [  # (batch, M, N, K)
    (1, 5, 7, 3),
    (1, 130, 70, 45),      # ragged in every dimension
    (3, 200, 129, 97),     # batched, two M tiles, three N tiles
    (1, 64, 40, 4000),     # long K: split across CTAs, partials reduced
    (2, 257, 33, 600),
]
TOL = {0: 1e-5, 1: 1e-5, 2: 1e-4}


def _case(kind, ta, tb, shape, seed):
    import torch
    batch, M, N, Kd = shape
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((batch, Kd, M) if ta else (batch, M, Kd)).astype(np.float32)
    b = rng.standard_normal((batch, N, Kd) if tb else (batch, Kd, N)).astype(np.float32)
    c0 = rng.standard_normal((batch, M, N)).astype(np.float32)
    alpha, beta = 0.75, -0.5
    opa = np.swapaxes(a, 1, 2) if ta else a
    opb = np.swapaxes(b, 1, 2) if tb else b
    ref = alpha * np.matmul(opa.astype(np.float64), opb.astype(np.float64)) + beta * c0.astype(np.float64)
    scale = np.abs(alpha) * np.matmul(np.abs(opa).astype(np.float64), np.abs(opb).astype(np.float64)) \
        + np.abs(beta * c0.astype(np.float64))
    ta_, tb_, tc_ = (torch.from_numpy(x).cuda() for x in (a, b, c0))
    return ta_, tb_, tc_, alpha, beta, ref, scale


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_contraction_gemm_elementwise(ctx, kind):
    seed = 10
    for ta in (False, True):
        for tb in (False, True):
            for shape in SHAPES:
                seed += 1
                a, b, c, alpha, beta, ref, scale = _case(kind, ta, tb, shape, seed)
                K.tt_gemm_f32(ctx, kind, ta, tb, a, b, c, alpha, beta)
                got = c.cpu().numpy().astype(np.float64)
                bad = np.abs(got - ref) > TOL[kind] * scale
                assert not bad.any(), (kind, ta, tb, shape, np.argwhere(bad)[:3],
                                       float(np.max(np.abs(got - ref) / scale)))


def test_bf16_split_beats_plain_bf16_rounding(ctx):
    # the three-term split must be far more accurate than one BF16 product
    import torch
    a, b, c, _, _, ref, scale = _case(2, False, False, (1, 130, 70, 300), 99)
    c.zero_()
    K.tt_gemm_f32(ctx, 2, False, False, a, b, c, 1.0, 0.0)
    ref1 = np.matmul(a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64))
    err_split = np.max(np.abs(c.cpu().numpy() - ref1))
    plain = torch.matmul(a.bfloat16().double(), b.bfloat16().double()).cpu().numpy()
    err_plain = np.max(np.abs(plain - ref1))
    assert err_split < 0.05 * err_plain, (err_split, err_plain)
