"""GPU parity of the TT_TF32_SPLIT path: the local-system contractions of the
linear solves run on the tcgen05 tensor cores (TF32 three-term split, FP32
accumulation) inside FP64 iterative refinement, so the solves and the
eigenpair meet the same FP64 targets as the all-FP64 path."""
import dataclasses

import numpy as np
import pytest

import keig_inputs as ki
from oracle import transport as T
from oracle import ttref as R

pytestmark = pytest.mark.gpu

K = pytest.importorskip("paper_2309_03347_gb300")


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _ones(ctx, modes):
    return K.tt_vec_create(ctx, [np.ones((1, m, 1)) for m in modes])


@pytest.mark.parametrize("rhs_rank", [9])
def test_solve_local_tf32_split_matches_sweep(ctx, rhs_rank):
    # the transport sweep H^-1 b of the oracle, reached by the tensor-core
    # solve to the FP64 tolerance of the all-FP64 solve
    p = ki.fissile_box(l=3, G=2, order=4, seed=41, half_width=2)
    A = K.tt_build_operator(ctx, p, 0, 1e-13)
    d = len(p.tt_modes)
    bc = ki.random_cores(p.tt_modes, [1] + [rhs_rank] * (d - 1) + [1], 33 + rhs_rank)
    x = _ones(ctx, p.tt_modes)
    ctx.reset_counters()
    ctx.set_profiling(True)
    try:
        info = K.tt_solve_local(ctx, A, K.tt_vec_create(ctx, bc), x, eps=1e-10, rmax=0, max_sweeps=40, kick=4,
                                prec=K.TT_TF32_SPLIT)
        launches, ms, flops = ctx.gemmtc_stats()
    finally:
        ctx.set_profiling(False)
    ref = T.OracleProblem(p).sweep(R.full(bc).reshape(p.psi_shape)).ravel()
    assert rel(x.dense_cuda().cpu().numpy().ravel(), ref) < 1e-7, info
    # the contractions did run on the tensor-core kernel
    assert launches > 0 and flops > 0 and ms > 0


def test_solve_local_tf32_split_agrees_with_fp64(ctx):
    # same operator and right-hand side: the two precisions agree to the
    # solve tolerance (both are within it of the exact solution)
    p = ki.homogeneous(l=3, G=2, order=4, seed=1000)
    A = K.tt_build_operator(ctx, p, 0, 1e-13)
    d = len(p.tt_modes)
    bc = ki.random_cores(p.tt_modes, [1] + [3] * (d - 1) + [1], 77)
    xs = []
    for prec in (K.TT_FP64, K.TT_TF32_SPLIT):
        x = _ones(ctx, p.tt_modes)
        K.tt_solve_local(ctx, A, K.tt_vec_create(ctx, bc), x, eps=1e-10, rmax=0, max_sweeps=40, kick=4, prec=prec)
        xs.append(x.dense_cuda().cpu().numpy().ravel())
    assert rel(xs[1], xs[0]) < 1e-7


def test_keig_tf32_split_matches_oracle(ctx):
    p = dataclasses.replace(ki.config(0), side=(2.0,) * 3)
    ref = T.OracleProblem(p).keig(tol_k=1e-12, max_iter=20000)
    o = K.keig_default_opts()
    o.eps, o.rmax, o.tol_k, o.tol_psi, o.max_iter = 1e-10, 0, 1e-11, 1e-7, 200
    o.solve_sweeps, o.mv_sweeps = 4, 4
    o.prec = K.TT_TF32_SPLIT
    res = K.keig_fixed_point(ctx, p, o, want_phi=True)
    assert abs(res["k"] - ref["k"]) / ref["k"] < 1e-6
    assert rel(res["phi"], ref["phi"]) < 1e-5
