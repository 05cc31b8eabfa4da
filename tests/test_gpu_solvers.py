"""The other members of the alternating TT solver family of Sec. 3.5 ("ALS,
DMRG, AMEn"): two-site DMRG (tt_solve_dmrg) and one-site ALS (tt_solve_local
with kick = 0), against the oracle's sweep (H^{-1} b on the full grid), and
DMRG inside the fixed point of Eq. (TT_k_eff_fixed_points) against the
oracle's k and scalar flux."""
import dataclasses

import numpy as np
import pytest

import keig_inputs as ki
from oracle import transport as T
from oracle import ttref as R

pytestmark = pytest.mark.gpu

K = pytest.importorskip("paper_2309_03347_gb300")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _vec(ctx, cores):
    return K.tt_vec_create(ctx, [np.ascontiguousarray(c, np.float64) for c in cores])


def _full_ranks(modes):
    """Largest useful TT ranks: min(product of modes left of the bond, right of it)."""
    d = len(modes)
    return [1] + [int(min(np.prod(modes[:k]), np.prod(modes[k:]))) for k in range(1, d)] + [1]


@pytest.mark.parametrize("hetero,prec", [(False, "fp64"), (True, "fp32")])
def test_dmrg_solve_matches_sweep(ctx, hetero, prec):
    p = ki.fissile_box(l=3, G=2, order=4, seed=41, half_width=2) if hetero else ki.homogeneous(l=2, G=2, order=4)
    A = K.tt_build_operator(ctx, p, 0, 1e-13)
    bc = ki.random_cores(p.tt_modes, [1] + [2] * (len(p.tt_modes) - 1) + [1], 33)
    x = _vec(ctx, [np.ones((1, m, 1)) for m in p.tt_modes])
    info = K.tt_solve_dmrg(ctx, A, _vec(ctx, bc), x, eps=1e-10, rmax=0, max_sweeps=30,
                           prec=K.TT_FP64 if prec == "fp64" else K.TT_FP32_REFINED)
    ref = T.OracleProblem(p).sweep(R.full(bc).reshape(p.psi_shape)).ravel()
    assert rel(x.dense_cuda().cpu().numpy().ravel(), ref) < 1e-7, info


def test_als_solve_matches_sweep(ctx):
    # one-site ALS keeps the ranks of its initial guess: start from full ranks
    p = ki.homogeneous(l=2, G=2, order=4, seed=1000)
    A = K.tt_build_operator(ctx, p, 0, 1e-13)
    bc = ki.random_cores(p.tt_modes, [1] + [2] * (len(p.tt_modes) - 1) + [1], 35)
    x = _vec(ctx, ki.random_cores(p.tt_modes, _full_ranks(p.tt_modes), 36))
    info = K.tt_solve_local(ctx, A, _vec(ctx, bc), x, eps=1e-10, rmax=0, max_sweeps=40, kick=0)
    ref = T.OracleProblem(p).sweep(R.full(bc).reshape(p.psi_shape)).ravel()
    assert rel(x.dense_cuda().cpu().numpy().ravel(), ref) < 1e-7, info


def test_als_does_not_grow_ranks(ctx):
    # from a rank-1 guess ALS stays at rank 1 (no enrichment), unlike AMEn
    p = ki.homogeneous(l=2, G=2, order=4, seed=1000)
    A = K.tt_build_operator(ctx, p, 0, 1e-13)
    bc = ki.random_cores(p.tt_modes, [1] + [2] * (len(p.tt_modes) - 1) + [1], 37)
    x = _vec(ctx, [np.ones((1, m, 1)) for m in p.tt_modes])
    K.tt_solve_local(ctx, A, _vec(ctx, bc), x, eps=1e-10, rmax=0, max_sweeps=3, kick=0, allow_noconv=True)
    assert max(x.ranks) == 1


def test_dmrg_reports_noconv(ctx):
    p = ki.homogeneous(l=2, G=2, order=4, seed=1000)
    A = K.tt_build_operator(ctx, p, 0, 1e-13)
    bc = ki.random_cores(p.tt_modes, [1] + [2] * (len(p.tt_modes) - 1) + [1], 32)
    x = _vec(ctx, [np.ones((1, m, 1)) for m in p.tt_modes])
    info = K.tt_solve_dmrg(ctx, A, _vec(ctx, bc), x, eps=1e-12, max_sweeps=1, allow_noconv=True)
    assert info["code"] == K.TT_ENOCONV


def test_fixed_point_with_dmrg(ctx):
    # the two-site solve adapts ranks itself inside the fixed point (one-site
    # ALS cannot: its ranks stay those of its initial guess)
    p = dataclasses.replace(ki.config(0), side=(2.0,) * 3)
    o = K.keig_default_opts()
    o.eps, o.rmax, o.tol_k, o.tol_psi, o.max_iter = 1e-10, 0, 1e-11, 1e-7, 600
    o.solve_sweeps, o.mv_sweeps = 4, 4
    o.solve_method = 2
    res = K.keig_fixed_point(ctx, p, o, want_phi=True)
    ref = T.OracleProblem(p).keig(tol_k=1e-12, max_iter=20000)
    assert abs(res["k"] - ref["k"]) / ref["k"] < 1e-6
    assert rel(res["phi"], ref["phi"]) < 1e-5
