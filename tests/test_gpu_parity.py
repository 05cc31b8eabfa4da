"""GPU parity: the CUDA tensor-train path (through the C-ABI) against the
FP64 CPU oracle (dense reconstruct, Kronecker assembly, full-grid sweep).

Tolerances: primitives that are exact in exact arithmetic (products, sums,
rounding at eps = 0, operator assembly) agree to 1e-12 relative (FP64
rounding of O(100) chained contractions); truncated results obey the
truncation bounds they are built to; the eigenvalue agrees with the oracle to
1e-6 relative and the scalar flux to 1e-5 relative L2 (the stated targets).
"""
import numpy as np
import pytest

import keig_inputs as ki
from oracle import operators as O
from oracle import transport as T
from oracle import ttref as R

pytestmark = pytest.mark.gpu

K = pytest.importorskip("paper_2309_03347_gb300")


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _vec(ctx, cores):
    return K.tt_vec_create(ctx, cores)


MODES = [3, 2, 4, 2, 2, 5, 2]


@pytest.mark.parametrize("rank,seed", [(1, 0), (3, 1), (7, 2)])
def test_vec_roundtrip_dense_dot_sum(ctx, rank, seed):
    ranks = [1] + [rank] * (len(MODES) - 1) + [1]
    cores = ki.random_cores(MODES, ranks, seed)
    x = _vec(ctx, cores)
    for a, b in zip(x.cores(), cores):
        assert np.array_equal(a, b)
    full = R.full(cores)
    dense = x.dense_cuda().cpu().numpy()
    assert rel(dense, full) < 1e-13
    cores2 = ki.random_cores(MODES, ranks, seed + 10)
    y = _vec(ctx, cores2)
    assert abs(x.dot(y) - np.vdot(full, R.full(cores2))) <= 1e-12 * np.linalg.norm(full) * np.linalg.norm(R.full(cores2))
    assert abs(x.norm() - np.linalg.norm(full)) <= 1e-12 * np.linalg.norm(full)
    assert abs(x.sum() - full.sum()) <= 1e-12 * np.abs(full).sum()


def test_axpby_scale(ctx):
    ranks = [1, 2, 3, 3, 2, 2, 4, 1]
    a = ki.random_cores(MODES, ranks, 3)
    b = ki.random_cores(MODES, ranks[::-1], 4)
    x = _vec(ctx, a)
    y = _vec(ctx, b)
    y.axpby(0.5, x, -2.0)
    assert rel(y.dense_cuda().cpu().numpy(), 0.5 * R.full(a) - 2.0 * R.full(b)) < 1e-13
    x.scale(3.0)
    assert rel(x.dense_cuda().cpu().numpy(), 3.0 * R.full(a)) < 1e-14


@pytest.mark.parametrize("seed", [0, 1])
def test_round_exact_at_zero_eps(ctx, seed):
    # a TT with redundant ranks: the sum x + x has ranks doubled, rounding at
    # eps = 0 must reproduce the tensor and bring the ranks back
    ranks = [1, 3, 4, 5, 4, 3, 2, 1]
    c = ki.random_cores(MODES, ranks, seed)
    x = _vec(ctx, c)
    x.axpby(1.0, _vec(ctx, c), 1.0)
    K.tt_round(ctx, x, 0.0)
    assert rel(x.dense_cuda().cpu().numpy(), 2 * R.full(c)) < 1e-12
    # a tolerance at the FP64 noise level removes the redundant half exactly
    K.tt_round(ctx, x, 1e-14)
    assert rel(x.dense_cuda().cpu().numpy(), 2 * R.full(c)) < 1e-12
    assert x.ranks == R.ranks(R.tt_round(c, 1e-14))


@pytest.mark.parametrize("eps", [1e-1, 1e-3, 1e-6])
def test_round_error_bound_and_singular_values(ctx, eps):
    ranks = [1, 3, 6, 8, 8, 6, 4, 1]
    c = ki.random_cores(MODES, ranks, 7)
    # give the spectrum a decay so truncation is meaningful
    c = [ci * (0.3 ** np.arange(ci.shape[2]))[None, None, :] for ci in c]
    full = R.full(c)
    x = _vec(ctx, c)
    K.tt_round(ctx, x, eps)
    xr = x.dense_cuda().cpu().numpy()
    assert rel(xr, full) <= eps * (1 + 1e-9)
    # ranks no larger than the oracle's rounding with the same rule
    ref = R.tt_round(c, eps)
    assert all(a <= b for a, b in zip(x.ranks, R.ranks(ref)))
    # singular values of every bond of the rounded tensor match the oracle's
    for k in range(1, len(MODES)):
        sv_gpu = np.linalg.svd(xr.reshape(int(np.prod(MODES[:k])), -1), compute_uv=False)[: x.ranks[k]]
        sv_ref = R.bond_singular_values(ref, k)[: x.ranks[k]]
        assert np.allclose(sv_gpu, sv_ref, rtol=1e-8, atol=1e-12 * sv_ref[0])


def test_round_rank_cap(ctx):
    ranks = [1, 3, 6, 8, 8, 6, 4, 1]
    c = ki.random_cores(MODES, ranks, 9)
    x = _vec(ctx, c)
    K.tt_round(ctx, x, 0.0, rmax=3)
    assert max(x.ranks) <= 3
    # the capped result is the oracle's capped rounding (same singular values kept)
    ref = R.tt_round(c, 0.0, 3)
    assert rel(x.dense_cuda().cpu().numpy(), R.full(ref)) < 1e-10


@pytest.mark.parametrize("eps", [0.0, 1e-9, 1e-4])
def test_round_large_ranks(ctx, eps):
    # bonds of 40-90 go through the mixed-precision SVD (FP32 rotations
    # refined by FP64 matrix products); the result must still be an
    # FP64-accurate rounding
    modes = [4, 8, 6, 4, 4, 2]
    ranks = [1, 4, 32, 90, 48, 8, 1]
    c = ki.random_cores(modes, ranks, 17)
    c = [ci * (0.8 ** np.arange(ci.shape[2]))[None, None, :] for ci in c]
    full = R.full(c)
    x = _vec(ctx, c)
    K.tt_round(ctx, x, eps)
    xr = x.dense_cuda().cpu().numpy()
    assert rel(xr, full) <= max(eps, 1e-13) * (1 + 1e-9)
    ref = R.tt_round(c, eps)
    assert x.ranks == R.ranks(ref)
    for k in range(1, len(modes)):
        sv_gpu = np.linalg.svd(xr.reshape(int(np.prod(modes[:k])), -1), compute_uv=False)[: x.ranks[k]]
        sv_ref = R.bond_singular_values(ref, k)[: x.ranks[k]]
        assert np.allclose(sv_gpu, sv_ref, rtol=1e-9, atol=1e-12 * sv_ref[0])
    # orthonormality of the non-first cores after rounding (right-orthogonal)
    for k, core in enumerate(x.cores()[1:], start=1):
        m = core.reshape(core.shape[0], -1)
        assert np.abs(m @ m.T - np.eye(m.shape[0])).max() < 1e-12


def test_round_large_redundant_ranks(ctx):
    # x + x with bonds of 60-80: half of every bond's singular values are
    # exactly zero; the mixed-precision SVD must resolve them to the FP64
    # noise level so that rounding at 1e-14 returns the original ranks
    modes = [4, 8, 6, 4, 4, 2]
    ranks = [1, 4, 30, 40, 30, 8, 1]
    c = ki.random_cores(modes, ranks, 23)
    c = [ci * (0.9 ** np.arange(ci.shape[2]))[None, None, :] for ci in c]
    x = _vec(ctx, c)
    x.axpby(1.0, _vec(ctx, c), 1.0)
    assert max(x.ranks) == 80
    K.tt_round(ctx, x, 1e-14)
    assert rel(x.dense_cuda().cpu().numpy(), 2 * R.full(c)) < 1e-12
    assert x.ranks == R.ranks(R.tt_round(c, 1e-14))


def _rand_op(modes, ranks, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((ranks[k], m, m, ranks[k + 1])) for k, m in enumerate(modes)]


def test_exact_matvec(ctx):
    modes = [3, 2, 4, 2, 2]
    A = _rand_op(modes, [1, 2, 3, 2, 2, 1], 11)
    xc = ki.random_cores(modes, [1, 2, 2, 3, 2, 1], 12)
    Ag = K.tt_op_create(ctx, A)
    x = _vec(ctx, xc)
    y = K.tt_matvec(ctx, Ag, x, scale=0.7)
    ref = 0.7 * (R.mat_full(A) @ R.full(xc).ravel())
    assert rel(y.dense_cuda().cpu().numpy(), ref) < 1e-13
    assert y.ranks == [1] + [a * b for a, b in zip([2, 3, 2, 2], [2, 2, 3, 2])] + [1]
    # with rounding
    y2 = K.tt_matvec(ctx, Ag, x, scale=1.0, eps=1e-12)
    assert rel(y2.dense_cuda().cpu().numpy(), ref / 0.7) < 1e-11


def test_amen_matvec(ctx):
    modes = [3, 2, 4, 2, 2, 2]
    A = _rand_op(modes, [1, 2, 3, 2, 2, 2, 1], 21)
    xc = ki.random_cores(modes, [1, 2, 2, 3, 2, 2, 1], 22)
    y = K.tt_matvec(ctx, K.tt_op_create(ctx, A), _vec(ctx, xc), method=K.TT_MV_AMEN, eps=1e-10, max_sweeps=10)
    ref = R.mat_full(A) @ R.full(xc).ravel()
    assert rel(y.dense_cuda().cpu().numpy(), ref) < 1e-8


def _tiny_problem(hetero=False):
    if hetero:
        return ki.fissile_box(l=3, G=2, order=4, seed=77, half_width=2)
    return ki.homogeneous(l=2, G=2, order=4, seed=1000)


def _op_modes(p):
    return p.tt_modes


@pytest.mark.parametrize("hetero", [False, True])
@pytest.mark.parametrize("kind", [0, 1, 2])
def test_build_operator_matches_kronecker_assembly(ctx, hetero, kind):
    p = _tiny_problem(hetero)
    H, S, F = O.assemble(p)
    ref = [H, S, F][kind].toarray()
    A = K.tt_build_operator(ctx, p, kind, 1e-13)
    m, n, _ = A.shape
    assert m == p.tt_modes and n == p.tt_modes
    dense = R.mat_full(A.cores())
    assert np.abs(dense - ref).max() <= 1e-11 * np.abs(ref).max()


def test_qtt_factor_ranks_are_low(ctx):
    # homogeneous H: every spatial bond carries the rank-2 QTT of the 1-D
    # factors summed over the octant terms; the rounded ranks stay small
    p = ki.homogeneous(l=4, G=2, order=4, seed=5)
    A = K.tt_build_operator(ctx, p, 0, 1e-12)
    _, _, Rk = A.shape
    assert max(Rk) <= 64


def test_solve_local_matches_sweep(ctx):
    p = ki.homogeneous(l=2, G=2, order=4, seed=1000)
    H, _, _ = O.assemble(p)
    A = K.tt_build_operator(ctx, p, 0, 1e-13)
    bc = ki.random_cores(p.tt_modes, [1] + [2] * (len(p.tt_modes) - 1) + [1], 31)
    b = _vec(ctx, bc)
    x = _vec(ctx, [np.ones((1, m, 1)) for m in p.tt_modes])
    info = K.tt_solve_local(ctx, A, b, x, eps=1e-10, rmax=0, max_sweeps=40, kick=4)
    ref = T.OracleProblem(p).sweep(R.full(bc).reshape(p.psi_shape)).ravel()
    got = x.dense_cuda().cpu().numpy().ravel()
    assert rel(got, ref) < 1e-7, info


def test_solve_local_mixed_precision_matches_sweep(ctx):
    # FP32 Krylov iterations inside FP64 iterative refinement reach the same
    # FP64 tolerance as the all-FP64 solve
    p = ki.fissile_box(l=3, G=2, order=4, seed=41, half_width=2)
    A = K.tt_build_operator(ctx, p, 0, 1e-13)
    bc = ki.random_cores(p.tt_modes, [1] + [2] * (len(p.tt_modes) - 1) + [1], 33)
    x = _vec(ctx, [np.ones((1, m, 1)) for m in p.tt_modes])
    info = K.tt_solve_local(ctx, A, _vec(ctx, bc), x, eps=1e-10, rmax=0, max_sweeps=40, kick=4,
                            prec=K.TT_FP32_REFINED)
    ref = T.OracleProblem(p).sweep(R.full(bc).reshape(p.psi_shape)).ravel()
    assert rel(x.dense_cuda().cpu().numpy().ravel(), ref) < 1e-7, info


def test_solve_local_reports_noconv(ctx):
    p = ki.homogeneous(l=2, G=2, order=4, seed=1000)
    A = K.tt_build_operator(ctx, p, 0, 1e-13)
    bc = ki.random_cores(p.tt_modes, [1] + [2] * (len(p.tt_modes) - 1) + [1], 32)
    x = _vec(ctx, [np.ones((1, m, 1)) for m in p.tt_modes])
    info = K.tt_solve_local(ctx, A, _vec(ctx, bc), x, eps=1e-12, max_sweeps=1, kick=1, allow_noconv=True)
    assert info["code"] == K.TT_ENOCONV


def test_rejects_bad_inputs(ctx):
    p = ki.homogeneous(l=2, G=2, order=4, seed=1000)
    bad = ki.homogeneous(l=2, G=2, order=4, seed=1000)
    bad.sig_t = bad.sig_t.copy()
    bad.sig_t[0, 0] = np.nan
    with pytest.raises(K.KeigError) as e:
        K.tt_build_operator(ctx, bad, 0)
    assert e.value.code == K.TT_EINVAL
    with pytest.raises(K.KeigError) as e:
        K.tt_build_operator(ctx, p.with_bc((1, 0, 0, 0, 0, 0)), 0)
    assert e.value.code == K.TT_EINVAL
    with pytest.raises(K.KeigError) as e:
        K.tt_vec_create(ctx, [np.full((1, 2, 1), np.inf)])
    assert e.value.code == K.TT_EINVAL


def _oracle_keig(p, tol=1e-12):
    return T.OracleProblem(p).keig(tol_k=tol, max_iter=20000)


def _keig_full_rank(ctx, p, max_iter, prec=0):
    o = K.keig_default_opts()
    o.eps, o.rmax, o.tol_k, o.tol_psi, o.max_iter = 1e-10, 0, 1e-11, 1e-7, max_iter
    o.solve_sweeps, o.mv_sweeps = 4, 4
    o.prec = prec
    return K.keig_fixed_point(ctx, p, o, want_phi=True)


def test_keig_mixed_precision_matches_oracle(ctx):
    import dataclasses
    p = dataclasses.replace(ki.config(0), side=(2.0,) * 3)
    ref = _oracle_keig(p)
    res = _keig_full_rank(ctx, p, 200, prec=K.TT_FP32_REFINED)
    assert abs(res["k"] - ref["k"]) / ref["k"] < 1e-6
    assert rel(res["phi"], ref["phi"]) < 1e-5


@pytest.mark.parametrize("case", ["homogeneous_side2", "fissile_box_side3"])
def test_keig_matches_oracle(ctx, case):
    # 8^3 grids at full TT rank (no truncation beyond 1e-10): the QTT fixed
    # point must reproduce the oracle's eigenpair
    import dataclasses
    if case == "homogeneous_side2":
        p = dataclasses.replace(ki.config(0), side=(2.0,) * 3)
    else:
        p = dataclasses.replace(ki.fissile_box(l=3, G=2, order=4, seed=1003, half_width=2), side=(3.0,) * 3)
    ref = _oracle_keig(p)
    res = _keig_full_rank(ctx, p, 200)
    assert abs(res["k"] - ref["k"]) / ref["k"] < 1e-6
    assert rel(res["phi"], ref["phi"]) < 1e-5


def test_keig_exact_product_matches_oracle(ctx):
    # solver variant: the exact TT product rounded at eps in place of the
    # AMEn product (Sec. 3.5 compares the two); same fixed point
    import dataclasses
    p = dataclasses.replace(ki.config(0), side=(2.0,) * 3)
    ref = _oracle_keig(p)
    o = K.keig_default_opts()
    o.eps, o.rmax, o.tol_k, o.tol_psi, o.max_iter = 1e-10, 0, 1e-11, 1e-7, 200
    o.solve_sweeps, o.mv_sweeps = 4, 4
    o.mv_kind = 1
    res = K.keig_fixed_point(ctx, p, o, want_phi=True)
    assert abs(res["k"] - ref["k"]) / ref["k"] < 1e-6
    assert rel(res["phi"], ref["phi"]) < 1e-5


@pytest.mark.parametrize("mu_bar", [-0.2, 0.25])
def test_keig_linear_anisotropy_matches_oracle(ctx, mu_bar):
    # linearly anisotropic scattering (N_s = 1): the S operator gains the
    # P1 terms; the QTT fixed point must reproduce the oracle's eigenpair
    import dataclasses
    p = ki.with_linear_anisotropy(
        dataclasses.replace(ki.fissile_box(l=3, G=2, order=4, seed=1003, half_width=2), side=(3.0,) * 3), mu_bar)
    H, S, F = O.assemble(p)
    A = K.tt_build_operator(ctx, p, 1, 1e-13)
    x = ki.random_cores(p.tt_modes, [1] + [2] * (len(p.tt_modes) - 1) + [1], 44)
    y = K.tt_matvec(ctx, A, _vec(ctx, x), 1.0, K.TT_MV_EXACT, -1.0)
    assert rel(y.dense_cuda().cpu().numpy().ravel(), S @ R.full(x).ravel()) < 1e-11
    ref = _oracle_keig(p)
    res = _keig_full_rank(ctx, p, 200, prec=K.TT_FP32_REFINED)
    assert abs(res["k"] - ref["k"]) / ref["k"] < 1e-6
    assert rel(res["phi"], ref["phi"]) < 1e-5


def test_higher_order_scattering_matches_oracle(ctx):
    # scattering orders 1-3: the TT S operator against the Kronecker assembly
    # (real spherical harmonics of the oracle, evaluated at the signed
    # directions), and the fixed point against the library eigensolve
    import dataclasses
    p = ki.with_anisotropy(
        dataclasses.replace(ki.fissile_box(l=3, G=2, order=4, seed=1003, half_width=2), side=(3.0,) * 3),
        0.2, 0.1, 0.05)
    H, S, F = O.assemble(p)
    A = K.tt_build_operator(ctx, p, 1, 1e-13)
    x = ki.random_cores(p.tt_modes, [1] + [2] * (len(p.tt_modes) - 1) + [1], 45)
    y = K.tt_matvec(ctx, A, _vec(ctx, x), 1.0, K.TT_MV_EXACT, -1.0)
    assert rel(y.dense_cuda().cpu().numpy().ravel(), S @ R.full(x).ravel()) < 1e-11
    k_ref, _ = O.ges_k(p, H, S, F)
    res = _keig_full_rank(ctx, p, 200, prec=K.TT_FP32_REFINED)
    assert abs(res["k"] - k_ref) / k_ref < 1e-6, (res["k"], k_ref)


@pytest.mark.slow
def test_keig_config0_vacuum(ctx):
    # dominance ratio 0.956: about 200 power iterations to 1e-7 in k
    p = ki.config(0)
    ref = _oracle_keig(p)
    res = _keig_full_rank(ctx, p, 600)
    assert abs(res["k"] - ref["k"]) / ref["k"] < 1e-6
    assert rel(res["phi"], ref["phi"]) < 1e-5


def test_keig_noconv_returns_best_iterate(ctx):
    p = ki.config(0)
    o = K.keig_default_opts()
    o.max_iter = 2
    res = K.keig_fixed_point(ctx, p, o, allow_noconv=True)
    assert res["code"] == K.TT_ENOCONV and res["iters"] == 2 and np.isfinite(res["k"])


@pytest.mark.parametrize("case", ["homogeneous_side2", "fissile_box_side3"])
def test_adjoint_sensitivities_match_finite_differences(ctx, case):
    # dk/d(every cross-section entry) from the adjoint QTT fixed point against
    # central finite differences of the oracle (step 1e-6 relative)
    import dataclasses
    from oracle import sensitivity as SE
    if case == "homogeneous_side2":
        p = dataclasses.replace(ki.config(0), side=(2.0,) * 3)
    else:
        p = dataclasses.replace(ki.fissile_box(l=3, G=2, order=4, seed=1003, half_width=2), side=(3.0,) * 3)
    o = K.keig_default_opts()
    o.eps, o.rmax, o.tol_k, o.tol_psi, o.max_iter = 1e-10, 0, 1e-12, 1e-8, 300
    o.solve_sweeps, o.mv_sweeps = 4, 4
    g = K.keig_sensitivities(ctx, p, o)
    assert abs(g["k"] - g["k_adjoint"]) < 1e-8 * g["k"]
    fd = SE.fd_gradients(p)
    # per entry: 1e-4 relative to that entry's finite difference, with an
    # absolute floor of 1e-7 x the largest derivative for the finite
    # difference's own noise (k converged to 1e-13, step 1e-6 relative)
    scale = max(np.abs(v).max() for v in fd.values())
    for f in SE.FIELDS:
        bad = np.abs(g[f] - fd[f]) > 1e-4 * np.abs(fd[f]) + 1e-7 * scale
        assert not bad.any(), (f, g[f][bad], fd[f][bad])


def test_autograd_function_backward(ctx):
    import dataclasses
    import torch
    p = dataclasses.replace(ki.config(0), side=(2.0,) * 3)
    o = K.keig_default_opts()
    o.eps, o.rmax, o.tol_k, o.tol_psi, o.max_iter = 1e-10, 0, 1e-12, 1e-8, 300
    o.solve_sweeps, o.mv_sweeps = 4, 4
    o.tol_k, o.tol_psi = 1e-9, 1e-6  # this test checks the plumbing of backward()
    KeigK = K.keig_k_function()
    t = {f: torch.tensor(getattr(p, f), dtype=torch.float64, requires_grad=True)
         for f in ("sig_t", "sig_s", "nu_sig_f", "chi")}
    k = KeigK.apply(t["sig_t"], t["sig_s"], t["nu_sig_f"], t["chi"], p, ctx, o)
    (2.0 * k).backward()
    g = K.keig_sensitivities(ctx, p, o)
    for f in ("sig_t", "sig_s", "nu_sig_f", "chi"):
        assert np.allclose(t[f].grad.numpy(), 2.0 * g[f], rtol=1e-9, atol=0)
