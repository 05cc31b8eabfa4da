"""Pins of the CPU oracle against what the paper and the mathematics fix,
independent of the oracle's own formulas:

* the 1-D factor matrices as Sec. 3.2.1 prints them (golden fixture);
* two independent constructions of the discrete operators — the vertex-by-
  vertex balance of Eq. (Discretized_kNTE) in C (``sweep.c``) and the sum of
  Kronecker products of Sec. 3.2 (``operators.py``) — agree entry by entry;
* the sweep is H^{-1} (library sparse solve of the assembled H);
* the power iteration of Eq. (k_eff_fixed_points) reaches the dominant
  eigenvalue of a library generalized eigensolver (GES, Sec. 4.1);
* the infinite-medium closed form k_inf = nsf^T (Sig_t - Sig_s)^{-1} chi is an
  exact eigenpair of the operators with mirror faces (flat flux);
* global neutron balance, cube symmetry, k < k_inf for vacuum faces;
* quadrature tables (Lewis & Miller, the discrete-ordinates reference of
  Appendix A.2) and the TT reference (TT-SVD, rounding, TT-matrix algebra,
  Algorithm 1) against brute force.
"""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import keig_inputs as ki
from oracle import operators as O
from oracle import transport as T
from oracle import ttref as R

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_factors():
    mats, name, rows = {}, None, []
    for line in open(os.path.join(GOLD, "paper_factor_matrices_n4.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line[0].isalpha():
            if name:
                mats[name] = np.array(rows, float)
            name, rows = line, []
        else:
            rows.append([float(v) for v in line.split()])
    mats[name] = np.array(rows, float)
    return mats


def test_factor_matrices_as_printed():
    g = _read_factors()
    assert np.array_equal(O.factor_D(4, 1.0, True), g["D+"])
    # the operator uses |mu| * Dt with Dt- = -D-
    assert np.array_equal(-O.factor_D(4, 1.0, False), g["D-"])
    assert np.array_equal(O.factor_Ip(4, True), g["Ip+"])
    assert np.array_equal(O.factor_Ip(4, False), g["Ip-"])
    assert np.array_equal(O.factor_Ip(4, True, True), g["Ip+noBC"])
    assert np.array_equal(O.factor_Ip(4, False, True), g["Ip-noBC"])


def test_quadrature_tables():
    for line in open(os.path.join(GOLD, "lqn_quadrature.txt")):
        if line.startswith("#") or not line.strip():
            continue
        tag, vals = line.split(":")
        order, kind = tag.split()
        q = ki.level_symmetric(int(order[1:]))
        vals = np.array([float(v) for v in vals.split()])
        if kind == "levels":
            assert np.allclose(np.unique(np.round(q.amu, 7)), vals, atol=2e-7)
        else:
            assert np.allclose(np.unique(np.round(8 * q.w8, 7)), np.sort(vals), atol=2e-7)
    for order in (4, 6, 8, 10, 12, 16):
        q = ki.level_symmetric(order)
        assert q.L == order * (order + 2)
        assert abs(q.w.sum() - 1.0) < 1e-12 and (q.w8 > 0).all()
        assert np.allclose(q.amu ** 2 + q.aeta ** 2 + q.axi ** 2, 1.0, atol=1e-6)
        # even moments of one cosine over the sphere: <mu^2> = 1/3, <mu^4> = 1/5
        assert abs(np.sum(q.w * q.mu ** 2) - 1 / 3) < 1e-6
        assert abs(np.sum(q.w * q.mu ** 4) - 1 / 5) < 1e-6
        assert abs(np.sum(q.w * q.mu)) < 1e-12
        # every even moment of one cosine up to degree N, and the mixed
        # moments an LQ_N set of order >= 6 integrates (the weights of S16
        # are not fixed by the single-cosine conditions; the table's are)
        for k in range(order // 2 + 1):
            assert abs(np.sum(q.w * q.mu ** (2 * k)) - 1 / (2 * k + 1)) < 1e-7
        if order >= 6:
            assert abs(np.sum(q.w * q.mu ** 2 * q.eta ** 2) - 1 / 15) < 1e-7
            assert abs(np.sum(q.w * q.mu ** 2 * q.eta ** 2 * q.xi ** 2) - 1 / 105) < 1e-7


@pytest.mark.parametrize("hetero", [False, True])
def test_stencil_equals_kronecker_assembly(hetero):
    p = ki.fissile_box(l=3, G=3, order=4, seed=3, half_width=2) if hetero else ki.homogeneous(l=2, G=2, order=4)
    op = T.OracleProblem(p)
    H, S, F = O.assemble(p)
    rng = np.random.default_rng(1)
    psi = rng.standard_normal(p.psi_shape)
    assert np.abs(op.apply_H(psi).ravel() - H @ psi.ravel()).max() < 1e-12 * np.abs(H).max() * 8
    s, f = op.apply_SF(psi)
    assert np.abs(s.ravel() - S @ psi.ravel()).max() < 1e-13
    assert np.abs(f.ravel() - F @ psi.ravel()).max() < 1e-13


def test_sweep_is_inverse_of_H():
    p = ki.fissile_box(l=3, G=2, order=4, seed=4, half_width=2)
    H, _, _ = O.assemble(p)
    b = np.random.default_rng(2).standard_normal(p.psi_shape)
    x = T.OracleProblem(p).sweep(b).ravel()
    ref = spla.spsolve(H.tocsc(), b.ravel())
    assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("hetero", [False, True])
def test_power_iteration_matches_ges(hetero):
    p = ki.fissile_box(l=3, G=2, order=4, seed=5, half_width=2) if hetero else ki.homogeneous(l=2, G=2, order=4)
    r = T.OracleProblem(p).keig(tol_k=1e-13, max_iter=50000, store_psi=True)
    kg, v = O.ges_k(p)
    assert abs(r["k"] - kg) < 1e-10 * kg
    psi = r["psi"].ravel()
    assert np.linalg.norm(psi - v) < 1e-6 * np.linalg.norm(v)


def test_mirror_rows_make_H_singular():
    """Config 0 with every face reflective: replacing the inflow rows of H by
    the mirror condition (the reading of reflective faces for the vertex
    diamond difference; the paper treats vacuum faces only) gives a singular
    H, so the fixed point of Eq. (k_eff_fixed_points), which applies H^{-1},
    is undefined there.  Inverse iteration with a library LU finds a unit
    vector in the numerical null space; the vacuum H is well conditioned."""
    p = ki.config(0, "reflective")
    H, _, _ = O.assemble(p)
    Hr = O.reflective_rows(p, H)
    x = np.random.default_rng(0).standard_normal(H.shape[0])
    lu = spla.splu(Hr.tocsc())
    for _ in range(3):
        x = lu.solve(x)
        x /= np.linalg.norm(x)
    assert np.linalg.norm(Hr @ x) < 1e-12
    assert np.linalg.norm(H @ x) > 1e-3
    b = np.random.default_rng(1).standard_normal(H.shape[0])
    xv = spla.splu(H.tocsc()).solve(b)
    assert np.linalg.norm(xv) < 1e3 * np.linalg.norm(b)


def test_infinite_medium_closed_form():
    p = ki.config(0, "reflective")
    kinf = O.k_infinity(p.sig_t[0], p.sig_s[0], p.nu_sig_f[0], p.chi[0])
    # flat group spectrum: the eigenvector of (Sig_t - Sig_s)^{-1} chi nsf^T
    c = np.linalg.solve(np.diag(p.sig_t[0]) - p.sig_s[0], p.chi[0])
    psi = np.broadcast_to(c[:, None, None, None, None], p.psi_shape).copy()
    H, S, F = O.assemble(p)
    Hr = O.reflective_rows(p, H)
    res = Hr @ psi.ravel() - (S @ psi.ravel() + F @ psi.ravel() / kinf)
    assert np.abs(res).max() < 1e-12 * np.abs(H @ psi.ravel()).max()
    # the C stencil reproduces the interior rows of the same identity
    op = T.OracleProblem(ki.config(0))
    s, f = op.apply_SF(psi)
    hp = op.apply_H(psi)
    rows = np.abs(s + f / kinf).ravel() > 0  # non-inflow rows
    assert np.abs((hp - s - f / kinf).ravel()[rows]).max() < 1e-12
    # and a vacuum cube leaks: its k lies below k_inf
    k_vac = op.keig(tol_k=1e-12)["k"]
    assert 0 < k_vac < kinf


def test_global_balance_and_symmetry():
    p = ki.config(0)
    op = T.OracleProblem(p)
    r = op.keig(tol_k=1e-13, max_iter=50000, store_psi=True)
    b = op.balance(r["psi"])
    k_bal = b["prod"] / (b["leak"] + b["absorb"] - b["scat_in"])
    assert abs(k_bal - r["k"]) < 1e-9 * r["k"]
    assert b["leak"] > 0
    phi = r["phi"]
    for g in range(p.G):
        f = phi[g]
        for t in (f[::-1], f[:, ::-1], f[:, :, ::-1], f.transpose(1, 0, 2), f.transpose(2, 1, 0)):
            assert np.abs(t - f).max() < 1e-9 * np.abs(f).max()
    # production identity used by the fixed point
    assert abs(T.production(p, phi) - 1.0) < 1e-12


# ----------------------------------------------------------------- TT reference

def test_full_of_rank1_is_outer_product():
    rng = np.random.default_rng(0)
    vs = [rng.standard_normal(n) for n in (3, 4, 2, 5)]
    cores = [v.reshape(1, -1, 1) for v in vs]
    ref = np.multiply.outer(np.multiply.outer(np.multiply.outer(vs[0], vs[1]), vs[2]), vs[3])
    assert np.allclose(R.full(cores), ref, rtol=0, atol=1e-14)
    # rank-2 cores built by hand: a sum of two outer products
    ws = [rng.standard_normal(n) for n in (3, 4, 2, 5)]
    c2 = [np.stack([vs[0], ws[0]], 1)[None], None, None, np.stack([vs[3], ws[3]], 0)[:, :, None]]
    for k in (1, 2):
        c = np.zeros((2, len(vs[k]), 2))
        c[0, :, 0] = vs[k]
        c[1, :, 1] = ws[k]
        c2[k] = c
    ref2 = ref + np.multiply.outer(np.multiply.outer(np.multiply.outer(ws[0], ws[1]), ws[2]), ws[3])
    assert np.allclose(R.full(c2), ref2, atol=1e-13)


def test_tt_svd_exact_and_ranks():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((3, 4, 5, 2, 3))
    cores = R.tt_svd(a, 0.0)
    assert np.allclose(R.full(cores), a, atol=1e-12)
    for k in range(1, 5):
        m = int(np.prod(a.shape[:k]))
        assert R.ranks(cores)[k] == np.linalg.matrix_rank(a.reshape(m, -1))


@pytest.mark.parametrize("eps", [0.0, 1e-2, 1e-6])
def test_tt_round_bound_and_idempotence(eps):
    c = ki.random_cores([3, 2, 4, 2, 3], [1, 3, 5, 5, 3, 1], 4)
    c = [ci * (0.2 ** np.arange(ci.shape[2]))[None, None, :] for ci in c]
    x = R.full(c)
    r1 = R.tt_round(c, eps)
    assert np.linalg.norm(R.full(r1) - x) <= max(eps, 1e-13) * np.linalg.norm(x) * (1 + 1e-9)
    r2 = R.tt_round(r1, eps)
    assert R.ranks(r2) == R.ranks(r1)
    assert np.linalg.norm(R.full(r2) - R.full(r1)) <= max(eps, 1e-13) * np.linalg.norm(x)
    if eps == 0.0:
        for k in range(1, 5):
            assert np.allclose(R.bond_singular_values(r1, k), R.bond_singular_values(c, k), atol=1e-12)


def test_tt_matrix_is_kronecker_product_and_matvec():
    rng = np.random.default_rng(2)
    fs = [rng.standard_normal((n, n)) for n in (2, 3, 4)]
    A = R.mat_rank1(fs)
    assert np.allclose(R.mat_full(A), np.kron(np.kron(fs[0], fs[1]), fs[2]), atol=1e-13)
    A2 = R.mat_add(A, R.mat_rank1([f.T for f in fs]), 1.0, -0.5)
    dense = np.kron(np.kron(fs[0], fs[1]), fs[2]) - 0.5 * np.kron(np.kron(fs[0].T, fs[1].T), fs[2].T)
    assert np.allclose(R.mat_full(A2), dense, atol=1e-12)
    x = ki.random_cores([2, 3, 4], [1, 2, 2, 1], 5)
    y = R.matvec(A2, x)
    assert np.allclose(R.full(y).ravel(), dense @ R.full(x).ravel(), atol=1e-12)


def test_qtt_of_paper_factors_has_rank_two():
    for l in (3, 5):
        n = 1 << l
        for pos in (True, False):
            for m in (O.factor_D(n, 0.7, pos), O.factor_Ip(n, pos)):
                q = R.qtt_matrix(m)
                assert max(c.shape[3] for c in q) == 2 and q[-1].shape[3] == 1
                assert np.allclose(R.mat_full(q), m, atol=1e-12)
            q = R.qtt_matrix(O.factor_Ip(n, pos, True))
            assert max(c.shape[3] for c in q) <= 3
            assert np.allclose(R.mat_full(q), O.factor_Ip(n, pos, True), atol=1e-12)


def test_projected_system_reproduces_galerkin_identity():
    rng = np.random.default_rng(3)
    x = R.left_orthogonalize(ki.random_cores([2, 3, 2, 2], [1, 2, 3, 2, 1], 6))
    A = rng.standard_normal((24, 24))
    Aloc, P = R.projected_system(A, x, 3)
    # the frames are orthonormal, so P^T P = I and full(x) = P vec(x_3)
    assert np.allclose(P.T @ P, np.eye(P.shape[1]), atol=1e-12)
    assert np.allclose(P @ x[3].ravel(), R.full(x).ravel(), atol=1e-12)
    assert np.allclose(Aloc, P.T @ A @ P)


def test_finite_difference_gradients_match_dense_adjoint():
    # two independent derivative computations of the oracle's k: central
    # differences of the power iteration and the dense adjoint formula with
    # exact operator derivatives (Kronecker assembly, linear in every entry)
    from oracle import sensitivity as SE
    import dataclasses
    p = dataclasses.replace(ki.config(0), l=2, mat=np.zeros((3, 3, 3), np.uint8), side=(2.0,) * 3)
    fd = SE.fd_gradients(p)
    ad, k1, k2 = SE.dense_adjoint_gradients(p)
    assert abs(k1 - k2) < 1e-10 * k1
    scale = max(np.abs(v).max() for v in ad.values())
    for f in SE.FIELDS:
        assert np.abs(fd[f] - ad[f]).max() < 1e-6 * scale, f


def test_functional_gradients_gpt_match_finite_differences():
    # the flux functional J (fissile-region group-1 flux of the
    # production-normalised eigenvector): central differences of the oracle's
    # J against generalised perturbation theory with the dense operators
    from oracle import sensitivity as SE
    import dataclasses
    p = dataclasses.replace(ki.fissile_box(l=2, G=2, order=4, seed=1003, half_width=1), side=(2.0,) * 3)
    rg, rv = ki.fissile_response(p, 0)
    fd = SE.fd_functional_gradients(p, rg, rv)
    gp, J, k = SE.dense_gpt_gradients(p, rg, rv)
    j_or, k_or = SE.oracle_functional(p, rg, rv)
    assert abs(J - j_or) < 1e-10 * abs(J) and abs(k - k_or) < 1e-10 * k
    scale = max(np.abs(v).max() for v in gp.values())
    for f in SE.FIELDS:
        assert np.abs(fd[f] - gp[f]).max() < 1e-7 * scale, f
    # the normalisation term matters: without -J sum(dF Psi) the fission
    # derivatives would be wrong
    assert np.abs(gp["nu_sig_f"]).max() > 1e-3 * scale


def test_linear_anisotropy_oracle():
    # linearly anisotropic scattering (N_s = 1): the stencil's per-direction
    # sources equal the Kronecker assembly, the power iteration equals the
    # library eigensolve, an isotropic flux feels no P1 source, mu_bar = 0
    # reproduces isotropic scattering exactly, and forward scattering (which
    # lowers the transport cross section) raises the leakage of a small bare
    # system, so k falls as mu_bar grows
    import dataclasses
    import scipy.sparse.linalg as spla
    p0 = dataclasses.replace(ki.fissile_box(l=2, G=2, order=4, seed=1003, half_width=1), side=(2.0,) * 3)
    ks = []
    for mu in (-0.2, 0.0, 0.2):
        p = ki.with_linear_anisotropy(p0, mu)
        o = T.OracleProblem(p)
        H, S, F = O.assemble(p)
        psi = np.random.default_rng(5).standard_normal(H.shape[0])
        s_c, _ = o.apply_SF(psi)
        assert np.abs(S @ psi - s_c.ravel()).max() < 1e-13
        iso = np.broadcast_to(np.random.default_rng(6).standard_normal((p.G, 1, p.n, p.n, p.n)),
                              p.psi_shape).ravel()
        s_iso, _ = o.apply_SF(iso)
        s_ref, _ = T.OracleProblem(p0).apply_SF(iso)
        assert np.abs(s_iso - s_ref).max() < 1e-13
        r = o.keig(tol_k=1e-13, max_iter=100000)
        lu = spla.splu((H - S).tocsc())
        N = H.shape[0]
        vals, _ = spla.eigs(spla.LinearOperator((N, N), matvec=lambda x: lu.solve(F @ x), dtype=np.float64), k=1,
                            which="LM", tol=1e-14, v0=np.ones(N))
        assert abs(r["k"] - np.real(vals[0])) < 1e-11 * r["k"]
        ks.append(r["k"])
    assert ks[0] > ks[1] > ks[2]
    k_iso = T.OracleProblem(p0).keig(tol_k=1e-13, max_iter=100000)["k"]
    assert abs(ks[1] - k_iso) < 1e-14 * k_iso


def test_higher_order_scattering_oracle():
    # orders 2-3 of the scattering expansion: the real spherical harmonics of
    # the oracle are orthonormal (unit mean square) under an exact product
    # rule, satisfy the addition theorem sum_m Y_nm Y_nm' = (2n+1) P_n, the
    # generic order-1 matrix equals the P1 form checked against the stencil,
    # and every order n >= 1 conserves particles (angular integral zero)
    from numpy.polynomial import legendre as Lg
    zt, wt = Lg.leggauss(12)
    ph = np.arange(24) * (2 * np.pi / 24)
    Z, P = np.meshgrid(zt, ph, indexing="ij")
    W = np.outer(wt, np.full(24, 1.0 / 24)) / 2.0  # weights of the unit sphere average
    X, Y = np.sqrt(1 - Z ** 2) * np.cos(P), np.sqrt(1 - Z ** 2) * np.sin(P)
    idx = [(n, m) for n in range(4) for m in range(-n, n + 1)]
    vals = {nm: O.real_sh(*nm, X, Y, Z) for nm in idx}
    for a in idx:
        for b in idx:
            assert abs(np.sum(W * vals[a] * vals[b]) - (a == b)) < 1e-12, (a, b)
    rng = np.random.default_rng(2)
    u = rng.standard_normal((3, 50)); u /= np.linalg.norm(u, axis=0)
    v = rng.standard_normal((3, 50)); v /= np.linalg.norm(v, axis=0)
    for n in range(4):
        s = sum(O.real_sh(n, m, *u) * O.real_sh(n, m, *v) for m in range(-n, n + 1))
        assert np.abs(s - (2 * n + 1) * Lg.legval(np.sum(u * v, axis=0), [0] * n + [1])).max() < 1e-12
    q = ki.level_symmetric(4)
    x, y, z = O.signed_directions(q)
    w = np.tile(q.w8, 8)
    A1 = O.aniso_angular(q, 1)
    assert np.abs(A1 - 3 * (np.outer(x, x * w) + np.outer(y, y * w) + np.outer(z, z * w))).max() < 1e-13
    for n in (1, 2, 3):
        assert np.abs(w @ O.aniso_angular(q, n)).max() < 1e-13, n
    # the assembled S: an isotropic flux sees no order-2/3 source
    import dataclasses
    p0 = dataclasses.replace(ki.fissile_box(l=2, G=2, order=4, seed=1003, half_width=1), side=(2.0,) * 3)
    p = ki.with_anisotropy(p0, 0.0, 0.15, 0.05)
    _, S0, _ = O.assemble(p0)
    _, S, _ = O.assemble(p)
    iso = np.broadcast_to(rng.standard_normal((p.G, 1, p.n, p.n, p.n)), p.psi_shape).ravel()
    assert np.abs(S @ iso - S0 @ iso).max() < 1e-12
    assert np.abs((S - S0) @ rng.standard_normal(S.shape[0])).max() > 1e-3
