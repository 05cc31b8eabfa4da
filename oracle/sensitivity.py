"""ORACLE (test infrastructure only): derivatives of k with respect to the
cross-section tables.

* ``fd_gradients``: central finite differences of the oracle's power iteration
  (Eq. (k_eff_fixed_points) in ``sweep.c``), step ``h = 1e-6 |p|`` or ``1e-6``
  when ``p = 0`` — the plain definition of the derivative.
* ``dense_adjoint_gradients``: the same derivatives from the dense
  operators of ``operators.assemble`` (Kronecker assembly): left and right
  eigenvectors of the generalized problem by a library eigensolver and
  ``dk/dp = -k^2 <psi_adj, (dH - dS - dF/k) psi> / <psi_adj, F psi>``, the
  operator derivatives taken exactly by linearity (the operators are linear in
  every table entry).  Used to pin the finite differences, not the GPU.
* ``fd_functional_gradients`` / ``dense_gpt_gradients``: the same two routes
  for the flux functional J (the fissile-region group-1 flux of the
  production-normalised eigenvector): central differences of the oracle's J,
  and generalised perturbation theory with the dense operators.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse.linalg as spla

from . import operators as O
from . import transport as T

FIELDS = ("sig_t", "sig_s", "nu_sig_f", "chi")


def _with(prob, field, idx, value):
    arr = getattr(prob, field).copy()
    arr[idx] = value
    return dataclasses.replace(prob, **{field: arr})


def oracle_k(prob, tol=1e-13):
    return T.OracleProblem(prob).keig(tol_k=tol, max_iter=100000)["k"]


def fd_gradients(prob, rel_step=1e-6, tol=1e-13):
    out = {}
    for field in FIELDS:
        base = getattr(prob, field)
        g = np.zeros_like(base, dtype=np.float64)
        for idx in np.ndindex(base.shape):
            p0 = float(base[idx])
            h = rel_step * abs(p0) if p0 != 0.0 else rel_step
            kp = oracle_k(_with(prob, field, idx, p0 + h), tol)
            km = oracle_k(_with(prob, field, idx, p0 - h), tol)
            g[idx] = (kp - km) / (2 * h)
        out[field] = g
    return out


def _eig(Aop_solve, N, v0):
    vals, vecs = spla.eigs(spla.LinearOperator((N, N), matvec=Aop_solve, dtype=np.float64), k=1, which="LM",
                           tol=1e-14, v0=v0)
    return float(np.real(vals[0])), np.real(vecs[:, 0])


def dense_adjoint_gradients(prob):
    H, S, F = O.assemble(prob)
    N = H.shape[0]
    A = (H - S).tocsc()
    lu = spla.splu(A)
    luT = spla.splu(A.T.tocsc())
    k, psi = _eig(lambda x: lu.solve(F @ x), N, np.ones(N))
    k2, adj = _eig(lambda x: luT.solve(F.T @ x), N, np.ones(N))
    denom = adj @ (F @ psi)
    out = {}
    for field in FIELDS:
        base = getattr(prob, field)
        g = np.zeros_like(base, dtype=np.float64)
        for idx in np.ndindex(base.shape):
            # exact derivative of a linear operator: A(p + 1) - A(p)
            pp = _with(prob, field, idx, float(base[idx]) + 1.0)
            H1, S1, F1 = O.assemble(pp)
            dH, dS, dF = H1 - H, S1 - S, F1 - F
            g[idx] = -k * k * (adj @ (dH @ psi - dS @ psi - (dF @ psi) / k)) / denom
        out[field] = g
    return out, k, k2


# ---------------------------------------------------------------- flux functional
# J = sum_g sum_v resp_g[g] resp_v[v] phi[g, v] of the eigenvector normalised
# so that its production sum(F Psi) is 1, and its derivatives.


def functional_from_phi(prob, phi, resp_g, resp_v):
    """J of a scalar flux phi[g, z, y, x], after normalising its production to 1."""
    phi = np.asarray(phi) / T.production(prob, phi)
    return float(np.einsum("g,gkji,kji->", resp_g, phi, resp_v))


def oracle_functional(prob, resp_g, resp_v, tol=1e-13):
    r = T.OracleProblem(prob).keig(tol_k=tol, max_iter=100000)
    return functional_from_phi(prob, r["phi"], resp_g, resp_v), r["k"]


def fd_functional_gradients(prob, resp_g, resp_v, rel_step=1e-6, tol=1e-13):
    """Central finite differences of J, step 1e-6 |p| (1e-6 when p = 0)."""
    out = {}
    for field in FIELDS:
        base = getattr(prob, field)
        g = np.zeros_like(base, dtype=np.float64)
        for idx in np.ndindex(base.shape):
            p0 = float(base[idx])
            h = rel_step * abs(p0) if p0 != 0.0 else rel_step
            jp, _ = oracle_functional(_with(prob, field, idx, p0 + h), resp_g, resp_v, tol)
            jm, _ = oracle_functional(_with(prob, field, idx, p0 - h), resp_g, resp_v, tol)
            g[idx] = (jp - jm) / (2 * h)
        out[field] = g
    return out


def dense_gpt_gradients(prob, resp_g, resp_v):
    """Generalised perturbation theory with the dense operators.

    With A = H - S - F/k, A Psi = 0, sum(F Psi) = <f, Psi> = 1 (f = F^T 1) and
    J = <j, Psi> (j = resp_g (x) w (x) resp_v), differentiating both
    constraints and J gives dJ/dp = <j, dPsi>; the generalised adjoint Gamma
    with A^T Gamma = j - J f and <Gamma, F Psi> = 0 turns it into
        dJ/dp = -<Gamma, (dH - dS - dF/k) Psi> - J sum(dF Psi).
    Gamma comes from the consistent bordered system [A^T; (F Psi)^T] Gamma =
    [j - J f; 0] solved by a dense least-squares routine (tiny grids only).
    Returns (gradients, J, k)."""
    H, S, F = O.assemble(prob)
    N = H.shape[0]
    A = (H - S).tocsc()
    lu = spla.splu(A)
    k, psi = _eig(lambda x: lu.solve(F @ x), N, np.ones(N))
    psi = psi / np.sum(F @ psi)
    j = np.einsum("g,l,v->glv", resp_g, prob.quad.w, np.asarray(resp_v).ravel()).ravel()
    f = np.asarray(F.T @ np.ones(N)).ravel()
    J = float(j @ psi)
    Ad = (H - S - F / k).toarray()
    Fpsi = np.asarray(F @ psi).ravel()
    M = np.vstack([Ad.T, Fpsi[None, :]])
    rhs = np.concatenate([j - J * f, [0.0]])
    gam = np.linalg.lstsq(M, rhs, rcond=None)[0]
    out = {}
    for field in FIELDS:
        base = getattr(prob, field)
        g = np.zeros_like(base, dtype=np.float64)
        for idx in np.ndindex(base.shape):
            pp = _with(prob, field, idx, float(base[idx]) + 1.0)
            H1, S1, F1 = O.assemble(pp)
            dH, dS, dF = H1 - H, S1 - S, F1 - F
            g[idx] = -(gam @ (dH @ psi - dS @ psi - (dF @ psi) / k)) - J * float(np.sum(dF @ psi))
        out[field] = g
    return out, J, k
