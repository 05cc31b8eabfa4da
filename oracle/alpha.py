"""ORACLE (test infrastructure only): the alpha-eigenvalue problem
(alpha V^{-1} + H) Psi = (S + F) Psi of Eq. (OpFormAlphaNTE).

* ``secant_alpha``: the paper's procedure (Eq. (alpha_eig_fixed_points)):
  k-eigenvalue solves of (H + alpha V^{-1}) Psi = (S + F/k) Psi by the
  oracle's power iteration, starting from alpha = 0 and alpha = 0.01, and the
  secant update on k(alpha) = 1.  The printed update is dimensionally garbled;
  it is read as the secant step
  alpha' = alpha_{-1} + (1 - k_{-1}) (alpha - alpha_{-1}) / (k - k_{-1}).
  V^{-1} = diag(1/v) (x) (octant selector (x) I) (x) Ip (x) Ip (x) Ip
  (Sec. 3.2.1) has the structure of the collision term of H, so
  H + alpha V^{-1} is H with sigma_t replaced by sigma_t + alpha / v.
* ``ges_alpha``: the fundamental alpha from the assembled operators:
  the rightmost real eigenvalue of V (S + F - H), library sparse eigensolve.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import operators as O
from . import transport as T


def _shifted(prob, inv_v, alpha):
    return dataclasses.replace(prob, sig_t=prob.sig_t + alpha * np.asarray(inv_v)[None, :])


def secant_alpha(prob, inv_v, tol_k=1e-10, max_steps=60, k_tol=1e-13):
    hist = []
    a0, a1 = 0.0, 0.01
    k0 = T.OracleProblem(_shifted(prob, inv_v, a0)).keig(tol_k=k_tol, max_iter=100000)["k"]
    k1 = T.OracleProblem(_shifted(prob, inv_v, a1)).keig(tol_k=k_tol, max_iter=100000)["k"]
    hist += [(a0, k0), (a1, k1)]
    for _ in range(max_steps):
        if abs(k1 - 1.0) < tol_k or k1 == k0:
            break
        a2 = a0 + (1.0 - k0) * (a1 - a0) / (k1 - k0)
        a0, k0 = a1, k1
        a1 = a2
        k1 = T.OracleProblem(_shifted(prob, inv_v, a1)).keig(tol_k=k_tol, max_iter=100000)["k"]
        hist.append((a1, k1))
    return a1, k1, hist


def assemble_vinv(prob, inv_v):
    """V^{-1}: the collision-term structure with diag(1/v) in the group core."""
    p0 = dataclasses.replace(prob, sig_t=np.zeros_like(prob.sig_t))
    p1 = dataclasses.replace(prob, sig_t=np.broadcast_to(np.asarray(inv_v)[None, :], prob.sig_t.shape).copy())
    H0, _, _ = O.assemble(p0)
    H1, _, _ = O.assemble(p1)
    return (H1 - H0).tocsc()


def ges_alpha(prob, inv_v):
    H, S, F = O.assemble(prob)
    Vinv = assemble_vinv(prob, inv_v)
    lu = spla.splu(Vinv)
    A = (S + F - H).tocsr()
    N = A.shape[0]
    op = spla.LinearOperator((N, N), matvec=lambda x: lu.solve(A @ x), dtype=np.float64)
    vals = spla.eigs(op, k=6, which="LR", return_eigenvectors=False, tol=1e-12, v0=np.ones(N))
    real = [v.real for v in vals if abs(v.imag) < 1e-8 * max(1.0, abs(v.real))]
    return float(max(real))
