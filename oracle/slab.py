"""ORACLE (test infrastructure only): the 1-D slab k-eigenvalue problem of
the paper's 1-D case study (Sec. 4.1), in FP64 on the CPU.

Vertex diamond difference restricted to x (the 1-D reading of the cell
balance of Eq. (Discretized_kNTE)): for mu > 0 and each cell c between
points i-1 and i,
    (mu / Delta) (psi_i - psi_{i-1}) + sigma_t(c) (psi_i + psi_{i-1}) / 2 = q_c,
    q_c = sum_g' [sigma_s(c)[g][g'] + chi(c)[g] nu_sigma_f(c)[g'] / k] (phi_{g'}(i-1) + phi_{g'}(i)) / 2,
with psi_0 = 0 (vacuum inflow), and the mirror image for mu < 0 (psi_{n-1} = 0,
cell c between i and i+1); phi = sum_d w_d (psi(mu_d) + psi(-mu_d)).

* ``SlabOracle.sweep``: H^-1 by marching each direction downstream.
* ``SlabOracle.keig``: the power iteration of Eq. (k_eff_fixed_points) with
  k' = k P(Psi') / P(Psi), P = sum(F Psi), Psi normalised to P = 1 (the
  paper's ISFM: the iterative solver on the full, matricized operators).
* ``assemble``: H, S, F as sparse matrices from Kronecker products of the
  1-D factors (the matrices of Sec. 3.2 restricted to x: D, Ip with and
  without the inflow row), for the library eigensolver ``ges`` (the paper's
  GES).
Index order of Psi: (g, hemisphere (0: mu < 0, 1: mu > 0), direction, x).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _cell_tables(s):
    m = np.asarray(s.mat, dtype=np.intp)
    return s.sig_t[m], s.sig_s[m], s.nu_sig_f[m], s.chi[m]  # per cell


class SlabOracle:
    def __init__(self, slab):
        self.s = slab
        self.st, self.ss, self.nsf, self.chi = _cell_tables(slab)

    def scalar_flux(self, psi):
        psi = np.asarray(psi).reshape(self.s.psi_shape)
        return np.einsum("d,ghdi->gi", self.s.w, psi)

    def source(self, phi, k):
        """q[g, c] for the cells from the scalar flux."""
        pbar = 0.5 * (phi[:, :-1] + phi[:, 1:])  # (G, cells)
        scat = np.einsum("cgh,hc->gc", self.ss, pbar)
        fis = np.einsum("cg,ch,hc->gc", self.chi, self.nsf, pbar)
        return scat + fis / k, scat, fis

    def sweep(self, q):
        """psi = H^-1 applied to the cell sources q[g, c] (vacuum faces)."""
        s = self.s
        G, nd, n = s.G, s.n_dir, s.n
        inv_d = 1.0 / s.delta
        mu = np.asarray(s.amu)[None, :]  # (1, nd)
        psi = np.zeros((G, 2, nd, n))
        st = self.st.T  # (G, cells)
        # mu > 0: march i = 1 .. n-1 through cell i-1
        up = np.zeros((G, nd))
        for i in range(1, n):
            c = i - 1
            a = mu * inv_d + 0.5 * st[:, c:c + 1]
            b = 0.5 * st[:, c:c + 1] - mu * inv_d
            up = (q[:, c:c + 1] - b * up) / a
            psi[:, 1, :, i] = up
        # mu < 0: march i = n-2 .. 0 through cell i
        up = np.zeros((G, nd))
        for i in range(n - 2, -1, -1):
            c = i
            a = mu * inv_d + 0.5 * st[:, c:c + 1]
            b = 0.5 * st[:, c:c + 1] - mu * inv_d
            up = (q[:, c:c + 1] - b * up) / a
            psi[:, 0, :, i] = up
        return psi

    def production(self, phi):
        """P = sum(F Psi): every direction contributes each non-inflow row,
        whose value is chi_g sum_g' nsf_g' phibar_g'(cell); each cell feeds one
        row per direction, so P = 2 n_dir sum_c sum_g chi_g sum_g' nsf phibar."""
        _, _, fis = self.source(phi, 1.0)
        return 2 * self.s.n_dir * float(np.sum(fis))

    def keig(self, tol_k=1e-12, max_iter=100000):
        s = self.s
        phi = np.ones((s.G, s.n))
        phi /= self.production(phi)
        k = 1.0
        hist = []
        for it in range(max_iter):
            q, _, _ = self.source(phi, k)
            psi = self.sweep(q)
            phi_new = self.scalar_flux(psi)
            pn = self.production(phi_new)
            k_new = k * pn
            phi = phi_new / pn
            hist.append(k_new)
            dk = abs(k_new - k)
            k = k_new
            if dk < tol_k * abs(k):
                break
        psi = psi / pn
        return dict(k=k, phi=phi, psi=psi, iters=it + 1, k_hist=np.array(hist))


# ---------------------------------------------------------------- matrices
def _factor_D(n, delta, pos):
    a = np.eye(n) / delta
    for i in range(n):
        if pos and i > 0:
            a[i, i - 1] = -1.0 / delta
        if not pos and i + 1 < n:
            a[i, i + 1] = -1.0 / delta
    return a


def _factor_Ip(n, pos, no_bc):
    a = 0.5 * np.eye(n)
    for i in range(n):
        if pos and i > 0:
            a[i, i - 1] = 0.5
        if not pos and i + 1 < n:
            a[i, i + 1] = 0.5
    if no_bc:
        a[0 if pos else n - 1, :] = 0.0
    return a


def _row_mask(s, m, pos):
    """Rows whose upstream cell (i-1 for mu > 0, i for mu < 0, clamped) has material m."""
    n = s.n
    cells = np.clip(np.arange(n) - (1 if pos else 0), 0, n - 2)
    return np.diag((np.asarray(s.mat)[cells] == m).astype(float))


def _kron(*mats):
    out = sp.csr_matrix(np.asarray(mats[0], dtype=np.float64))
    for m in mats[1:]:
        out = sp.kron(out, sp.csr_matrix(np.asarray(m, dtype=np.float64)), format="csr")
    return out


def assemble(s):
    """H, S, F (sparse CSR) with the index order of Psi."""
    G, nd, n = s.G, s.n_dir, s.n
    H = sp.csr_matrix((G * 2 * nd * n,) * 2)
    S = H.copy()
    F = H.copy()
    w_row = np.tile(s.w, (nd, 1))  # every direction row sums the weighted directions
    for h in (0, 1):
        pos = h == 1
        E = np.zeros((2, 2))
        E[h, h] = 1.0
        Intg = np.zeros((2, 2))
        Intg[h, :] = 1.0
        D = _factor_D(n, s.delta, pos)
        Ip = _factor_Ip(n, pos, False)
        IpN = _factor_Ip(n, pos, True)
        H = H + _kron(np.eye(G), E, np.diag(s.amu), D)
        for m in range(s.n_mat):
            M = _row_mask(s, m, pos)
            H = H + _kron(np.diag(s.sig_t[m]), E, np.eye(nd), M @ Ip)
            S = S + _kron(s.sig_s[m], Intg, w_row, M @ IpN)
            F = F + _kron(np.outer(s.chi[m], s.nu_sig_f[m]), Intg, w_row, M @ IpN)
    return H.tocsr(), S.tocsr(), F.tocsr()


def ges(s):
    """k and Psi from a library eigensolver on (H - S)^-1 F (largest magnitude)."""
    H, S, F = assemble(s)
    lu = spla.splu((H - S).tocsc())
    N = H.shape[0]
    vals, vecs = spla.eigs(spla.LinearOperator((N, N), matvec=lambda x: lu.solve(F @ x), dtype=np.float64), k=1,
                           which="LM", tol=1e-14, v0=np.ones(N))
    psi = np.real(vecs[:, 0])
    psi = psi / np.sum(F @ psi)
    return float(np.real(vals[0])), psi
