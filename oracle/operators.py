"""ORACLE (test infrastructure only): the transport operators assembled as
sums of Kronecker products of one-dimensional factors (arXiv 2309.03347,
Sec. 3.2), as sparse matrices for tiny grids, plus the generalized
eigensolve (GES) of Sec. 4.1 used as an independent check of the sweep.

Readings of the paper used here (each is a place where the printed text is
ambiguous or garbled):

* D+ = (1/Delta) lower-bidiagonal(1 on the diagonal, -1 below) and
  D- = (1/Delta) upper-bidiagonal(-1 on the diagonal, +1 above), Sec. 3.2.1;
  with signed cosines mu*D^{sign(mu)} = |mu| * Dt where Dt+ = D+, Dt- = -D-.
  The inflow of mu > 0 is at i = 0 (the matrices and Eq. (discreteBCs)), the
  sentence that puts it at i = M is read as reversed.
* Ip+ = (1/2) lower-bidiagonal(1, 1), Ip- = (1/2) upper-bidiagonal(1, 1); the
  noBC variants zero the inflow row (row 0 for +, row n-1 for -).
* Octant selector E_o = e_o e_o^T; integral operator
  Intg^o = (e_o 1_8^T) (x) (1_{L/8} w8^T): rows of octant o, columns all
  directions weighted by w (the printed C_1 (x) (1 (x) w) has the wrong shape).
* Group matrices: Sigma_s[g, g'] = sigma_s(g' -> g) and chi nu_sigma_f^T
  (the printed diag() is only right for one group); F = fission,
  S = scattering (Eq. (OpFormkNTE)).
* Heterogeneous cross sections: each row of octant o takes the material of
  its upstream cell (cell i-1 along an axis with a positive cosine, cell i
  with a negative one, clamped at the faces), through a diagonal row mask.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def factor_D(n, delta, positive):
    """Dt^{+/-}: differentiation with the inflow boundary row embedded."""
    a = np.eye(n)
    if positive:
        a -= np.eye(n, k=-1)
    else:
        a -= np.eye(n, k=1)
    return a / delta


def factor_Ip(n, positive, no_bc=False):
    """Ip^{+/-} (and the noBC variants that zero the inflow row)."""
    a = np.eye(n) + (np.eye(n, k=-1) if positive else np.eye(n, k=1))
    a *= 0.5
    if no_bc:
        a[0 if positive else n - 1, :] = 0.0
    return a


def row_cells(n, positive):
    """Upstream cell of every vertex along one axis (clamped at the faces)."""
    v = np.arange(n)
    c = v - 1 if positive else v.copy()
    return np.clip(c, 0, n - 2)


def material_mask(prob, o, m):
    """Diagonal of the row mask M^o_m over vertices (k, j, i)."""
    n = prob.n
    ck = row_cells(n, bool(o & 4))
    cj = row_cells(n, bool(o & 2))
    ci = row_cells(n, bool(o & 1))
    mat = prob.mat[np.ix_(ck, cj, ci)]
    return (mat == m).astype(np.float64).ravel()


def _kron(*mats):
    out = sp.csr_matrix(np.ones((1, 1)))
    for m in mats:
        out = sp.kron(out, sp.csr_matrix(m), format="csr")
    return out


def _oct_sel(o):
    e = np.zeros((8, 8))
    e[o, o] = 1.0
    return e


def real_sh(n, m, x, y, z):
    """Real spherical harmonic of degree n, order m (m > 0 cosine type, m < 0
    sine type) with unit mean square over the sphere (Y_00 = 1), written out
    as Cartesian polynomials for n <= 3 at the direction (x, y, z)."""
    r3, r5, r7 = np.sqrt(3.0), np.sqrt(5.0), np.sqrt(7.0)
    table = {
        (0, 0): lambda: np.ones_like(np.asarray(x, dtype=np.float64)),
        (1, 1): lambda: r3 * x, (1, -1): lambda: r3 * y, (1, 0): lambda: r3 * z,
        (2, 0): lambda: r5 / 2 * (3 * z * z - 1), (2, 1): lambda: np.sqrt(15.0) * x * z,
        (2, -1): lambda: np.sqrt(15.0) * y * z, (2, 2): lambda: np.sqrt(15.0) / 2 * (x * x - y * y),
        (2, -2): lambda: np.sqrt(15.0) * x * y,
        (3, 0): lambda: r7 / 2 * (5 * z ** 3 - 3 * z), (3, 1): lambda: np.sqrt(42.0) / 4 * x * (5 * z * z - 1),
        (3, -1): lambda: np.sqrt(42.0) / 4 * y * (5 * z * z - 1),
        (3, 2): lambda: np.sqrt(105.0) / 2 * z * (x * x - y * y), (3, -2): lambda: np.sqrt(105.0) * x * y * z,
        (3, 3): lambda: np.sqrt(70.0) / 4 * x * (x * x - 3 * y * y),
        (3, -3): lambda: np.sqrt(70.0) / 4 * y * (3 * x * x - y * y),
    }
    return table[(n, m)]()


def signed_directions(q):
    """(x, y, z) cosines of all L directions, octant-major (octant o has
    positive x if o & 1, y if o & 2, z if o & 4)."""
    m8 = q.n_per_octant
    xs, ys, zs = [], [], []
    for o in range(8):
        xs.append(np.asarray(q.amu) * (1 if o & 1 else -1))
        ys.append(np.asarray(q.aeta) * (1 if o & 2 else -1))
        zs.append(np.asarray(q.axi) * (1 if o & 4 else -1))
    return np.concatenate(xs), np.concatenate(ys), np.concatenate(zs)


def aniso_angular(q, n):
    """L x L angular matrix of the order-n scattering term: entry (l, l') =
    sum_m Y_nm(Omega_l) Y_nm(Omega_l') w_l' (the moment operators
    L_n^+ L_n of Appendix A.2 with weights summing to 1)."""
    x, y, z = signed_directions(q)
    w = np.tile(q.w8, 8)
    A = np.zeros((x.size, x.size))
    for m in range(-n, n + 1):
        v = real_sh(n, m, x, y, z)
        A += np.outer(v, v * w)
    return A


def assemble(prob):
    """Sparse H, S, F (the matrices of Eq. (OpFormkNTE)) for a small grid."""
    n, G = prob.n, prob.G
    q = prob.quad
    dx, dy, dz = prob.delta
    m8 = q.n_per_octant
    IG = np.eye(G)
    Id = np.eye(m8)
    H = None
    S = None
    F = None
    for o in range(8):
        px, py, pz = bool(o & 1), bool(o & 2), bool(o & 4)
        E = _oct_sel(o)
        Ipx, Ipy, Ipz = factor_Ip(n, px), factor_Ip(n, py), factor_Ip(n, pz)
        Dx, Dy, Dz = factor_D(n, dx, px), factor_D(n, dy, py), factor_D(n, dz, pz)
        terms = [
            _kron(IG, E, np.diag(q.amu), Ipz, Ipy, Dx),
            _kron(IG, E, np.diag(q.aeta), Ipz, Dy, Ipx),
            _kron(IG, E, np.diag(q.axi), Dz, Ipy, Ipx),
        ]
        spat = _kron(Ipz, Ipy, Ipx)
        Nx = factor_Ip(n, px, True)
        Ny = factor_Ip(n, py, True)
        Nz = factor_Ip(n, pz, True)
        spat_nobc = _kron(Nz, Ny, Nx)
        intg = np.zeros((8, 8))
        intg[o, :] = 1.0
        dirm = np.outer(np.ones(m8), q.w8)
        for m in range(prob.n_mat):
            mask = sp.diags(material_mask(prob, o, m))
            terms.append(_kron(np.diag(prob.sig_t[m]), E, Id, mask @ spat))
            s_t = _kron(prob.sig_s[m], intg, dirm, mask @ spat_nobc)
            f_t = _kron(np.outer(prob.chi[m], prob.nu_sig_f[m]), intg, dirm, mask @ spat_nobc)
            S = s_t if S is None else S + s_t
            F = f_t if F is None else F + f_t
            for nord, field in ((2, "sig_s2"), (3, "sig_s3")):
                sn = getattr(prob, field, None)
                if sn is not None:
                    # order-n term: the L x L angular matrix restricted to the
                    # rows of octant o, with the order-n group matrix
                    A = aniso_angular(q, nord)
                    rows = np.zeros_like(A)
                    rows[o * m8:(o + 1) * m8, :] = A[o * m8:(o + 1) * m8, :]
                    S = S + _kron(np.asarray(sn[m]), rows, mask @ spat_nobc)
            s1 = getattr(prob, "sig_s1", None)
            if s1 is not None:
                # linear anisotropy (N_s = 1 of the moment operators, weights
                # summing to 1): row (o, d) gains 3 Omega_a(o, d) sum_{o', d'}
                # w_d' Omega_a(o', d') for each axis a, with the P1 group matrix
                for bit, cos in ((1, q.amu), (2, q.aeta), (4, q.axi)):
                    sgn = np.array([1.0 if (oo & bit) else -1.0 for oo in range(8)])
                    octm = np.zeros((8, 8))
                    octm[o, :] = sgn[o] * sgn
                    dirp = np.outer(cos, cos * q.w8)
                    S = S + _kron(3.0 * np.asarray(s1[m]), octm, dirp, mask @ spat_nobc)
        for t in terms:
            H = t if H is None else H + t
    return H.tocsr(), S.tocsr(), F.tocsr()


def reflective_rows(prob, H):
    """H with the rows of reflective inflow faces replaced by the mirror
    condition psi(l, v) - psi(l_R, v) = 0 (paper silent: it treats vacuum
    faces only).  l_R flips the cosines of every inflow face through v; a
    vertex on any vacuum inflow face keeps its vacuum row."""
    n, G, m8 = prob.n, prob.G, prob.quad.n_per_octant
    L = 8 * m8
    n3 = n ** 3
    H = H.tolil()
    kk, jj, ii = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    kk, jj, ii = kk.ravel(), jj.ravel(), ii.ravel()
    for o in range(8):
        px, py, pz = o & 1, o & 2, o & 4
        on = [(ii == 0) if px else (ii == n - 1),
              (jj == 0) if py else (jj == n - 1),
              (kk == 0) if pz else (kk == n - 1)]
        face = [0 if px else 1, 2 if py else 3, 4 if pz else 5]
        for v in range(n3):
            flip, vac, any_in = 0, False, False
            for a, bit in zip(range(3), (1, 2, 4)):
                if on[a][v]:
                    any_in = True
                    if prob.bc[face[a]]:
                        flip |= bit
                    else:
                        vac = True
            if not any_in or vac:
                continue
            for g in range(G):
                for d in range(m8):
                    row = (g * L + o * m8 + d) * n3 + v
                    col = (g * L + (o ^ flip) * m8 + d) * n3 + v
                    H.rows[row] = [row, col]
                    H.data[row] = [1.0, -1.0]
    return H.tocsr()


def ges_k(prob, H=None, S=None, F=None, tol=1e-13):
    """Dominant eigenvalue k of H psi = (S + F/k) psi, i.e. the largest
    eigenvalue of (H - S)^{-1} F, by a library sparse LU + Arnoldi (GES)."""
    if H is None:
        H, S, F = assemble(prob)
    lu = spla.splu((H - S).tocsc())
    N = H.shape[0]
    op = spla.LinearOperator((N, N), matvec=lambda x: lu.solve(F @ x), dtype=np.float64)
    vals, vecs = spla.eigs(op, k=1, which="LM", tol=tol, v0=np.ones(N))
    k = float(np.real(vals[0]))
    v = np.real(vecs[:, 0])
    v = v / (np.sum(F @ v))  # sum(F psi) = 1
    return k, v


def k_infinity(sig_t, sig_s, nu_sig_f, chi):
    """Closed form for an infinite homogeneous medium:
    k_inf = nu_sig_f^T (Sigma_t - Sigma_s)^{-1} chi."""
    A = np.diag(sig_t) - sig_s
    return float(nu_sig_f @ np.linalg.solve(A, chi))
