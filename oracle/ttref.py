"""ORACLE (test infrastructure only): dense-reconstruct tensor-train reference
in plain numpy FP64.

Follows arXiv 2309.03347, Sec. 2.2 (TT format, Eq. (TT_def_element),
TT-matrix format, Eq. (TT-matrix-componentwise), index-pair permutation
Eq. (permute), QTT of vectors and matrices, Algorithm 1) and the
TT-SVD / TT-rounding procedures of the TT paper the method cites
(Oseledets 2011, Algorithms 1 and 2), whose truncation rule we read as
``delta = eps * ||x||_F / sqrt(d - 1)`` per bond.

Layouts: a TT vector is a list of cores ``G_k`` of shape ``(r_{k-1}, n_k, r_k)``
with ``r_0 = r_d = 1``; a TT matrix is a list of cores ``A_k`` of shape
``(R_{k-1}, m_k, n_k, R_k)`` (output index ``i_k`` = m, input index ``j_k`` = n).
Flattening is row-major (the first core is the slowest index).
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np


# --------------------------------------------------------------------- TT vectors

def full(cores: Sequence[np.ndarray]) -> np.ndarray:
    """Dense tensor of a TT vector, Eq. (TT_def_element)."""
    out = np.ones((1, 1))
    shape = []
    for c in cores:
        r0, n, r1 = c.shape
        out = out.reshape(-1, r0) @ c.reshape(r0, n * r1)
        shape.append(n)
    return out.reshape(shape)


def ranks(cores) -> List[int]:
    return [1] + [c.shape[2] for c in cores]


def truncation_rank(s: np.ndarray, delta: float, rmax: int) -> int:
    """Smallest r with sqrt(sum_{i>=r} s_i^2) <= delta, at least 1, at most rmax."""
    tail = np.sqrt(np.cumsum((s ** 2)[::-1]))[::-1]  # tail[i] = ||s[i:]||
    r = len(s)
    for i in range(len(s)):
        if tail[i] <= delta:
            r = i
            break
    return int(max(1, min(r, rmax)))


def tt_svd(a: np.ndarray, eps: float = 0.0, rmax: int = 1 << 30) -> List[np.ndarray]:
    """TT decomposition of a dense tensor by sequential truncated SVDs."""
    shape = a.shape
    d = len(shape)
    delta = eps * np.linalg.norm(a) / np.sqrt(max(d - 1, 1))
    cores = []
    r = 1
    c = a.reshape(1, -1)
    for k in range(d - 1):
        c = c.reshape(r * shape[k], -1)
        u, s, vt = np.linalg.svd(c, full_matrices=False)
        rk = truncation_rank(s, delta, rmax)
        cores.append(u[:, :rk].reshape(r, shape[k], rk))
        c = s[:rk, None] * vt[:rk]
        r = rk
    cores.append(c.reshape(r, shape[-1], 1))
    return cores


def left_orthogonalize(cores):
    """QR sweep from the first core to the last (left-orthogonal cores 1..d-1)."""
    cores = [c.copy() for c in cores]
    for k in range(len(cores) - 1):
        r0, n, r1 = cores[k].shape
        q, rr = np.linalg.qr(cores[k].reshape(r0 * n, r1))
        cores[k] = q.reshape(r0, n, q.shape[1])
        cores[k + 1] = np.einsum("ab,bjc->ajc", rr, cores[k + 1])
    return cores


def tt_round(cores, eps: float = 0.0, rmax: int = 1 << 30):
    """TT rounding: left-to-right QR sweep, then right-to-left truncated SVD
    sweep with per-bond threshold eps * ||x|| / sqrt(d - 1) and rank cap."""
    d = len(cores)
    cores = left_orthogonalize(cores)
    nrm = np.linalg.norm(cores[-1])
    delta = eps * nrm / np.sqrt(max(d - 1, 1))
    for k in range(d - 1, 0, -1):
        r0, n, r1 = cores[k].shape
        u, s, vt = np.linalg.svd(cores[k].reshape(r0, n * r1), full_matrices=False)
        rk = truncation_rank(s, delta, rmax)
        cores[k] = vt[:rk].reshape(rk, n, r1)
        cores[k - 1] = np.einsum("ajb,bc->ajc", cores[k - 1], u[:, :rk] * s[:rk])
    return cores


def bond_singular_values(cores, k: int) -> np.ndarray:
    """Singular values of the unfolding (n_1..n_k) x (n_{k+1}..n_d) of the
    dense tensor (gauge-invariant; used to check rounding)."""
    a = full(cores)
    m = int(np.prod(a.shape[:k]))
    return np.linalg.svd(a.reshape(m, -1), compute_uv=False)


def dot(x, y) -> float:
    """<x, y> by left-to-right contraction of the cores."""
    v = np.ones((1, 1))
    for a, b in zip(x, y):
        v = np.einsum("ab,ajc,bjd->cd", v, a, b, optimize=True)  # pairwise contraction order
    return float(v[0, 0])


def norm(x) -> float:
    return float(np.sqrt(max(dot(x, x), 0.0)))


def add(x, y, alpha=1.0, beta=1.0):
    """alpha x + beta y by block-diagonal core concatenation (ranks add)."""
    d = len(x)
    out = []
    for k in range(d):
        a, b = x[k], y[k]
        if k == 0:
            out.append(np.concatenate([alpha * a, beta * b], axis=2))
        elif k == d - 1:
            out.append(np.concatenate([a, b], axis=0))
        else:
            c = np.zeros((a.shape[0] + b.shape[0], a.shape[1], a.shape[2] + b.shape[2]))
            c[: a.shape[0], :, : a.shape[2]] = a
            c[a.shape[0]:, :, a.shape[2]:] = b
            out.append(c)
    if d == 1:
        out = [alpha * x[0] + beta * y[0]]
    return out


# --------------------------------------------------------------------- TT matrices

def mat_full(cores) -> np.ndarray:
    """Dense matrix of a TT matrix, Eq. (TT-matrix-componentwise): row index
    (i_1..i_d), column index (j_1..j_d), both row-major."""
    out = np.ones((1, 1, 1))  # (rows, cols, R)
    for c in cores:
        R0, m, n, R1 = c.shape
        out = np.einsum("xyr,rijs->xiyjs", out, c)
        out = out.reshape(out.shape[0] * m, out.shape[2] * n, R1)
    return out[:, :, 0]


def mat_rank1(factors) -> List[np.ndarray]:
    """Rank-1 TT matrix of a Kronecker product of square matrices
    (the tensor product of univariate operators, Eq. (TT_matrices))."""
    return [f.reshape(1, f.shape[0], f.shape[1], 1).astype(np.float64) for f in factors]


def matvec(a_cores, x_cores):
    """Exact TT-matrix times TT-vector: core-wise Kronecker products
    Y_k[(a,b), i, (a',b')] = sum_j A_k[a, i, j, a'] X_k[b, j, b'] (ranks multiply)."""
    out = []
    for A, X in zip(a_cores, x_cores):
        R0, m, n, R1 = A.shape
        r0, n2, r1 = X.shape
        assert n == n2
        y = np.einsum("aijc,bjd->abicd", A, X).reshape(R0 * r0, m, R1 * r1)
        out.append(y)
    return out


def mat_add(a, b, alpha=1.0, beta=1.0):
    """alpha A + beta B for TT matrices (block-diagonal concatenation)."""
    d = len(a)
    out = []
    for k in range(d):
        x, y = a[k], b[k]
        if d == 1:
            out.append(alpha * x + beta * y)
        elif k == 0:
            out.append(np.concatenate([alpha * x, beta * y], axis=3))
        elif k == d - 1:
            out.append(np.concatenate([x, y], axis=0))
        else:
            c = np.zeros((x.shape[0] + y.shape[0], x.shape[1], x.shape[2], x.shape[3] + y.shape[3]))
            c[: x.shape[0], :, :, : x.shape[3]] = x
            c[x.shape[0]:, :, :, x.shape[3]:] = y
            out.append(c)
    return out


def mat_round(cores, eps=0.0, rmax=1 << 30):
    """Round a TT matrix by treating (i_k, j_k) as one mode of size m_k n_k."""
    shp = [(c.shape[1], c.shape[2]) for c in cores]
    v = [c.reshape(c.shape[0], c.shape[1] * c.shape[2], c.shape[3]) for c in cores]
    v = tt_round(v, eps, rmax)
    return [c.reshape(c.shape[0], m, n, c.shape[2]) for c, (m, n) in zip(v, shp)]


def qtt_matrix(m: np.ndarray, eps: float = 1e-14) -> List[np.ndarray]:
    """Algorithm 1 for one 2^l x 2^l matrix: reshape to a 2x...x2 tensor,
    permute the index pairs to (i_1, j_1, ..., i_l, j_l), TT-decompose with
    modes of size 4 = (i_k, j_k), then split each mode back into (2, 2)."""
    n = m.shape[0]
    l = int(round(np.log2(n)))
    assert 1 << l == n and m.shape == (n, n)
    t = m.reshape((2,) * (2 * l))
    perm = [x for k in range(l) for x in (k, l + k)]
    t = t.transpose(perm).reshape((4,) * l)
    cores = tt_svd(t, eps)
    return [c.reshape(c.shape[0], 2, 2, c.shape[2]) for c in cores]


def qtt_vector(v: np.ndarray, eps: float = 1e-14) -> List[np.ndarray]:
    """QTT of a length-2^l vector: reshape to 2x...x2 (first bit slowest)."""
    l = int(round(np.log2(v.size)))
    return tt_svd(v.reshape((2,) * l), eps)


# --------------------------------------------------------------------- local systems

def interface_frames(x, k):
    """Left frame U (prod n_<k, r_{k-1}) and right frame V (r_k, prod n_>k) of
    a TT vector around core k, so that full(x) = U . X_k . V."""
    left = np.ones((1, 1))
    for c in x[:k]:
        left = (left @ c.reshape(c.shape[0], -1)).reshape(-1, c.shape[2])
    right = np.ones((1, 1))
    for c in reversed(x[k + 1:]):
        right = (c.reshape(-1, c.shape[2]) @ right).reshape(c.shape[0], -1)
    return left, right


def projected_system(a_dense, x, k):
    """Galerkin local system (U (x) I (x) V)^T A (U (x) I (x) V) at core k."""
    U, V = interface_frames(x, k)
    n = x[k].shape[1]
    P = np.kron(np.kron(U, np.eye(n)), V.T)
    return P.T @ a_dense @ P, P
