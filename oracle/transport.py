"""ORACLE (test infrastructure only): ctypes driver for ``oracle/sweep.c``.

Full-grid FP64 vertex diamond-difference transport (arXiv 2309.03347,
Eq. (Discretized_kNTE), Sec. 2.1.5 and Appendix A) and the k fixed point of
Eq. (k_eff_fixed_points).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sweep.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle_sweep.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile sweep.c with gcc -O2 -fopenmp into oracle/_build/."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [
        ("l", C.c_int), ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
        ("G", C.c_int), ("n_mat", C.c_int),
        ("sig_t", C.POINTER(C.c_double)), ("sig_s", C.POINTER(C.c_double)),
        ("nu_sig_f", C.POINTER(C.c_double)), ("chi", C.POINTER(C.c_double)),
        ("mat", C.POINTER(C.c_uint8)), ("L", C.c_int),
        ("amu", C.POINTER(C.c_double)), ("aeta", C.POINTER(C.c_double)),
        ("axi", C.POINTER(C.c_double)), ("w8", C.POINTER(C.c_double)),
        ("bc", C.c_int * 6), ("threads", C.c_int), ("sig_s1", C.POINTER(C.c_double)),
    ]


class _Opts(C.Structure):
    _fields_ = [("tol_k", C.c_double), ("max_iter", C.c_int), ("k0", C.c_double),
                ("store_psi", C.c_int)]


class _Res(C.Structure):
    _fields_ = [("k", C.c_double), ("iters", C.c_int), ("dk_last", C.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER(_Problem)
            D = C.POINTER(C.c_double)
            lib.oracle_apply_H.argtypes = [P, D, D]
            lib.oracle_sweep.argtypes = [P, D, D]
            lib.oracle_apply_SF.argtypes = [P, D, D, D]
            lib.oracle_keig.argtypes = [P, C.POINTER(_Opts), D, D, D, D, D, C.POINTER(_Res)]
            lib.oracle_keig.restype = C.c_int
            lib.oracle_balance.argtypes = [P, D, D, D, D, D, D]
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class OracleProblem:
    """Holds contiguous copies of a ``keig_inputs.Problem``'s tables."""

    def __init__(self, prob, threads: int = 0):
        self.prob = prob
        q = prob.quad
        self._keep = dict(
            sig_t=np.ascontiguousarray(prob.sig_t, dtype=np.float64),
            sig_s=np.ascontiguousarray(prob.sig_s, dtype=np.float64),
            nsf=np.ascontiguousarray(prob.nu_sig_f, dtype=np.float64),
            chi=np.ascontiguousarray(prob.chi, dtype=np.float64),
            mat=np.ascontiguousarray(prob.mat, dtype=np.uint8),
            amu=np.ascontiguousarray(q.amu, dtype=np.float64),
            aeta=np.ascontiguousarray(q.aeta, dtype=np.float64),
            axi=np.ascontiguousarray(q.axi, dtype=np.float64),
            w8=np.ascontiguousarray(q.w8, dtype=np.float64),
        )
        k = self._keep
        dx, dy, dz = prob.delta
        s = _Problem()
        s.l, s.dx, s.dy, s.dz = prob.l, dx, dy, dz
        s.G, s.n_mat = prob.G, prob.n_mat
        s.sig_t, s.sig_s, s.nu_sig_f, s.chi = _dp(k["sig_t"]), _dp(k["sig_s"]), _dp(k["nsf"]), _dp(k["chi"])
        s.mat = k["mat"].ctypes.data_as(C.POINTER(C.c_uint8))
        s.L = q.L
        s.amu, s.aeta, s.axi, s.w8 = _dp(k["amu"]), _dp(k["aeta"]), _dp(k["axi"]), _dp(k["w8"])
        for i in range(6):
            s.bc[i] = int(prob.bc[i])
        s.threads = int(threads)
        if getattr(prob, "sig_s2", None) is not None or getattr(prob, "sig_s3", None) is not None:
            raise NotImplementedError("the stencil oracle covers scattering orders N_s <= 1; use "
                                      "operators.assemble and operators.ges_k for higher orders")
        if getattr(prob, "sig_s1", None) is not None:
            self._keep["sig_s1"] = np.ascontiguousarray(prob.sig_s1, dtype=np.float64)
            s.sig_s1 = _dp(self._keep["sig_s1"])
        else:
            s.sig_s1 = None
        self.s = s
        self.shape = prob.psi_shape

    def _vec(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.shape)
        return x

    def apply_H(self, psi):
        psi = self._vec(psi)
        out = np.empty_like(psi)
        _load().oracle_apply_H(C.byref(self.s), _dp(psi), _dp(out))
        return out

    def sweep(self, b):
        """H^{-1} b (downstream substitution for every (g, l))."""
        b = self._vec(b)
        out = np.empty_like(b)
        _load().oracle_sweep(C.byref(self.s), _dp(b), _dp(out))
        return out

    def apply_SF(self, psi):
        psi = self._vec(psi)
        s = np.empty_like(psi)
        f = np.empty_like(psi)
        _load().oracle_apply_SF(C.byref(self.s), _dp(psi), _dp(s), _dp(f))
        return s, f

    def keig(self, psi0=None, phi0=None, tol_k=1e-8, max_iter=10000, k0=1.0,
             store_psi=False, history=False):
        """Power iteration; returns dict(k, iters, dk, phi, psi, k_hist)."""
        G, L, n = self.prob.G, self.prob.L, self.prob.n
        if psi0 is None and phi0 is None:
            phi0 = np.ones((G, n, n, n))
        p0 = self._vec(psi0) if psi0 is not None else None
        f0 = np.ascontiguousarray(phi0, dtype=np.float64) if phi0 is not None else None
        phi = np.empty((G, n, n, n))
        psi = np.empty(self.shape) if store_psi else None
        hist = np.zeros(max_iter) if history else None
        o = _Opts(tol_k, int(max_iter), k0, int(store_psi))
        r = _Res()
        rc = _load().oracle_keig(
            C.byref(self.s), C.byref(o),
            _dp(p0) if p0 is not None else None,
            _dp(f0) if f0 is not None else None,
            _dp(phi), _dp(psi) if psi is not None else None,
            _dp(hist) if hist is not None else None, C.byref(r))
        if rc < 0:
            raise ValueError("oracle_keig: only vacuum faces are supported")
        return dict(k=r.k, iters=r.iters, dk=r.dk_last, phi=phi, psi=psi,
                    converged=(rc == 0),
                    k_hist=hist[: r.iters] if hist is not None else None)

    def balance(self, psi):
        """(leakage, absorption, in-scatter, production) of a solution."""
        psi = self._vec(psi)
        v = [C.c_double() for _ in range(5)]
        _load().oracle_balance(C.byref(self.s), _dp(psi), *[C.byref(x) for x in v])
        return dict(leak=v[0].value, absorb=v[1].value, scat_in=v[3].value, prod=v[4].value)


def scalar_flux(prob, psi):
    """phi[g, v] = sum_l w_l psi[g, l, v] (isotropic moment, Appendix A.3)."""
    psi = np.asarray(psi).reshape(prob.psi_shape)
    return np.einsum("l,glkji->gkji", prob.quad.w, psi)


def production(prob, phi):
    """sum(F Psi) expressed through the scalar flux: every direction of
    octant o contributes each non-inflow row, whose value is
    chi_g * sum_g' nu_sig_f_g' * (8-corner average of phi_g') of the row's
    upstream cell; each cell is the upstream cell of exactly one row per
    octant, so the sum is L * sum_c sum_g chi_g sum_g' nsf_g' phibar_g'(c)."""
    phi = np.asarray(phi)
    pbar = 0.125 * sum(phi[:, a:a + prob.n - 1, b:b + prob.n - 1, c:c + prob.n - 1]
                       for a in (0, 1) for b in (0, 1) for c in (0, 1))
    m = prob.mat
    chi_sum = prob.chi.sum(axis=1)[m]
    nsf = prob.nu_sig_f[m]  # (cz, cy, cx, G)
    src = np.einsum("kjig,gkji->kji", nsf, pbar)
    return prob.L * float(np.sum(chi_sum * src))
