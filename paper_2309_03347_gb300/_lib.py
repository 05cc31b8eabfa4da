"""ctypes marshalling for libkeig_tt.so.  Names follow include/keig.h."""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import List, Optional, Sequence

import numpy as np

TT_OK, TT_EINVAL, TT_ENOMEM, TT_ECUDA, TT_ENOCONV, TT_ETIMEOUT, TT_ENONFINITE = 0, -1, -2, -3, -4, -5, -6
TT_OP_H, TT_OP_S, TT_OP_F = 0, 1, 2
TT_MV_EXACT, TT_MV_AMEN = 0, 1
TT_FP64 = 0
TT_FP32_REFINED = 3
TT_TF32_SPLIT = 1
TT_BF16_SPLIT = 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_FILE = os.path.join(_HERE, "_build", "libkeig_tt.so")
_lock = threading.Lock()
_lib = None

D = C.POINTER(C.c_double)
I = C.POINTER(C.c_int)
# keig.h: tt_alloc_fn / tt_free_fn
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class KeigError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class TTProblem(C.Structure):
    _fields_ = [
        ("l", C.c_int), ("side", C.c_double * 3), ("G", C.c_int), ("n_mat", C.c_int),
        ("sig_t", D), ("sig_s", D), ("nu_sig_f", D), ("chi", D), ("inv_v", D),
        ("mat", C.POINTER(C.c_uint8)), ("n_dir", C.c_int),
        ("amu", D), ("aeta", D), ("axi", D), ("w", D), ("bc", C.c_int * 6), ("sig_s1", D), ("sig_s2", D),
        ("sig_s3", D),
    ]


class KeigOpts(C.Structure):
    _fields_ = [
        ("eps", C.c_double), ("rmax", C.c_int), ("tol_k", C.c_double), ("tol_psi", C.c_double),
        ("max_iter", C.c_int), ("solve_sweeps", C.c_int), ("mv_sweeps", C.c_int), ("kick", C.c_int),
        ("scheme", C.c_int), ("prec", C.c_int), ("eps_op", C.c_double), ("psi0_cores", D),
        ("mv_kind", C.c_int), ("local_form", C.c_int), ("solve_method", C.c_int),
    ]


class KeigResult(C.Structure):
    _fields_ = [
        ("k", C.c_double), ("iters", C.c_int), ("dk_last", C.c_double), ("wall_ms", C.c_double),
        ("max_rank", C.c_int), ("k_hist", C.c_double * 512), ("t_hist", C.c_double * 512),
    ]


def lib_path() -> str:
    return _LIB_FILE


def load():
    """Load libkeig_tt.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_FILE):
            raise ImportError(f"libkeig_tt.so not built ({_LIB_FILE}); run __graft_entry__.build()")
        lib = C.CDLL(_LIB_FILE)
        P = C.c_void_p
        sig = {
            "tt_ctx_create": ([C.POINTER(P), P, ALLOC_FN, FREE_FN, P], C.c_int),
            "tt_ctx_destroy": ([P], C.c_int),
            "tt_last_error": ([P], C.c_char_p),
            "tt_version": ([], C.c_char_p),
            "tt_ctx_counters": ([P, C.POINTER(C.c_int64), D], C.c_int),
            "tt_ctx_reset_counters": ([P], C.c_int),
            "tt_ctx_set_wait_limit": ([P, C.c_longlong], C.c_int),
            "tt_measure_fma_peak": ([P, C.c_int, C.c_int, C.c_int, D], C.c_int),
            "tt_gemm_f32": ([P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float, P, C.c_int,
                             C.c_longlong, P, C.c_int, C.c_longlong, C.c_float, P, C.c_int, C.c_longlong, C.c_int],
                            C.c_int),
            "tt_ctx_set_profiling": ([P, C.c_int], C.c_int),
            "tt_ctx_gemm_stats": ([P, C.POINTER(C.c_int64), D, D], C.c_int),
            "tt_ctx_gemm32_stats": ([P, C.POINTER(C.c_int64), D, D], C.c_int),
            "tt_ctx_gemmtc_stats": ([P, C.POINTER(C.c_int64), D, D], C.c_int),
            "tt_ctx_gmres_stats": ([P, C.POINTER(C.c_int64), D, D], C.c_int),
            "tt_vec_create": ([P, C.c_int, I, I, D, C.c_int, C.POINTER(P)], C.c_int),
            "tt_vec_destroy": ([P], C.c_int),
            "tt_vec_shape": ([P, I, I, I], C.c_int),
            "tt_vec_numel": ([P, C.POINTER(C.c_size_t)], C.c_int),
            "tt_vec_get_cores": ([P, P, D, C.c_int], C.c_int),
            "tt_vec_to_dense": ([P, P, D, C.c_size_t], C.c_int),
            "tt_vec_axpby": ([P, C.c_double, P, C.c_double, P], C.c_int),
            "tt_vec_scale": ([P, P, C.c_double], C.c_int),
            "tt_vec_dot": ([P, P, P, D], C.c_int),
            "tt_vec_norm": ([P, P, D], C.c_int),
            "tt_vec_sum": ([P, P, D], C.c_int),
            "tt_round": ([P, P, C.c_double, C.c_int], C.c_int),
            "tt_op_create": ([P, C.c_int, I, I, I, D, C.c_int, C.POINTER(P)], C.c_int),
            "tt_op_destroy": ([P], C.c_int),
            "tt_op_shape": ([P, I, I, I, I], C.c_int),
            "tt_op_numel": ([P, C.POINTER(C.c_size_t)], C.c_int),
            "tt_op_get_cores": ([P, P, D, C.c_int], C.c_int),
            "tt_op_axpby": ([P, C.c_double, P, C.c_double, P, C.c_double, C.c_int, C.POINTER(P)], C.c_int),
            "tt_build_operator": ([P, C.POINTER(TTProblem), C.c_int, C.c_double, C.POINTER(P)], C.c_int),
            "tt_matvec": ([P, P, P, C.c_double, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, C.POINTER(P)],
                          C.c_int),
            "tt_solve_local": ([P, P, P, P, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, I, D], C.c_int),
            "tt_solve_dmrg": ([P, P, P, P, C.c_double, C.c_int, C.c_int, C.c_int, I, D], C.c_int),
            "keig_default_opts": ([C.POINTER(KeigOpts)], C.c_int),
            "keig_fixed_point": ([P, C.POINTER(TTProblem), C.POINTER(KeigOpts), C.POINTER(KeigResult),
                                  C.POINTER(P), D], C.c_int),
            "tt_scalar_flux": ([P, P, D, C.c_int, C.POINTER(P)], C.c_int),
            "tt_dot_noalloc": ([D, I, D, I, C.c_int, I, D, P, C.c_char_p, C.c_size_t], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(D)


def _ip(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(I)


class TorchCachingAllocator:
    """Device allocator hooks (keig.h tt_alloc_fn / tt_free_fn) that draw on
    PyTorch's caching allocator, so the library shares torch's memory pool.
    alloc(bytes, stream) returns a device address or 0; free(ptr, stream)."""

    def __init__(self, device=None):
        import torch
        self.device = torch.cuda.current_device() if device is None else int(device)

    def alloc(self, nbytes: int, stream: int) -> int:
        import torch
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream))
        except RuntimeError:  # out of memory
            return 0

    def free(self, ptr: int, stream: int) -> None:
        import torch
        torch.cuda.caching_allocator_delete(ptr)


class Context:
    """A tt_ctx bound to the current CUDA device and a torch CUDA stream.
    allocator: None (the device's stream-ordered pool) or an object with
    alloc(nbytes, stream) -> address (0 on failure) and free(address, stream),
    e.g. TorchCachingAllocator()."""

    def __init__(self, stream=None, allocator=None):
        import torch
        if not torch.cuda.is_available():
            raise KeigError(TT_ECUDA, "CUDA device required (no CPU fallback)")
        self.lib = load()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.allocator = allocator
        if allocator is not None:
            def _alloc(nbytes, strm, user):
                return allocator.alloc(nbytes, strm or 0) or None

            def _free(ptr, strm, user):
                allocator.free(ptr, strm or 0)
            # the callbacks must outlive the context
            self._hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
        else:
            self._hooks = (ALLOC_FN(), FREE_FN())
        h = C.c_void_p()
        self._check(self.lib.tt_ctx_create(C.byref(h), C.c_void_p(stream.cuda_stream), self._hooks[0],
                                           self._hooks[1], None), None)
        self.h = h

    def _check(self, rc, h="self"):
        if rc != TT_OK:
            hh = self.h if h == "self" else None
            msg = self.lib.tt_last_error(hh).decode() if hh else "tt_ctx_create failed"
            raise KeigError(rc, msg)

    def check(self, rc):
        self._check(rc)

    def close(self):
        if getattr(self, "h", None):
            self.lib.tt_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def counters(self):
        n = C.c_int64()
        f = C.c_double()
        self.check(self.lib.tt_ctx_counters(self.h, C.byref(n), C.byref(f)))
        return int(n.value), float(f.value)

    def reset_counters(self):
        self.check(self.lib.tt_ctx_reset_counters(self.h))

    def set_wait_limit(self, spins: int):
        """Spin limit of the bounded device waits (keig.h); < 0: default."""
        self.check(self.lib.tt_ctx_set_wait_limit(self.h, int(spins)))

    def set_profiling(self, on: bool):
        self.check(self.lib.tt_ctx_set_profiling(self.h, int(bool(on))))

    def gemm_stats(self):
        n = C.c_int64()
        ms = C.c_double()
        f = C.c_double()
        self.check(self.lib.tt_ctx_gemm_stats(self.h, C.byref(n), C.byref(ms), C.byref(f)))
        return int(n.value), float(ms.value), float(f.value)

    def gmres_stats(self):
        n = C.c_int64()
        ms = C.c_double()
        f = C.c_double()
        self.check(self.lib.tt_ctx_gmres_stats(self.h, C.byref(n), C.byref(ms), C.byref(f)))
        return int(n.value), float(ms.value), float(f.value)

    def gemmtc_stats(self):
        n = C.c_int64()
        ms = C.c_double()
        f = C.c_double()
        self.check(self.lib.tt_ctx_gemmtc_stats(self.h, C.byref(n), C.byref(ms), C.byref(f)))
        return int(n.value), float(ms.value), float(f.value)

    def gemm32_stats(self):
        n = C.c_int64()
        ms = C.c_double()
        f = C.c_double()
        self.check(self.lib.tt_ctx_gemm32_stats(self.h, C.byref(n), C.byref(ms), C.byref(f)))
        return int(n.value), float(ms.value), float(f.value)


class TTVec:
    """Owning wrapper of a tt_vec handle."""

    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.h = handle

    def __del__(self):
        if getattr(self, "h", None):
            self.ctx.lib.tt_vec_destroy(self.h)
            self.h = None

    @property
    def shape(self):
        d = C.c_int()
        self.ctx.check(self.ctx.lib.tt_vec_shape(self.h, C.byref(d), None, None))
        n = np.zeros(d.value, np.int32)
        r = np.zeros(d.value + 1, np.int32)
        self.ctx.check(self.ctx.lib.tt_vec_shape(self.h, C.byref(d), n.ctypes.data_as(I), r.ctypes.data_as(I)))
        return list(n), list(r)

    @property
    def ranks(self):
        return self.shape[1]

    def cores(self) -> List[np.ndarray]:
        n, r = self.shape
        cnt = C.c_size_t()
        self.ctx.check(self.ctx.lib.tt_vec_numel(self.h, C.byref(cnt)))
        buf = np.empty(cnt.value)
        self.ctx.check(self.ctx.lib.tt_vec_get_cores(self.ctx.h, self.h, _dp(buf), 0))
        out, off = [], 0
        for k in range(len(n)):
            sz = r[k] * n[k] * r[k + 1]
            out.append(buf[off:off + sz].reshape(r[k], n[k], r[k + 1]).copy())
            off += sz
        return out

    def dense_cuda(self):
        import torch
        n, _ = self.shape
        t = torch.empty(int(np.prod(n)), dtype=torch.float64, device="cuda")
        self.ctx.check(self.ctx.lib.tt_vec_to_dense(self.ctx.h, self.h, C.cast(t.data_ptr(), D), t.numel()))
        return t.reshape([int(v) for v in n])

    def dot(self, other: "TTVec") -> float:
        v = C.c_double()
        self.ctx.check(self.ctx.lib.tt_vec_dot(self.ctx.h, self.h, other.h, C.byref(v)))
        return v.value

    def norm(self) -> float:
        v = C.c_double()
        self.ctx.check(self.ctx.lib.tt_vec_norm(self.ctx.h, self.h, C.byref(v)))
        return v.value

    def sum(self) -> float:
        v = C.c_double()
        self.ctx.check(self.ctx.lib.tt_vec_sum(self.ctx.h, self.h, C.byref(v)))
        return v.value

    def scale(self, a: float):
        self.ctx.check(self.ctx.lib.tt_vec_scale(self.ctx.h, self.h, float(a)))

    def axpby(self, a: float, x: "TTVec", b: float):
        """self = a x + b self (ranks add)."""
        self.ctx.check(self.ctx.lib.tt_vec_axpby(self.ctx.h, float(a), x.h, float(b), self.h))


class TTOp:
    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.h = handle

    def __del__(self):
        if getattr(self, "h", None):
            self.ctx.lib.tt_op_destroy(self.h)
            self.h = None

    @property
    def shape(self):
        d = C.c_int()
        self.ctx.check(self.ctx.lib.tt_op_shape(self.h, C.byref(d), None, None, None))
        m = np.zeros(d.value, np.int32)
        n = np.zeros(d.value, np.int32)
        R = np.zeros(d.value + 1, np.int32)
        self.ctx.check(self.ctx.lib.tt_op_shape(self.h, C.byref(d), m.ctypes.data_as(I), n.ctypes.data_as(I),
                                                R.ctypes.data_as(I)))
        return list(m), list(n), list(R)

    def cores(self) -> List[np.ndarray]:
        m, n, R = self.shape
        cnt = C.c_size_t()
        self.ctx.check(self.ctx.lib.tt_op_numel(self.h, C.byref(cnt)))
        buf = np.empty(cnt.value)
        self.ctx.check(self.ctx.lib.tt_op_get_cores(self.ctx.h, self.h, _dp(buf), 0))
        out, off = [], 0
        for k in range(len(m)):
            sz = R[k] * m[k] * n[k] * R[k + 1]
            out.append(buf[off:off + sz].reshape(R[k], m[k], n[k], R[k + 1]).copy())
            off += sz
        return out


# ---------------------------------------------------------------- C-ABI names

def tt_ctx_create(stream=None, allocator=None) -> Context:
    return Context(stream, allocator)


def _cat(cores: Sequence):
    """Concatenate cores given as numpy arrays (host) or torch CUDA tensors (device)."""
    first = cores[0]
    if hasattr(first, "is_cuda") and first.is_cuda:
        import torch
        flat = torch.cat([c.reshape(-1).to(torch.float64) for c in cores]).contiguous()
        return flat, C.cast(flat.data_ptr(), D), 1
    flat = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.float64).ravel() for c in cores]))
    return flat, _dp(flat), 0


def tt_vec_create(ctx: Context, cores: Sequence) -> TTVec:
    n = [int(c.shape[1]) for c in cores]
    r = [1] + [int(c.shape[2]) for c in cores]
    na, npp = _ip(n)
    ra, rp = _ip(r)
    flat, ptr, dev = _cat(cores)
    h = C.c_void_p()
    ctx.check(ctx.lib.tt_vec_create(ctx.h, len(n), npp, rp, ptr, dev, C.byref(h)))
    return TTVec(ctx, h)


def tt_op_create(ctx: Context, cores: Sequence) -> TTOp:
    m = [int(c.shape[1]) for c in cores]
    n = [int(c.shape[2]) for c in cores]
    R = [1] + [int(c.shape[3]) for c in cores]
    ma, mp = _ip(m)
    na, npp = _ip(n)
    Ra, Rp = _ip(R)
    flat, ptr, dev = _cat(cores)
    h = C.c_void_p()
    ctx.check(ctx.lib.tt_op_create(ctx.h, len(m), mp, npp, Rp, ptr, dev, C.byref(h)))
    return TTOp(ctx, h)


def tt_round(ctx: Context, x: TTVec, eps: float, rmax: int = 0) -> TTVec:
    ctx.check(ctx.lib.tt_round(ctx.h, x.h, float(eps), int(rmax)))
    return x


def tt_op_axpby(ctx: Context, a: float, A: TTOp, b: float, B: TTOp, eps: float = -1.0, rmax: int = 0) -> TTOp:
    h = C.c_void_p()
    ctx.check(ctx.lib.tt_op_axpby(ctx.h, float(a), A.h, float(b), B.h, float(eps), int(rmax), C.byref(h)))
    return TTOp(ctx, h)


def tt_matvec(ctx: Context, A: TTOp, x: TTVec, scale: float = 1.0, method: int = TT_MV_EXACT,
              eps: float = -1.0, rmax: int = 0, max_sweeps: int = 4, prec: int = TT_FP64) -> TTVec:
    h = C.c_void_p()
    ctx.check(ctx.lib.tt_matvec(ctx.h, A.h, x.h, float(scale), int(method), float(eps), int(rmax),
                                int(max_sweeps), int(prec), C.byref(h)))
    return TTVec(ctx, h)


def tt_solve_local(ctx: Context, A: TTOp, b: TTVec, x: TTVec, eps: float, rmax: int = 0,
                   max_sweeps: int = 10, kick: int = 4, prec: int = TT_FP64, allow_noconv: bool = False):
    sw = C.c_int()
    dx = C.c_double()
    rc = ctx.lib.tt_solve_local(ctx.h, A.h, b.h, x.h, float(eps), int(rmax), int(max_sweeps), int(kick),
                                int(prec), C.byref(sw), C.byref(dx))
    if not (allow_noconv and rc == TT_ENOCONV):
        ctx.check(rc)
    return dict(sweeps=sw.value, rel_change=dx.value, code=rc)


def tt_solve_dmrg(ctx: Context, A: TTOp, b: TTVec, x: TTVec, eps: float, rmax: int = 0,
                  max_sweeps: int = 10, prec: int = TT_FP64, allow_noconv: bool = False):
    """Two-site DMRG solve of A x = b (keig.h tt_solve_dmrg); x: guess in, solution out."""
    sw = C.c_int()
    dx = C.c_double()
    rc = ctx.lib.tt_solve_dmrg(ctx.h, A.h, b.h, x.h, float(eps), int(rmax), int(max_sweeps), int(prec),
                               C.byref(sw), C.byref(dx))
    if not (allow_noconv and rc == TT_ENOCONV):
        ctx.check(rc)
    return dict(sweeps=sw.value, rel_change=dx.value, code=rc)


class _ProblemArrays:
    """Keeps the contiguous arrays a TTProblem points into alive."""

    def __init__(self, prob):
        q = prob.quad
        self.arrays = dict(
            sig_t=np.ascontiguousarray(prob.sig_t, np.float64),
            sig_s=np.ascontiguousarray(prob.sig_s, np.float64),
            nsf=np.ascontiguousarray(prob.nu_sig_f, np.float64),
            chi=np.ascontiguousarray(prob.chi, np.float64),
            mat=np.ascontiguousarray(prob.mat, np.uint8),
            amu=np.ascontiguousarray(q.amu, np.float64),
            aeta=np.ascontiguousarray(q.aeta, np.float64),
            axi=np.ascontiguousarray(q.axi, np.float64),
            w=np.ascontiguousarray(q.w8, np.float64),
        )
        a = self.arrays
        s = TTProblem()
        s.l = prob.l
        for i in range(3):
            s.side[i] = float(prob.side[i])
        s.G, s.n_mat = prob.G, prob.n_mat
        s.sig_t, s.sig_s, s.nu_sig_f, s.chi = _dp(a["sig_t"]), _dp(a["sig_s"]), _dp(a["nsf"]), _dp(a["chi"])
        if getattr(prob, "inv_v", None) is not None:
            a["inv_v"] = np.ascontiguousarray(prob.inv_v, np.float64)
            s.inv_v = _dp(a["inv_v"])
        else:
            s.inv_v = None
        s.mat = a["mat"].ctypes.data_as(C.POINTER(C.c_uint8))
        s.n_dir = q.n_per_octant
        s.amu, s.aeta, s.axi, s.w = _dp(a["amu"]), _dp(a["aeta"]), _dp(a["axi"]), _dp(a["w"])
        for i in range(6):
            s.bc[i] = int(prob.bc[i])
        for f in ("sig_s1", "sig_s2", "sig_s3"):
            if getattr(prob, f, None) is not None:
                a[f] = np.ascontiguousarray(getattr(prob, f), np.float64)
                setattr(s, f, _dp(a[f]))
            else:
                setattr(s, f, None)
        self.s = s


def tt_build_operator(ctx: Context, prob, kind: int, eps_op: float = 1e-12) -> TTOp:
    pa = _ProblemArrays(prob)
    h = C.c_void_p()
    ctx.check(ctx.lib.tt_build_operator(ctx.h, C.byref(pa.s), int(kind), float(eps_op), C.byref(h)))
    return TTOp(ctx, h)


def keig_default_opts() -> KeigOpts:
    o = KeigOpts()
    load().keig_default_opts(C.byref(o))
    return o


def keig_fixed_point(ctx: Context, prob, opts: Optional[KeigOpts] = None, want_psi: bool = False,
                     want_phi: bool = False, allow_noconv: bool = False, psi0=None, phi_out=None):
    """Run the QTT fixed point; returns dict(k, iters, dk, wall_ms, max_rank,
    k_hist, t_hist, psi (TTVec or None), phi (host array or None), code).
    phi_out: optional preallocated host array (G, n, n, n) float64 for the
    scalar flux (e.g. in pinned memory); implies want_phi."""
    pa = _ProblemArrays(prob)
    o = opts if opts is not None else keig_default_opts()
    keep = None
    if psi0 is not None:
        keep = np.ascontiguousarray(np.concatenate([np.asarray(c, np.float64).ravel() for c in psi0]))
        o.psi0_cores = _dp(keep)
    res = KeigResult()
    h = C.c_void_p()
    if phi_out is not None:
        if phi_out.dtype != np.float64 or not phi_out.flags.c_contiguous or phi_out.size != prob.G * prob.n ** 3:
            raise KeigError(TT_EINVAL, "keig_fixed_point: phi_out must be a contiguous float64 (G, n, n, n) array")
        phi = phi_out
    else:
        phi = np.empty((prob.G, prob.n, prob.n, prob.n)) if want_phi else None
    rc = ctx.lib.keig_fixed_point(ctx.h, C.byref(pa.s), C.byref(o), C.byref(res),
                                  C.byref(h) if want_psi else None, _dp(phi) if phi is not None else None)
    if not (allow_noconv and rc == TT_ENOCONV):
        ctx.check(rc)
    it = min(res.iters, 512)
    return dict(k=res.k, iters=res.iters, dk=res.dk_last, wall_ms=res.wall_ms, max_rank=res.max_rank,
                k_hist=np.array(res.k_hist[:it]), t_hist=np.array(res.t_hist[:it]),
                psi=TTVec(ctx, h) if want_psi and h.value else None, phi=phi, code=rc)


class TTSlab(C.Structure):
    _fields_ = [
        ("l", C.c_int), ("width", C.c_double), ("G", C.c_int), ("n_mat", C.c_int),
        ("sig_t", D), ("sig_s", D), ("nu_sig_f", D), ("chi", D), ("mat", C.POINTER(C.c_uint8)),
        ("n_dir", C.c_int), ("amu", D), ("w", D),
    ]


class _SlabArrays:
    """Keeps the contiguous arrays a TTSlab points into alive."""

    def __init__(self, slab):
        self.arrays = a = dict(
            sig_t=np.ascontiguousarray(slab.sig_t, np.float64), sig_s=np.ascontiguousarray(slab.sig_s, np.float64),
            nsf=np.ascontiguousarray(slab.nu_sig_f, np.float64), chi=np.ascontiguousarray(slab.chi, np.float64),
            mat=np.ascontiguousarray(slab.mat, np.uint8), amu=np.ascontiguousarray(slab.amu, np.float64),
            w=np.ascontiguousarray(slab.w, np.float64))
        s = TTSlab()
        s.l, s.width, s.G, s.n_mat = int(slab.l), float(slab.width), int(slab.G), int(slab.n_mat)
        s.sig_t, s.sig_s, s.nu_sig_f, s.chi = _dp(a["sig_t"]), _dp(a["sig_s"]), _dp(a["nsf"]), _dp(a["chi"])
        s.mat = a["mat"].ctypes.data_as(C.POINTER(C.c_uint8))
        s.n_dir = int(a["amu"].size)
        s.amu, s.w = _dp(a["amu"]), _dp(a["w"])
        self.s = s


def keig_slab_fixed_point(ctx: Context, slab, opts: Optional[KeigOpts] = None, want_phi: bool = False,
                          allow_noconv: bool = False):
    """The k fixed point on a 1-D slab (keig.h: keig_slab_fixed_point);
    returns dict(k, iters, dk, wall_ms, max_rank, k_hist, phi, code)."""
    lib = load()
    if not getattr(lib.keig_slab_fixed_point, "_marshalled", False):
        lib.keig_slab_fixed_point.argtypes = [C.c_void_p, C.POINTER(TTSlab), C.POINTER(KeigOpts),
                                              C.POINTER(KeigResult), D]
        lib.keig_slab_fixed_point.restype = C.c_int
        lib.keig_slab_fixed_point._marshalled = True
    sa = _SlabArrays(slab)
    o = opts if opts is not None else keig_default_opts()
    res = KeigResult()
    phi = np.empty((slab.G, slab.n)) if want_phi else None
    rc = lib.keig_slab_fixed_point(ctx.h, C.byref(sa.s), C.byref(o), C.byref(res),
                                   _dp(phi) if phi is not None else None)
    if not (allow_noconv and rc == TT_ENOCONV):
        ctx.check(rc)
    it = min(res.iters, 512)
    return dict(k=res.k, iters=res.iters, dk=res.dk_last, wall_ms=res.wall_ms, max_rank=res.max_rank,
                k_hist=np.array(res.k_hist[:it]), phi=phi, code=rc)


def tt_scalar_flux(ctx: Context, psi: TTVec, w8) -> TTVec:
    w = np.ascontiguousarray(w8, np.float64)
    h = C.c_void_p()
    ctx.check(ctx.lib.tt_scalar_flux(ctx.h, psi.h, _dp(w), len(w), C.byref(h)))
    return TTVec(ctx, h)


def tt_dot_noalloc(x_cores, rx, y_cores, ry, n, out, stream=None) -> None:
    """<x, y> into the one-element CUDA tensor `out`, for callers that cannot
    allocate device memory where they need the product (a fixed memory
    budget, or a loop where an allocation would stall the device).
    x_cores / y_cores: contiguous float64 CUDA tensors holding all cores back
    to back; rx, ry, n: ranks and modes (host ints).  The sizes are checked
    against the tensors before the call; the library allocates nothing and
    shares one scratch array between all calls (keig.h)."""
    import torch
    lib = load()
    n = [int(v) for v in n]
    rx = [int(v) for v in rx]
    ry = [int(v) for v in ry]
    d = len(n)
    if d < 1 or len(rx) != d + 1 or len(ry) != d + 1:
        raise KeigError(TT_EINVAL, "tt_dot_noalloc: rx and ry need len(n) + 1 entries")
    if min(n + rx + ry) < 1:
        raise KeigError(TT_EINVAL, "tt_dot_noalloc: ranks and modes must be positive")
    for t in (x_cores, y_cores, out):
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise KeigError(TT_EINVAL, "tt_dot_noalloc: expects contiguous float64 CUDA tensors")
    for name, t, r in (("x_cores", x_cores, rx), ("y_cores", y_cores, ry)):
        need = sum(r[k] * n[k] * r[k + 1] for k in range(d))
        if t.numel() != need:
            raise KeigError(TT_EINVAL, f"tt_dot_noalloc: {name} holds {t.numel()} doubles, the ranks and "
                                       f"modes need {need}")
    if out.numel() < 1:
        raise KeigError(TT_EINVAL, "tt_dot_noalloc: out needs one element")
    if stream is None:
        stream = torch.cuda.current_stream()
    rxa, rxp = _ip(rx)
    rya, ryp = _ip(ry)
    na, npp = _ip(n)
    err = C.create_string_buffer(256)
    rc = lib.tt_dot_noalloc(C.cast(x_cores.data_ptr(), D), rxp, C.cast(y_cores.data_ptr(), D), ryp, len(na), npp,
                            C.cast(out.data_ptr(), D), C.c_void_p(stream.cuda_stream), err, 256)
    if rc != TT_OK:
        raise KeigError(rc, err.value.decode() or "tt_dot_noalloc failed")


class KeigSensInfo(C.Structure):
    _fields_ = [("k", C.c_double), ("k_adjoint", C.c_double), ("iters", C.c_int), ("iters_adjoint", C.c_int),
                ("adjoint_production", C.c_double), ("wall_ms", C.c_double)]


def keig_sensitivities(ctx: Context, prob, opts: Optional[KeigOpts] = None, allow_noconv: bool = False):
    """dk/d(table entry) for sig_t, sig_s, nu_sig_f and chi by the adjoint
    fixed point (keig.h); returns dict of arrays shaped like the tables plus
    the run information."""
    lib = load()
    sig = getattr(lib.keig_sensitivities, "_marshalled", False)
    if not sig:
        lib.keig_sensitivities.argtypes = [C.c_void_p, C.POINTER(TTProblem), C.POINTER(KeigOpts), D, D, D, D,
                                           C.POINTER(KeigSensInfo)]
        lib.keig_sensitivities.restype = C.c_int
        lib.keig_sensitivities._marshalled = True
    pa = _ProblemArrays(prob)
    o = opts if opts is not None else keig_default_opts()
    nm, G = prob.n_mat, prob.G
    gt, gs, gn, gc = np.zeros((nm, G)), np.zeros((nm, G, G)), np.zeros((nm, G)), np.zeros((nm, G))
    info = KeigSensInfo()
    rc = lib.keig_sensitivities(ctx.h, C.byref(pa.s), C.byref(o), _dp(gt), _dp(gs), _dp(gn), _dp(gc), C.byref(info))
    if not (allow_noconv and rc == TT_ENOCONV):
        ctx.check(rc)
    return dict(sig_t=gt, sig_s=gs, nu_sig_f=gn, chi=gc, k=info.k, k_adjoint=info.k_adjoint, iters=info.iters,
                iters_adjoint=info.iters_adjoint, adjoint_production=info.adjoint_production,
                wall_ms=info.wall_ms, code=rc)


class KeigGptInfo(C.Structure):
    _fields_ = [("J", C.c_double), ("k", C.c_double), ("iters", C.c_int), ("iters_adjoint", C.c_int),
                ("iters_gpt", C.c_int), ("gpt_change", C.c_double), ("wall_ms", C.c_double)]


def keig_gpt(ctx: Context, prob, resp_g, resp_v, opts: Optional[KeigOpts] = None, tol_gpt: float = 1e-8,
             max_gpt: int = 500, allow_noconv: bool = False):
    """dJ/d(table entry) of the flux functional J = sum resp_g[g] resp_v[v]
    phi[g, v] by generalised perturbation theory (keig.h: keig_gpt); returns
    dict of arrays shaped like the tables plus J and the run information."""
    lib = load()
    if not getattr(lib.keig_gpt, "_marshalled", False):
        lib.keig_gpt.argtypes = [C.c_void_p, C.POINTER(TTProblem), C.POINTER(KeigOpts), D, D, C.c_double, C.c_int,
                                 D, D, D, D, C.POINTER(KeigGptInfo)]
        lib.keig_gpt.restype = C.c_int
        lib.keig_gpt._marshalled = True
    pa = _ProblemArrays(prob)
    o = opts if opts is not None else keig_default_opts()
    nm, G = prob.n_mat, prob.G
    rg = np.ascontiguousarray(resp_g, dtype=np.float64).ravel()
    rv = np.ascontiguousarray(resp_v, dtype=np.float64).ravel()
    if rg.size != G or rv.size != prob.n ** 3:
        raise KeigError(TT_EINVAL, "keig_gpt: response sizes must be G and (2^l)^3")
    gt, gs, gn, gc = np.zeros((nm, G)), np.zeros((nm, G, G)), np.zeros((nm, G)), np.zeros((nm, G))
    info = KeigGptInfo()
    rc = lib.keig_gpt(ctx.h, C.byref(pa.s), C.byref(o), _dp(rg), _dp(rv), float(tol_gpt), int(max_gpt), _dp(gt),
                      _dp(gs), _dp(gn), _dp(gc), C.byref(info))
    if not (allow_noconv and rc == TT_ENOCONV):
        ctx.check(rc)
    return dict(sig_t=gt, sig_s=gs, nu_sig_f=gn, chi=gc, J=info.J, k=info.k, iters=info.iters,
                iters_adjoint=info.iters_adjoint, iters_gpt=info.iters_gpt, gpt_change=info.gpt_change,
                wall_ms=info.wall_ms, code=rc)


def keig_batch(problems, opts_list, n_workers: int = 8, contexts=None):
    """Solve independent problems side by side (keig.h: keig_batch).  One
    context per worker, each on its own torch CUDA stream.  Returns a list of
    result dicts (k, iters, dk, wall_ms, max_rank, code)."""
    import torch
    lib = load()
    if not getattr(lib.keig_batch, "_marshalled", False):
        lib.keig_batch.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.POINTER(TTProblem), C.POINTER(KeigOpts), C.c_int,
                                   C.POINTER(KeigResult), C.POINTER(C.c_int)]
        lib.keig_batch.restype = C.c_int
        lib.keig_batch._marshalled = True
    n = len(problems)
    if contexts is None:
        contexts = [Context(torch.cuda.Stream()) for _ in range(max(1, min(n_workers, n)))]
    handles = (C.c_void_p * len(contexts))(*[c.h.value for c in contexts])
    arrays = [_ProblemArrays(p) for p in problems]
    probs = (TTProblem * n)(*[a.s for a in arrays])
    opts = (KeigOpts * n)(*opts_list)
    res = (KeigResult * n)()
    status = (C.c_int * n)()
    lib.keig_batch(handles, len(contexts), probs, opts, n, res, status)
    torch.cuda.synchronize()
    gl, gs = C.c_longlong(), C.c_longlong()
    lib.keig_batch_stats.argtypes = [C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
    lib.keig_batch_stats(C.byref(gl), C.byref(gs))
    keig_batch.last_group_launches, keig_batch.last_group_systems = gl.value, gs.value
    out = []
    for i in range(n):
        r = res[i]
        it = min(r.iters, 512)
        out.append(dict(k=r.k, iters=r.iters, dk=r.dk_last, wall_ms=r.wall_ms, max_rank=r.max_rank,
                        k_hist=np.array(r.k_hist[:it]), code=int(status[i])))
    return out, contexts


class KeigAlphaResult(C.Structure):
    _fields_ = [("alpha", C.c_double), ("k", C.c_double), ("steps", C.c_int), ("outer_iters", C.c_int),
                ("wall_ms", C.c_double), ("alpha_hist", C.c_double * 64), ("k_hist", C.c_double * 64)]


def keig_alpha(ctx: Context, prob, opts: Optional[KeigOpts] = None, tol_k1: float = 1e-9, max_steps: int = 30,
               allow_noconv: bool = False):
    """The alpha eigenvalue by secant steps on k(alpha) = 1 (keig.h); the
    problem must carry inv_v."""
    lib = load()
    if not getattr(lib.keig_alpha, "_marshalled", False):
        lib.keig_alpha.argtypes = [C.c_void_p, C.POINTER(TTProblem), C.POINTER(KeigOpts), C.c_double, C.c_int,
                                   C.POINTER(KeigAlphaResult)]
        lib.keig_alpha.restype = C.c_int
        lib.keig_alpha._marshalled = True
    pa = _ProblemArrays(prob)
    o = opts if opts is not None else keig_default_opts()
    r = KeigAlphaResult()
    rc = lib.keig_alpha(ctx.h, C.byref(pa.s), C.byref(o), float(tol_k1), int(max_steps), C.byref(r))
    if not (allow_noconv and rc == TT_ENOCONV):
        ctx.check(rc)
    n = min(r.steps, 64)
    return dict(alpha=r.alpha, k=r.k, steps=r.steps, outer_iters=r.outer_iters, wall_ms=r.wall_ms,
                alpha_hist=np.array(r.alpha_hist[:n]), k_hist=np.array(r.k_hist[:n]), code=rc)


def keig_k_function():
    """A torch.autograd.Function computing k from the cross-section tables
    (sig_t, sig_s, nu_sig_f, chi) of a problem template; its backward uses the
    adjoint sensitivities computed in the forward call."""
    import dataclasses

    import torch

    class KeigK(torch.autograd.Function):
        @staticmethod
        def forward(fctx, sig_t, sig_s, nu_sig_f, chi, problem, ctx, opts):
            p = dataclasses.replace(problem, sig_t=sig_t.detach().cpu().double().numpy(),
                                    sig_s=sig_s.detach().cpu().double().numpy(),
                                    nu_sig_f=nu_sig_f.detach().cpu().double().numpy(),
                                    chi=chi.detach().cpu().double().numpy())
            r = keig_sensitivities(ctx, p, opts)
            grads = [torch.from_numpy(r[f]).to(sig_t.device, sig_t.dtype)
                     for f in ("sig_t", "sig_s", "nu_sig_f", "chi")]
            fctx.save_for_backward(*grads)
            return torch.tensor(r["k"], dtype=sig_t.dtype, device=sig_t.device)

        @staticmethod
        def backward(fctx, gk):
            gt, gs, gn, gc = fctx.saved_tensors
            return gk * gt, gk * gs, gk * gn, gk * gc, None, None, None

    return KeigK


def keig_j_function():
    """A torch.autograd.Function computing the flux functional
    J = sum_g sum_v resp_g[g] resp_v[v] phi[g, v] of the production-normalised
    eigenvector from the cross-section tables (sig_t, sig_s, nu_sig_f, chi) of
    a problem template; its backward uses the GPT gradients that keig_gpt
    returns with J (one adjoint fixed point and one fixed-source iteration in
    the forward call)."""
    import dataclasses

    import torch

    class KeigJ(torch.autograd.Function):
        @staticmethod
        def forward(fctx, sig_t, sig_s, nu_sig_f, chi, problem, resp_g, resp_v, ctx, opts, tol_gpt=1e-8,
                    max_gpt=500):
            p = dataclasses.replace(problem, sig_t=sig_t.detach().cpu().double().numpy(),
                                    sig_s=sig_s.detach().cpu().double().numpy(),
                                    nu_sig_f=nu_sig_f.detach().cpu().double().numpy(),
                                    chi=chi.detach().cpu().double().numpy())
            r = keig_gpt(ctx, p, resp_g, resp_v, opts, tol_gpt=tol_gpt, max_gpt=max_gpt)
            grads = [torch.from_numpy(r[f]).to(sig_t.device, sig_t.dtype)
                     for f in ("sig_t", "sig_s", "nu_sig_f", "chi")]
            fctx.save_for_backward(*grads)
            return torch.tensor(r["J"], dtype=sig_t.dtype, device=sig_t.device)

        @staticmethod
        def backward(fctx, gj):
            gt, gs, gn, gc = fctx.saved_tensors
            return gj * gt, gj * gs, gj * gn, gj * gc, None, None, None, None, None, None, None

    return KeigJ


def tt_measure_fma_peak(fp64: bool, iters: int = 4096, reps: int = 5, stream=None) -> float:
    """Peak FMA rate of the current device in flop/s (keig.h)."""
    import torch
    lib = load()
    if stream is None:
        stream = torch.cuda.current_stream()
    out = C.c_double()
    rc = lib.tt_measure_fma_peak(C.c_void_p(stream.cuda_stream), int(bool(fp64)), int(iters), int(reps),
                                 C.byref(out))
    if rc != TT_OK:
        raise KeigError(rc, "tt_measure_fma_peak failed")
    return float(out.value)


def tt_gemm_f32(ctx: Context, kind: int, ta: bool, tb: bool, a, b, out, alpha: float = 1.0, beta: float = 0.0) -> None:
    """out[i] = alpha op(a[i]) op(b[i]) + beta out[i] on float32 CUDA tensors of
    shape (batch, rows, cols) (keig.h tt_gemm_f32; kind 0 SIMT, 1 TF32 split,
    2 BF16 split).  Sizes are checked here before the call."""
    import torch
    for t in (a, b, out):
        if not (t.is_cuda and t.dtype == torch.float32 and t.dim() == 3 and t.is_contiguous()):
            raise KeigError(TT_EINVAL, "tt_gemm_f32: expects contiguous float32 CUDA tensors (batch, rows, cols)")
    batch = a.shape[0]
    M, K = (a.shape[2], a.shape[1]) if ta else (a.shape[1], a.shape[2])
    Kb, N = (b.shape[2], b.shape[1]) if tb else (b.shape[1], b.shape[2])
    if b.shape[0] != batch or out.shape[0] != batch or Kb != K or tuple(out.shape[1:]) != (M, N):
        raise KeigError(TT_EINVAL, "tt_gemm_f32: inconsistent shapes")
    vp = lambda t: C.c_void_p(t.data_ptr())
    ctx.check(ctx.lib.tt_gemm_f32(ctx.h, int(kind), int(bool(ta)), int(bool(tb)), M, N, K, float(alpha), vp(a),
                                  a.shape[2], a.shape[1] * a.shape[2], vp(b), b.shape[2], b.shape[1] * b.shape[2],
                                  float(beta), vp(out), out.shape[2], out.shape[1] * out.shape[2], batch))
