"""Caller-supplied device allocator (keig.h tt_ctx_create hooks): the
library's buffers drawn from PyTorch's caching allocator give the same
result as the built-in stream-ordered pool, and an allocator that returns
NULL makes the running call fail with TT_ENOMEM while the context stays
usable (failure injected on the host, no device fault)."""
import dataclasses

import pytest

import keig_inputs as ki

pytestmark = pytest.mark.gpu

K = pytest.importorskip("paper_2309_03347_gb300")


def _problem_and_opts():
    p = dataclasses.replace(ki.config(0), side=(2.0,) * 3)
    o = K.keig_default_opts()
    o.eps, o.rmax, o.tol_k, o.tol_psi, o.max_iter = 1e-10, 0, 1e-11, 1e-7, 600
    o.solve_sweeps, o.mv_sweeps = 4, 4
    o.prec = K.TT_FP32_REFINED
    return p, o


class FailingAllocator(K.TorchCachingAllocator):
    """Serves `budget` allocations, then returns NULL until reset."""

    def __init__(self, budget):
        super().__init__()
        self.budget = budget
        self.served = 0
        self.live = set()

    def alloc(self, nbytes, stream):
        if self.served >= self.budget:
            return 0
        self.served += 1
        ptr = super().alloc(nbytes, stream)
        if ptr:
            self.live.add(ptr)
        return ptr

    def free(self, ptr, stream):
        self.live.discard(ptr)
        super().free(ptr, stream)


def test_torch_caching_allocator_matches_pool(ctx):
    p, o = _problem_and_opts()
    ref = K.keig_fixed_point(ctx, p, o)
    c2 = K.tt_ctx_create(allocator=K.TorchCachingAllocator())
    got = K.keig_fixed_point(c2, p, o)
    assert got["iters"] == ref["iters"]
    assert abs(got["k"] - ref["k"]) <= 1e-13 * abs(ref["k"])


def test_allocator_null_gives_enomem_and_context_survives(ctx):
    p, o = _problem_and_opts()
    ref = K.keig_fixed_point(ctx, p, o)
    a = FailingAllocator(budget=400)
    c2 = K.tt_ctx_create(allocator=a)
    with pytest.raises(K.KeigError) as e:
        K.keig_fixed_point(c2, p, o)
    assert e.value.code == K.TT_ENOMEM and "NULL" in str(e.value)
    # everything the failed call allocated has been handed back (the context
    # keeps only its own small buffers)
    kept = len(a.live)
    assert kept <= 16, kept
    a.budget = 1 << 60
    got = K.keig_fixed_point(c2, p, o)
    assert abs(got["k"] - ref["k"]) <= 1e-13 * abs(ref["k"])


def test_half_given_allocator_is_rejected():
    import ctypes as C
    import torch
    lib = K.load()
    h = C.c_void_p()
    from paper_2309_03347_gb300._lib import ALLOC_FN, FREE_FN
    keep = ALLOC_FN(lambda n, s, u: None)
    rc = lib.tt_ctx_create(C.byref(h), C.c_void_p(torch.cuda.current_stream().cuda_stream), keep, FREE_FN(), None)
    assert rc == K.TT_EINVAL and not h.value
