"""Failure detection without a device fault: the bounded waits of the
persistent GMRES kernel (its grid barriers) are made to run out by a spin
limit of zero, so every barrier gives up at once.  The kernel records
TT_ETIMEOUT and returns, the host reads the status, the whole call fails
with TT_ETIMEOUT, and the same context then solves the problem normally."""
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
    o.prec = K.TT_FP32_REFINED  # the local solves run in the persistent GMRES kernel
    return p, o


def test_barrier_wait_runs_out_and_context_survives(ctx):
    p, o = _problem_and_opts()
    ref = K.keig_fixed_point(ctx, p, o)
    c2 = K.tt_ctx_create()
    c2.set_wait_limit(0)
    with pytest.raises(K.KeigError) as e:
        K.keig_fixed_point(c2, p, o)
    assert e.value.code == K.TT_ETIMEOUT and "barrier" in str(e.value)
    c2.set_wait_limit(-1)
    got = K.keig_fixed_point(c2, p, o)
    assert got["iters"] == ref["iters"] and abs(got["k"] - ref["k"]) <= 1e-13 * abs(ref["k"])
