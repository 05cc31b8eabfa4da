"""GPU parity of the flux-functional gradient by generalised perturbation
theory (keig_gpt) against central finite differences of the oracle's
functional (the oracle's own GPT and finite differences are pinned against
each other in tests/test_oracle.py)."""
import dataclasses

import numpy as np
import pytest

import keig_inputs as ki

pytestmark = pytest.mark.gpu

K = pytest.importorskip("paper_2309_03347_gb300")


def test_gpt_functional_gradient_matches_finite_differences(ctx):
    from oracle import sensitivity as SE
    p = dataclasses.replace(ki.fissile_box(l=3, G=2, order=4, seed=1003, half_width=2), side=(3.0,) * 3)
    rg, rv = ki.fissile_response(p, 0)
    o = K.keig_default_opts()
    o.eps, o.rmax, o.tol_k, o.tol_psi, o.max_iter = 1e-10, 0, 1e-12, 1e-8, 300
    o.solve_sweeps, o.mv_sweeps = 4, 4
    g = K.keig_gpt(ctx, p, rg, rv, o, tol_gpt=1e-9, max_gpt=500)
    j_or, k_or = SE.oracle_functional(p, rg, rv)
    assert abs(g["k"] - k_or) < 1e-8 * k_or
    assert abs(g["J"] - j_or) < 1e-7 * abs(j_or), (g["J"], j_or)
    fd = SE.fd_functional_gradients(p, rg, rv)
    # per entry: 1e-4 relative to that entry's finite difference, with an
    # absolute floor of 1e-7 x the largest derivative for the finite
    # difference's own noise
    scale = max(np.abs(v).max() for v in fd.values())
    for f in SE.FIELDS:
        bad = np.abs(g[f] - fd[f]) > 1e-4 * np.abs(fd[f]) + 1e-7 * scale
        assert not bad.any(), (f, g[f][bad], fd[f][bad])


def test_gpt_rejects_bad_response(ctx):
    p = dataclasses.replace(ki.fissile_box(l=3, G=2, order=4, seed=1003, half_width=2), side=(3.0,) * 3)
    rg, rv = ki.fissile_response(p, 0)
    rv = rv.copy()
    rv.flat[5] = np.nan
    with pytest.raises(K.KeigError) as e:
        K.keig_gpt(ctx, p, rg, rv)
    assert e.value.code == K.TT_EINVAL


def test_j_autograd_function_backward(ctx):
    # the autograd wrapper returns keig_gpt's J and hands its GPT gradients to backward()
    import torch
    p = dataclasses.replace(ki.fissile_box(l=3, G=2, order=4, seed=1003, half_width=2), side=(3.0,) * 3)
    rg, rv = ki.fissile_response(p, 0)
    o = K.keig_default_opts()
    o.eps, o.rmax, o.tol_k, o.tol_psi, o.max_iter = 1e-10, 0, 1e-12, 1e-8, 300
    o.solve_sweeps, o.mv_sweeps = 4, 4
    KeigJ = K.keig_j_function()
    t = {f: torch.tensor(getattr(p, f), dtype=torch.float64, requires_grad=True)
         for f in ("sig_t", "sig_s", "nu_sig_f", "chi")}
    o.tol_k, o.tol_psi = 1e-9, 1e-6  # this test checks the plumbing of backward()
    j = KeigJ.apply(t["sig_t"], t["sig_s"], t["nu_sig_f"], t["chi"], p, rg, rv, ctx, o, 1e-6, 500)
    (3.0 * j).backward()
    g = K.keig_gpt(ctx, p, rg, rv, o, tol_gpt=1e-6, max_gpt=500)
    assert abs(float(j.detach()) - g["J"]) <= 1e-12 * abs(g["J"])
    for f in ("sig_t", "sig_s", "nu_sig_f", "chi"):
        assert np.allclose(t[f].grad.numpy(), 3.0 * g[f], rtol=1e-9, atol=0)
