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
    scale = max(np.abs(v).max() for v in fd.values())
    for f in SE.FIELDS:
        err = np.abs(g[f] - fd[f]).max() / scale
        assert err < 1e-4, (f, err, g[f], fd[f])


def test_gpt_rejects_bad_response(ctx):
    p = dataclasses.replace(ki.fissile_box(l=3, G=2, order=4, seed=1003, half_width=2), side=(3.0,) * 3)
    rg, rv = ki.fissile_response(p, 0)
    rv = rv.copy()
    rv.flat[5] = np.nan
    with pytest.raises(K.KeigError) as e:
        K.keig_gpt(ctx, p, rg, rv)
    assert e.value.code == K.TT_EINVAL
