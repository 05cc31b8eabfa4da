"""The alpha-eigenvalue problem (NEXT row of the hot-path table): the
oracle's secant over power iterations is pinned by a dense generalized
eigensolve; the GPU secant over QTT fixed points matches the oracle."""
import dataclasses

import numpy as np
import pytest

import keig_inputs as ki
from oracle import alpha as A


def _problem(l=2, side=6.0):
    p = ki.homogeneous(l=l, G=2, order=4, seed=1000, side=side)
    p = dataclasses.replace(p, nu_sig_f=p.nu_sig_f * 4.0, inv_v=np.array([0.5, 2.0]))
    return p


def test_oracle_secant_alpha_matches_dense_eigenvalue():
    p = _problem()
    a, k, hist = A.secant_alpha(p, p.inv_v)
    assert abs(k - 1.0) < 1e-10
    assert abs(a - A.ges_alpha(p, p.inv_v)) < 1e-9 * max(1.0, abs(a))
    # k(alpha) decreases with alpha (more absorption), so the secant brackets 1
    ks = [h[1] for h in hist[:2]]
    assert ks[1] < ks[0]


@pytest.mark.gpu
def test_gpu_alpha_matches_oracle(ctx):
    import paper_2309_03347_gb300 as K
    p = _problem(l=2, side=6.0)
    a_ref, _, _ = A.secant_alpha(p, p.inv_v)
    o = K.keig_default_opts()
    o.eps, o.rmax, o.tol_k, o.tol_psi, o.max_iter = 1e-10, 0, 1e-11, 1e-7, 300
    o.solve_sweeps, o.mv_sweeps = 4, 4
    r = K.keig_alpha(ctx, p, o, tol_k1=1e-9, max_steps=30)
    assert abs(r["k"] - 1.0) < 1e-9
    assert abs(r["alpha"] - a_ref) < 1e-6 * max(1.0, abs(a_ref))
