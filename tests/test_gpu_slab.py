"""GPU parity of the 1-D slab fixed point (the paper's ISTT, Sec. 4.1)
against the slab oracle (ISFM), and its approach to the exact k = 1 of the
critical Pu-239 slab at the paper's 1024 points."""
import dataclasses

import numpy as np
import pytest

import keig_inputs as ki
from oracle import slab as SL

pytestmark = pytest.mark.gpu

K = pytest.importorskip("paper_2309_03347_gb300")


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _opts(prec=0):
    o = K.keig_default_opts()
    o.eps, o.rmax, o.tol_k, o.tol_psi, o.max_iter = 1e-10, 0, 1e-12, 1e-8, 300
    o.solve_sweeps, o.mv_sweeps = 4, 4
    o.prec = prec
    return o


@pytest.mark.parametrize("L", [2, 8, 32])
def test_slab_matches_oracle(ctx, L):
    s = ki.pu239_slab(l=10, L=L)
    ref = SL.SlabOracle(s).keig(tol_k=1e-13)
    res = K.keig_slab_fixed_point(ctx, s, _opts(), want_phi=True)
    assert abs(res["k"] - ref["k"]) < 1e-6 * ref["k"], (res["k"], ref["k"])
    assert rel(res["phi"], ref["phi"]) < 1e-5


def test_slab_approaches_critical(ctx):
    # the paper's Panel A: the TT eigenvalue converges to the exact k = 1
    errs = [abs(K.keig_slab_fixed_point(ctx, ki.pu239_slab(l=10, L=L), _opts())["k"] - 1.0) for L in (2, 8, 32)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 5e-4, errs


def test_slab_two_materials_mixed_precision(ctx):
    s = ki.pu239_slab(l=8, L=8)
    mat = np.zeros(s.n - 1, np.uint8)
    mat[: s.n // 4] = 1
    s = dataclasses.replace(s, sig_t=np.array([[0.3264], [0.5]]), sig_s=np.array([[[0.225216]], [[0.45]]]),
                            nu_sig_f=np.array([[0.264384], [0.0]]), chi=np.array([[1.0], [1.0]]), mat=mat)
    ref = SL.SlabOracle(s).keig(tol_k=1e-13)
    res = K.keig_slab_fixed_point(ctx, s, _opts(K.TT_FP32_REFINED), want_phi=True)
    assert abs(res["k"] - ref["k"]) < 1e-6 * ref["k"]
    assert rel(res["phi"], ref["phi"]) < 1e-5


def test_slab_rejects_bad_input(ctx):
    s = ki.pu239_slab(l=6, L=4)
    bad = dataclasses.replace(s, amu=-s.amu)
    with pytest.raises(K.KeigError) as e:
        K.keig_slab_fixed_point(ctx, bad)
    assert e.value.code == K.TT_EINVAL
