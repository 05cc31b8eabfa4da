"""The QTT fixed point in the truncating regime: a 16^3 bare cube (config-0
cross sections, 2 groups, S4, 20 cm, vacuum) whose converged angular flux
needs TT ranks up to about 200 at 1e-6, solved with a rank cap of 112 that
binds.  The oracle's own truncated power iteration (exact sweep, TT-SVD to
rank 112 each iteration) reaches k within 3e-8 and the scalar flux within
3e-6 there, so the GPU fixed point must meet the parity bar in spite of the
cap: k within 1e-6 and the scalar flux within 1e-5 (relative L2, both fluxes
normalised to sum(F Psi) = 1).  The local systems take the least-squares
form of Eq. (linear_system_obj): with Galerkin systems this problem needs
about eight times longer per outer iteration and its k wanders around the
tolerance (the symmetric part of H is indefinite)."""
import numpy as np
import pytest

import keig_inputs as ki
from oracle import transport as T

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

K = pytest.importorskip("paper_2309_03347_gb300")

CAP = 112


@pytest.fixture(scope="module")
def oracle16():
    p = ki.homogeneous(l=4, G=2, order=4, side=20.0, seed=1000, name="cube16_g2_s4_20cm")
    ref = T.OracleProblem(p).keig(tol_k=1e-13, max_iter=100000)
    phi = ref["phi"] / T.production(p, ref["phi"])
    return p, ref["k"], phi


def test_rank_capped_fixed_point_matches_oracle(ctx, oracle16):
    p, k_ref, phi_ref = oracle16
    o = K.keig_default_opts()
    o.eps, o.rmax, o.tol_k, o.tol_psi, o.max_iter = 1e-9, CAP, 1e-10, 1e-6, 600
    o.solve_sweeps, o.mv_sweeps = 2, 2
    o.prec = K.TT_FP32_REFINED
    o.local_form = 1
    r = K.keig_fixed_point(ctx, p, o, want_phi=True, allow_noconv=True)
    assert CAP - 16 <= r["max_rank"] <= CAP + o.kick  # the cap binds
    phi = r["phi"] / T.production(p, r["phi"])
    dk = abs(r["k"] - k_ref) / k_ref
    dphi = float(np.linalg.norm(phi - phi_ref) / np.linalg.norm(phi_ref))
    assert dk < 1e-6, (dk, r["iters"])
    assert dphi < 1e-5, dphi
