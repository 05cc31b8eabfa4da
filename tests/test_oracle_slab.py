"""Pins of the 1-D slab oracle (Sec. 4.1): the printed benchmark data, the
sweep against the assembled operator, the power iteration (the paper's ISFM)
against a library eigensolver (GES), and convergence of k to the exact value
1 of the critical Pu-239 slab as the number of ordinates grows."""
import os

import numpy as np
import pytest

import keig_inputs as ki
from oracle import slab as SL

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    vals = {}
    with open(os.path.join(HERE, "golden", "pu239_slab.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_slab_inputs_are_the_printed_benchmark():
    g = _golden()
    s = ki.pu239_slab(l=10, L=8)
    assert s.sig_t[0, 0] == g["sigma_t"] and s.sig_s[0, 0, 0] == g["sigma_s"]
    assert abs(s.nu_sig_f[0, 0] - g["nu"] * g["sigma_f"]) < 1e-15
    assert s.width == g["width_cm"] and s.n == int(g["points"])
    # half-range Gauss-Legendre: weights of both halves sum to 1, nodes in (0, 1)
    assert abs(2 * s.w.sum() - 1.0) < 1e-14 and np.all((s.amu > 0) & (s.amu < 1))


def test_slab_sweep_inverts_the_assembled_operator():
    s = ki.pu239_slab(l=6, L=4)
    o = SL.SlabOracle(s)
    H, _, _ = SL.assemble(s)
    q = np.random.default_rng(3).standard_normal((s.G, s.n - 1))
    psi = o.sweep(q)
    rhs = np.zeros(s.psi_shape)
    rhs[:, 1, :, 1:] = q[:, None, :]      # mu > 0: row i carries cell i-1
    rhs[:, 0, :, :-1] = q[:, None, :]     # mu < 0: row i carries cell i
    assert np.abs(H @ psi.ravel() - rhs.ravel()).max() < 1e-12


@pytest.mark.parametrize("two_materials", [False, True])
def test_slab_power_iteration_matches_library_eigensolver(two_materials):
    s = ki.pu239_slab(l=6, L=4)
    if two_materials:
        import dataclasses
        mat = np.zeros(s.n - 1, np.uint8)
        mat[: s.n // 4] = 1
        s = dataclasses.replace(s, sig_t=np.array([[0.3264], [0.5]]), sig_s=np.array([[[0.225216]], [[0.45]]]),
                                nu_sig_f=np.array([[0.264384], [0.0]]), chi=np.array([[1.0], [1.0]]), mat=mat)
    r = SL.SlabOracle(s).keig(tol_k=1e-14)
    k, psi = SL.ges(s)
    assert abs(r["k"] - k) < 1e-11 * k
    assert np.linalg.norm(r["psi"].ravel() - psi) < 1e-8 * np.linalg.norm(psi)


def test_slab_k_converges_to_the_critical_value():
    # the paper's discretisation: 1024 points, growing ordinate sets; the
    # exact transport eigenvalue of this slab is 1
    g = _golden()
    errs = []
    for L in (2, 4, 8, 16, 32):
        k = SL.SlabOracle(ki.pu239_slab(l=10, L=L)).keig(tol_k=1e-13)["k"]
        errs.append(abs(k - g["k_eff"]))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 5e-4, errs
