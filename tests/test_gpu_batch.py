"""Batched problems (keig_batch): every problem of a batch solved side by
side reaches the same eigenvalue as the oracle and, with grouped GMRES
launches, as a lone solve."""
import dataclasses

import numpy as np
import pytest

import keig_inputs as ki
from oracle import transport as T

pytestmark = pytest.mark.gpu

K = pytest.importorskip("paper_2309_03347_gb300")


def _problems():
    out = []
    for i in range(6):
        side = 2.0 + 0.5 * (i % 3)
        if i % 2:
            p = ki.fissile_box(l=3, G=2, order=4, seed=2000 + i, half_width=2)
        else:
            p = ki.homogeneous(l=3, G=2, order=4, seed=2000 + i)
        out.append(dataclasses.replace(p, side=(side,) * 3))
    return out


def _opts():
    o = K.keig_default_opts()
    o.eps, o.rmax, o.tol_k, o.tol_psi, o.max_iter = 1e-10, 0, 1e-11, 1e-7, 200
    o.solve_sweeps, o.mv_sweeps = 4, 4
    return o


def test_batch_matches_oracle(ctx):
    probs = _problems()[:4]
    res, _ = K.keig_batch(probs, [_opts() for _ in probs], n_workers=3)
    for p, r in zip(probs, res):
        assert r["code"] == K.TT_OK
        ref = T.OracleProblem(p).keig(tol_k=1e-12, max_iter=20000)["k"]
        assert abs(r["k"] - ref) / ref < 1e-6


def test_grouped_gmres_launches_match_oracle(ctx):
    # FP32-refined local solves: the workers' persistent-GMRES systems share
    # grouped cooperative launches (several systems per launch, each on its
    # own range of CTAs), and every problem still reaches the oracle's k
    probs = _problems()[:4]
    opts = []
    for _ in probs:
        o = _opts()
        o.prec = K.TT_FP32_REFINED
        opts.append(o)
    res, _ = K.keig_batch(probs, opts, n_workers=4)
    launches, systems = K.keig_batch.last_group_launches, K.keig_batch.last_group_systems
    assert launches > 0 and systems > launches, (launches, systems)  # some launches carried several systems
    for p, r, o in zip(probs, res, opts):
        assert r["code"] == K.TT_OK
        ref = T.OracleProblem(p).keig(tol_k=1e-12, max_iter=20000)["k"]
        assert abs(r["k"] - ref) / ref < 1e-6
        single = K.keig_fixed_point(ctx, p, o)
        assert abs(single["k"] - r["k"]) < 1e-9 * abs(single["k"])
