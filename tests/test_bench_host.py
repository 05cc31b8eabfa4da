"""Host-side logic of the benchmark (no GPU): the stored oracle references it
reads, the iteration rule of its timed steps, and its workload table."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import keig_inputs as ki  # noqa: E402
from oracle import transport as T  # noqa: E402


def test_first_within_rule():
    k = 2.0
    hist = k * (1 + np.array([1e-2, 1e-4, 5e-7, 2e-6, 9e-7, 3e-7, 1e-8]))
    assert bench.first_within(hist, k) == 5          # 2e-6 at index 3 breaks the run before
    assert bench.first_within(hist, k, 4e-7) == 6
    assert bench.first_within(hist, k, 1e-9) is None
    assert bench.first_within(k * (1 + np.array([1e-7])), k) == 1


def test_stored_oracle_reference_reproduces():
    # the stored 64^3 reference is the oracle's own result (regenerated here)
    k, n_ok = bench.golden_reference("cube64_g2_s4_10cm")
    p = ki.bare_cube(6)
    r = T.OracleProblem(p).keig(tol_k=1e-13, max_iter=100000, history=True)
    assert abs(r["k"] - k) <= 1e-12 * k
    ks = r["k_hist"]
    assert n_ok == next(i for i in range(len(ks)) if np.all(np.abs(ks[i:] - r["k"]) < 1e-6 * r["k"])) + 1


def test_benchmark_workloads_have_references():
    for name, (make, cap, eps, lf, sweeps, note) in bench.WORKLOADS.items():
        p = make()
        assert p.name == name or name == "box32_g4_s8"
        assert cap >= 1 and 0 < eps < 1 and lf in (0, 1) and sweeps >= 1 and note
        if name.startswith("cube"):
            assert bench.golden_reference(name) is not None, name
    assert bench.DEFAULT_WORKLOAD in bench.WORKLOADS


def test_batch_mix_is_seeded():
    a = bench.batch_problems(5)
    b = bench.batch_problems(5)
    for (pa, ca), (pb, cb) in zip(a, b):
        assert ca == cb and pa.n == pb.n and pa.G == pb.G and pa.L == pb.L
        assert np.array_equal(pa.sig_t, pb.sig_t)
