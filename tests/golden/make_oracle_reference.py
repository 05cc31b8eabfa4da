"""Writes tests/golden/oracle_reference.txt: the oracle's converged k of the
workloads whose full-grid solve takes too long to repeat in every benchmark
run (power iteration of Eq. (k_eff_fixed_points) to |dk| < 1e-13, all host
cores), its iteration count, and the first iteration from which every
iterate is within 1e-6 (relative) of that k.  Calls only oracle/ and
keig_inputs/.

usage: python tests/golden/make_oracle_reference.py cube128_g2_s4_10cm [...]
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import keig_inputs as ki  # noqa: E402
from oracle import transport as T  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_reference.txt")
WORKLOADS = {
    "cube64_g2_s4_10cm": lambda: ki.bare_cube(6),
    "cube128_g2_s4_10cm": lambda: ki.bare_cube(7),
    "cube256_g2_s4_10cm": lambda: ki.bare_cube(8),
}


def read():
    """{name: (k, iterations)} of the stored entries."""
    out = {}
    if os.path.exists(OUT):
        for line in open(OUT):
            if line.strip() and not line.startswith("#"):
                name, k, it, ok = line.split()[:4]
                out[name] = (float(k), int(it), int(ok))
    return out


def main(names):
    have = read()
    for name in names:
        p = WORKLOADS[name]()
        t0 = time.time()
        r = T.OracleProblem(p).keig(tol_k=1e-13, max_iter=100000, history=True)
        ks = r["k_hist"]
        n_ok = next(i for i in range(len(ks)) if all(abs(x - r["k"]) < 1e-6 * r["k"] for x in ks[i:])) + 1
        have[name] = (r["k"], r["iters"], n_ok)
        print(f"{name}: k = {r['k']:.15f} after {r['iters']} iterations ({time.time() - t0:.0f} s)", flush=True)
        with open(OUT, "w") as f:
            f.write("# workload  k (oracle power iteration, |dk| < 1e-13)  iterations  "
                    "first iteration within 1e-6 for good\n")
            f.write("# written by tests/golden/make_oracle_reference.py (oracle only)\n")
            for n in sorted(have):
                f.write(f"{n} {have[n][0]:.15f} {have[n][1]} {have[n][2]}\n")


if __name__ == "__main__":
    main(sys.argv[1:])
