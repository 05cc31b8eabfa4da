"""Benchmark: time to a k-eigenvalue solution within 1e-6 of the FP64 oracle,
with the dominant contraction kernel's throughput against its roofline.

One step = one call of keig_fixed_point (operator construction, then the
QTT fixed point of Eq. (TT_k_eff_fixed_points)) run for the number of outer
iterations after which every iterate stays within 1e-6 of the oracle's k
(found in the first warm-up solve).  `value` is seconds per such solve,
measured with CUDA events on the library stream, problem tables resident on
the host side of the library (a few KB, copied inside the call); `e2e` is the
same call timed on the host with the tables in pinned host memory and the
scalar flux copied back to pinned host memory.

The default workload is the paper's 3-D benchmark geometry (Sec. 4.2): a bare
homogeneous cube of 10 cm with vacuum faces at 256 grid points per axis (its
middle grid), with seeded synthetic 2-group cross sections and an S4
level-symmetric set in place of the unavailable 256-group data and the S8
square set.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload NAME] [--prec mixed|tf32|bf16|fp64]
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import keig_inputs as ki  # noqa: E402

METRIC = "time to k within 1e-6 of FP64 oracle; TT contraction TFLOP/s and % of peak"
UNIT = "s"
GOLDEN = os.path.join(ROOT, "tests", "golden", "oracle_reference.txt")

# name -> (problem, rank cap, eps, local form (0 Galerkin, 1 least squares),
#          AMEn sweeps per product and per solve, note)
WORKLOADS = {
    "cube128_g2_s4_10cm": (lambda: ki.bare_cube(7), 96, 1e-5, 1, 1,
                           "bare homogeneous 10 cm cube, 128^3 grid points (the paper's Sec. 4.2 geometry at its "
                           "smallest grid), 2 groups, S4 level-symmetric (24 directions), vacuum"),
    "cube256_g2_s4_10cm": (lambda: ki.bare_cube(8), 96, 1e-5, 1, 1,
                           "bare homogeneous 10 cm cube, 256^3 grid points (the paper's middle grid), 2 groups, S4, "
                           "vacuum"),
    "cube64_g2_s4_10cm": (lambda: ki.bare_cube(6), 96, 1e-5, 1, 1,
                          "bare homogeneous 10 cm cube, 64^3 grid points, 2 groups, S4, vacuum"),
    "box32_g4_s8": (lambda: ki.config(1), 64, 1e-7, 0, 2,
                    "fissile box in a c = 0.9 reflector, 32^3, 4 groups, S8 (its rank cap 64 limits k to about "
                    "5e-5 of the oracle: this workload cannot reach 1e-6)"),
}
DEFAULT_WORKLOAD = "cube256_g2_s4_10cm"

PRECISION_TEXT = {
    "mixed": "FP32 Krylov contractions (SIMT) in FP64 iterative refinement; FP64 products, rounding, k",
    "tf32": ("FP32 Krylov contractions on tcgen05 tensor cores (TF32 three-term split, FP32 accumulation) "
             "in FP64 iterative refinement; FP64 products, rounding, k"),
    "bf16": ("FP32 Krylov contractions on tcgen05 tensor cores (BF16 three-term split, FP32 accumulation) "
             "in FP64 iterative refinement; FP64 products, rounding, k"),
    "fp64": "FP64 throughout",
}
DTYPE_TEXT = {"mixed": "f64+f32", "tf32": "f64+tf32x3", "bf16": "f64+bf16x3", "fp64": "f64"}


def golden_reference(name):
    """(k, oracle iterations to 1e-6) stored by tests/golden/make_oracle_reference.py, or None."""
    if os.path.exists(GOLDEN):
        for line in open(GOLDEN):
            if line.strip() and not line.startswith("#"):
                f = line.split()
                if f[0] == name:
                    return float(f[1]), int(f[3])
    return None


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo; 'unknown' if absent)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu part", "hardware"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine() or "unknown"


def oracle_ref(p, name, threads=0):
    """k of the oracle (stored for the large workloads, else computed here)
    and the oracle iterations after which its k stays within 1e-6."""
    g = golden_reference(name)
    if g is not None:
        return g[0], g[1], "stored (tests/golden/oracle_reference.txt)"
    from oracle import transport as T
    r = T.OracleProblem(p, threads=threads).keig(tol_k=1e-13, max_iter=100000, history=True)
    ks = r["k_hist"]
    n_ok = next(i for i in range(len(ks)) if np.all(np.abs(ks[i:] - r["k"]) < 1e-6 * r["k"])) + 1
    return r["k"], n_ok, "computed by the oracle in this run"


def oracle_sample(p, n_iter, threads):
    """Seconds per oracle power iteration on `threads` host cores, timed over
    n_iter iterations of the same workload (a bounded sample)."""
    from oracle import transport as T
    op = T.OracleProblem(p, threads=threads)
    t0 = time.time()
    op.keig(tol_k=0.0, max_iter=n_iter)
    return (time.time() - t0) / n_iter


class Clocks:
    """nvidia-smi sampler during the timed region."""

    def __init__(self, index=0):
        self.samples = []
        self.proc = None
        self.index = index

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 3 + i and s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def max_over_ranks(value, dist=None, device="cpu"):
    """The job's step time is the slowest rank's (replicas run the same
    problem; no collective touches the data path)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, name):
    """The oracle (plain FP64 CPU power iteration, the paper's fixed point on
    the full grid) on the same workload: time per iteration from a bounded
    sample of iterations, times the iterations the oracle needs to stay
    within 1e-6 of its converged k."""
    p = WORKLOADS[name][0]()
    cores = os.cpu_count() or 1
    kref, n_ok, src = oracle_ref(p, name, threads=cores)
    sample_it = max(2, min(10, int(20.0 / max(1e-9, 4e-9 * p.G * p.L * p.n ** 3))))
    times = [oracle_sample(p, sample_it, cores) * n_ok for _ in range(max(1, args.steps))]
    v = float(np.median(times))
    sample = (f"{sample_it} oracle iterations per step on {cores} cores, scaled to the {n_ok} iterations after "
              f"which its k stays within 1e-6 of its converged value (k {src})")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "grid": f"{p.n}^3", "groups": p.G, "directions": p.L,
                       "side_cm": p.side[0]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "k": kref}


def measured_peaks(K):
    """Live roofline denominators (TFLOP/s): the library's FP64 and FP32 FMA
    streams and the cuBLAS TF32 and BF16 GEMM rates (torch.matmul)."""
    from paper_2309_03347_gb300.peaks import measure_peaks
    return measure_peaks(gemms=True)


def make_opts(K, name, prec, max_iter):
    _, cap, eps, lf, sweeps, _ = WORKLOADS[name]
    o = K.keig_default_opts()
    o.eps, o.rmax = eps, cap
    o.tol_k, o.tol_psi, o.max_iter = 1e-10, 1e-7, max_iter
    o.solve_sweeps, o.mv_sweeps, o.kick = sweeps, sweeps, 4
    o.scheme = 0
    o.local_form = lf
    o.prec = {"mixed": K.TT_FP32_REFINED, "tf32": K.TT_TF32_SPLIT, "bf16": K.TT_BF16_SPLIT,
              "fp64": K.TT_FP64}[prec]
    return o


def first_within(k_hist, k_ref, tol=1e-6):
    """1-based index of the first iterate from which every later k stays
    within tol (relative) of k_ref, or None."""
    err = np.abs(np.asarray(k_hist) - k_ref) / abs(k_ref)
    for i in range(len(err)):
        if np.all(err[i:] < tol):
            return i + 1
    return None


def roof(name, n, gms, gfl, peak, source, ms_step, bound="alu"):
    """Roofline entry of one kernel from its per-launch CUDA-event times."""
    avg = gms / max(n, 1)
    ach = (gfl / max(n, 1)) / (avg * 1e-3) / 1e12 if n and avg > 0 else 0.0
    return {"bound": bound, "kernel": name, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak if peak else None, "traffic": None, "peak_source": source, "launches": n,
            "avg_launch_us": avg * 1e3, "ms_in_step": gms, "share_of_step": gms / ms_step if ms_step else None}


def batch_problems(n):
    """Seeded mix of independent problems for the batched mode: bare 10 cm cubes
    of 16^3 or 32^3 points, 2 or 4 groups, S4, S6 or S8, rank caps 16-64."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(2000 + i)
        l = int(rng.choice([4, 5]))
        G = int(rng.choice([2, 4]))
        order = int(rng.choice([4, 6, 8]))
        prob = ki.homogeneous(l=l, G=G, order=order, side=10.0, seed=2000 + i, name=f"batch{i}")
        out.append((prob, int(rng.integers(16, 65))))
    return out


def run_batch(args):
    """Batched mode: problems/s of keig_batch over a seeded mix, grouped
    persistent-GMRES launches against one whole-GPU launch per system, and the
    per-problem k error against the oracle."""
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2309_03347_gb300 as K
    from oracle import transport as T
    probs = batch_problems(args.batch)
    opts = []
    for prob, cap in probs:
        o = K.keig_default_opts()
        o.eps, o.rmax, o.tol_k, o.tol_psi, o.max_iter = 1e-8, cap, 1e-9, 1e-5, 150
        o.solve_sweeps = o.mv_sweeps = 1
        o.local_form = 1
        o.prec = K.TT_FP32_REFINED
        opts.append(o)
    plist = [p for p, _ in probs]
    out = {}
    for mode in ("grouped", "ungrouped"):
        if mode == "ungrouped":
            os.environ["KEIG_BATCH_UNGROUPED"] = "1"
        else:
            os.environ.pop("KEIG_BATCH_UNGROUPED", None)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res, _ = K.keig_batch(plist, opts, n_workers=args.batch_workers)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        out[mode] = {"s": wall, "problems_per_s": len(plist) / wall,
                     "group_launches": K.keig_batch.last_group_launches,
                     "group_systems": K.keig_batch.last_group_systems, "res": res}
    os.environ.pop("KEIG_BATCH_UNGROUPED", None)
    errs = []
    for (prob, _), r in zip(probs, out["grouped"]["res"]):
        kref = T.OracleProblem(prob).keig(tol_k=1e-12, max_iter=100000)["k"]
        errs.append(abs(r["k"] - kref) / kref)
    line = {"metric": "problems per second (batched k-eigenvalue solves)", "value": out["grouped"]["problems_per_s"],
            "unit": "problems/s", "higher_is_better": True, "n_problems": len(plist),
            "workers": args.batch_workers,
            "config": {"workload": "bare 10 cm cubes 16^3/32^3, G 2/4, S4-S8, rank caps 16-64, seeds 2000+p",
                       "local_systems": "least squares", "precision": PRECISION_TEXT["mixed"]},
            "grouped": {k: v for k, v in out["grouped"].items() if k != "res"},
            "one_launch_per_system": {k: v for k, v in out["ungrouped"].items() if k != "res"},
            "k_rel_err": {"max": float(np.max(errs)), "median": float(np.median(errs)),
                          "within_1e-6": int(np.sum(np.array(errs) < 1e-6))}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="mixed", choices=["mixed", "tf32", "bf16", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=0,
                    help="batched mode: solve this many independent problems with keig_batch (problems/s)")
    ap.add_argument("--batch-workers", type=int, default=8)
    ap.add_argument("--max-iter", type=int, default=None,
                    help="run every solve for this many outer iterations (short runs for profiler captures)")
    args = ap.parse_args()

    if args.batch:
        run_batch(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    name = args.workload
    p = WORKLOADS[name][0]()

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, name)))
        return

    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import __graft_entry__ as g
    g.build()
    import paper_2309_03347_gb300 as K

    peaks = measured_peaks(K)
    kref, n_ok_oracle, kref_src = oracle_ref(p, name, threads=os.cpu_count() or 1)
    ctx = K.tt_ctx_create()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)

    def step(o, phi_out=None, prob=p):
        return K.keig_fixed_point(ctx, prob, o, allow_noconv=True, phi_out=phi_out)

    # ---- warm-up: the first solve runs to the solver's own stop and fixes the
    # number of outer iterations after which k stays within 1e-6 of the oracle
    full = make_opts(K, name, args.prec, args.max_iter or 150)
    flush.fill_(1.0)
    r0 = step(full)
    n_ok = first_within(r0["k_hist"], kref)
    # the timed steps run to the first iterate from which k stays within 7e-7:
    # a margin under 1e-6 for rounding differences between runs (the GMRES
    # grid-size tuner may pick other grids in later runs)
    n_safe = first_within(r0["k_hist"], kref, 7e-7)
    if args.max_iter:
        n_it = args.max_iter
    else:
        n_it = n_safe if n_safe is not None else (n_ok if n_ok is not None else r0["iters"])
    opts = make_opts(K, name, args.prec, n_it)
    for _ in range(max(0, args.warmup - 1)):
        flush.fill_(1.0)
        step(opts)
    torch.cuda.synchronize()

    # ---- device-timed steps
    ev, results = [], []
    ctx.reset_counters()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            results.append(step(opts))
            b.record(stream)
            ev.append((a, b))
        torch.cuda.synchronize()
    launches, cflops = ctx.counters()
    if dist:
        dist.barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    ms_step = max_over_ranks(float(np.median(ms)), dist, "cuda")
    errs = [abs(r["k"] - kref) / kref for r in results]

    # ---- end to end: host wall time of the same call through the public API,
    # problem tables in pinned host memory (copied to the device inside the
    # call) and the scalar flux copied back into a pinned host buffer
    pins = []  # keep the pinned tensors alive for the arrays that view them

    def pinned(a):
        a = np.ascontiguousarray(a)
        t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
        pins.append(t)
        out = t.numpy()
        out[...] = a
        return out
    p_pin = dataclasses.replace(p, sig_t=pinned(p.sig_t), sig_s=pinned(p.sig_s), nu_sig_f=pinned(p.nu_sig_f),
                                chi=pinned(p.chi), mat=pinned(p.mat))
    phi_pin = pinned(np.zeros((p.G, p.n, p.n, p.n)))
    e2e = []
    for _ in range(max(1, min(args.steps, 2))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(opts, phi_out=phi_pin, prob=p_pin)
        e2e.append(time.perf_counter() - t0)
    phi_bytes = phi_pin.nbytes
    in_bytes = sum(x.nbytes for x in (p.sig_t, p.sig_s, p.nu_sig_f, p.chi, p.mat)) + 4 * p.quad.amu.nbytes

    # ---- one instrumented step: per-launch device time of the contraction kernels
    ctx.set_profiling(True)
    flush.fill_(1.0)
    step(opts)
    n_gemm, gemm_ms, gemm_flops = ctx.gemm_stats()
    n32, gemm32_ms, gemm32_flops = ctx.gemm32_stats()
    ntc, gemmtc_ms, gemmtc_flops = ctx.gemmtc_stats()
    npg, pg_ms, pg_flops = ctx.gmres_stats()
    ctx.set_profiling(False)

    if rank != 0:
        return
    res = results[-1]
    _, cap, eps, lf, sweeps, note = WORKLOADS[name]
    line = {
        "metric": METRIC, "value": ms_step / 1e3, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE_TEXT[args.prec], "data": "synthetic",
        "config": {"workload": name, "description": note, "grid": f"{p.n}^3", "groups": p.G, "directions": p.L,
                   "side_cm": p.side[0], "rank_cap": cap, "eps": eps, "scheme": "paper",
                   "local_systems": "least squares (Eq. (linear_system_obj))" if lf else "Galerkin",
                   "amen_sweeps": sweeps,
                   "outer_iterations": n_it,
                   "outer_iterations_rule": "first iterate from which k stays within 7e-7 of the oracle "
                                            "(1e-6 with a margin for run-to-run rounding)",
                   "precision": PRECISION_TEXT[args.prec],
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "k": res["k"], "k_oracle": kref, "k_oracle_source": kref_src,
        "k_rel_err": float(np.max(errs)), "within_1e-6": bool(n_ok is not None and max(errs) < 1e-6),
        "time_to_1e-6_ms": ms_step if (n_ok is not None and not args.max_iter) else None,
        "first_solve": {"iters": r0["iters"], "k_rel_err": abs(r0["k"] - kref) / kref, "wall_ms": r0["wall_ms"],
                        "first_within_1e-6": n_ok,
                        "t_at_first_within_ms": float(r0["t_hist"][n_ok - 1]) if n_ok else None},
        "max_rank": res["max_rank"],
        "gpu_launches": int(launches // max(args.steps, 1)),
        "e2e": {"value": float(np.median(e2e)), "unit": UNIT, "h2d_bytes_per_step": int(in_bytes),
                "d2h_bytes_per_step": int(phi_bytes)},
        "peaks_tflops": {k: v for k, v in peaks.items() if isinstance(v, float)},
    }
    src_fma = "measured live: the library's FMA-stream kernel (tt_measure_fma_peak)"
    tc_peak = peaks["bf16_gemm"] if args.prec == "bf16" else peaks["tf32_gemm"]
    r64 = roof("dgemm_kernel (FP64 contraction GEMM)", n_gemm, gemm_ms, gemm_flops, peaks["fp64_fma"],
               src_fma + ", FP64", ms_step)
    r32 = roof("sgemm_kernel (FP32 SIMT contraction GEMM)", n32, gemm32_ms, gemm32_flops, peaks["fp32_fma"],
               src_fma + ", FP32", ms_step)
    rtc = roof("tc_gemm_kernel (tcgen05 three-term split GEMM; 3 MMA passes per product, so frac <= 1/3)",
               ntc, gemmtc_ms, gemmtc_flops, tc_peak,
               "measured live: cuBLAS " + ("BF16" if args.prec == "bf16" else "TF32") + " GEMM 8192^3",
               ms_step, bound="tensor")
    rpg = roof("pgmres_kernel (persistent FP32 GMRES of the local systems: local matvecs + Gram-Schmidt)", npg,
               pg_ms, pg_flops, peaks["fp32_fma"], src_fma + ", FP32", ms_step)
    roofs = sorted([(gemm_ms, r64), (gemm32_ms, r32), (gemmtc_ms, rtc), (pg_ms, rpg)], key=lambda t: -t[0])
    line["roofline"] = roofs[0][1]
    line["roofline_other"] = [r for _, r in roofs[1:] if r["launches"]]
    line["contraction_tflops_step"] = cflops / max(args.steps, 1) / (ms_step * 1e-3) / 1e12
    line["clocks"] = clk.summary()
    if not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        it_all = max(2, min(10, int(20.0 / max(1e-9, 4e-9 * p.G * p.L * p.n ** 3))))
        t_all = oracle_sample(p, it_all, cores)
        t_one = oracle_sample(p, 1, 1)
        line["cpu_baseline"] = {
            "value": t_all * n_ok_oracle, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"{it_all} oracle power iterations timed on {cores} cores ({t_all:.3f} s each), scaled to "
                       f"the {n_ok_oracle} iterations after which the oracle's k stays within 1e-6 of its "
                       f"converged value"),
            "cpu_model": cpu_model(),
            "one_core": {"value": t_one * n_ok_oracle, "unit": UNIT, "cores": 1,
                         "sample": f"1 iteration timed on 1 core ({t_one:.3f} s), scaled likewise"}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
