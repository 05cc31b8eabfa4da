"""Benchmark: time to a k-eigenvalue solution within 1e-6 of the FP64 oracle,
with the contraction kernel's FP64 throughput against its roofline.

One step = one call of keig_fixed_point on the synthetic workload (operator
construction, QTT fixed point to the solver's own stop), inputs resident on
the device side of the library when the timed region starts (the problem
tables are a few KB and are copied inside the call).  `value` is seconds per
solve measured with CUDA events on the library stream; `e2e` is the same call
timed on the host with the scalar flux copied back to host memory.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
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
FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 rate from the profiling recipe's table (nominal)


def workload():
    p = ki.config(1)
    return p


def opts_for(K, p, prec="mixed"):
    o = K.keig_default_opts()
    o.eps, o.rmax = p.eps, p.rmax
    o.tol_k, o.tol_psi, o.max_iter = 1e-9, 1e-5, 20
    o.solve_sweeps, o.mv_sweeps, o.kick = 2, 2, 4
    o.scheme = 0
    o.prec = {"mixed": K.TT_FP32_REFINED, "tf32": K.TT_TF32_SPLIT, "fp64": K.TT_FP64}[prec]
    return o


PRECISION_TEXT = {
    "mixed": "FP32 Krylov contractions (SIMT) in FP64 iterative refinement; FP64 products, rounding, k",
    "tf32": ("FP32 Krylov contractions on tcgen05 tensor cores (TF32 three-term split, FP32 accumulation) "
             "in FP64 iterative refinement; FP64 products, rounding, k"),
    "fp64": "FP64 throughout",
}
DTYPE_TEXT = {"mixed": "f64+f32", "tf32": "f64+tf32x3", "fp64": "f64"}


def tf32_tensor_peak_tflops():
    """Dense TF32 tensor rate: the measured sustained bf16 cuBLAS rate of
    MEASURED_PEAKS.json times the nominal tf32/bf16 ratio (1.1 / 2.25)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16 = float(json.load(f)["bf16_tflops_sustained"])
        src = "measured sustained bf16 x 1.1/2.25 (nominal tf32/bf16)"
    except (OSError, KeyError, ValueError):
        bf16 = 1700.0
        src = "fallback sustained bf16 x 1.1/2.25 (nominal tf32/bf16)"
    return bf16 * 1.1 / 2.25, src


# FP32 SIMT peak of the part from its unit counts and clock: 152 SMs x 128
# FP32 lanes x 2 flops (FMA) x the maximum SM clock.
def fp32_simt_peak_tflops(sm_mhz=2070.0, sms=152):
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


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


def oracle_reference(p, threads=0, tol=1e-10):
    from oracle import transport as T
    t0 = time.time()
    r = T.OracleProblem(p, threads=threads).keig(tol_k=tol, max_iter=20000, history=True)
    return r, time.time() - t0


def first_within(k_hist, t_hist, k_ref, tol=1e-6):
    """Time (ms) of the first iterate from which k stays within tol of k_ref."""
    err = np.abs(np.asarray(k_hist) - k_ref) / abs(k_ref)
    ok = err < tol
    for i in range(len(ok)):
        if ok[i:].all():
            return float(t_hist[i]), i + 1
    return None, None


def cpu_model():
    """The host CPU's model name (from /proc/cpuinfo; 'unknown' if absent)."""
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu part", "hardware"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine() or "unknown"


def run_reference(args, p):
    """The oracle (plain FP64 CPU power iteration) on the same workload; the
    CPU program keeps no state between runs, so it needs no warm-up."""
    cores = os.cpu_count() or 1
    times, kref = [], None
    for _ in range(args.steps):
        r, dt = oracle_reference(p, threads=cores, tol=1e-9)
        # time to k within 1e-6 of its own converged value
        ks = r["k_hist"]
        kref = r["k"]
        n_ok = next(i for i in range(len(ks)) if np.all(np.abs(ks[i:] - kref) / kref < 1e-6)) + 1
        times.append(dt * n_ok / max(r["iters"], 1))
    v = float(np.median(times))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": p.name, "grid": f"{p.n}^3", "groups": p.G, "directions": p.L,
                       "side_cm": p.side[0]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "full power iteration to |dk| < 1e-9; time scaled to the first "
                                       "iterate within 1e-6 of the converged k"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "k": kref}
    line["cpu_baseline"]["cpu_model"] = cpu_model()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--max-iter", type=int, default=None,
                    help="cap the outer iterations (short runs for profiler captures)")
    ap.add_argument("--prec", default="mixed", choices=["mixed", "tf32", "fp64"])
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    p = workload()

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, p)))
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

    ctx = K.tt_ctx_create()
    opts = opts_for(K, p, args.prec)
    if args.max_iter:
        opts.max_iter = args.max_iter
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)

    def step(want_phi=False):
        return K.keig_fixed_point(ctx, p, opts, want_phi=want_phi, allow_noconv=True)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()

    # ---- device-timed steps
    ev = []
    results = []
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
            results.append(step())
            b.record(stream)
            ev.append((a, b))
        torch.cuda.synchronize()
    launches, cflops = ctx.counters()
    if dist:
        dist.barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    ms_step = max_over_ranks(float(np.median(ms)), dist, "cuda")

    # ---- end to end: host wall time including the scalar-flux readback
    # inputs (the problem tables) and the scalar-flux result in pinned host memory
    pins = []  # keep the pinned tensors alive for the arrays that view them

    def pinned(a):
        a = np.ascontiguousarray(a)
        t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
        pins.append(t)
        out = t.numpy()
        out[...] = a
        return out
    import dataclasses
    p_pin = dataclasses.replace(p, sig_t=pinned(p.sig_t), sig_s=pinned(p.sig_s), nu_sig_f=pinned(p.nu_sig_f),
                                chi=pinned(p.chi), mat=pinned(p.mat))
    phi_pin = pinned(np.zeros((p.G, p.n, p.n, p.n)))
    e2e = []
    for _ in range(max(1, args.steps)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = K.keig_fixed_point(ctx, p_pin, opts, allow_noconv=True, phi_out=phi_pin)
        e2e.append(time.perf_counter() - t0)
    phi_bytes = phi_pin.nbytes
    in_bytes = sum(x.nbytes for x in (p.sig_t, p.sig_s, p.nu_sig_f, p.chi, p.mat)) + 4 * p.quad.amu.nbytes

    # ---- one instrumented step: per-launch device time of the contraction GEMM
    ctx.set_profiling(True)
    step()
    n_gemm, gemm_ms, gemm_flops = ctx.gemm_stats()
    n32, gemm32_ms, gemm32_flops = ctx.gemm32_stats()
    ntc, gemmtc_ms, gemmtc_flops = ctx.gemmtc_stats()
    npg, pg_ms, pg_flops = ctx.gmres_stats()
    ctx.set_profiling(False)

    if rank != 0:
        return
    res = results[-1]
    line = {
        "metric": METRIC, "value": ms_step / 1e3, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE_TEXT[args.prec], "data": "synthetic",
        "config": {"workload": p.name, "grid": f"{p.n}^3", "groups": p.G, "directions": p.L,
                   "side_cm": p.side[0], "rank_cap": p.rmax, "eps": p.eps, "scheme": "paper",
                   "precision": PRECISION_TEXT[args.prec],
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "k": res["k"], "iters": res["iters"], "max_rank": res["max_rank"], "converged": res["code"] == 0,
        "gpu_launches": int(launches // max(args.steps, 1)),
        "e2e": {"value": float(np.median(e2e)), "unit": UNIT, "h2d_bytes_per_step": int(in_bytes),
                "d2h_bytes_per_step": int(phi_bytes)},
    }
    def roof(name, n, gms, gfl, peak, source, bound="alu"):
        avg = gms / max(n, 1)
        ach = (gfl / max(n, 1)) / (avg * 1e-3) / 1e12 if n else 0.0
        return {"bound": bound, "kernel": name, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None, "peak_source": source, "launches": n,
                "avg_launch_us": avg * 1e3, "ms_in_step": gms, "share_of_step": gms / ms_step if ms_step else None}

    sm_max = clk.summary().get("sm_max_mhz") or 2070.0
    r64 = roof("dgemm_kernel (FP64 contraction GEMM)", n_gemm, gemm_ms, gemm_flops, FP64_NOMINAL_TFLOPS,
               "nominal FP64 rate of the recipe table (MEASURED_PEAKS.json has no FP64 entry)")
    r32 = roof("sgemm_kernel (FP32 contraction GEMM of the mixed-precision solves)", n32, gemm32_ms, gemm32_flops,
               fp32_simt_peak_tflops(sm_max),
               "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock (MEASURED_PEAKS.json has no FP32 entry)")
    tf32_peak, tf32_src = tf32_tensor_peak_tflops()
    rtc = roof("tc_gemm_kernel (tcgen05 TF32 three-term contraction GEMM; 3 MMA passes per product, "
               "so frac <= 1/3)", ntc, gemmtc_ms, gemmtc_flops, tf32_peak, tf32_src, bound="tensor")
    rpg = roof("pgmres_kernel (persistent FP32 GMRES of the local systems: local matvecs + Gram-Schmidt)", npg,
               pg_ms, pg_flops, fp32_simt_peak_tflops(sm_max),
               "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock (MEASURED_PEAKS.json has no FP32 entry)")
    # the dominant contraction kernel of the step (by device time) carries the roofline
    roofs = sorted([(gemm_ms, r64), (gemm32_ms, r32), (gemmtc_ms, rtc), (pg_ms, rpg)], key=lambda t: -t[0])
    line["roofline"] = roofs[0][1]
    line["roofline_other_gemm"] = [r for t, r in roofs[1:] if r["launches"]]
    line["contraction_tflops_step"] = cflops / max(args.steps, 1) / (ms_step * 1e-3) / 1e12
    line["clocks"] = clk.summary()
    if not args.no_cpu_baseline:
        r, dt = oracle_reference(p, threads=os.cpu_count() or 1, tol=1e-10)
        kref = r["k"]
        t_ok, it_ok = first_within(res["k_hist"], res["t_hist"], kref)
        line["k_oracle"] = kref
        line["k_rel_err"] = abs(res["k"] - kref) / kref
        line["time_to_1e-6_ms"] = t_ok
        ks = r["k_hist"]
        n_ok = next(i for i in range(len(ks)) if np.all(np.abs(ks[i:] - kref) / kref < 1e-6)) + 1
        line["cpu_baseline"] = {"value": dt * n_ok / max(r["iters"], 1), "unit": UNIT,
                                "cores": os.cpu_count() or 1, "kind": "oracle",
                                "sample": f"full FP64 power iteration ({r['iters']} iterations, {dt:.2f} s); "
                                          f"time scaled to the first of {n_ok} iterates within 1e-6"}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
