"""Measured arithmetic peaks of the current GPU: the roofline denominators of
the library's FP64 and FP32 SIMT kernels (tt_measure_fma_peak, the
library's own FMA-stream kernel) and, for context, the library GEMM rates of
cuBLAS through torch.matmul (FP64, FP32 without TF32, TF32, BF16).

python -m paper_2309_03347_gb300.peaks  prints one JSON line.
"""
from __future__ import annotations

import json


def _gemm_tflops(dtype, n, reps=5, tf32=False):
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = tf32
    try:
        a = torch.randn(n, n, device="cuda").to(dtype)
        b = torch.randn(n, n, device="cuda").to(dtype)
        c = a @ b
        torch.cuda.synchronize()
        best = 0.0
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            c = a @ b
            e1.record()
            e1.synchronize()
            best = max(best, 2.0 * n ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
        del c
        return best
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def measure_peaks(gemms: bool = True) -> dict:
    """TFLOP/s: fp64_fma, fp32_fma (the library's FMA streams), and with
    gemms the cuBLAS rates dgemm, sgemm (no TF32), tf32_gemm, bf16_gemm."""
    import torch

    from ._lib import tt_measure_fma_peak
    out = {
        "fp64_fma": tt_measure_fma_peak(True, iters=512) / 1e12,
        "fp32_fma": tt_measure_fma_peak(False, iters=4096) / 1e12,
        "how": "fma: 4 CTAs x 256 threads per SM, 8 independent FMA chains per thread, best of 5 launches "
               "(CUDA events); gemm: torch.matmul (cuBLAS), best of 5",
        "device": torch.cuda.get_device_name(),
    }
    if gemms:
        out["dgemm"] = _gemm_tflops(torch.float64, 4096)
        out["sgemm"] = _gemm_tflops(torch.float32, 8192, tf32=False)
        out["tf32_gemm"] = _gemm_tflops(torch.float32, 8192, tf32=True)
        out["bf16_gemm"] = _gemm_tflops(torch.bfloat16, 8192)
    return out


if __name__ == "__main__":
    print(json.dumps(measure_peaks()))
