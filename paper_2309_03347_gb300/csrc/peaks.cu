// Peak arithmetic rates of the device the library runs on, measured by
// dependent-free fused multiply-add streams (the roofline denominators of
// the FP64 and FP32 SIMT kernels).  Each thread runs kChains independent FMA
// chains for `iters` rounds; every SM gets four CTAs of 256 threads, enough
// warps to hide the FMA latency.  flops = 2 x threads x chains x iters.
#include "common.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) fma_stream_kernel(T *out, int iters, T seed) {
  T a[kChains];
  const T b = seed * (T)0.999999, c = (T)1e-7;
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = seed + (T)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  // never true for the seeds used; keeps the chains live
  if (s == (T)-12345.0) out[blockIdx.x * kThreads + threadIdx.x] = s;
}

template <class T>
double measure(cudaStream_t st, int sms, int iters, int reps) {
  const int blocks = sms * 4;
  T *out = nullptr;
  TT_CHECK_CUDA(cudaMallocAsync(&out, sizeof(T) * blocks * kThreads, st));
  cudaEvent_t e0, e1;
  TT_CHECK_CUDA(cudaEventCreate(&e0));
  TT_CHECK_CUDA(cudaEventCreate(&e1));
  fma_stream_kernel<T><<<blocks, kThreads, 0, st>>>(out, iters, (T)1.0);  // warm-up
  double best = 0.0;
  for (int r = 0; r < reps; ++r) {
    TT_CHECK_CUDA(cudaEventRecord(e0, st));
    fma_stream_kernel<T><<<blocks, kThreads, 0, st>>>(out, iters, (T)1.0);
    TT_CHECK_CUDA(cudaEventRecord(e1, st));
    TT_CHECK_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    TT_CHECK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    const double flops = 2.0 * blocks * kThreads * (double)kChains * 16.0 * iters;
    best = std::max(best, flops / (ms * 1e-3));
  }
  TT_CHECK_CUDA(cudaGetLastError());
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  TT_CHECK_CUDA(cudaFreeAsync(out, st));
  TT_CHECK_CUDA(cudaStreamSynchronize(st));
  return best;
}

}  // namespace

extern "C" int tt_measure_fma_peak(void *cuda_stream, int fp64, int iters, int reps, double *flops_per_s) {
  if (!flops_per_s || iters < 1 || reps < 1) return TT_EINVAL;
  try {
    int dev = 0, sms = 0;
    TT_CHECK_CUDA(cudaGetDevice(&dev));
    TT_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    *flops_per_s = fp64 ? measure<double>(st, sms, iters, reps) : measure<float>(st, sms, iters, reps);
    return TT_OK;
  } catch (const tt::Error &e) {
    return e.code;
  }
}
