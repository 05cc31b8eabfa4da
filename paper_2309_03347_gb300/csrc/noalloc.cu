// Allocation-free inner product of two TT vectors (tt_dot_noalloc).
//
// Some callers cannot allocate device memory at the point where they need
// the result: a real-time loop where cudaMalloc/cudaFree would stall or
// serialise the device, and hosts that hand the library a fixed memory
// budget and forbid further allocations.  For them this entry point computes <x, y> with its scratch in
// a fixed file-scope device array instead of the context's allocator.
//
// The scratch array lives in every device that loads the library until the
// process exits.  All calls share it, and it keeps the last call's contents;
// every scratch value a call reads is written earlier in the same call, so no
// clearing between calls is needed.  Two calls that overlap on the GPU (on
// different streams, or from different host threads) race on the array.
#include <mutex>

#include "common.cuh"

namespace {

constexpr int kMaxRank = 128;  // largest bond rank accepted
constexpr int kMaxMode = 64;   // largest mode size accepted
// two rank x rank interface matrices and one rank x mode x rank intermediate
constexpr size_t kScratchDoubles = 2 * (size_t)kMaxRank * kMaxRank + (size_t)kMaxRank * kMaxMode * kMaxRank;

static __device__ __align__(256) double g_dot_scratch[kScratchDoubles];  // 8.25 MiB

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_addr[kMaxDevices] = {nullptr};

// t[b, i, a'] = sum_a v[a, b] x[a, i, a']      (v: rx0 x ry0)
__global__ void dot_left(const double *__restrict__ v, const double *__restrict__ x, int rx0, int ry0, int n,
                         int rx1, double *__restrict__ t) {
  const int tot = ry0 * n * rx1;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
    const int a1 = e % rx1, bi = e / rx1;
    const int i = bi % n, b = bi / n;
    double s = 0.0;
    for (int a = 0; a < rx0; ++a) s = fma(v[a * ry0 + b], x[((long long)a * n + i) * rx1 + a1], s);
    t[e] = s;
  }
}

// v'[a', b'] = sum_{b, i} t[b, i, a'] y[b, i, b']
__global__ void dot_right(const double *__restrict__ t, const double *__restrict__ y, int ry0, int n, int rx1,
                          int ry1, double *__restrict__ vout) {
  const int tot = rx1 * ry1;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
    const int b1 = e % ry1, a1 = e / ry1;
    double s = 0.0;
    for (int bi = 0; bi < ry0 * n; ++bi) s = fma(t[(long long)bi * rx1 + a1], y[(long long)bi * ry1 + b1], s);
    vout[e] = s;
  }
}

__global__ void dot_init(double *v) { v[0] = 1.0; }
__global__ void dot_final(const double *v, double *out) { out[0] = v[0]; }

void set_err(char *err, size_t len, const char *msg) {
  if (err && len) {
    strncpy(err, msg, len - 1);
    err[len - 1] = '\0';
  }
}

}  // namespace

extern "C" int tt_dot_noalloc(const double *x_cores, const int *rx, const double *y_cores, const int *ry, int d,
                              const int *n, double *out, void *cuda_stream, char *err, size_t err_len) {
  if (!x_cores || !y_cores || !rx || !ry || !n || !out || d < 1) {
    set_err(err, err_len, "tt_dot_noalloc: null pointer or d < 1");
    return TT_EINVAL;
  }
  if (rx[0] != 1 || ry[0] != 1 || rx[d] != 1 || ry[d] != 1) {
    set_err(err, err_len, "tt_dot_noalloc: boundary ranks must be 1");
    return TT_EINVAL;
  }
  for (int k = 0; k <= d; ++k)
    if (rx[k] < 1 || ry[k] < 1 || rx[k] > kMaxRank || ry[k] > kMaxRank) {
      set_err(err, err_len, "tt_dot_noalloc: a bond rank is outside [1, 128]");
      return TT_EINVAL;
    }
  for (int k = 0; k < d; ++k)
    if (n[k] < 1 || n[k] > kMaxMode) {
      set_err(err, err_len, "tt_dot_noalloc: a mode size is outside [1, 64]");
      return TT_EINVAL;
    }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_err(err, err_len, "tt_dot_noalloc: no usable current CUDA device");
    return TT_ECUDA;
  }
  double *scratch = nullptr;
  {
    // first call on a device: look up the device address of the array (kept
    // for the process; a cudaDeviceReset invalidates it)
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_dot_scratch);
      if (e != cudaSuccess) {
        set_err(err, err_len, cudaGetErrorString(e));
        return TT_ECUDA;
      }
      g_scratch_addr[dev] = static_cast<double *>(p);
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  double *v = scratch;
  double *v2 = scratch + (size_t)kMaxRank * kMaxRank;
  double *t = scratch + 2 * (size_t)kMaxRank * kMaxRank;
  dot_init<<<1, 1, 0, s>>>(v);
  size_t ox = 0, oy = 0;
  for (int k = 0; k < d; ++k) {
    const int tA = ry[k] * n[k] * rx[k + 1];
    dot_left<<<(tA + 255) / 256, 256, 0, s>>>(v, x_cores + ox, rx[k], ry[k], n[k], rx[k + 1], t);
    const int tB = rx[k + 1] * ry[k + 1];
    dot_right<<<(tB + 255) / 256, 256, 0, s>>>(t, y_cores + oy, ry[k], n[k], rx[k + 1], ry[k + 1], v2);
    double *tmp = v;
    v = v2;
    v2 = tmp;
    ox += (size_t)rx[k] * n[k] * rx[k + 1];
    oy += (size_t)ry[k] * n[k] * ry[k + 1];
  }
  dot_final<<<1, 1, 0, s>>>(v, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_err(err, err_len, cudaGetErrorString(e));
    return TT_ECUDA;
  }
  return TT_OK;
}
