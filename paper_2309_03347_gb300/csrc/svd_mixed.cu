// Mixed-precision one-sided Jacobi SVD of a small square matrix.
//
// The rotations of a one-sided Jacobi SVD (Hestenes) are first found in FP32
// (an SM's FP32 rate is 64x its FP64 rate on this part), giving V32 with
// R V32 ~ U S to FP32 accuracy.  V32 is promoted to FP64 and made orthogonal
// to FP64 accuracy by two Newton-Schulz steps V <- V (3 I - V^T V) / 2 (each
// squares the orthogonality error; multi-SM FP64 GEMMs).  The FP64 one-sided
// Jacobi then runs on B = R V, whose columns are already orthogonal to FP32
// accuracy, so it converges quadratically in about two sweeps; the result is
// R = U S (V Q)^T with Q the FP64 rotations.
#include "common.cuh"

namespace tt {

namespace {

constexpr int J32_THREADS = 1024;
constexpr int J32_MAX_SWEEPS = 12;

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// B (n x n, column-major, FP64 input) -> V (n x n column-major FP32 rotations)
__global__ void __launch_bounds__(J32_THREADS) jacobi32_kernel(const double *__restrict__ Bin, int n,
                                                               float *__restrict__ Vout) {
  extern __shared__ float sm[];
  float *B = sm;
  float *V = sm + (size_t)n * n;
  __shared__ int s_rot;
  const long long nn = (long long)n * n;
  for (long long e = threadIdx.x; e < nn; e += blockDim.x) {
    B[e] = (float)Bin[e];
    V[e] = ((e % n) == (e / n)) ? 1.f : 0.f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int np = (n + 1) & ~1;
  const float tol = fmaxf(1e-6f, 1.2e-7f * sqrtf((float)n));
  for (int sweep = 0; sweep < J32_MAX_SWEEPS; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      for (int t = warp; t < np / 2; t += nwarp) {
        int p, q;
        if (t == 0) {
          p = np - 1;
          q = round;
        } else {
          p = (round + t) % (np - 1);
          q = (round - t + (np - 1)) % (np - 1);
        }
        if (p >= n || q >= n) continue;
        float *bp = B + (long long)p * n, *bq = B + (long long)q * n;
        float al = 0.f, be = 0.f, ga = 0.f;
        for (int i = lane; i < n; i += 32) {
          const float x = bp[i], y = bq[i];
          al = fmaf(x, x, al);
          be = fmaf(y, y, be);
          ga = fmaf(x, y, ga);
        }
        al = warp_sum_f(al);
        be = warp_sum_f(be);
        ga = warp_sum_f(ga);
        if (ga == 0.f || al == 0.f || be == 0.f) continue;
        if (fabsf(ga) <= tol * sqrtf(al * be)) continue;
        const float zeta = (be - al) / (2.f * ga);
        const float tt = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
        const float cs = 1.f / sqrtf(1.f + tt * tt);
        const float sn = cs * tt;
        float *vp = V + (long long)p * n, *vq = V + (long long)q * n;
        for (int i = lane; i < n; i += 32) {
          const float x = bp[i], y = bq[i];
          bp[i] = cs * x - sn * y;
          bq[i] = sn * x + cs * y;
          const float u = vp[i], w = vq[i];
          vp[i] = cs * u - sn * w;
          vq[i] = sn * u + cs * w;
        }
        if (lane == 0) atomicAdd(&s_rot, 1);
      }
      __syncthreads();
    }
    if (s_rot == 0) break;
    __syncthreads();
  }
  for (long long e = threadIdx.x; e < nn; e += blockDim.x) Vout[e] = V[e];
}

__global__ void f2d_kernel(const float *__restrict__ x, double *__restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

}  // namespace

bool jacobi_svd_mixed_fits(int n) { return 2LL * n * n * (long long)sizeof(float) <= 200 * 1024; }

// Same contract as jacobi_svd: B (n x n column-major, destroyed) = U S V^T.
void jacobi_svd_mixed(Ctx *c, double *B, int n, double *U, double *S, double *V) {
  TT_REQUIRE(jacobi_svd_mixed_fits(n), "jacobi_svd_mixed: matrix too large");
  const size_t nn = (size_t)n * n;
  DBuf v32(c, (nn + 1) / 2), vd(c, nn), g(c, nn), w(c, nn), rb(c, nn), q(c, nn);
  const size_t smem = 2 * nn * sizeof(float);
  TT_CHECK_CUDA(cudaFuncSetAttribute(jacobi32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  jacobi32_kernel<<<1, J32_THREADS, smem, c->stream>>>(B, n, reinterpret_cast<float *>(v32.p()));
  c->count();
  TT_CHECK_CUDA(cudaGetLastError());
  f2d_kernel<<<(unsigned)std::min<size_t>((nn + 255) / 256, 1024), 256, 0, c->stream>>>(
      reinterpret_cast<const float *>(v32.p()), vd.p(), nn);
  c->count();
  TT_CHECK_CUDA(cudaGetLastError());
  // Column-major products with the row-major GEMM: Z = X Y  <=>  Z^T = Y^T X^T.
  for (int it = 0; it < 2; ++it) {
    // g = V^T V  (symmetric)
    gemm(c, false, true, n, n, n, 1.0, vd.p(), n, 0, vd.p(), n, 0, 0.0, g.p(), n, 0);
    // w = V g ;  V = 1.5 V - 0.5 w
    gemm(c, false, false, n, n, n, 1.0, g.p(), n, 0, vd.p(), n, 0, 0.0, w.p(), n, 0);
    axpby(c, nn, -0.5, w.p(), 1.5, vd.p());
  }
  // rb = B V  (columns orthogonal to FP32 accuracy)
  gemm(c, false, false, n, n, n, 1.0, vd.p(), n, 0, B, n, 0, 0.0, rb.p(), n, 0);
  // FP64 Jacobi on rb: rb = U S Q^T, then V_final = V Q
  jacobi_svd(c, rb.p(), n, U, S, q.p());
  gemm(c, false, false, n, n, n, 1.0, q.p(), n, 0, vd.p(), n, 0, 0.0, V, n, 0);
}

}  // namespace tt
