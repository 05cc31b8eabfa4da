// Mixed-precision SVD of a small square matrix R (column-major).
//
// FP64 arithmetic on this part runs at 1/64 of the FP32 rate, so a one-CTA
// FP64 Jacobi sweep over a 64 x 64 matrix costs about half a millisecond.
// Here the rotations are found by a one-sided (Hestenes) Jacobi in FP32 on
// one CTA, and every FP64 step afterwards is a multi-SM matrix product:
//
//   1. V32: FP32 Jacobi rotations with R V32 ~ U S to FP32 accuracy.
//   2. Refinement by matrix multiplication (the approach of Ogita & Aishima's
//      iterative refinement of eigen/singular vectors, specialised to the
//      one-sided form), twice:
//        V <- V (3 I - V^T V) / 2                       (Newton-Schulz: V orthogonal)
//        B = R V,  G = B^T B,  d = diag G
//        X_ij = G_ij / (d_j - d_i) for well-separated pairs, 0 otherwise
//        V <- V (I + X)                                 (first-order rotation)
//      then a last Newton-Schulz step and B = R V.
//   3. S_i = ||B_i||, sorted; U = B S^-1.
//
// V is orthogonal to FP64 rounding, and R = B V^T holds to FP64 rounding, so
// truncating to the leading columns has error exactly ||B_dropped||_F.  The
// X step removes the leakage of large columns into small ones (which would
// otherwise inflate the tail estimate to ~1e-6 of the norm); pairs whose
// squared norms are within a factor 2 are left as they are: mixing them
// changes neither column norm by more than their cosine squared.  So U is
// orthonormal only to the cosine left between such near pairs; callers that
// need an exactly orthonormal left factor ask for it and the routine then
// runs on R^T and swaps the factors.
#include "common.cuh"

namespace tt {

namespace {

constexpr int J32_THREADS = 1024;
constexpr int J32_MAX_SWEEPS = 12;

// B (n x n, column-major, FP64 input) -> V (n x n column-major FP32 rotations)
__global__ void __launch_bounds__(J32_THREADS) jacobi32_kernel(const double *__restrict__ Bin, int n,
                                                               float *__restrict__ Vout) {
  extern __shared__ float sm[];
  float *B = sm;
  float *V = sm + (size_t)n * n;
  __shared__ int s_rot;
  __shared__ double s_max[32];
  const long long nn = (long long)n * n;
  // scale by a power of two that brings the largest entry near 1, so that
  // small matrices do not underflow in FP32 (rotations are scale-free)
  double mx = 0.0;
  for (long long e = threadIdx.x; e < nn; e += blockDim.x) mx = fmax(mx, fabs(Bin[e]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = threadIdx.x < (blockDim.x >> 5) ? s_max[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0) s_max[0] = mx;
  }
  __syncthreads();
  int ex = 0;
  if (s_max[0] > 0.0 && isfinite(s_max[0])) frexp(s_max[0], &ex);
  const double scl = ldexp(1.0, -ex);
  for (long long e = threadIdx.x; e < nn; e += blockDim.x) {
    B[e] = (float)(Bin[e] * scl);
    V[e] = ((e % n) == (e / n)) ? 1.f : 0.f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int np = (n + 1) & ~1;
  const float tol = fmaxf(2e-6f, 1.2e-7f * sqrtf((float)n));
  // a group of 8 lanes per column pair (4 pairs per warp): vectors of a few
  // dozen entries leave a full warp mostly idle, and a round's cost is its
  // instruction count
  const int sl = lane & 7;
  for (int sweep = 0; sweep < J32_MAX_SWEEPS; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      for (int t0 = warp * 4; t0 < np / 2; t0 += nwarp * 4) {
        const int t = t0 + (lane >> 3);
        int p = 0, q = 0;
        if (t == 0) {
          p = np - 1;
          q = round;
        } else {
          p = (round + t) % (np - 1);
          q = (round - t + (np - 1)) % (np - 1);
        }
        const bool valid = t < np / 2 && p < n && q < n;
        float *bp = B + (long long)p * n, *bq = B + (long long)q * n;
        float al = 0.f, be = 0.f, ga = 0.f;
        if (valid)
          for (int i = sl; i < n; i += 8) {
            const float x = bp[i], y = bq[i];
            al = fmaf(x, x, al);
            be = fmaf(y, y, be);
            ga = fmaf(x, y, ga);
          }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (!valid || ga == 0.f || al == 0.f || be == 0.f) continue;
        if (fabsf(ga) <= tol * sqrtf(al * be)) continue;
        const float zeta = (be - al) / (2.f * ga);
        const float tt = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
        const float cs = 1.f / sqrtf(1.f + tt * tt);
        const float sn = cs * tt;
        float *vp = V + (long long)p * n, *vq = V + (long long)q * n;
        for (int i = sl; i < n; i += 8) {
          const float x = bp[i], y = bq[i];
          bp[i] = cs * x - sn * y;
          bq[i] = sn * x + cs * y;
          const float u = vp[i], w = vq[i];
          vp[i] = cs * u - sn * w;
          vq[i] = sn * u + cs * w;
        }
        if (sl == 0) atomicAdd(&s_rot, 1);
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

// X (n x n column-major) from G = B^T B: the first-order rotation
// X_ij = G_ij / (d_j - d_i) that diagonalises G, for pairs whose diagonal
// entries differ by at least half the larger one and whose rotation is small
// (|X_ij| <= 1e-3: the first-order step is accurate and V (I + X) stays in
// the convergence region of the Newton-Schulz step); zero elsewhere.  A
// column that only carries leakage from a large one has a large cosine with
// it but a small X_ij, and is cleaned; columns at the noise floor with large
// mutual cosines are left as they are.  X is antisymmetric.
__global__ void xstep_kernel(const double *__restrict__ G, int n, double *__restrict__ X) {
  const long long nn = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    double x = 0.0;
    if (i != j) {
      const double di = G[(long long)i * n + i], dj = G[(long long)j * n + j];
      const double gap = dj - di;
      const double g = G[e];
      if (fabs(gap) >= 0.5 * fmax(di, dj) && gap != 0.0 && fabs(g) <= 1e-3 * fabs(gap)) x = g / gap;
    }
    X[e] = x;
  }
}

// Column norms of B (n x n column-major) -> S sorted decreasing; U[:, r] =
// B[:, j] / S_r and Vo[:, r] = V[:, j] for the column j of rank r (ties by index).
__global__ void __launch_bounds__(1024) colnorm_sort_kernel(const double *__restrict__ B,
                                                            const double *__restrict__ V, int n,
                                                            double *__restrict__ U, double *__restrict__ S,
                                                            double *__restrict__ Vo) {
  extern __shared__ double sh[];
  double *sv = sh;
  int *rank = reinterpret_cast<int *>(sh + n);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int j = warp; j < n; j += nwarp) {
    const double *bj = B + (long long)j * n;
    double acc = 0.0;
    for (int i = lane; i < n; i += 32) acc = fma(bj[i], bj[i], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) sv[j] = sqrt(acc);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double v = sv[j];
    int r = 0;
    for (int i = 0; i < n; ++i) {
      const double u = sv[i];
      r += (u > v) || (u == v && i < j);
    }
    rank[j] = r;
    S[r] = v;
  }
  __syncthreads();
  const long long nn = (long long)n * n;
  for (long long e = threadIdx.x; e < nn; e += blockDim.x) {
    const int j = (int)(e / n), i = (int)(e % n), r = rank[j];
    const double v = sv[j];
    U[(long long)r * n + i] = v > 0.0 ? B[e] / v : 0.0;
    Vo[(long long)r * n + i] = V[e];
  }
}

__global__ void transpose_sq_kernel(const double *__restrict__ A, int n, double *__restrict__ T) {
  const long long nn = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn;
       e += (long long)gridDim.x * blockDim.x)
    T[(e % n) * n + e / n] = A[e];
}

}  // namespace

bool jacobi_svd_mixed_fits(int n) { return 2LL * n * n * (long long)sizeof(float) <= 200 * 1024 && n <= 4096; }

// Same contract as jacobi_svd except for orthogonality: V (or U when
// exact_u) is orthonormal to FP64 rounding, the other factor to the cosine
// left between near pairs (see the top of this file); B = U S V^T to FP64
// rounding either way.  B is not modified.
void jacobi_svd_mixed(Ctx *c, double *B, int n, double *U, double *S, double *V, bool exact_u) {
  TT_REQUIRE(jacobi_svd_mixed_fits(n), "jacobi_svd_mixed: matrix too large");
  const size_t nn = (size_t)n * n;
  const unsigned ew = (unsigned)std::min<size_t>((nn + 255) / 256, 1024);
  DBuf rt, v32(c, (nn + 1) / 2), vd(c, nn), g(c, nn), w(c, nn), rb(c, nn);
  const double *R = B;
  if (exact_u) {
    // R^T = U' S V'^T with V' exact  ->  R = V' S U'^T: run on R^T, swap the factors
    rt.ensure(c, nn);
    transpose_sq_kernel<<<ew, 256, 0, c->stream>>>(B, n, rt.p());
    c->count();
    TT_CHECK_CUDA(cudaGetLastError());
    R = rt.p();
  }
  const size_t smem = 2 * nn * sizeof(float);
  {
    PhaseTimer pt0(c, "svd.j32");
    TT_CHECK_CUDA(cudaFuncSetAttribute(jacobi32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    jacobi32_kernel<<<1, J32_THREADS, smem, c->stream>>>(R, n, reinterpret_cast<float *>(v32.p()));
    c->count();
    TT_CHECK_CUDA(cudaGetLastError());
  }
  PhaseTimer pt1(c, "svd.refine");
  f2d_kernel<<<ew, 256, 0, c->stream>>>(reinterpret_cast<const float *>(v32.p()), vd.p(), nn);
  c->count();
  TT_CHECK_CUDA(cudaGetLastError());
  // Column-major products with the row-major GEMM: Z = X Y  <=>  Z^T = Y^T X^T.
  auto newton_schulz = [&]() {
    // g = V^T V ; w = V g ; V = 1.5 V - 0.5 w
    gemm(c, false, true, n, n, n, 1.0, vd.p(), n, 0, vd.p(), n, 0, 0.0, g.p(), n, 0);
    gemm(c, false, false, n, n, n, 1.0, g.p(), n, 0, vd.p(), n, 0, 0.0, w.p(), n, 0);
    axpby(c, nn, -0.5, w.p(), 1.5, vd.p());
  };
  for (int it = 0; it < 2; ++it) {
    newton_schulz();
    // rb = R V ; g = rb^T rb ; w = X(g) ; V += V w
    gemm(c, false, false, n, n, n, 1.0, vd.p(), n, 0, R, n, 0, 0.0, rb.p(), n, 0);
    gemm(c, false, true, n, n, n, 1.0, rb.p(), n, 0, rb.p(), n, 0, 0.0, g.p(), n, 0);
    xstep_kernel<<<ew, 256, 0, c->stream>>>(g.p(), n, w.p());
    c->count();
    TT_CHECK_CUDA(cudaGetLastError());
    gemm(c, false, false, n, n, n, 1.0, w.p(), n, 0, vd.p(), n, 0, 0.0, g.p(), n, 0);
    axpby(c, nn, 1.0, g.p(), 1.0, vd.p());
  }
  newton_schulz();
  gemm(c, false, false, n, n, n, 1.0, vd.p(), n, 0, R, n, 0, 0.0, rb.p(), n, 0);
  const size_t sh = (size_t)n * sizeof(double) + (size_t)n * sizeof(int);
  double *Uo = exact_u ? V : U, *Vo = exact_u ? U : V;
  colnorm_sort_kernel<<<1, 1024, sh, c->stream>>>(rb.p(), vd.p(), n, Uo, S, Vo);
  c->count();
  TT_CHECK_CUDA(cudaGetLastError());
}

}  // namespace tt
