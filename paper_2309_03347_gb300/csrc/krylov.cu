// Device-resident pieces of the restarted FP32 GMRES of the mixed-precision
// local solves: the Gram-Schmidt products spread over many CTAs, and the
// Hessenberg column, Givens rotation, residual estimate and normalisation of
// each Arnoldi step computed on the device, so that the host can queue the
// next step before it reads the residual of the current one.
//
// All reductions accumulate in FP64 in a fixed order (deterministic).
#include "common.cuh"

namespace tt {

namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum_d(double v, double *sh) {
  v = warp_sum_d(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[l] : 0.0;
  if (w == 0) v = warp_sum_d(v);
  __syncthreads();
  return v;
}

// part[j * S + s] = sum over split s of V_j . w      grid (S, nv)
__global__ void mdot_kernel(const float *__restrict__ V, size_t ldv, const float *__restrict__ w, size_t n,
                            size_t chunk, double *__restrict__ part) {
  __shared__ double sh[32];
  const int j = blockIdx.y, s = blockIdx.x, S = gridDim.x;
  const float *v = V + (size_t)j * ldv;
  const size_t lo = (size_t)s * chunk, hi = min(n, lo + chunk);
  double acc = 0.0;
  for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) acc = fma((double)v[i], (double)w[i], acc);
  acc = block_sum_d(acc, sh);
  if (threadIdx.x == 0) part[(size_t)j * S + s] = acc;
}

// h_j = sum_s part[j S + s];  w -= sum_j h_j V_j;  hout = h (block 0);
// npart[block] = sum of the new w^2 over the block's elements (when npart)
__global__ void maxpy_kernel(const float *__restrict__ V, size_t ldv, int nv, const double *__restrict__ part, int S,
                             float *__restrict__ w, size_t n, double *__restrict__ hout,
                             double *__restrict__ npart) {
  __shared__ double h[64];
  __shared__ double sh[32];
  for (int j = threadIdx.x; j < nv; j += blockDim.x) {
    double a = 0.0;
    for (int s = 0; s < S; ++s) a += part[(size_t)j * S + s];
    h[j] = a;
    if (blockIdx.x == 0 && hout) hout[j] = a;
  }
  __syncthreads();
  double sq = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int j = 0; j < nv; ++j) a = fma((double)V[(size_t)j * ldv + i], h[j], a);
    const float nw = (float)((double)w[i] - a);
    w[i] = nw;
    sq = fma((double)nw, (double)nw, sq);
  }
  if (npart) {
    sq = block_sum_d(sq, sh);
    if (threadIdx.x == 0) npart[blockIdx.x] = sq;
  }
}

__global__ void sumsq_kernel(const float *__restrict__ x, size_t n, double *__restrict__ npart) {
  __shared__ double sh[32];
  double sq = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    sq = fma((double)x[i], (double)x[i], sq);
  sq = block_sum_d(sq, sh);
  if (threadIdx.x == 0) npart[blockIdx.x] = sq;
}

// one warp: sum the partial squares in a fixed order
__device__ double warp_total(const double *__restrict__ npart, int nb) {
  double a = 0.0;
  for (int i = threadIdx.x; i < nb; i += 32) a += npart[i];
  return warp_sum_d(a);
}

// Arnoldi step j: column j of H from the two Gram-Schmidt passes and the
// norm; earlier rotations applied, the new one formed; g updated.
// st[2j] = |g[j+1]| (residual estimate), st[2j+1] = h_{j+1,j};
// inv = 1 / h_{j+1,j} (1 on breakdown: the vector is left as it is).
__global__ void arnoldi_kernel(int j, int mr, const double *__restrict__ h1, const double *__restrict__ h2,
                               const double *__restrict__ npart, int nb, double *__restrict__ H,
                               double *__restrict__ cs, double *__restrict__ sn, double *__restrict__ g,
                               double *__restrict__ st, double *__restrict__ inv) {
  const double hn2 = warp_total(npart, nb);
  if (threadIdx.x != 0) return;
  const double hn = sqrt(fmax(hn2, 0.0));
  for (int i = 0; i <= j; ++i) H[(size_t)i * mr + j] = h1[i] + h2[i];
  H[(size_t)(j + 1) * mr + j] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = H[(size_t)i * mr + j], b = H[(size_t)(i + 1) * mr + j];
    H[(size_t)i * mr + j] = cs[i] * a + sn[i] * b;
    H[(size_t)(i + 1) * mr + j] = -sn[i] * a + cs[i] * b;
  }
  const double a = H[(size_t)j * mr + j], b = H[(size_t)(j + 1) * mr + j];
  const double den = hypot(a, b);
  cs[j] = den == 0.0 ? 1.0 : a / den;
  sn[j] = den == 0.0 ? 0.0 : b / den;
  H[(size_t)j * mr + j] = den;
  H[(size_t)(j + 1) * mr + j] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  st[2 * j] = fabs(g[j + 1]);
  st[2 * j + 1] = hn;
  inv[0] = hn > 1e-30 ? 1.0 / hn : 1.0;
}

// beta = ||r|| ; g = (beta, 0, ...) ; st = beta ; inv = 1 / beta (0 if beta = 0)
__global__ void gmres_start_kernel(const double *__restrict__ npart, int nb, int mr, double *__restrict__ g,
                                   double *__restrict__ st, double *__restrict__ inv) {
  const double b2 = warp_total(npart, nb);
  const double beta = sqrt(fmax(b2, 0.0));
  for (int i = threadIdx.x; i <= mr; i += 32) g[i] = i == 0 ? beta : 0.0;
  if (threadIdx.x == 0) {
    st[0] = beta;
    inv[0] = beta > 0.0 ? 1.0 / beta : 0.0;
  }
}

// y = -(H[:kk, :kk])^-1 g[:kk]  (upper triangular back substitution)
__global__ void trisolve_kernel(int kk, int mr, const double *__restrict__ H, const double *__restrict__ g,
                                double *__restrict__ y) {
  if (threadIdx.x != 0) return;
  for (int i = kk - 1; i >= 0; --i) {
    double s = g[i];
    for (int l = i + 1; l < kk; ++l) s += H[(size_t)i * mr + l] * y[l];  // y holds -solution
    const double d = H[(size_t)i * mr + i];
    y[i] = d != 0.0 ? -s / d : 0.0;
  }
}

__global__ void scale_dev_kernel(const float *__restrict__ x, float *__restrict__ y, size_t n,
                                 const double *__restrict__ s) {
  const float f = (float)s[0];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = f * x[i];
}

unsigned kry_blocks(Ctx *c, size_t n) {
  return (unsigned)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, (size_t)c->sm_count * 4));
}

}  // namespace

int kry_mdot(Ctx *c, const float *V, size_t ldv, int nv, const float *w, size_t n, double *part) {
  TT_REQUIRE(nv >= 1 && nv <= KRY_MAX_VECS, "kry_mdot: too many vectors");
  int S = (int)std::min<size_t>((size_t)std::max(1, (2 * c->sm_count + nv - 1) / nv), (n + 1023) / 1024);
  S = std::max(1, std::min(S, KRY_MAX_SPLIT));
  const size_t chunk = (n + S - 1) / S;
  mdot_kernel<<<dim3(S, nv), 256, 0, c->stream>>>(V, ldv, w, n, chunk, part);
  c->count();
  TT_CHECK_CUDA(cudaGetLastError());
  return S;
}

int kry_maxpy(Ctx *c, const float *V, size_t ldv, int nv, const double *part, int S, float *w, size_t n,
              double *hout, double *npart) {
  TT_REQUIRE(nv >= 1 && nv <= KRY_MAX_VECS, "kry_maxpy: too many vectors");
  const unsigned nb = kry_blocks(c, n);
  maxpy_kernel<<<nb, 256, 0, c->stream>>>(V, ldv, nv, part, S, w, n, hout, npart);
  c->count();
  TT_CHECK_CUDA(cudaGetLastError());
  return (int)nb;
}

int kry_sumsq(Ctx *c, const float *x, size_t n, double *npart) {
  const unsigned nb = kry_blocks(c, n);
  sumsq_kernel<<<nb, 256, 0, c->stream>>>(x, n, npart);
  c->count();
  TT_CHECK_CUDA(cudaGetLastError());
  return (int)nb;
}

void kry_arnoldi(Ctx *c, int j, int mr, const double *h1, const double *h2, const double *npart, int nb, double *H,
                 double *cs, double *sn, double *g, double *st, double *inv) {
  arnoldi_kernel<<<1, 32, 0, c->stream>>>(j, mr, h1, h2, npart, nb, H, cs, sn, g, st, inv);
  c->count();
  TT_CHECK_CUDA(cudaGetLastError());
}

void kry_start(Ctx *c, const double *npart, int nb, int mr, double *g, double *st, double *inv) {
  gmres_start_kernel<<<1, 32, 0, c->stream>>>(npart, nb, mr, g, st, inv);
  c->count();
  TT_CHECK_CUDA(cudaGetLastError());
}

void kry_trisolve(Ctx *c, int kk, int mr, const double *H, const double *g, double *y) {
  trisolve_kernel<<<1, 32, 0, c->stream>>>(kk, mr, H, g, y);
  c->count();
  TT_CHECK_CUDA(cudaGetLastError());
}

void kry_scale(Ctx *c, const float *x, float *y, size_t n, const double *s) {
  if (!n) return;
  scale_dev_kernel<<<kry_blocks(c, n), 256, 0, c->stream>>>(x, y, n, s);
  c->count();
  TT_CHECK_CUDA(cudaGetLastError());
}

}  // namespace tt
