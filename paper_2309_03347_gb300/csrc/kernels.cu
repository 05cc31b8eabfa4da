// FP64 building blocks of the tensor-train path: tiled strided-batched GEMM
// with split-K, tensor permutation, reductions, Householder QR and one-sided
// Jacobi SVD.  Every kernel bounds-checks its indices against the sizes it is
// given; none waits on another block.
#include <chrono>

#include "common.cuh"

namespace tt {

// ----------------------------------------------------------------- DBuf
void DBuf::alloc(Ctx *c, size_t n) {
  release();
  ctx_ = c;
  if (n == 0) n = 1;
  void *p = nullptr;
  if (c->alloc_fn) {
    p = c->alloc_fn(n * sizeof(double), (void *)c->stream, c->alloc_user);
    if (!p) throw Error(TT_ENOMEM, "caller allocator returned NULL for " + std::to_string(n * 8) + " bytes");
  } else {
    cudaError_t e = cudaMallocAsync(&p, n * sizeof(double), c->stream);
    if (e != cudaSuccess)
      throw Error(e == cudaErrorMemoryAllocation ? TT_ENOMEM : TT_ECUDA,
                  std::string("cudaMallocAsync(") + std::to_string(n * 8) + "): " + cudaGetErrorString(e));
  }
  p_ = static_cast<double *>(p);
  n_ = cap_ = n;
}

void DBuf::release() {
  if (p_ && ctx_) {
    if (ctx_->free_fn)
      ctx_->free_fn(p_, (void *)ctx_->stream, ctx_->alloc_user);
    else
      cudaFreeAsync(p_, ctx_->stream);
  }
  p_ = nullptr;
  n_ = cap_ = 0;
}

static double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

PhaseTimer::PhaseTimer(Ctx *cc, const char *n) : c(cc), name(n) {
  if (c->phase_timing) {
    cudaStreamSynchronize(c->stream);
    t0 = now_ms();
  }
}

PhaseTimer::~PhaseTimer() {
  if (c->phase_timing) {
    cudaStreamSynchronize(c->stream);
    c->phase_add(name, now_ms() - t0);
  }
}

void Ctx::prof_begin(cudaEvent_t *b, cudaEvent_t *e, int tag) {
  if (ev_used == ev_pool.size()) {
    if (ev_pool.size() >= 8192) prof_fold();
    if (ev_used == ev_pool.size()) {
      cudaEvent_t x, y;
      TT_CHECK_CUDA(cudaEventCreate(&x));
      TT_CHECK_CUDA(cudaEventCreate(&y));
      ev_pool.push_back({x, y});
      ev_tag.push_back(0);
    }
  }
  *b = ev_pool[ev_used].first;
  *e = ev_pool[ev_used].second;
  ev_tag[ev_used] = tag;
  ++ev_used;
}

void Ctx::prof_fold() {
  if (!ev_used) return;
  TT_CHECK_CUDA(cudaStreamSynchronize(stream));
  for (size_t i = 0; i < ev_used; ++i) {
    float ms = 0.f;
    TT_CHECK_CUDA(cudaEventElapsedTime(&ms, ev_pool[i].first, ev_pool[i].second));
    (ev_tag[i] == 3 ? pg_ms_done : ev_tag[i] == 2 ? gemmtc_ms_done : ev_tag[i] == 1 ? gemm32_ms_done : gemm_ms_done) +=
        ms;
  }
  ev_used = 0;
}

#define LAUNCH_CHECK(c)                                   \
  do {                                                    \
    (c)->count();                                         \
    TT_CHECK_CUDA(cudaGetLastError());                    \
  } while (0)

// ----------------------------------------------------------------- GEMM
// 64 x 64 output tile, K step 16, 256 threads; each thread owns a 4 x 4
// sub-tile with stride 16 (conflict-free shared-memory reads).
constexpr int GBM = 64, GBN = 64, GBK = 16;

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) dgemm_kernel(int M, int N, int K, double alpha,
                                                    const double *__restrict__ A, int lda, long long sA,
                                                    const double *__restrict__ B, int ldb, long long sB,
                                                    double beta, double *__restrict__ C, int ldc,
                                                    long long sC, int splitk, int kchunk,
                                                    double *__restrict__ ws) {
  __shared__ double As[GBK][GBM + 1];
  __shared__ double Bs[GBK][GBN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int bz = blockIdx.z;
  const int batch = bz / splitk, split = bz % splitk;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int kbeg = split * kchunk;
  const int kend = min(K, kbeg + kchunk);
  A += batch * sA;
  B += batch * sB;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int k0 = kbeg; k0 < kend; k0 += GBK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      int mm, kk;
      if (TA) {
        mm = e & 63;
        kk = e >> 6;
      } else {
        kk = e & 15;
        mm = e >> 4;
      }
      const int gm = m0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < M && gk < kend) v = TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
      As[kk][mm] = v;
      int nn, kb;
      if (TB) {
        kb = e & 15;
        nn = e >> 4;
      } else {
        nn = e & 63;
        kb = e >> 6;
      }
      const int gn = n0 + nn, gkb = k0 + kb;
      double w = 0.0;
      if (gn < N && gkb < kend) w = TB ? B[(long long)gn * ldb + gkb] : B[(long long)gkb * ldb + gn];
      Bs[kb][nn] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (splitk == 1) {
    double *Cb = C + batch * sC;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gm = m0 + ty + 16 * i;
      if (gm >= M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gn = n0 + tx + 16 * j;
        if (gn >= N) continue;
        double *cp = Cb + (long long)gm * ldc + gn;
        *cp = beta == 0.0 ? alpha * acc[i][j] : alpha * acc[i][j] + beta * *cp;
      }
    }
  } else {
    double *W = ws + (long long)bz * M * N;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gm = m0 + ty + 16 * i;
      if (gm >= M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gn = n0 + tx + 16 * j;
        if (gn < N) W[(long long)gm * N + gn] = acc[i][j];
      }
    }
  }
}

// Small-tile FP64 GEMM for products too small to fill the GPU with 64 x 64
// tiles.  FP64 issues at about 2 FMA per clock per SM on this part, so a
// GEMM's time is its FMA count divided by the SMs it reaches: 16 x 16 output
// tiles (one output per thread) and a K split give every SM work.  K step
// 16 with the next step's operands loaded into registers during the current
// step's products.
constexpr int SBM = 16, SBN = 16, SBK = 16;

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) dgemm16_kernel(int M, int N, int K, double alpha,
                                                      const double *__restrict__ A, int lda, long long sA,
                                                      const double *__restrict__ B, int ldb, long long sB,
                                                      double beta, double *__restrict__ C, int ldc, long long sC,
                                                      int splitk, int kchunk, double *__restrict__ ws) {
  __shared__ double As[SBK][SBM + 1];
  __shared__ double Bs[SBK][SBN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int bz = blockIdx.z, bb = bz / splitk, split = bz % splitk;
  const int m0 = blockIdx.y * SBM, n0 = blockIdx.x * SBN;
  const int kbeg = split * kchunk, kend = min(K, kbeg + kchunk);
  A += bb * sA;
  B += bb * sB;
  // element loaded by this thread: A (row am, k ak), B (k bk, column bn)
  const int am = TA ? (tid & 15) : (tid >> 4), ak = TA ? (tid >> 4) : (tid & 15);
  const int bn = TB ? (tid >> 4) : (tid & 15), bk = TB ? (tid & 15) : (tid >> 4);
  auto ldA = [&](int k0) {
    const int gm = m0 + am, gk = k0 + ak;
    return (gm < M && gk < kend) ? (TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk]) : 0.0;
  };
  auto ldB = [&](int k0) {
    const int gn = n0 + bn, gk = k0 + bk;
    return (gn < N && gk < kend) ? (TB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn]) : 0.0;
  };
  double acc = 0.0;
  double ra = kbeg < kend ? ldA(kbeg) : 0.0, rb = kbeg < kend ? ldB(kbeg) : 0.0;
  for (int k0 = kbeg; k0 < kend; k0 += SBK) {
    As[ak][am] = ra;
    Bs[bk][bn] = rb;
    __syncthreads();
    if (k0 + SBK < kend) {
      ra = ldA(k0 + SBK);
      rb = ldB(k0 + SBK);
    }
#pragma unroll
    for (int kk = 0; kk < SBK; ++kk) acc = fma(As[kk][ty], Bs[kk][tx], acc);
    __syncthreads();
  }
  const int gm = m0 + ty, gn = n0 + tx;
  if (gm < M && gn < N) {
    if (splitk == 1) {
      double *cp = C + bb * sC + (long long)gm * ldc + gn;
      *cp = beta == 0.0 ? alpha * acc : alpha * acc + beta * *cp;
    } else {
      ws[(long long)bz * M * N + (long long)gm * N + gn] = acc;
    }
  }
}

__global__ void splitk_reduce(int M, int N, int splitk, int batch, const double *__restrict__ ws,
                              double alpha, double beta, double *__restrict__ C, int ldc, long long sC) {
  const long long tot = (long long)batch * M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e / ((long long)M * N));
    const long long r = e % ((long long)M * N);
    const int m = (int)(r / N), n = (int)(r % N);
    double s = 0.0;
    for (int q = 0; q < splitk; ++q) s += ws[((long long)b * splitk + q) * M * N + r];
    double *cp = C + b * sC + (long long)m * ldc + n;
    *cp = beta == 0.0 ? alpha * s : alpha * s + beta * *cp;
  }
}

void gemm(Ctx *c, bool ta, bool tb, int M, int N, int K, double alpha, const double *A, int lda,
          long long sA, const double *B, int ldb, long long sB, double beta, double *C, int ldc,
          long long sC, int batch) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (K <= 0) {
    // C = beta C
    for (int b = 0; b < batch; ++b) {
      if (beta == 0.0) {
        for (int m = 0; m < M; ++m) fill(c, C + b * sC + (long long)m * ldc, N, 0.0);
      } else if (beta != 1.0) {
        for (int m = 0; m < M; ++m) scale(c, C + b * sC + (long long)m * ldc, N, beta);
      }
    }
    return;
  }
  const long long tiles = (long long)((M + GBM - 1) / GBM) * ((N + GBN - 1) / GBN) * batch;
  const long long target = 2LL * c->sm_count;
  // too few 64 x 64 tiles to reach every SM: 16 x 16 tiles with a K split
  const bool small = tiles < c->sm_count;
  const int TM = small ? SBM : GBM, TN = small ? SBN : GBN, TK = small ? SBK : GBK;
  const long long tl = (long long)((M + TM - 1) / TM) * ((N + TN - 1) / TN) * batch;
  int splitk = 1;
  if (small) {
    if (tl < target && K > TK) splitk = (int)std::min<long long>((target + tl - 1) / tl, (K + TK - 1) / TK);
  } else if (tl < target && K > 4 * TK) {
    splitk = (int)std::min<long long>((target + tl - 1) / tl, (K + 63) / 64);
  }
  splitk = std::max(1, std::min(splitk, 64));
  int kchunk = (K + splitk - 1) / splitk;
  kchunk = (kchunk + TK - 1) / TK * TK;
  splitk = (K + kchunk - 1) / kchunk;
  TT_REQUIRE((long long)batch * splitk <= 65535, "gemm: batch too large");
  TT_REQUIRE((M + TM - 1) / TM <= 65535, "gemm: M too large");
  double *ws = nullptr;
  if (splitk > 1) {
    c->ws_gemm.ensure(c, (size_t)batch * splitk * M * N);
    ws = c->ws_gemm.p();
  }
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, batch * splitk);
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (c->profiling) {
    c->prof_begin(&ev0, &ev1);
    TT_CHECK_CUDA(cudaEventRecord(ev0, c->stream));
  }
#define GEMM_LAUNCH(TA_, TB_)                                                                                   \
  do {                                                                                                          \
    if (small)                                                                                                  \
      dgemm16_kernel<TA_, TB_><<<grid, 256, 0, c->stream>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, \
                                                            sC, splitk, kchunk, ws);                            \
    else                                                                                                        \
      dgemm_kernel<TA_, TB_><<<grid, 256, 0, c->stream>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc,   \
                                                          sC, splitk, kchunk, ws);                              \
  } while (0)
  if (ta && tb) GEMM_LAUNCH(true, true);
  else if (ta) GEMM_LAUNCH(true, false);
  else if (tb) GEMM_LAUNCH(false, true);
  else GEMM_LAUNCH(false, false);
#undef GEMM_LAUNCH
  LAUNCH_CHECK(c);
  if (splitk > 1) {
    const long long tot = (long long)batch * M * N;
    const unsigned blocks = (unsigned)std::min<long long>((tot + 255) / 256, 4LL * c->sm_count * 8);
    splitk_reduce<<<blocks, 256, 0, c->stream>>>(M, N, splitk, batch, ws, alpha, beta, C, ldc, sC);
    LAUNCH_CHECK(c);
  }
  if (c->profiling) {
    TT_CHECK_CUDA(cudaEventRecord(ev1, c->stream));
    c->gemm_flops += 2.0 * M * (double)N * K * batch;
    c->gemm_launches += 1;
  }
}

// ----------------------------------------------------------------- permute
constexpr int PERM_MAX_DIMS = 24;
struct PermArgs {
  int ndim;
  long long out_stride_in[PERM_MAX_DIMS];  // stride in the input of each output dimension
  long long out_shape[PERM_MAX_DIMS];
};

__global__ void permute_kernel(const double *__restrict__ in, double *__restrict__ out, long long total,
                               PermArgs a) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long rem = e, src = 0;
    for (int d = a.ndim - 1; d >= 0; --d) {
      const long long i = rem % a.out_shape[d];
      rem /= a.out_shape[d];
      src += i * a.out_stride_in[d];
    }
    out[e] = in[src];
  }
}

void permute(Ctx *c, const double *in, double *out, int ndim, const int *shape, const int *perm) {
  TT_REQUIRE(ndim >= 1 && ndim <= PERM_MAX_DIMS, "permute: ndim");
  long long stride[PERM_MAX_DIMS];
  long long total = 1;
  for (int d = ndim - 1; d >= 0; --d) {
    stride[d] = total;
    total *= shape[d];
  }
  if (total == 0) return;
  PermArgs a;
  a.ndim = ndim;
  for (int d = 0; d < ndim; ++d) {
    TT_REQUIRE(perm[d] >= 0 && perm[d] < ndim, "permute: perm");
    a.out_shape[d] = shape[perm[d]];
    a.out_stride_in[d] = stride[perm[d]];
  }
  const unsigned blocks = (unsigned)std::min<long long>((total + 255) / 256, 16LL * c->sm_count * 8);
  permute_kernel<<<blocks, 256, 0, c->stream>>>(in, out, total, a);
  LAUNCH_CHECK(c);
}

__global__ void transpose_kernel(const double *__restrict__ in, double *__restrict__ out, int rows,
                                 int cols) {
  __shared__ double t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int r = r0 + k, cc = c0 + threadIdx.x;
    if (r < rows && cc < cols) t[k][threadIdx.x] = in[(long long)r * cols + cc];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += 8) {
    const int cc = c0 + k, r = r0 + threadIdx.x;
    if (r < rows && cc < cols) out[(long long)cc * rows + r] = t[threadIdx.x][k];
  }
}

void transpose(Ctx *c, const double *in, double *out, int rows, int cols) {
  if (rows <= 0 || cols <= 0) return;
  TT_REQUIRE((rows + 31) / 32 <= 65535, "transpose: too many rows");
  dim3 grid((cols + 31) / 32, (rows + 31) / 32);
  transpose_kernel<<<grid, dim3(32, 8), 0, c->stream>>>(in, out, rows, cols);
  LAUNCH_CHECK(c);
}

// ----------------------------------------------------------------- elementwise
__global__ void fill_kernel(double *p, size_t n, double v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    p[i] = v;
}
__global__ void scale_kernel(double *p, size_t n, double a) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    p[i] *= a;
}
__global__ void axpby_kernel(size_t n, double a, const double *x, double b, double *y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = b == 0.0 ? a * x[i] : a * x[i] + b * y[i];
}
__global__ void copy2d_kernel(double *dst, int ldd, const double *src, int lds, int rows, int cols,
                              double alpha) {
  const long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / cols), cc = (int)(e % cols);
    dst[(long long)r * ldd + cc] = alpha * src[(long long)r * lds + cc];
  }
}
__global__ void scale_rows_kernel(double *a, int rows, int cols, const double *s) {
  const long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x)
    a[e] *= s[e / cols];
}

static unsigned ew_blocks(Ctx *c, size_t n) {
  return (unsigned)std::min<size_t>((n + 255) / 256, (size_t)c->sm_count * 16);
}

void fill(Ctx *c, double *p, size_t n, double v) {
  if (!n) return;
  fill_kernel<<<ew_blocks(c, n), 256, 0, c->stream>>>(p, n, v);
  LAUNCH_CHECK(c);
}
void copy(Ctx *c, double *dst, const double *src, size_t n) {
  if (!n || dst == src) return;
  TT_CHECK_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
}
void scale(Ctx *c, double *p, size_t n, double a) {
  if (!n || a == 1.0) return;
  scale_kernel<<<ew_blocks(c, n), 256, 0, c->stream>>>(p, n, a);
  LAUNCH_CHECK(c);
}
void axpby(Ctx *c, size_t n, double a, const double *x, double b, double *y) {
  if (!n) return;
  axpby_kernel<<<ew_blocks(c, n), 256, 0, c->stream>>>(n, a, x, b, y);
  LAUNCH_CHECK(c);
}
void copy2d(Ctx *c, double *dst, int ldd, const double *src, int lds, int rows, int cols, double alpha) {
  if (rows <= 0 || cols <= 0) return;
  copy2d_kernel<<<ew_blocks(c, (size_t)rows * cols), 256, 0, c->stream>>>(dst, ldd, src, lds, rows, cols,
                                                                            alpha);
  LAUNCH_CHECK(c);
}
void scale_rows(Ctx *c, double *a, int rows, int cols, const double *s) {
  if (rows <= 0 || cols <= 0) return;
  scale_rows_kernel<<<ew_blocks(c, (size_t)rows * cols), 256, 0, c->stream>>>(a, rows, cols, s);
  LAUNCH_CHECK(c);
}

// ----------------------------------------------------------------- reductions
// Two-pass deterministic dot product: fixed grid, per-block partials, then one
// block sums the partials in a fixed order.
constexpr int RED_BLOCKS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v, double *sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) v = warp_sum(v);
  return v;  // valid in thread 0
}

__global__ void dot_partial(const double *__restrict__ x, const double *__restrict__ y, size_t n,
                            double *__restrict__ part) {
  __shared__ double sh[32];
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s = fma(x[i], y[i], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void sum_partials(const double *__restrict__ part, int np, double *__restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[0] = s;
}

void dot_dev(Ctx *c, const double *x, const double *y, size_t n, double *out) {
  c->scratch[7].ensure(c, RED_BLOCKS);
  if (n == 0) {
    fill(c, out, 1, 0.0);
    return;
  }
  const int nb = (int)std::min<size_t>(RED_BLOCKS, (n + 255) / 256);
  dot_partial<<<nb, 256, 0, c->stream>>>(x, y, n, c->scratch[7].p());
  LAUNCH_CHECK(c);
  sum_partials<<<1, 256, 0, c->stream>>>(c->scratch[7].p(), nb, out);
  LAUNCH_CHECK(c);
}

double dot(Ctx *c, const double *x, const double *y, size_t n) {
  dot_dev(c, x, y, n, c->d_scalar);
  TT_CHECK_CUDA(cudaMemcpyAsync(c->h_pinned, c->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  c->sync();
  return c->h_pinned[0];
}

double nrm2(Ctx *c, const double *x, size_t n) {
  // scaled to avoid overflow: ||x|| = s * ||x / s|| with s = max|x| is not
  // needed for the magnitudes met here; plain sum of squares in FP64.
  const double s = dot(c, x, x, n);
  return std::sqrt(std::max(s, 0.0));
}

// h[j] = <V_j, w>, one block per j
__global__ void multi_dot_kernel(const double *__restrict__ V, size_t ldv, const double *__restrict__ w,
                                 size_t n, double *__restrict__ h) {
  __shared__ double sh[32];
  const double *v = V + blockIdx.x * ldv;
  double s = 0.0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(v[i], w[i], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) h[blockIdx.x] = s;
}

__global__ void multi_axpy_kernel(const double *__restrict__ V, size_t ldv, int nv, const double *__restrict__ h,
                                  double *__restrict__ w, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < nv; ++j) s = fma(V[j * ldv + i], h[j], s);
    w[i] -= s;
  }
}

void multi_dot(Ctx *c, const double *V, size_t ldv, int nv, const double *w, size_t n, double *h) {
  if (nv <= 0) return;
  multi_dot_kernel<<<nv, 256, 0, c->stream>>>(V, ldv, w, n, h);
  LAUNCH_CHECK(c);
}
void multi_axpy(Ctx *c, const double *V, size_t ldv, int nv, const double *h, double *w, size_t n) {
  if (nv <= 0 || n == 0) return;
  multi_axpy_kernel<<<ew_blocks(c, n), 256, 0, c->stream>>>(V, ldv, nv, h, w, n);
  LAUNCH_CHECK(c);
}

__global__ void nonfinite_kernel(const double *x, size_t n, double *flag) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) flag[0] = 1.0;
}

bool has_nonfinite(Ctx *c, const double *x, size_t n) {
  fill(c, c->d_scalar + 1, 1, 0.0);
  if (n) {
    nonfinite_kernel<<<ew_blocks(c, n), 256, 0, c->stream>>>(x, n, c->d_scalar + 1);
    LAUNCH_CHECK(c);
  }
  TT_CHECK_CUDA(cudaMemcpyAsync(c->h_pinned, c->d_scalar + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  c->sync();
  return c->h_pinned[0] != 0.0;
}

// ----------------------------------------------------------------- Householder QR
// One block per matrix.  Column-major A (m x n).  Reflector j: v = [1; A[j+1:, j]],
// tau[j]; R[j][j] = beta.  Q is formed by backward accumulation.
constexpr int QR_THREADS = 512;

__global__ void __launch_bounds__(QR_THREADS) householder_qr_kernel(double *__restrict__ A, int m, int n,
                                                                    double *__restrict__ tau,
                                                                    double *__restrict__ Q,
                                                                    double *__restrict__ R, int form_q) {
  __shared__ double sh[32];
  __shared__ double s_beta, s_tau, s_scale;
  const int k = min(m, n);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int j = 0; j < k; ++j) {
    double *col = A + (long long)j * m;
    // ||x[1:]||^2
    double s = 0.0;
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) s = fma(col[i], col[i], s);
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
      const double alpha = col[j];
      if (s == 0.0) {
        s_tau = 0.0;
        s_beta = alpha;
        s_scale = 0.0;
      } else {
        const double nr = sqrt(alpha * alpha + s);
        const double beta = alpha >= 0.0 ? -nr : nr;
        s_tau = (beta - alpha) / beta;
        s_scale = 1.0 / (alpha - beta);
        s_beta = beta;
      }
    }
    __syncthreads();
    const double tj = s_tau, sc = s_scale;
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) col[i] *= sc;
    if (threadIdx.x == 0) {
      col[j] = s_beta;
      tau[j] = tj;
    }
    __syncthreads();
    if (tj != 0.0) {
      // apply H_j to columns j+1..n-1: one warp per column
      for (int cidx = j + 1 + warp; cidx < n; cidx += nwarp) {
        double *cc = A + (long long)cidx * m;
        double w = 0.0;
        for (int i = j + 1 + lane; i < m; i += 32) w = fma(col[i], cc[i], w);
        w = warp_sum(w);
        w += cc[j];
        w *= tj;
        if (lane == 0) cc[j] -= w;
        for (int i = j + 1 + lane; i < m; i += 32) cc[i] -= w * col[i];
      }
    }
    __syncthreads();
  }
  // R (k x n, column-major)
  for (long long e = threadIdx.x; e < (long long)k * n; e += blockDim.x) {
    const int r = (int)(e % k), cc = (int)(e / k);
    R[e] = (r <= cc) ? A[(long long)cc * m + r] : 0.0;
  }
  if (!form_q) return;
  // Q (m x k) = H_0 ... H_{k-1} I
  for (long long e = threadIdx.x; e < (long long)m * k; e += blockDim.x) {
    const int r = (int)(e % m), cc = (int)(e / m);
    Q[e] = (r == cc) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const double tj = tau[j];
    if (tj == 0.0) continue;
    const double *col = A + (long long)j * m;
    for (int cidx = j + warp; cidx < k; cidx += nwarp) {
      double *qc = Q + (long long)cidx * m;
      double w = 0.0;
      for (int i = j + 1 + lane; i < m; i += 32) w = fma(col[i], qc[i], w);
      w = warp_sum(w);
      w += qc[j];
      w *= tj;
      if (lane == 0) qc[j] -= w;
      for (int i = j + 1 + lane; i < m; i += 32) qc[i] -= w * col[i];
    }
    __syncthreads();
  }
}

// V (m x k, column-major): the Householder vectors left below the diagonal of
// A with the implicit unit diagonal; a reflector with tau = 0 (H = I) gets v = 0.
__global__ void wy_v_kernel(const double *__restrict__ A, const double *__restrict__ tau, int m, int k,
                            double *__restrict__ V) {
  const long long tot = (long long)m * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    V[e] = tau[j] == 0.0 ? 0.0 : (i < j ? 0.0 : (i == j ? 1.0 : A[e]));
  }
}

// X = S^-1 V1^T with S = strictly-upper(W) + diag(1/tau) (W = V^T V, row-major
// k x k) and V1 the top k x k block of V: one thread per column of X, back
// substitution (X row-major k x k).  H_0 ... H_{k-1} = I - V S^-1 V^T (the UT
// form of a product of Householder reflectors).
__global__ void ut_solve_kernel(const double *__restrict__ W, const double *__restrict__ tau,
                                const double *__restrict__ V, int m, int k, double *__restrict__ X) {
  const int cc = blockIdx.x * blockDim.x + threadIdx.x;
  if (cc >= k) return;
  for (int i = k - 1; i >= 0; --i) {
    double acc = V[cc + (long long)i * m];  // V1^T[i][cc] = V1[cc][i]
    for (int l = i + 1; l < k; ++l) acc -= W[(long long)i * k + l] * X[(long long)l * k + cc];
    const double t = tau[i];
    X[(long long)i * k + cc] = t == 0.0 ? 0.0 : acc * t;
  }
}

__global__ void eye_kernel(double *__restrict__ Q, int m, int k) {
  const long long tot = (long long)m * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x)
    Q[e] = (e % m) == (e / m) ? 1.0 : 0.0;
}

void qr_colmajor(Ctx *c, double *A, int m, int n, double *Q, double *R) {
  TT_REQUIRE(m > 0 && n > 0, "qr: empty matrix");
  const int k = std::min(m, n);
  c->scratch[6].ensure(c, (size_t)k);
  double *tau = c->scratch[6].p();
  // Q from the UT form with multi-SM FP64 products for 8 <= k <= 128; the
  // one-CTA backward accumulation otherwise
  const bool ut = k >= 8 && k <= 128;
  householder_qr_kernel<<<1, QR_THREADS, 0, c->stream>>>(A, m, n, tau, Q, R, ut ? 0 : 1);
  LAUNCH_CHECK(c);
  if (!ut) return;
  const size_t mk = (size_t)m * k, kk = (size_t)k * k;
  DBuf V(c, mk), W(c, kk), X(c, kk);
  wy_v_kernel<<<ew_blocks(c, mk), 256, 0, c->stream>>>(A, tau, m, k, V.p());
  LAUNCH_CHECK(c);
  // W = V^T V (V column-major m x k is row-major V^T, ld m)
  gemm(c, false, true, k, k, m, 1.0, V.p(), m, 0, V.p(), m, 0, 0.0, W.p(), k, 0);
  ut_solve_kernel<<<(k + 63) / 64, 64, 0, c->stream>>>(W.p(), tau, V.p(), m, k, X.p());
  LAUNCH_CHECK(c);
  // Q = I - V X: Q column-major is row-major Q^T (k x m, ld m); Q^T -= X^T V^T
  eye_kernel<<<ew_blocks(c, mk), 256, 0, c->stream>>>(Q, m, k);
  LAUNCH_CHECK(c);
  gemm(c, true, false, k, m, k, -1.0, X.p(), k, 0, V.p(), m, 0, 1.0, Q, m, 0);
}

// ----------------------------------------------------------------- Jacobi SVD
// One-sided (Hestenes) Jacobi on the columns of a square n x n matrix with
// the round-robin pair ordering; rotation from the classical formulas
// zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)).
// The matrix is staged in shared memory when it fits, V stays in global memory.
constexpr int JAC_THREADS = 1024;
constexpr int JAC_SMEM_DOUBLES = 24 * 1024;  // 192 KB
constexpr int JAC_MAX_SWEEPS = 40;

// One-sided (Hestenes) Jacobi SVD of an n x n column-major matrix on one CTA:
// one warp per column pair of a round-robin round, B (and V when both fit)
// in shared memory.  A pair is rotated while its columns' cosine exceeds
// n * 2^-52, the level below which FP64 rounding of the dot products makes
// the cosine noise (a tighter threshold never stops rotating).
__global__ void __launch_bounds__(JAC_THREADS) jacobi_svd_kernel(double *__restrict__ Bg, int n,
                                                                 double *__restrict__ U,
                                                                 double *__restrict__ S,
                                                                 double *__restrict__ V,
                                                                 double *__restrict__ Vscr,
                                                                 int smem_mode) {
  extern __shared__ double smem[];
  __shared__ int s_rot;
  const long long nn = (long long)n * n;
  // smem_mode: 0 both in global memory, 1 B in shared memory, 2 B and V in shared memory
  double *B = smem_mode >= 1 ? smem : Bg;
  double *Vtmp = smem_mode == 2 ? smem + nn : Vscr;
  if (smem_mode >= 1)
    for (long long e = threadIdx.x; e < nn; e += blockDim.x) B[e] = Bg[e];
  for (long long e = threadIdx.x; e < nn; e += blockDim.x) Vtmp[e] = ((e % n) == (e / n)) ? 1.0 : 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int np = (n + 1) & ~1;  // players (padded to even)
  const double tol = fmax(1e-15, 2.220446049250313e-16 * n);
  for (int sweep = 0; sweep < JAC_MAX_SWEEPS; ++sweep) {
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
        if (p > q) {
          const int tmp = p;
          p = q;
          q = tmp;
        }
        double *bp = B + (long long)p * n, *bq = B + (long long)q * n;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = lane; i < n; i += 32) {
          const double x = bp[i], y = bq[i];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga == 0.0 || al == 0.0 || be == 0.0) continue;
        if (fabs(ga) <= tol * sqrt(al * be)) continue;
        const double zeta = (be - al) / (2.0 * ga);
        const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + tt * tt);
        const double sn = cs * tt;
        for (int i = lane; i < n; i += 32) {
          const double x = bp[i], y = bq[i];
          bp[i] = cs * x - sn * y;
          bq[i] = sn * x + cs * y;
        }
        double *vp = Vtmp + (long long)p * n, *vq = Vtmp + (long long)q * n;
        for (int i = lane; i < n; i += 32) {
          const double x = vp[i], y = vq[i];
          vp[i] = cs * x - sn * y;
          vq[i] = sn * x + cs * y;
        }
        if (lane == 0) atomicAdd(&s_rot, 1);
      }
      __syncthreads();
    }
    if (s_rot == 0) break;
    __syncthreads();
  }
  // singular values = column norms; sort descending (rank by counting, ties by index)
  double *sv = Vscr + nn;  // n scratch doubles after the V scratch
  for (int j = warp; j < n; j += nwarp) {
    const double *bj = B + (long long)j * n;
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s = fma(bj[i], bj[i], s);
    s = warp_sum(s);
    if (lane == 0) sv[j] = sqrt(s);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double v = sv[j];
    int r = 0;
    for (int i = 0; i < n; ++i) {
      const double u = sv[i];
      r += (u > v) || (u == v && i < j);
    }
    S[r] = v;
    // column r of the outputs takes column j
    const double inv = v > 0.0 ? 1.0 / v : 0.0;
    for (int i = 0; i < n; ++i) {
      U[(long long)r * n + i] = B[(long long)j * n + i] * inv;
      V[(long long)r * n + i] = Vtmp[(long long)j * n + i];
    }
  }
}

void jacobi_svd(Ctx *c, double *B, int n, double *U, double *S, double *V) {
  TT_REQUIRE(n > 0, "jacobi_svd: empty");
  c->scratch[5].ensure(c, (size_t)n * n + n);
  const long long nn = (long long)n * n;
  const int mode = 2 * nn <= JAC_SMEM_DOUBLES ? 2 : nn <= JAC_SMEM_DOUBLES ? 1 : 0;
  const size_t bytes = (size_t)mode * nn * sizeof(double);
  if (mode)
    TT_CHECK_CUDA(cudaFuncSetAttribute(jacobi_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(JAC_SMEM_DOUBLES * sizeof(double))));
  jacobi_svd_kernel<<<1, JAC_THREADS, bytes, c->stream>>>(B, n, U, S, V, c->scratch[5].p(), mode);
  LAUNCH_CHECK(c);
}

// ----------------------------------------------------------------- TT core kernels
// Y[(a,b), i, (c,e)] = sum_j A[a,i,j,c] X[b,j,e]
__global__ void kron_core_kernel(const double *__restrict__ A, int R0, int m, int n, int R1,
                                 const double *__restrict__ X, int r0, int r1, double *__restrict__ Y) {
  const long long tot = (long long)R0 * r0 * m * R1 * r1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    long long rem = e;
    const int ee = (int)(rem % r1);
    rem /= r1;
    const int cc = (int)(rem % R1);
    rem /= R1;
    const int i = (int)(rem % m);
    rem /= m;
    const int b = (int)(rem % r0);
    const int a = (int)(rem / r0);
    double s = 0.0;
    for (int j = 0; j < n; ++j)
      s = fma(A[(((long long)a * m + i) * n + j) * R1 + cc], X[((long long)b * n + j) * r1 + ee], s);
    Y[e] = s;
  }
}

void kron_core(Ctx *c, const double *A, int R0, int m, int n, int R1, const double *X, int r0, int r1,
               double *Y) {
  const long long tot = (long long)R0 * r0 * m * R1 * r1;
  if (!tot) return;
  kron_core_kernel<<<ew_blocks(c, (size_t)tot), 256, 0, c->stream>>>(A, R0, m, n, R1, X, r0, r1, Y);
  LAUNCH_CHECK(c);
  c->flops += 2.0 * (double)tot * n;
}

__global__ void contract_mode_kernel(const double *__restrict__ G, int r0, int n, int r1,
                                     const double *__restrict__ w, double *__restrict__ out) {
  const long long tot = (long long)r0 * r1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(e / r1), b = (int)(e % r1);
    double s = 0.0;
    for (int i = 0; i < n; ++i) s = fma(w[i], G[((long long)a * n + i) * r1 + b], s);
    out[e] = s;
  }
}

void contract_mode(Ctx *c, const double *G, int r0, int n, int r1, const double *w, double *out) {
  const long long tot = (long long)r0 * r1;
  if (!tot) return;
  contract_mode_kernel<<<ew_blocks(c, (size_t)tot), 256, 0, c->stream>>>(G, r0, n, r1, w, out);
  LAUNCH_CHECK(c);
}

}  // namespace tt

namespace tt {

// ----------------------------------------------------------------- FP32 building blocks
// Same tiling as the FP64 GEMM, FP32 operands and accumulation (the FP32 SIMT
// rate of an SM is 64x its FP64 rate on this part).
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, float alpha, const float *__restrict__ A,
                                                    int lda, long long sA, const float *__restrict__ B, int ldb,
                                                    long long sB, float beta, float *__restrict__ C, int ldc,
                                                    long long sC, int splitk, int kchunk, float *__restrict__ ws) {
  __shared__ float As[GBK][GBM + 1];
  __shared__ float Bs[GBK][GBN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int bz = blockIdx.z;
  const int batch = bz / splitk, split = bz % splitk;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int kbeg = split * kchunk;
  const int kend = min(K, kbeg + kchunk);
  A += batch * sA;
  B += batch * sB;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = kbeg; k0 < kend; k0 += GBK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      int mm, kk;
      if (TA) {
        mm = e & 63;
        kk = e >> 6;
      } else {
        kk = e & 15;
        mm = e >> 4;
      }
      const int gm = m0 + mm, gk = k0 + kk;
      float v = 0.f;
      if (gm < M && gk < kend) v = TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
      As[kk][mm] = v;
      int nn, kb;
      if (TB) {
        kb = e & 15;
        nn = e >> 4;
      } else {
        nn = e & 63;
        kb = e >> 6;
      }
      const int gn = n0 + nn, gkb = k0 + kb;
      float w = 0.f;
      if (gn < N && gkb < kend) w = TB ? B[(long long)gn * ldb + gkb] : B[(long long)gkb * ldb + gn];
      Bs[kb][nn] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (splitk == 1) {
    float *Cb = C + batch * sC;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gm = m0 + ty + 16 * i;
      if (gm >= M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gn = n0 + tx + 16 * j;
        if (gn >= N) continue;
        float *cp = Cb + (long long)gm * ldc + gn;
        *cp = beta == 0.f ? alpha * acc[i][j] : alpha * acc[i][j] + beta * *cp;
      }
    }
  } else {
    float *W = ws + (long long)bz * M * N;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gm = m0 + ty + 16 * i;
      if (gm >= M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gn = n0 + tx + 16 * j;
        if (gn < N) W[(long long)gm * N + gn] = acc[i][j];
      }
    }
  }
}

__global__ void splitk_reduce_f(int M, int N, int splitk, int batch, const float *__restrict__ ws, float alpha,
                                float beta, float *__restrict__ C, int ldc, long long sC) {
  const long long tot = (long long)batch * M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e / ((long long)M * N));
    const long long r = e % ((long long)M * N);
    const int m = (int)(r / N), n = (int)(r % N);
    float s = 0.f;
    for (int q = 0; q < splitk; ++q) s += ws[((long long)b * splitk + q) * M * N + r];
    float *cp = C + b * sC + (long long)m * ldc + n;
    *cp = beta == 0.f ? alpha * s : alpha * s + beta * *cp;
  }
}

void gemm_f32(Ctx *c, bool ta, bool tb, int M, int N, int K, float alpha, const float *A, int lda, long long sA,
              const float *B, int ldb, long long sB, float beta, float *C, int ldc, long long sC, int batch) {
  if (M <= 0 || N <= 0 || batch <= 0 || K <= 0) return;
  const long long tiles = (long long)((M + GBM - 1) / GBM) * ((N + GBN - 1) / GBN) * batch;
  const long long target = 2LL * c->sm_count;
  // too few 64 x 64 tiles to reach every SM: 16 x 16 tiles with a K split
  const bool small = tiles < c->sm_count;
  const int TM = small ? SBM : GBM, TN = small ? SBN : GBN, TK = small ? SBK : GBK;
  const long long tl = (long long)((M + TM - 1) / TM) * ((N + TN - 1) / TN) * batch;
  int splitk = 1;
  if (small) {
    if (tl < target && K > TK) splitk = (int)std::min<long long>((target + tl - 1) / tl, (K + TK - 1) / TK);
  } else if (tl < target && K > 4 * TK) {
    splitk = (int)std::min<long long>((target + tl - 1) / tl, (K + 63) / 64);
  }
  splitk = std::max(1, std::min(splitk, 64));
  int kchunk = (K + splitk - 1) / splitk;
  kchunk = (kchunk + TK - 1) / TK * TK;
  splitk = (K + kchunk - 1) / kchunk;
  TT_REQUIRE((long long)batch * splitk <= 65535, "gemm_f32: batch too large");
  float *ws = nullptr;
  if (splitk > 1) {
    c->ws_gemm32.ensure(c, ((size_t)batch * splitk * M * N + 1) / 2);
    ws = reinterpret_cast<float *>(c->ws_gemm32.p());
  }
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, batch * splitk);
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (c->profiling) {
    c->prof_begin(&ev0, &ev1, 1);
    TT_CHECK_CUDA(cudaEventRecord(ev0, c->stream));
  }
#define SGEMM_LAUNCH(TA_, TB_)                                                                      \
  sgemm_kernel<TA_, TB_><<<grid, 256, 0, c->stream>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, \
                                                      C, ldc, sC, splitk, kchunk, ws)
  if (ta && tb) SGEMM_LAUNCH(true, true);
  else if (ta) SGEMM_LAUNCH(true, false);
  else if (tb) SGEMM_LAUNCH(false, true);
  else SGEMM_LAUNCH(false, false);
#undef SGEMM_LAUNCH
  LAUNCH_CHECK(c);
  if (splitk > 1) {
    const long long tot = (long long)batch * M * N;
    const unsigned blocks = (unsigned)std::min<long long>((tot + 255) / 256, 4LL * c->sm_count * 8);
    splitk_reduce_f<<<blocks, 256, 0, c->stream>>>(M, N, splitk, batch, ws, alpha, beta, C, ldc, sC);
    LAUNCH_CHECK(c);
  }
  if (c->profiling) {
    TT_CHECK_CUDA(cudaEventRecord(ev1, c->stream));
    c->gemm32_flops += 2.0 * M * (double)N * K * batch;
    c->gemm32_launches += 1;
  }
}

__global__ void d2f_kernel(const double *__restrict__ x, float *__restrict__ y, size_t n, double s) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (float)(s * x[i]);
}
__global__ void f2d_axpy_kernel(const float *__restrict__ x, double *__restrict__ y, size_t n, double a) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] += a * (double)x[i];
}
__global__ void axpby_f_kernel(size_t n, float a, const float *x, float b, float *y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = b == 0.f ? a * x[i] : a * x[i] + b * y[i];
}
__global__ void multi_dot_f_kernel(const float *__restrict__ V, size_t ldv, const float *__restrict__ w, size_t n,
                                   double *__restrict__ h) {
  __shared__ double sh[32];
  const float *v = V + blockIdx.x * ldv;
  double s = 0.0;
  for (size_t i = threadIdx.x; i < n; i += blockDim.x) s = fma((double)v[i], (double)w[i], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) h[blockIdx.x] = s;
}
__global__ void multi_axpy_f_kernel(const float *__restrict__ V, size_t ldv, int nv, const double *__restrict__ h,
                                    float *__restrict__ w, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < nv; ++j) s = fma((double)V[j * ldv + i], h[j], s);
    w[i] = (float)((double)w[i] - s);
  }
}
__global__ void dot_f_partial(const float *__restrict__ x, const float *__restrict__ y, size_t n,
                              double *__restrict__ part) {
  __shared__ double sh[32];
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    s = fma((double)x[i], (double)y[i], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

void d2f(Ctx *c, const double *x, float *y, size_t n, double s) {
  if (!n) return;
  d2f_kernel<<<ew_blocks(c, n), 256, 0, c->stream>>>(x, y, n, s);
  LAUNCH_CHECK(c);
}
void f2d_axpy(Ctx *c, const float *x, double *y, size_t n, double a) {
  if (!n) return;
  f2d_axpy_kernel<<<ew_blocks(c, n), 256, 0, c->stream>>>(x, y, n, a);
  LAUNCH_CHECK(c);
}
void axpby_f(Ctx *c, size_t n, float a, const float *x, float b, float *y) {
  if (!n) return;
  axpby_f_kernel<<<ew_blocks(c, n), 256, 0, c->stream>>>(n, a, x, b, y);
  LAUNCH_CHECK(c);
}
void multi_dot_f(Ctx *c, const float *V, size_t ldv, int nv, const float *w, size_t n, double *h) {
  if (nv <= 0) return;
  multi_dot_f_kernel<<<nv, 256, 0, c->stream>>>(V, ldv, w, n, h);
  LAUNCH_CHECK(c);
}
void multi_axpy_f(Ctx *c, const float *V, size_t ldv, int nv, const double *h, float *w, size_t n) {
  if (nv <= 0 || n == 0) return;
  multi_axpy_f_kernel<<<ew_blocks(c, n), 256, 0, c->stream>>>(V, ldv, nv, h, w, n);
  LAUNCH_CHECK(c);
}
void dot_f_dev(Ctx *c, const float *x, const float *y, size_t n, double *out) {
  c->scratch[7].ensure(c, RED_BLOCKS);
  if (n == 0) {
    fill(c, out, 1, 0.0);
    return;
  }
  const int nb = (int)std::min<size_t>(RED_BLOCKS, (n + 255) / 256);
  dot_f_partial<<<nb, 256, 0, c->stream>>>(x, y, n, c->scratch[7].p());
  LAUNCH_CHECK(c);
  sum_partials<<<1, 256, 0, c->stream>>>(c->scratch[7].p(), nb, out);
  LAUNCH_CHECK(c);
}

}  // namespace tt
