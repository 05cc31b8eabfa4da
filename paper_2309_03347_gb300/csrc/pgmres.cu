// Restarted FP32 GMRES of one local system as a single persistent
// cooperative kernel: the local matvec (three tiled GEMMs), the two
// classical Gram-Schmidt passes, the Arnoldi/Givens update, the restarts and
// the convergence tests all run on the device, in phases separated by a grid
// barrier.  One launch replaces about a dozen launches and a host round trip
// per Arnoldi step.
//
// Local matvec (the Galerkin-projected operator of a core):
//   T1 = Phi_L (r0 R1 x r0) . v (r0 x m r1)
//   T2[a] = A^T (m R2 x R1 m) . T1[a] (R1 m x r1)          a < r0
//   w  = T2 (r0 m x R2 r1) . Phi_R^T (R2 r1 x r1)          (split over K)
// Basis vectors are stored unnormalised with their scale s_j; all inner
// products and updates use s_j V_j.  Reductions are in FP64, in a fixed
// order.  The grid barrier spins a bounded number of times and then sets an
// error code, so a kernel that cannot make progress returns.
#include "common.cuh"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <mutex>

namespace tt {

namespace {

constexpr int PG_THREADS = 256;
constexpr int TBM = 64, TBN = 64, TBK = 32;
constexpr int PG_CHUNK = 2048;  // largest per-CTA slice of a vector
constexpr long long BAR_LIMIT = 1LL << 24;
constexpr int PG_MAXR = 32;  // longest restart cycle

struct PGArgs {
  const float *PL, *A, *PR, *b;
  float *x, *V, *T1, *T2, *ws;
  double *D;
  int *st;         // [0] steps, [1] error, [2] cycle end, [3] done
  unsigned *bar;   // [0] arrivals, [1] generation
  int r0, R1, m, R2, r1, N, mr, maxit, split3, kchunk3, chunk, gv;
  double tol;
  long long bar_limit;  // spins of a CTA waiting at the grid barrier before it gives up
  int cta0, ncta;       // this system's CTAs: blockIdx.x in [cta0, cta0 + ncta)
  int cta;              // blockIdx.x - cta0 (set on the device)
};

// offsets into the device state D (doubles) for restart mr and G CTAs
struct PGLayout {
  size_t H, cs, sn, g, y, s, h1, h2, part, part2, npart, misc, total;
  __host__ __device__ PGLayout(int mr, int G) {
    H = 0;
    cs = H + (size_t)(mr + 1) * mr;
    sn = cs + mr;
    g = sn + mr;
    y = g + mr + 1;
    s = y + mr + 1;
    h1 = s + mr + 1;
    h2 = h1 + mr + 1;
    part = h2 + mr + 1;
    part2 = part + (size_t)(mr + 1) * G;
    npart = part2 + (size_t)(mr + 1) * G;
    misc = npart + G;
    total = misc + 8;
  }
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Grid barrier over co-resident CTAs (cooperative launch); bounded spin.
__device__ bool grid_sync(unsigned *bar, int *err, long long limit, unsigned nct) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *vgen = bar + 1;
    const unsigned g = *vgen;
    int ok = 1;
    __threadfence();
    if (atomicAdd(bar, 1u) == nct - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*vgen == g) {
        if (++spins > limit) {
          ok = 0;
          atomicExch(err, TT_ETIMEOUT);
          break;
        }
        __nanosleep(40);
      }
    }
    __threadfence();
    s_ok = ok && *(volatile int *)err == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// Tiled GEMM work items (tile row, tile column, split, batch) spread over the
// grid; C (+ q * sSplit for split q) = alpha op(A) op(B) over split q's K range.
template <bool TA, bool TB>
__device__ void gemm_phase(int M, int N, int K, float alpha, const float *__restrict__ A, int lda, long long sA,
                           const float *__restrict__ B, int ldb, long long sB, float *__restrict__ C, int ldc,
                           long long sC, int batch, int splits, int kchunk, long long sSplit, float (*As)[TBM + 1],
                           float (*Bs)[TBN + 1], int cta, int ncta) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int tm = (M + TBM - 1) / TBM, tn = (N + TBN - 1) / TBN;
  const long long items = (long long)tm * tn * splits * batch;
  for (long long item = cta; item < items; item += ncta) {
    long long t = item;
    const int bx = (int)(t % tn);
    t /= tn;
    const int by = (int)(t % tm);
    t /= tm;
    const int q = (int)(t % splits);
    const int bb = (int)(t / splits);
    const float *Ab = A + bb * sA;
    const float *Bb = B + bb * sB;
    float *Cb = C + bb * sC + q * sSplit;
    const int m0 = by * TBM, n0 = bx * TBN;
    const int kbeg = q * kchunk, kend = min(K, kbeg + kchunk);
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    float ra[8], rb[8];
    auto gload = [&](int k0) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = tid + PG_THREADS * u;
        int mm, kk;
        if (TA) {
          mm = e & 63;
          kk = e >> 6;
        } else {
          kk = e & 31;
          mm = e >> 5;
        }
        const int gm = m0 + mm, gk = k0 + kk;
        ra[u] = (gm < M && gk < kend) ? __ldcg(TA ? Ab + (long long)gk * lda + gm : Ab + (long long)gm * lda + gk)
                                      : 0.f;
        int nn, kb;
        if (TB) {
          kb = e & 31;
          nn = e >> 5;
        } else {
          nn = e & 63;
          kb = e >> 6;
        }
        const int gn = n0 + nn, gkb = k0 + kb;
        rb[u] = (gn < N && gkb < kend) ? __ldcg(TB ? Bb + (long long)gn * ldb + gkb : Bb + (long long)gkb * ldb + gn)
                                       : 0.f;
      }
    };
    if (kbeg < kend) gload(kbeg);
    for (int k0 = kbeg; k0 < kend; k0 += TBK) {
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int e = tid + PG_THREADS * u;
        if (TA) As[e >> 6][e & 63] = ra[u];
        else As[e & 31][e >> 5] = ra[u];
        if (TB) Bs[e & 31][e >> 5] = rb[u];
        else Bs[e >> 6][e & 63] = rb[u];
      }
      __syncthreads();
      if (k0 + TBK < kend) gload(k0 + TBK);
#pragma unroll 8
      for (int kk = 0; kk < TBK; ++kk) {
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
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gm = m0 + ty + 16 * i;
      if (gm >= M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gn = n0 + tx + 16 * j;
        if (gn < N) Cb[(long long)gm * ldc + gn] = alpha * acc[i][j];
      }
    }
  }
}

// GEMM2 and GEMM3 of the local matvec (T1 -> T2 -> split partials of w in ws)
__device__ bool matvec_tail(const PGArgs &P, float (*As)[TBM + 1], float (*Bs)[TBN + 1]) {
  const int r0 = P.r0, R1 = P.R1, m = P.m, R2 = P.R2, r1 = P.r1;
  gemm_phase<true, false>(m * R2, r1, R1 * m, 1.f, P.A, m * R2, 0, P.T1, r1, (long long)R1 * m * r1, P.T2, r1,
                          (long long)m * R2 * r1, r0, 1, R1 * m, 0, As, Bs, P.cta, P.ncta);
  if (!grid_sync(P.bar, P.st + 1, P.bar_limit, (unsigned)P.ncta)) return false;
  gemm_phase<false, true>(r0 * m, r1, R2 * r1, 1.f, P.T2, R2 * r1, 0, P.PR, R2 * r1, 0, P.ws, r1, 0, 1, P.split3,
                          P.kchunk3, (long long)P.N, As, Bs, P.cta, P.ncta);
  return grid_sync(P.bar, P.st + 1, P.bar_limit, (unsigned)P.ncta);
}

// w-partials of the matvec of v (scale alpha) into ws (split3 slices of N)
__device__ bool matvec_phases(const PGArgs &P, const float *v, float alpha, float (*As)[TBM + 1],
                              float (*Bs)[TBN + 1]) {
  const int r0 = P.r0, R1 = P.R1, m = P.m, r1 = P.r1;
  gemm_phase<false, false>(r0 * R1, m * r1, r0, alpha, P.PL, r0, 0, v, m * r1, 0, P.T1, m * r1, 0, 1, 1, r0, 0, As,
                           Bs, P.cta, P.ncta);
  if (!grid_sync(P.bar, P.st + 1, P.bar_limit, (unsigned)P.ncta)) return false;
  return matvec_tail(P, As, Bs);
}

// The GMRES of one system on its CTAs (P.cta = this CTA's index among them).
__device__ __forceinline__ void pgmres_body(const PGArgs &P) {
  __shared__ float As[TBK][TBM + 1];
  __shared__ float Bs[TBK][TBN + 1];
  __shared__ float wsh[PG_CHUNK];
  __shared__ float hsc[PG_MAXR + 1];   // Gram-Schmidt coefficients of the stored vectors
  __shared__ double ss[PG_MAXR + 1];   // scales s_v of the stored vectors (same in every CTA)
  __shared__ double red[PG_THREADS / 32];
  // Arnoldi state, used by CTA 0 only
  __shared__ double sH[(PG_MAXR + 1) * PG_MAXR];
  __shared__ double scs[PG_MAXR], ssn[PG_MAXR], sg[PG_MAXR + 1], sh1[PG_MAXR + 1], sh2[PG_MAXR + 1];
  __shared__ double s_hn;
  const int bid = P.cta, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarp = PG_THREADS / 32;
  const int Gv = P.gv;
  const PGLayout L(P.mr, Gv);
  double *D = P.D;
  const int N = P.N, mr = P.mr;
  const size_t lo = (size_t)bid * P.chunk, hi = bid < Gv ? min((size_t)N, lo + (size_t)P.chunk) : lo;
  const int cn = hi > lo ? (int)(hi - lo) : 0;
  int *err = P.st + 1;

  // block sum (all threads get the result)
  auto block_total = [&](double v) {
    v = warp_sum_d(v);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < nwarp; ++i) t += red[i];
    __syncthreads();
    return t;
  };
  // sum of the Gv partials of vector v, fixed order (one warp)
  auto warp_part_sum = [&](const double *part, int v) {
    double a = 0.0;
#pragma unroll 4
    for (int b = lane; b < Gv; b += 32) a += __ldcg(part + (size_t)v * Gv + b);
    return warp_sum_d(a);
  };
  // sum_{v <= j} V_v[i] c_v for the slice (c in hsc, FP32 products and sums:
  // the Krylov vectors are FP32), eight loads in flight
  auto sub_comb = [&](int i, int j) {
    const float *base = P.V + lo + i;
    float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int v = 0;
    for (; v + 7 <= j; v += 8) {
      float xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) xv[u] = __ldcg(base + (size_t)(v + u) * N);
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = fmaf(xv[u], hsc[v + u], a[u]);
    }
    for (; v <= j; ++v) a[0] = fmaf(__ldcg(base + (size_t)v * N), hsc[v], a[0]);
    return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
  };
  // partial inner products of the slice of w (in wsh) with the stored vectors
  // v <= j: FP32 products summed per lane, FP64 across lanes and CTAs
  auto inner = [&](double *part, int j) {
    for (int v = warp; v <= j; v += nwarp) {
      const float *vv = P.V + (size_t)v * N + lo;
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
      int i = lane;
      for (; i + 96 < cn; i += 128) {
        const float x0 = __ldcg(vv + i), x1 = __ldcg(vv + i + 32), x2 = __ldcg(vv + i + 64), x3 = __ldcg(vv + i + 96);
        a0 = fmaf(x0, wsh[i], a0);
        a1 = fmaf(x1, wsh[i + 32], a1);
        a2 = fmaf(x2, wsh[i + 64], a2);
        a3 = fmaf(x3, wsh[i + 96], a3);
      }
      for (; i < cn; i += 32) a0 = fmaf(__ldcg(vv + i), wsh[i], a0);
      const double a = warp_sum_d((double)a0 + (double)a1 + ((double)a2 + (double)a3));
      if (lane == 0 && bid < Gv) part[(size_t)v * Gv + bid] = a * ss[v];
    }
  };
  // h_{j+1,j} from the norm partials: every CTA forms the same value
  auto norm_from_partials = [&]() {
    if (warp == 0) {
      double a = 0.0;
      for (int b = lane; b < Gv; b += 32) a += __ldcg(D + L.npart + b);
      a = warp_sum_d(a);
      if (lane == 0) s_hn = sqrt(fmax(a, 0.0));
    }
    __syncthreads();
    return s_hn;
  };
  // CTA 0, one thread: column j of H, Givens rotations, residual; sets the cycle flags
  auto givens = [&](int j, double hn, int nsteps) {
    for (int i = 0; i <= j; ++i) sH[i * mr + j] = sh1[i] + sh2[i];
    sH[(j + 1) * mr + j] = hn;
    for (int i = 0; i < j; ++i) {
      const double a = sH[i * mr + j], bb = sH[(i + 1) * mr + j];
      sH[i * mr + j] = scs[i] * a + ssn[i] * bb;
      sH[(i + 1) * mr + j] = -ssn[i] * a + scs[i] * bb;
    }
    const double a = sH[j * mr + j], bb = sH[(j + 1) * mr + j];
    const double den = hypot(a, bb);
    scs[j] = den == 0.0 ? 1.0 : a / den;
    ssn[j] = den == 0.0 ? 0.0 : bb / den;
    sH[j * mr + j] = den;
    sH[(j + 1) * mr + j] = 0.0;
    sg[j + 1] = -ssn[j] * sg[j];
    sg[j] = scs[j] * sg[j];
    const double res = fabs(sg[j + 1]);
    const bool breakdown = hn <= 1e-30;
    P.st[0] = nsteps;
    if (!isfinite(hn) || !isfinite(res)) atomicExch(err, TT_ENONFINITE);
    P.st[2] = (res <= P.tol || nsteps >= P.maxit || breakdown || j == mr - 1) ? 1 : 0;
    P.st[3] = (res <= P.tol || nsteps >= P.maxit) ? 1 : 0;
  };

  int steps = 0;
  bool first = true;
  while (true) {
    // ---- r = b - M x into V_0 (x = 0 on the first cycle: r = b, x zeroed here)
    if (!first && !matvec_phases(P, P.x, 1.f, As, Bs)) return;
    {
      double sq = 0.0;
      for (int i = tid; i < cn; i += PG_THREADS) {
        const size_t gi = lo + i;
        float r = P.b[gi];
        if (first) {
          P.x[gi] = 0.f;
        } else {
          for (int q = 0; q < P.split3; ++q) r -= __ldcg(P.ws + (size_t)q * N + gi);
        }
        P.V[gi] = r;
        sq = fma((double)r, (double)r, sq);
      }
      sq = block_total(sq);
      if (tid == 0 && bid < Gv) D[L.npart + bid] = sq;
    }
    first = false;
    if (!grid_sync(P.bar, err, P.bar_limit, (unsigned)P.ncta)) return;
    {
      const double beta = norm_from_partials();
      if (tid == 0) {
        ss[0] = beta > 0.0 ? 1.0 / beta : 0.0;
        if (bid == 0) {
          for (int i = 0; i <= mr; ++i) sg[i] = 0.0;
          sg[0] = beta;
          if (!isfinite(beta)) atomicExch(err, TT_ENONFINITE);
        }
      }
      __syncthreads();
      if (!(beta > P.tol) || steps >= P.maxit || !isfinite(beta)) break;  // same decision in every CTA
    }
    // ---- Arnoldi steps; the Givens update of step j - 1 runs at the top of step j
    int jend = mr - 1;
    for (int j = 0; j <= mr; ++j) {
      if (j > 0) {
        const double hn = norm_from_partials();
        if (tid == 0) {
          ss[j] = hn <= 1e-30 ? 1.0 : 1.0 / hn;
          if (bid == 0) givens(j - 1, hn, steps + 1);
        }
        __syncthreads();
        ++steps;
      }
      if (j == mr) {
        if (!grid_sync(P.bar, err, P.bar_limit, (unsigned)P.ncta)) return;
        break;
      }
      // T1 = Phi_L (s_j V_j), then the flags of step j - 1 are visible
      {
        const int r0 = P.r0, R1 = P.R1, m = P.m, r1 = P.r1;
        gemm_phase<false, false>(r0 * R1, m * r1, r0, (float)ss[j], P.PL, r0, 0, P.V + (size_t)j * N, m * r1, 0,
                                 P.T1, m * r1, 0, 1, 1, r0, 0, As, Bs, P.cta, P.ncta);
        if (!grid_sync(P.bar, err, P.bar_limit, (unsigned)P.ncta)) return;
      }
      if (j > 0 && __ldcg(P.st + 2)) {
        jend = j - 1;
        break;
      }
      if (!matvec_tail(P, As, Bs)) return;
      // w = sum of the split partials (kept in shared memory); first pass of inner products
      float *w = P.V + (size_t)(j + 1) * N;
      for (int i = tid; i < cn; i += PG_THREADS) {
        const float *wp = P.ws + lo + i;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        int q = 0;
        for (; q + 3 < P.split3; q += 4) {
          a0 += __ldcg(wp + (size_t)q * N);
          a1 += __ldcg(wp + (size_t)(q + 1) * N);
          a2 += __ldcg(wp + (size_t)(q + 2) * N);
          a3 += __ldcg(wp + (size_t)(q + 3) * N);
        }
        for (; q < P.split3; ++q) a0 += __ldcg(wp + (size_t)q * N);
        wsh[i] = (a0 + a1) + (a2 + a3);
      }
      __syncthreads();
      inner(D + L.part, j);
      if (!grid_sync(P.bar, err, P.bar_limit, (unsigned)P.ncta)) return;
      // two subtraction passes; the second also forms the norm partials and stores w
      for (int pass = 0; pass < 2; ++pass) {
        const double *part = D + (pass == 0 ? L.part : L.part2);
        for (int v = warp; v <= j; v += nwarp) {
          const double h = warp_part_sum(part, v);
          if (lane == 0) {
            hsc[v] = (float)(h * ss[v]);
            if (bid == 0) (pass == 0 ? sh1 : sh2)[v] = h;
          }
        }
        __syncthreads();
        float sqf = 0.f;
        for (int i = tid; i < cn; i += PG_THREADS) {
          const float nw = wsh[i] - sub_comb(i, j);
          wsh[i] = nw;
          sqf = fmaf(nw, nw, sqf);
        }
        double sq = (double)sqf;
        __syncthreads();
        if (pass == 0) {
          inner(D + L.part2, j);
        } else {
          for (int i = tid; i < cn; i += PG_THREADS) w[lo + i] = wsh[i];
          sq = block_total(sq);
          if (tid == 0 && bid < Gv) D[L.npart + bid] = sq;
        }
        if (!grid_sync(P.bar, err, P.bar_limit, (unsigned)P.ncta)) return;
      }
    }
    // ---- x += sum_v y_v s_v V_v with y = H^-1 g over the columns 0..jend
    if (bid == 0 && tid == 0) {
      const int kk = jend + 1;
      double *y = D + L.y;
      for (int i = kk - 1; i >= 0; --i) {
        double sacc = sg[i];
        for (int l = i + 1; l < kk; ++l) sacc -= sH[i * mr + l] * y[l];
        const double dg = sH[i * mr + i];
        y[i] = dg != 0.0 ? sacc / dg : 0.0;
      }
      for (int i = 0; i < kk; ++i) y[i] *= ss[i];
    }
    if (!grid_sync(P.bar, err, P.bar_limit, (unsigned)P.ncta)) return;
    for (int v = tid; v <= jend; v += PG_THREADS) hsc[v] = (float)__ldcg(D + L.y + v);
    __syncthreads();
    for (int i = tid; i < cn; i += PG_THREADS) P.x[lo + i] += sub_comb(i, jend);
    if (!grid_sync(P.bar, err, P.bar_limit, (unsigned)P.ncta)) return;
    if (__ldcg(P.st + 3)) break;
  }
}

__global__ void __launch_bounds__(PG_THREADS, 1) pgmres_kernel(PGArgs P) {
  P.cta = (int)blockIdx.x - P.cta0;
  pgmres_body(P);
}

// Several independent systems in one cooperative launch: system g owns the
// CTAs [list[g].cta0, list[g].cta0 + list[g].ncta) (list sorted by cta0) and
// runs on them with its own barrier words, buffers and status.
__global__ void __launch_bounds__(PG_THREADS, 1) pgmres_group_kernel(const PGArgs *__restrict__ list, int n) {
  __shared__ PGArgs sp;
  if (threadIdx.x == 0) {
    int g = 0;
    while (g + 1 < n && list[g + 1].cta0 <= (int)blockIdx.x) ++g;
    sp = list[g];
    sp.cta = (int)blockIdx.x - sp.cta0;
  }
  __syncthreads();
  pgmres_body(sp);
}

}  // namespace

// The parameters of a system that depend on the CTAs it runs on: the CTAs
// of the vector phases (slices of about 256 entries, at most PG_CHUNK) and
// the K split of the third GEMM (fill the CTAs, K slices of >= 2 tiles).
void pg_shape(PGArgs &P, int ncta) {
  const int N = P.N;
  P.ncta = ncta;
  P.gv = std::max(1, std::min(ncta, (N + 255) / 256));
  P.chunk = (N + P.gv - 1) / P.gv;
  const int K3 = P.R2 * P.r1;
  const int tiles3 = ((P.r0 * P.m + TBM - 1) / TBM) * ((P.r1 + TBN - 1) / TBN);
  int split3 = std::max(1, std::min(32, ncta / std::max(1, tiles3)));
  int kchunk3 = (K3 + split3 - 1) / split3;
  kchunk3 = std::max(2 * TBK, (kchunk3 + TBK - 1) / TBK * TBK);
  P.split3 = (K3 + kchunk3 - 1) / kchunk3;
  P.kchunk3 = kchunk3;
}

// Shape class of a local system for the grid-size tuner: log2 of its size,
// its mode and (capped) operator ranks.
uint64_t pg_shape_class(int N, int m, int R1, int R2) {
  int lb = 0;
  while ((1 << (lb + 1)) <= N) ++lb;
  return (uint64_t)lb | ((uint64_t)std::min(m, 4095) << 8) | ((uint64_t)std::min(R1, 1023) << 20) |
         ((uint64_t)std::min(R2, 1023) << 30);
}

bool pgmres32_fits(Ctx *c, int N, int restart) {
  return restart >= 1 && restart <= PG_MAXR && N > 0 && (long long)N <= (long long)PG_CHUNK * c->sm_count;
}

// ----------------------------------------------------------------- grouped launches
// Local systems of independent problems (keig_batch: one worker thread and
// context per problem stream) are gathered into one cooperative launch of
// pgmres_group_kernel instead of one whole-GPU launch each.  A worker
// submits its prepared system and waits; the first waiting worker becomes
// the leader, waits until every active worker has submitted or a short
// window has passed, gives each gathered system CTAs in proportion to its
// size (at least enough for slices of PG_CHUNK entries), launches them
// together on the group's stream after the submitters' streams, and copies
// every system's status back.  Systems that do not fit in one grid wait for
// the next launch.
struct PGGroup {
  struct Item {
    PGArgs P;
    cudaEvent_t ready = nullptr;
    int hs[2] = {0, 0};
    bool done = false;
    int err = 0;
  };
  std::mutex mu;
  std::condition_variable cv;
  int active = 0;
  bool launching = false;
  std::vector<Item *> pending;
  std::chrono::steady_clock::time_point first_arrival;
  int device = 0, sm_count = 152;
  cudaStream_t stream = nullptr;
  PGArgs *d_list = nullptr, *h_list = nullptr;
  int *h_st = nullptr;
  double window_us = 300.0;
  long long launches = 0, systems = 0;
};

PGGroup *pg_group_create(int device, int sm_count) {
  PGGroup *g = new PGGroup();
  g->device = device;
  g->sm_count = sm_count;
  TT_CHECK_CUDA(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
  TT_CHECK_CUDA(cudaMalloc(&g->d_list, sizeof(PGArgs) * 1024));
  TT_CHECK_CUDA(cudaMallocHost(&g->h_list, sizeof(PGArgs) * 1024));
  TT_CHECK_CUDA(cudaMallocHost(&g->h_st, sizeof(int) * 2 * 1024));
  return g;
}

void pg_group_destroy(PGGroup *g) {
  if (!g) return;
  cudaStreamSynchronize(g->stream);
  cudaFree(g->d_list);
  cudaFreeHost(g->h_list);
  cudaFreeHost(g->h_st);
  cudaStreamDestroy(g->stream);
  delete g;
}

void pg_group_set_active(PGGroup *g, int n) {
  std::lock_guard<std::mutex> lk(g->mu);
  g->active = n;
  g->cv.notify_all();
}

void pg_group_join(PGGroup *g) {
  std::lock_guard<std::mutex> lk(g->mu);
  ++g->active;
}

void pg_group_leave(PGGroup *g) {
  std::lock_guard<std::mutex> lk(g->mu);
  --g->active;
  g->cv.notify_all();
}

void pg_group_stats(PGGroup *g, long long *launches, long long *systems) {
  std::lock_guard<std::mutex> lk(g->mu);
  *launches = g->launches;
  *systems = g->systems;
}

namespace {

// Launch the gathered items (called by the leader without the lock held).
void pg_group_launch(PGGroup *g, std::vector<PGGroup::Item *> &items) {
  const int n = (int)items.size();
  long long total_n = 0;
  for (auto *it : items) total_n += it->P.N;
  std::vector<int> need(n), give(n);
  int used = 0;
  for (int i = 0; i < n; ++i) {
    need[i] = std::max(1, (items[i]->P.N + PG_CHUNK - 1) / PG_CHUNK);
    used += need[i];
  }
  int spare = g->sm_count - used;
  for (int i = 0; i < n; ++i) {
    const int extra = (int)((double)spare * items[i]->P.N / std::max<long long>(1, total_n));
    give[i] = need[i] + std::max(0, extra);
  }
  int cta = 0;
  for (int i = 0; i < n; ++i) {
    PGArgs &P = items[i]->P;
    pg_shape(P, give[i]);
    P.cta0 = cta;
    P.cta = 0;
    cta += give[i];
    g->h_list[i] = P;
    TT_CHECK_CUDA(cudaStreamWaitEvent(g->stream, items[i]->ready, 0));
  }
  TT_CHECK_CUDA(cudaMemcpyAsync(g->d_list, g->h_list, sizeof(PGArgs) * n, cudaMemcpyHostToDevice, g->stream));
  const PGArgs *dl = g->d_list;
  void *args[] = {(void *)&dl, (void *)&n};
  TT_CHECK_CUDA(cudaLaunchCooperativeKernel((const void *)pgmres_group_kernel, dim3(cta), dim3(PG_THREADS), args, 0,
                                            g->stream));
  for (int i = 0; i < n; ++i)
    TT_CHECK_CUDA(cudaMemcpyAsync(g->h_st + 2 * i, items[i]->P.st, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                                  g->stream));
  TT_CHECK_CUDA(cudaStreamSynchronize(g->stream));
  for (int i = 0; i < n; ++i) {
    items[i]->hs[0] = g->h_st[2 * i];
    items[i]->hs[1] = g->h_st[2 * i + 1];
  }
}

}  // namespace

// Submit one prepared system (its status words already cleared on the
// worker's stream) and wait until a grouped launch has run it.
void pg_group_solve(PGGroup *g, Ctx *c, PGArgs P, int hs[2]) {
  PGGroup::Item item;
  item.P = P;
  TT_CHECK_CUDA(cudaEventCreateWithFlags(&item.ready, cudaEventDisableTiming));
  TT_CHECK_CUDA(cudaEventRecord(item.ready, c->stream));
  std::unique_lock<std::mutex> lk(g->mu);
  if (g->pending.empty()) g->first_arrival = std::chrono::steady_clock::now();
  g->pending.push_back(&item);
  g->cv.notify_all();
  while (!item.done) {
    if (!g->launching && !g->pending.empty()) {
      // lead: wait for the other active workers or the window, then launch
      const auto until = g->first_arrival + std::chrono::microseconds((long long)g->window_us);
      while ((int)g->pending.size() < g->active && std::chrono::steady_clock::now() < until)
        g->cv.wait_until(lk, until);
      if (g->launching || g->pending.empty()) continue;
      std::vector<PGGroup::Item *> batch;
      std::vector<PGGroup::Item *> rest;
      int used = 0;
      for (auto *it : g->pending) {
        const int need = std::max(1, (it->P.N + PG_CHUNK - 1) / PG_CHUNK);
        if (used + need <= g->sm_count && (int)batch.size() < 1024) {
          batch.push_back(it);
          used += need;
        } else {
          rest.push_back(it);
        }
      }
      g->pending.swap(rest);
      if (!g->pending.empty()) g->first_arrival = std::chrono::steady_clock::now();
      g->launching = true;
      lk.unlock();
      int err = 0;
      try {
        pg_group_launch(g, batch);
      } catch (const Error &e) {
        err = e.code;
      }
      lk.lock();
      g->launching = false;
      g->launches += 1;
      g->systems += (long long)batch.size();
      for (auto *it : batch) {
        it->err = err;
        it->done = true;
      }
      g->cv.notify_all();
    } else {
      g->cv.wait_for(lk, std::chrono::milliseconds(50));
    }
  }
  lk.unlock();
  cudaEventDestroy(item.ready);
  if (item.err) throw Error(item.err, "pgmres32: grouped launch failed");
  hs[0] = item.hs[0];
  hs[1] = item.hs[1];
}

int pgmres32(Ctx *c, const float *PL, const float *A32, const float *PR, int r0, int R1, int m, int R2, int r1,
             const float *b, float *x, double tol, int restart, int maxit, PGWork &W) {
  const int N = r0 * m * r1;
  TT_REQUIRE(pgmres32_fits(c, N, restart), "pgmres32: system too large for the persistent solver");
  int occ = 0;
  TT_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pgmres_kernel, PG_THREADS, 0));
  TT_REQUIRE(occ >= 1, "pgmres32: kernel does not fit on an SM");
  // one CTA per SM; the vector phases use the CTAs needed for slices of about 256
  const int G = c->sm_count;
  const int gv = std::max(1, std::min(G, (N + 255) / 256));
  const int chunk = (N + gv - 1) / gv;
  TT_REQUIRE(chunk <= PG_CHUNK, "pgmres32: vector slice too long");
  // split of the third GEMM: fill the grid, K slices of at least two tiles of K
  const int K3 = R2 * r1;
  const int tiles3 = ((r0 * m + TBM - 1) / TBM) * ((r1 + TBN - 1) / TBN);
  int split3 = std::max(1, std::min(32, G / std::max(1, tiles3)));
  int kchunk3 = (K3 + split3 - 1) / split3;
  kchunk3 = std::max(2 * TBK, (kchunk3 + TBK - 1) / TBK * TBK);
  split3 = (K3 + kchunk3 - 1) / kchunk3;
  const PGLayout L(restart, gv);
  W.V.ensure(c, ((size_t)(restart + 1) * N + 1) / 2);
  W.T1.ensure(c, ((size_t)r0 * R1 * m * r1 + 1) / 2);
  W.T2.ensure(c, ((size_t)r0 * m * R2 * r1 + 1) / 2);
  W.ws.ensure(c, ((size_t)split3 * N + 1) / 2);
  W.D.ensure(c, L.total);
  W.st.ensure(c, 4);  // 8 ints + 2 barrier words
  TT_CHECK_CUDA(cudaMemsetAsync(W.st.p(), 0, 4 * sizeof(double), c->stream));
  PGArgs P;
  P.PL = PL;
  P.A = A32;
  P.PR = PR;
  P.b = b;
  P.x = x;
  P.V = reinterpret_cast<float *>(W.V.p());
  P.T1 = reinterpret_cast<float *>(W.T1.p());
  P.T2 = reinterpret_cast<float *>(W.T2.p());
  P.ws = reinterpret_cast<float *>(W.ws.p());
  P.D = W.D.p();
  P.st = reinterpret_cast<int *>(W.st.p());
  P.bar = reinterpret_cast<unsigned *>(P.st + 4);
  P.r0 = r0;
  P.R1 = R1;
  P.m = m;
  P.R2 = R2;
  P.r1 = r1;
  P.N = N;
  P.mr = restart;
  P.maxit = maxit;
  P.split3 = split3;
  P.kchunk3 = kchunk3;
  P.chunk = chunk;
  P.gv = gv;
  P.tol = tol;
  P.bar_limit = c->wait_limit >= 0 ? c->wait_limit : BAR_LIMIT;
  P.cta0 = 0;
  P.ncta = G;
  P.cta = 0;
  // grid size of a single-system launch: picked per shape class by the tuner
  const uint64_t key = pg_shape_class(N, m, R1, R2);
  int Gl = G;
  const int gmin = std::max(1, (N + PG_CHUNK - 1) / PG_CHUNK);
  bool trial = false;
  if (!c->group && c->pg_tune) {
    auto it = c->pg_tuned.find(key);
    if (it != c->pg_tuned.end()) {
      Gl = std::max(it->second, gmin);
    } else {
      auto &tr = c->pg_trials[key];
      const int cand = G >> tr.size();  // G, G/2, G/4, G/8
      Gl = std::max(cand, gmin);
      trial = true;
    }
  }
  pg_shape(P, Gl);
  int hs[2];
  if (c->group) {
    // batched problems: this system joins the next grouped launch
    pg_group_solve(c->group, c, P, hs);
  } else {
    void *args[] = {&P};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (c->profiling) {
      c->prof_begin(&ev0, &ev1, 3);
      TT_CHECK_CUDA(cudaEventRecord(ev0, c->stream));
    }
    if (trial) TT_CHECK_CUDA(cudaEventRecord(c->tune_ev[0], c->stream));
    TT_CHECK_CUDA(cudaLaunchCooperativeKernel((const void *)pgmres_kernel, dim3(Gl), dim3(PG_THREADS), args, 0,
                                              c->stream));
    c->count();
    if (trial) TT_CHECK_CUDA(cudaEventRecord(c->tune_ev[1], c->stream));
    if (c->profiling) TT_CHECK_CUDA(cudaEventRecord(ev1, c->stream));
    TT_CHECK_CUDA(cudaMemcpyAsync(hs, W.st.p(), 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    c->sync();
    if (trial) {
      // time per Arnoldi step of this grid size; after the last candidate keep the fastest
      float ms = 0.f;
      TT_CHECK_CUDA(cudaEventElapsedTime(&ms, c->tune_ev[0], c->tune_ev[1]));
      auto &tr = c->pg_trials[key];
      tr.push_back({Gl, ms / std::max(1, hs[0])});
      if (tr.size() >= 4 || Gl == gmin) {
        auto best = *std::min_element(tr.begin(), tr.end(),
                                      [](const std::pair<int, double> &a, const std::pair<int, double> &b) {
                                        return a.second < b.second;
                                      });
        c->pg_tuned[key] = best.first;
      }
    }
  }
  // algorithmic work: one local matvec per Arnoldi step plus the restart residuals
  // (2 n r0 r1 (r0 R1 + n R1 R2 + r1 R2) each), and the two Gram-Schmidt passes
  // (4 N flops per stored vector per pass, counted with the mean basis size)
  const double mv = 2.0 * m * (double)r0 * r1 * ((double)r0 * R1 + (double)m * R1 * R2 + (double)r1 * R2);
  const int steps = std::max(hs[0], 0);
  const int cycles = (steps + restart - 1) / std::max(restart, 1);
  c->flops32 += mv * (steps + std::max(cycles - 1, 0));
  if (c->profiling) {
    c->pg_launches += 1;
    c->pg_flops += mv * (steps + std::max(cycles - 1, 0)) + 8.0 * N * steps * (0.5 * (std::min(steps, restart) + 1));
  }
  if (hs[1] == TT_ETIMEOUT) throw Error(TT_ETIMEOUT, "pgmres32: grid barrier gave up waiting");
  if (hs[1] != 0) throw Error(TT_ENONFINITE, "pgmres32: non-finite Krylov vector");
  return hs[0];
}

}  // namespace tt
