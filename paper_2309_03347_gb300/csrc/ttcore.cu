// TT vectors: construction, SVD/QR wrappers, orthogonalisation, rounding,
// dot products, sums and the exact operator-core x vector-core product.
#include <algorithm>
#include <numeric>

#include "tt.cuh"

namespace tt {

void tt_check(const TT &x) {
  TT_REQUIRE(x.d >= 1 && (int)x.n.size() == x.d && (int)x.r.size() == x.d + 1 &&
                 (int)x.core.size() == x.d,
             "TT: inconsistent metadata");
  TT_REQUIRE(x.r[0] == 1 && x.r[x.d] == 1, "TT: boundary ranks must be 1");
  for (int k = 0; k < x.d; ++k) TT_REQUIRE(x.n[k] >= 1 && x.r[k] >= 1, "TT: mode and rank >= 1");
}

TT tt_zeros(Ctx *c, const std::vector<int> &n, const std::vector<int> &r) {
  TT x;
  x.d = (int)n.size();
  x.n = n;
  x.r = r;
  x.core.resize(x.d);
  for (int k = 0; k < x.d; ++k) {
    x.core[k].alloc(c, x.csize(k));
    fill(c, x.core[k].p(), x.csize(k), 0.0);
  }
  return x;
}

TT tt_clone(Ctx *c, const TT &x) {
  TT y;
  y.d = x.d;
  y.n = x.n;
  y.r = x.r;
  y.mo = x.mo;
  y.mi = x.mi;
  y.core.resize(x.d);
  for (int k = 0; k < x.d; ++k) {
    y.core[k].alloc(c, x.csize(k));
    copy(c, y.core[k].p(), x.core[k].p(), x.csize(k));
  }
  return y;
}

TT tt_ones(Ctx *c, const std::vector<int> &n) {
  std::vector<int> r(n.size() + 1, 1);
  TT x = tt_zeros(c, n, r);
  for (int k = 0; k < x.d; ++k) fill(c, x.core[k].p(), x.csize(k), 1.0);
  return x;
}

// counter-based uniform(-1, 1) from the splitmix64 finaliser (Steele, Lea,
// Flood 2014) of (seed, index)
__global__ void random_kernel(double *p, size_t n, uint64_t seed) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    p[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}

TT tt_random(Ctx *c, const std::vector<int> &n, int rank, uint64_t seed) {
  const int d = (int)n.size();
  std::vector<int> r(d + 1, 1);
  // cap ranks by the sizes of the unfoldings so every bond is attainable
  for (int k = 1; k < d; ++k) {
    double left = 1, right = 1;
    for (int i = 0; i < k; ++i) left = std::min(left * n[i], 1e9);
    for (int i = k; i < d; ++i) right = std::min(right * n[i], 1e9);
    r[k] = (int)std::min<double>(rank, std::min(left, right));
  }
  TT x = tt_zeros(c, n, r);
  for (int k = 0; k < d; ++k) {
    random_kernel<<<64, 256, 0, c->stream>>>(x.core[k].p(), x.csize(k), seed * 1000003ull + k);
    c->count();
    TT_CHECK_CUDA(cudaGetLastError());
  }
  return x;
}

// ----------------------------------------------------------------- SVD / QR
int trunc_rank(const std::vector<double> &s, double delta, int rmax) {
  const int k = (int)s.size();
  int r = k;
  double tail = 0.0;
  // smallest r with ||s[r:]|| <= delta
  for (int i = k - 1; i >= 0; --i) {
    tail += s[i] * s[i];
    if (std::sqrt(tail) <= delta)
      r = i;
    else
      break;
  }
  if (rmax > 0) r = std::min(r, rmax);
  return std::max(1, r);
}

void qr_rm_from_t(Ctx *c, double *At, int m, int n, DBuf &Q, DBuf &R, int &k) {
  k = std::min(m, n);
  DBuf Qc(c, (size_t)m * k), Rc(c, (size_t)k * n);
  qr_colmajor(c, At, m, n, Qc.p(), Rc.p());
  // Qc col-major m x k == row-major k x m ; R col-major k x n == row-major n x k
  Q.ensure(c, (size_t)m * k);
  transpose(c, Qc.p(), Q.p(), k, m);
  R.ensure(c, (size_t)k * n);
  transpose(c, Rc.p(), R.p(), n, k);
}

// SVD of the small square R factor: mixed precision above 24 columns (FP32
// rotations refined by FP64 products), plain FP64 Jacobi below.  exact_u asks
// for U orthonormal to FP64 rounding (V is, otherwise).
static void small_svd(Ctx *c, double *R, int k, double *U, double *S, double *V, bool exact_u) {
  if (c->mixed_svd && k >= 24 && jacobi_svd_mixed_fits(k))
    jacobi_svd_mixed(c, R, k, U, S, V, exact_u);
  else
    jacobi_svd(c, R, k, U, S, V);
}

void svd_rm(Ctx *c, const double *A, int m, int n, SVD &o, int orth) {
  if (m <= 0 || n <= 0)
    throw Error(TT_EINVAL, "svd: empty matrix (" + std::to_string(m) + " x " + std::to_string(n) + ")");
  o.m = m;
  o.n = n;
  const int k = std::min(m, n);
  o.k = k;
  o.Ut.ensure(c, (size_t)k * m);
  o.Vt.ensure(c, (size_t)k * n);
  o.S.ensure(c, (size_t)k);
  DBuf work(c, (size_t)m * n), Q(c, (size_t)std::max(m, n) * k), Rm(c, (size_t)k * k);
  DBuf Ur(c, (size_t)k * k), Vr(c, (size_t)k * k);
  if (n >= m) {
    // X = A^T (n x m) column-major is A's memory: X = Q R, R = Ur S Vr^T
    // A = Vr S (Q Ur)^T  ->  Ut = Vr^T (Vr col-major memory), Vt = Ur^T Q^T
    copy(c, work.p(), A, (size_t)m * n);
    {
      PhaseTimer pt(c, "svd.qr");
      qr_colmajor(c, work.p(), n, m, Q.p(), Rm.p());
    }
    {
      PhaseTimer pt(c, "svd.small");
      small_svd(c, Rm.p(), k, Ur.p(), o.S.p(), Vr.p(), orth == SVD_ORTH_V);
    }
    copy(c, o.Ut.p(), Vr.p(), (size_t)k * k);
    // Vt (k x n row-major) = Ur^T (row-major view of Ur col-major: k x k) * Q^T (row-major view k x n)
    gemm(c, false, false, k, n, k, 1.0, Ur.p(), k, 0, Q.p(), n, 0, 0.0, o.Vt.p(), n, 0);
  } else {
    // A column-major = transpose of memory: A = Q R, R = Ur S Vr^T
    // A = (Q Ur) S Vr^T -> Ut = Ur^T Q^T, Vt = Vr^T (Vr col-major memory)
    transpose(c, A, work.p(), m, n);
    {
      PhaseTimer pt(c, "svd.qr");
      qr_colmajor(c, work.p(), m, n, Q.p(), Rm.p());
    }
    {
      PhaseTimer pt(c, "svd.small");
      small_svd(c, Rm.p(), k, Ur.p(), o.S.p(), Vr.p(), orth == SVD_ORTH_U);
    }
    gemm(c, false, false, k, m, k, 1.0, Ur.p(), k, 0, Q.p(), m, 0, 0.0, o.Ut.p(), m, 0);
    copy(c, o.Vt.p(), Vr.p(), (size_t)k * k);
  }
  o.Sh.resize(k);
  TT_CHECK_CUDA(cudaMemcpyAsync(c->h_pinned, o.S.p(), sizeof(double) * std::min(k, 4096), cudaMemcpyDeviceToHost,
                                c->stream));
  c->sync();
  for (int i = 0; i < std::min(k, 4096); ++i) o.Sh[i] = c->h_pinned[i];
  for (int i = 4096; i < k; ++i) o.Sh[i] = 0.0;
}

// ----------------------------------------------------------------- orthogonalisation
void orth_left(Ctx *c, TT &x, int upto) {
  for (int k = 0; k < upto && k < x.d - 1; ++k) {
    const int m = x.r[k] * x.n[k], nn = x.r[k + 1];
    DBuf At(c, (size_t)m * nn);
    transpose(c, x.core[k].p(), At.p(), m, nn);
    DBuf Q, R;
    int kk;
    qr_rm_from_t(c, At.p(), m, nn, Q, R, kk);
    // next core = R (kk x nn) * core_{k+1} (nn x n r2)
    const int cols = x.n[k + 1] * x.r[k + 2];
    DBuf nxt(c, (size_t)kk * cols);
    gemm(c, false, false, kk, cols, nn, 1.0, R.p(), nn, 0, x.core[k + 1].p(), cols, 0, 0.0, nxt.p(), cols, 0);
    Q.set_size((size_t)m * kk);
    x.core[k] = std::move(Q);
    x.core[k + 1] = std::move(nxt);
    x.r[k + 1] = kk;
  }
}

void orth_right(Ctx *c, TT &x, int downto) {
  for (int k = x.d - 1; k > downto && k > 0; --k) {
    const int m = x.r[k], nn = x.n[k] * x.r[k + 1];
    // core (m x nn) row-major; QR of its transpose (nn x m) whose column-major
    // storage is the core's memory: core^T = Q R -> core = R^T Q^T
    DBuf work(c, (size_t)m * nn);
    copy(c, work.p(), x.core[k].p(), (size_t)m * nn);
    const int kk = std::min(m, nn);
    DBuf Qc(c, (size_t)nn * kk), Rc(c, (size_t)kk * m);
    qr_colmajor(c, work.p(), nn, m, Qc.p(), Rc.p());
    // new core = Q^T (kk x nn row-major) = Qc memory; prev = prev * R^T
    // R col-major (kk x m) = row-major R^T (m x kk)
    const int rows = x.r[k - 1] * x.n[k - 1];
    DBuf prv(c, (size_t)rows * kk);
    gemm(c, false, false, rows, kk, m, 1.0, x.core[k - 1].p(), m, 0, Rc.p(), kk, 0, 0.0, prv.p(), kk, 0);
    Qc.set_size((size_t)kk * nn);
    x.core[k] = std::move(Qc);
    x.core[k - 1] = std::move(prv);
    x.r[k] = kk;
  }
}

void round(Ctx *c, TT &x, double eps, int rmax) {
  tt_check(x);
  if (x.d == 1) return;
  orth_left(c, x, x.d - 1);
  const double nrm = nrm2(c, x.core[x.d - 1].p(), x.csize(x.d - 1));
  const double delta = eps * nrm / std::sqrt((double)(x.d - 1));
  for (int k = x.d - 1; k >= 1; --k) {
    const int r0 = x.r[k], cols = x.n[k] * x.r[k + 1];
    SVD s;
    svd_rm(c, x.core[k].p(), r0, cols, s, SVD_ORTH_V);
    const int rk = trunc_rank(s.Sh, delta, rmax);
    DBuf nc(c, (size_t)rk * cols);
    copy(c, nc.p(), s.Vt.p(), (size_t)rk * cols);
    scale_rows(c, s.Ut.p(), rk, r0, s.S.p());
    const int rows = x.r[k - 1] * x.n[k - 1];
    DBuf prv(c, (size_t)rows * rk);
    // prev (rows x r0) * (Ut[:rk])^T (r0 x rk)
    gemm(c, false, true, rows, rk, r0, 1.0, x.core[k - 1].p(), r0, 0, s.Ut.p(), r0, 0, 0.0, prv.p(), rk, 0);
    x.core[k] = std::move(nc);
    x.core[k - 1] = std::move(prv);
    x.r[k] = rk;
  }
}

// ----------------------------------------------------------------- dot, sum, add
double dot(Ctx *c, const TT &x, const TT &y) {
  TT_REQUIRE(x.d == y.d, "dot: d mismatch");
  DBuf v(c, 1), t, v2;
  fill(c, v.p(), 1, 1.0);
  int rx = 1, ry = 1;
  for (int k = 0; k < x.d; ++k) {
    TT_REQUIRE(x.n[k] == y.n[k], "dot: mode mismatch");
    const int n = x.n[k], rx1 = x.r[k + 1], ry1 = y.r[k + 1];
    // t[b, (i a')] = sum_a v[a, b] x[a, (i a')]
    t.ensure(c, (size_t)ry * n * rx1);
    gemm(c, true, false, ry, n * rx1, rx, 1.0, v.p(), ry, 0, x.core[k].p(), n * rx1, 0, 0.0, t.p(), n * rx1, 0);
    // v'[a', b'] = sum_{b,i} t[(b i), a'] y[(b i), b']
    v2.ensure(c, (size_t)rx1 * ry1);
    gemm(c, true, false, rx1, ry1, ry * n, 1.0, t.p(), rx1, 0, y.core[k].p(), ry1, 0, 0.0, v2.p(), ry1, 0);
    v.swap(v2);
    rx = rx1;
    ry = ry1;
  }
  TT_CHECK_CUDA(cudaMemcpyAsync(c->h_pinned, v.p(), sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  c->sync();
  return c->h_pinned[0];
}

double norm(Ctx *c, const TT &x) {
  // orthogonalise a copy so the norm is the Frobenius norm of one core
  TT y = tt_clone(c, x);
  orth_left(c, y, y.d - 1);
  return nrm2(c, y.core[y.d - 1].p(), y.csize(y.d - 1));
}

double sum(Ctx *c, const TT &x) {
  TT o = tt_ones(c, x.n);
  return dot(c, x, o);
}

void scale(Ctx *c, TT &x, double a) { tt::scale(c, x.core[0].p(), x.csize(0), a); }

TT add(Ctx *c, double a, const TT &x, double b, const TT &y) {
  TT_REQUIRE(x.d == y.d, "add: d mismatch");
  for (int k = 0; k < x.d; ++k) TT_REQUIRE(x.n[k] == y.n[k], "add: mode mismatch");
  const int d = x.d;
  TT z;
  z.d = d;
  z.n = x.n;
  z.mo = x.mo;
  z.mi = x.mi;
  z.r.assign(d + 1, 1);
  for (int k = 1; k < d; ++k) z.r[k] = x.r[k] + y.r[k];
  z.core.resize(d);
  if (d == 1) {
    z.core[0].alloc(c, x.csize(0));
    copy(c, z.core[0].p(), y.core[0].p(), x.csize(0));
    axpby(c, x.csize(0), a, x.core[0].p(), b, z.core[0].p());
    return z;
  }
  for (int k = 0; k < d; ++k) {
    const int n = x.n[k];
    const size_t sz = z.csize(k);
    z.core[k].alloc(c, sz);
    fill(c, z.core[k].p(), sz, 0.0);
    const int zc = z.r[k + 1];
    if (k == 0) {
      copy2d(c, z.core[k].p(), zc, x.core[k].p(), x.r[1], n, x.r[1], a);
      copy2d(c, z.core[k].p() + x.r[1], zc, y.core[k].p(), y.r[1], n, y.r[1], b);
    } else if (k == d - 1) {
      copy(c, z.core[k].p(), x.core[k].p(), x.csize(k));
      copy(c, z.core[k].p() + x.csize(k), y.core[k].p(), y.csize(k));
    } else {
      copy2d(c, z.core[k].p(), zc, x.core[k].p(), x.r[k + 1], x.r[k] * n, x.r[k + 1]);
      copy2d(c, z.core[k].p() + (size_t)x.r[k] * n * zc + x.r[k + 1], zc, y.core[k].p(), y.r[k + 1],
             y.r[k] * n, y.r[k + 1]);
    }
  }
  return z;
}

// ----------------------------------------------------------------- operators on vectors
TT matvec_exact(Ctx *c, const TT &A, const TT &x) {
  TT_REQUIRE(A.is_matrix() && A.d == x.d, "matvec: operator/vector mismatch");
  TT y;
  y.d = x.d;
  y.n.resize(x.d);
  y.r.assign(x.d + 1, 1);
  y.core.resize(x.d);
  for (int k = 0; k < x.d; ++k) {
    TT_REQUIRE(A.mi[k] == x.n[k], "matvec: mode mismatch");
    y.n[k] = A.mo[k];
    y.r[k + 1] = A.r[k + 1] * x.r[k + 1];
  }
  for (int k = 0; k < x.d; ++k) {
    y.core[k].alloc(c, y.csize(k));
    kron_core(c, A.core[k].p(), A.r[k], A.mo[k], A.mi[k], A.r[k + 1], x.core[k].p(), x.r[k], x.r[k + 1],
              y.core[k].p());
  }
  return y;
}

TT transpose_op(Ctx *c, const TT &A) {
  TT B;
  B.d = A.d;
  B.r = A.r;
  B.mo = A.mi;
  B.mi = A.mo;
  B.n = A.n;
  B.core.resize(A.d);
  for (int k = 0; k < A.d; ++k) {
    B.core[k].alloc(c, A.csize(k));
    const int shape[4] = {A.r[k], A.mo[k], A.mi[k], A.r[k + 1]};
    const int perm[4] = {0, 2, 1, 3};
    permute(c, A.core[k].p(), B.core[k].p(), 4, shape, perm);
  }
  return B;
}

// A^T B of two TT matrices, core by core (ranks multiply):
//   C_k[(a, b), i, j, (a', b')] = sum_l A_k[a, l, i, a'] B_k[b, l, j, b'],
// one GEMM over the shared index l per core between the permuted cores
// A' (l; a i a') and B' (l; b j b'), then a permute of the product
// (a i a', b j b') into (a b, i, j, a' b').
TT op_matmul_tn(Ctx *c, const TT &A, const TT &B) {
  TT_REQUIRE(A.d == B.d && A.is_matrix() && B.is_matrix(), "op_matmul_tn: operands must be TT matrices of one d");
  const int d = A.d;
  TT C;
  C.d = d;
  C.r.resize(d + 1);
  C.mo.resize(d);
  C.mi.resize(d);
  C.n.resize(d);
  C.core.resize(d);
  for (int k = 0; k <= d; ++k) C.r[k] = A.r[k] * B.r[k];
  DBuf Ap, Bp, P;
  for (int k = 0; k < d; ++k) {
    TT_REQUIRE(A.mo[k] == B.mo[k], "op_matmul_tn: the shared (row) modes differ");
    const int ra = A.r[k], rb = B.r[k], ra1 = A.r[k + 1], rb1 = B.r[k + 1];
    const int L = A.mo[k], mi = A.mi[k], mj = B.mi[k];
    C.mo[k] = mi;
    C.mi[k] = mj;
    C.n[k] = mi * mj;
    const int shA[4] = {ra, L, mi, ra1}, shB[4] = {rb, L, mj, rb1};
    const int pl[4] = {1, 0, 2, 3};
    Ap.ensure(c, A.csize(k));
    Bp.ensure(c, B.csize(k));
    permute(c, A.core[k].p(), Ap.p(), 4, shA, pl);  // (l, a, i, a')
    permute(c, B.core[k].p(), Bp.p(), 4, shB, pl);  // (l, b, j, b')
    const int M = ra * mi * ra1, N = rb * mj * rb1;
    P.ensure(c, (size_t)M * N);
    gemm(c, true, false, M, N, L, 1.0, Ap.p(), M, 0, Bp.p(), N, 0, 0.0, P.p(), N, 0);
    // (a, i, a', b, j, b') -> (a, b, i, j, a', b')
    const int shP[6] = {ra, mi, ra1, rb, mj, rb1};
    const int pp[6] = {0, 3, 1, 4, 2, 5};
    C.core[k].alloc(c, (size_t)M * N);
    permute(c, P.p(), C.core[k].p(), 6, shP, pp);
  }
  return C;
}

void TTOp::prepare(Ctx *c) {
  if (prepared) return;
  a_ajib.resize(t.d);
  a_jbai.resize(t.d);
  for (int k = 0; k < t.d; ++k) {
    const int shape[4] = {t.r[k], t.mo[k], t.mi[k], t.r[k + 1]};
    a_ajib[k].alloc(c, t.csize(k));
    const int p1[4] = {0, 2, 1, 3};
    permute(c, t.core[k].p(), a_ajib[k].p(), 4, shape, p1);
    a_jbai[k].alloc(c, t.csize(k));
    const int p2[4] = {2, 3, 0, 1};
    permute(c, t.core[k].p(), a_jbai[k].p(), 4, shape, p2);
  }
  prepared = true;
}

void TTOp::prepare32(Ctx *c) {
  prepare(c);
  if (prepared32) return;
  a_ajib32.resize(t.d);
  for (int k = 0; k < t.d; ++k) {
    a_ajib32[k].alloc(c, (t.csize(k) + 1) / 2);
    d2f(c, a_ajib[k].p(), reinterpret_cast<float *>(a_ajib32[k].p()), t.csize(k));
  }
  prepared32 = true;
}

void to_dense(Ctx *c, const TT &x, double *dst, size_t len) {
  size_t total = 1;
  for (int k = 0; k < x.d; ++k) total *= (size_t)x.n[k];
  TT_REQUIRE(len >= total, "to_dense: destination too small");
  TT_REQUIRE(total <= (size_t)1 << 28, "to_dense: tensor too large");
  DBuf a(c, x.csize(0)), b;
  copy(c, a.p(), x.core[0].p(), x.csize(0));
  size_t rows = x.n[0];
  for (int k = 1; k < x.d; ++k) {
    const int rk = x.r[k], cols = x.n[k] * x.r[k + 1];
    b.ensure(c, rows * cols);
    // row blocks keep every GEMM launch inside its grid limit
    const size_t blk = (size_t)1 << 21;
    for (size_t r0 = 0; r0 < rows; r0 += blk) {
      const int mr = (int)std::min(blk, rows - r0);
      gemm(c, false, false, mr, cols, rk, 1.0, a.p() + r0 * rk, rk, 0, x.core[k].p(), cols, 0, 0.0,
           b.p() + r0 * cols, cols, 0);
    }
    a.swap(b);
    rows *= x.n[k];
  }
  copy(c, dst, a.p(), total);
}

TT tt_svd_dense(Ctx *c, const double *a, const std::vector<int> &modes, double eps, int rmax) {
  const int d = (int)modes.size();
  size_t total = 1;
  for (int m : modes) total *= (size_t)m;
  const double nrm = nrm2(c, a, total);
  const double delta = eps * nrm / std::sqrt((double)std::max(d - 1, 1));
  TT x;
  x.d = d;
  x.n = modes;
  x.r.assign(d + 1, 1);
  x.core.resize(d);
  DBuf cur(c, total);
  copy(c, cur.p(), a, total);
  int r = 1;
  size_t rest = total;
  for (int k = 0; k < d - 1; ++k) {
    const int rows = r * modes[k];
    rest /= (size_t)modes[k];
    TT_REQUIRE(rest <= (size_t)INT32_MAX, "tt_svd: unfolding too large");
    SVD s;
    svd_rm(c, cur.p(), rows, (int)rest, s, SVD_ORTH_U);
    const int rk = trunc_rank(s.Sh, delta, rmax);
    x.core[k].alloc(c, (size_t)rows * rk);
    transpose(c, s.Ut.p(), x.core[k].p(), rk, rows);
    DBuf nxt(c, (size_t)rk * rest);
    copy(c, nxt.p(), s.Vt.p(), (size_t)rk * rest);
    scale_rows(c, nxt.p(), rk, (int)rest, s.S.p());
    cur = std::move(nxt);
    x.r[k + 1] = rk;
    r = rk;
  }
  x.core[d - 1] = std::move(cur);
  return x;
}

}  // namespace tt
