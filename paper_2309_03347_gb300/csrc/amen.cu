// Alternating local solves over the TT cores (Sec. 3.5: the linear system of
// Eq. (linear_system_obj) and the product of Eq. (mv_obj) solved one core at
// a time, "AMEn" family), with the contractions of the local systems:
//
//   local matvec   y = Phi_L . A_k . Phi_R . x            (three GEMMs)
//   left update    Phi_L' = y^T . Phi_L . A_k . x          (three GEMMs)
//   right update   Phi_R' = y . A_k . x . Phi_R            (three GEMMs + 2 permutes)
//
// Interfaces: Phi (ry, RA, rx) for operator frames, Psi (ry, rb) for vector
// frames; all row-major.  The local systems are Galerkin projections onto the
// current interfaces (x left-orthogonal before core k, right-orthogonal
// after it) solved by restarted GMRES; the enrichment follows the residual
// of the current solution projected onto a low-rank TT z updated alongside.
#include <algorithm>

#include "tt.cuh"

namespace tt {

namespace {

double contraction_flops_local(int ry1, int R1, int rx1, int n, int m, int R2, int rx2, int ry2) {
  return 2.0 * ry1 * R1 * rx1 * n * rx2 + 2.0 * ry1 * m * R2 * rx2 * R1 * n + 2.0 * ry1 * m * ry2 * R2 * rx2;
}

// T1 = Phi_L (ry1 R1 x rx1) . x (rx1 x n rx2);  T2[a] = Ap^T . T1[a]  -> (ry1, m, R2, rx2)
void left_two_steps(Ctx *c, const double *PhiL, int ry1, int R1, int rx1, const double *Aajib, int m, int n,
                    int R2, const double *x, int rx2, DBuf &T1, DBuf &T2) {
  T1.ensure(c, (size_t)ry1 * R1 * n * rx2);
  gemm(c, false, false, ry1 * R1, n * rx2, rx1, 1.0, PhiL, rx1, 0, x, n * rx2, 0, 0.0, T1.p(), n * rx2, 0);
  T2.ensure(c, (size_t)ry1 * m * R2 * rx2);
  gemm(c, true, false, m * R2, rx2, R1 * n, 1.0, Aajib, m * R2, 0, T1.p(), rx2, (long long)R1 * n * rx2, 0.0,
       T2.p(), rx2, (long long)m * R2 * rx2, ry1);
}

}  // namespace

// y (ry1, m, ry2) = Phi_L (ry1, R1, rx1) A (R1, m, n, R2) Phi_R (ry2, R2, rx2) x (rx1, n, rx2)
void local_matvec(Ctx *c, const double *PhiL, const double *Aajib, const double *PhiR, const double *x, int ry1,
                  int R1, int rx1, int m, int n, int R2, int ry2, int rx2, double *y, DBuf &T1, DBuf &T2) {
  left_two_steps(c, PhiL, ry1, R1, rx1, Aajib, m, n, R2, x, rx2, T1, T2);
  gemm(c, false, true, ry1 * m, ry2, R2 * rx2, 1.0, T2.p(), R2 * rx2, 0, PhiR, R2 * rx2, 0, 0.0, y, ry2, 0);
  c->flops += contraction_flops_local(ry1, R1, rx1, n, m, R2, rx2, ry2);
}

// FP32 version of local_matvec (operands converted once per local system);
// tc selects the tcgen05 TF32 three-term GEMM instead of the FP32 SIMT GEMM
void local_matvec32(Ctx *c, const float *PhiL, const float *Aajib, const float *PhiR, const float *x, int ry1,
                    int R1, int rx1, int m, int n, int R2, int ry2, int rx2, float *y, DBuf &T1, DBuf &T2,
                    int tc = 0) {
  T1.ensure(c, ((size_t)ry1 * R1 * n * rx2 + 1) / 2);
  T2.ensure(c, ((size_t)ry1 * m * R2 * rx2 + 1) / 2);
  float *t1 = reinterpret_cast<float *>(T1.p()), *t2 = reinterpret_cast<float *>(T2.p());
  // tc: 0 FP32 SIMT GEMM, 1 tcgen05 TF32 three-term split, 2 tcgen05 BF16 three-term split
  auto g = [&](bool ta, bool tb, int M, int N, int K, float al, const float *A, int lda, long long sA, const float *B,
               int ldb, long long sB, float be, float *C, int ldc, long long sC, int batch) {
    if (tc)
      gemm_f32_tc(c, ta, tb, M, N, K, al, A, lda, sA, B, ldb, sB, be, C, ldc, sC, batch, tc == 2);
    else
      gemm_f32(c, ta, tb, M, N, K, al, A, lda, sA, B, ldb, sB, be, C, ldc, sC, batch);
  };
  g(false, false, ry1 * R1, n * rx2, rx1, 1.f, PhiL, rx1, 0, x, n * rx2, 0, 0.f, t1, n * rx2, 0, 1);
  g(true, false, m * R2, rx2, R1 * n, 1.f, Aajib, m * R2, 0, t1, rx2, (long long)R1 * n * rx2, 0.f, t2, rx2,
    (long long)m * R2 * rx2, ry1);
  g(false, true, ry1 * m, ry2, R2 * rx2, 1.f, t2, R2 * rx2, 0, PhiR, R2 * rx2, 0, 0.f, y, ry2, 0, 1);
  c->flops32 += contraction_flops_local(ry1, R1, rx1, n, m, R2, rx2, ry2);
}

// Phi_L' (ry2, R2, rx2) from Phi_L (ry1, R1, rx1), y (ry1, m, ry2), A, x (rx1, n, rx2)
void left_update(Ctx *c, const double *PhiL, const double *y, const double *Aajib, const double *x, int ry1,
                 int R1, int rx1, int m, int n, int R2, int ry2, int rx2, DBuf &out, DBuf &T1, DBuf &T2) {
  left_two_steps(c, PhiL, ry1, R1, rx1, Aajib, m, n, R2, x, rx2, T1, T2);
  out.ensure(c, (size_t)ry2 * R2 * rx2);
  gemm(c, true, false, ry2, R2 * rx2, ry1 * m, 1.0, y, ry2, 0, T2.p(), R2 * rx2, 0, 0.0, out.p(), R2 * rx2, 0);
  c->flops += contraction_flops_local(ry1, R1, rx1, n, m, R2, rx2, ry2);
}

// Phi_R' (ry1, R1, rx1) from Phi_R (ry2, R2, rx2), y (ry1, m, ry2), A, x (rx1, n, rx2)
void right_update(Ctx *c, const double *PhiR, const double *y, const double *Ajbai, const double *x, int ry1,
                  int R1, int rx1, int m, int n, int R2, int ry2, int rx2, DBuf &out, DBuf &T1, DBuf &T2) {
  // U1 [c][j][a'][b] = x (rx1 n x rx2) . Phi_R^T (rx2 x ry2 R2)
  T1.ensure(c, (size_t)rx1 * n * ry2 * R2);
  gemm(c, false, true, rx1 * n, ry2 * R2, rx2, 1.0, x, rx2, 0, PhiR, rx2, 0, 0.0, T1.p(), ry2 * R2, 0);
  // U1p [c][a'][j][b]
  T2.ensure(c, (size_t)rx1 * n * ry2 * R2);
  {
    const int shape[4] = {rx1, n, ry2, R2};
    const int perm[4] = {0, 2, 1, 3};
    permute(c, T1.p(), T2.p(), 4, shape, perm);
  }
  // U2 [c][a'][alpha][i] = U1p (rx1 ry2 x n R2) . Aq (n R2 x R1 m)
  T1.ensure(c, (size_t)rx1 * ry2 * R1 * m);
  gemm(c, false, false, rx1 * ry2, R1 * m, n * R2, 1.0, T2.p(), n * R2, 0, Ajbai, R1 * m, 0, 0.0, T1.p(), R1 * m,
       0);
  // U2p [i][a'][alpha][c]
  T2.ensure(c, (size_t)rx1 * ry2 * R1 * m);
  {
    const int shape[4] = {rx1, ry2, R1, m};
    const int perm[4] = {3, 1, 2, 0};
    permute(c, T1.p(), T2.p(), 4, shape, perm);
  }
  out.ensure(c, (size_t)ry1 * R1 * rx1);
  gemm(c, false, false, ry1, R1 * rx1, m * ry2, 1.0, y, m * ry2, 0, T2.p(), R1 * rx1, 0, 0.0, out.p(), R1 * rx1, 0);
  c->flops += 2.0 * rx1 * n * ry2 * R2 * rx2 + 2.0 * rx1 * ry2 * R1 * m * n * R2 + 2.0 * ry1 * R1 * rx1 * m * ry2;
}

// Psi_L' (ry2, rb2) from Psi_L (ry1, rb1), y (ry1, m, ry2), b (rb1, m, rb2)
void vleft_update(Ctx *c, const double *PsiL, const double *y, const double *b, int ry1, int rb1, int m, int ry2,
                  int rb2, DBuf &out, DBuf &T) {
  T.ensure(c, (size_t)ry1 * m * rb2);
  gemm(c, false, false, ry1, m * rb2, rb1, 1.0, PsiL, rb1, 0, b, m * rb2, 0, 0.0, T.p(), m * rb2, 0);
  out.ensure(c, (size_t)ry2 * rb2);
  gemm(c, true, false, ry2, rb2, ry1 * m, 1.0, y, ry2, 0, T.p(), rb2, 0, 0.0, out.p(), rb2, 0);
}

// Psi_R' (ry1, rb1) from Psi_R (ry2, rb2), y (ry1, m, ry2), b (rb1, m, rb2)
void vright_update(Ctx *c, const double *PsiR, const double *y, const double *b, int ry1, int rb1, int m, int ry2,
                   int rb2, DBuf &out, DBuf &T) {
  T.ensure(c, (size_t)rb1 * m * ry2);
  gemm(c, false, true, rb1 * m, ry2, rb2, 1.0, b, rb2, 0, PsiR, rb2, 0, 0.0, T.p(), ry2, 0);
  out.ensure(c, (size_t)ry1 * rb1);
  gemm(c, false, true, ry1, rb1, m * ry2, 1.0, y, m * ry2, 0, T.p(), m * ry2, 0, 0.0, out.p(), rb1, 0);
}

// rhs (ry1, m, ry2) = Psi_L (ry1, rb1) b (rb1, m, rb2) Psi_R^T (rb2, ry2)
void vlocal(Ctx *c, const double *PsiL, const double *b, const double *PsiR, int ry1, int rb1, int m, int rb2,
            int ry2, double *out, DBuf &T) {
  T.ensure(c, (size_t)ry1 * m * rb2);
  gemm(c, false, false, ry1, m * rb2, rb1, 1.0, PsiL, rb1, 0, b, m * rb2, 0, 0.0, T.p(), m * rb2, 0);
  gemm(c, false, true, ry1 * m, ry2, rb2, 1.0, T.p(), rb2, 0, PsiR, rb2, 0, 0.0, out, ry2, 0);
}

namespace {

// ----------------------------------------------------------------- local GMRES
struct Gmres {
  int restart = 30;
  int maxit = 300;
  DBuf V, hbuf, r, y;
  std::vector<double> H, cs, sn, g, hh;
};

// Solve M x = b (N unknowns) by restarted GMRES with classical Gram-Schmidt
// applied twice; x holds the initial guess.  Returns iterations.
template <class MV>
int gmres(Ctx *c, Gmres &G, MV &&mv, const double *b, double *x, size_t N, double tol) {
  const int mr = G.restart;
  G.V.ensure(c, (size_t)(mr + 1) * N);
  G.hbuf.ensure(c, (size_t)2 * (mr + 1) + 4);
  G.r.ensure(c, N);
  G.y.ensure(c, (size_t)mr + 1);
  G.H.assign((size_t)(mr + 1) * mr, 0.0);
  G.cs.assign(mr, 0.0);
  G.sn.assign(mr, 0.0);
  G.g.assign(mr + 1, 0.0);
  const double nb = nrm2(c, b, N);
  if (nb == 0.0) {
    fill(c, x, N, 0.0);
    return 0;
  }
  int it = 0;
  double *hd = G.hbuf.p();
  double *hp = c->h_pinned;
  while (true) {
    mv(x, G.r.p());
    axpby(c, N, 1.0, b, -1.0, G.r.p());  // r = b - A x
    const double beta = nrm2(c, G.r.p(), N);
    if (!(beta > tol * nb) || it >= G.maxit) return it;
    double *V = G.V.p();
    axpby(c, N, 1.0 / beta, G.r.p(), 0.0, V);
    std::fill(G.g.begin(), G.g.end(), 0.0);
    G.g[0] = beta;
    int jend = -1;
    double res = beta;
    for (int j = 0; j < mr; ++j) {
      double *w = V + (size_t)(j + 1) * N;
      mv(V + (size_t)j * N, w);
      ++it;
      multi_dot(c, V, N, j + 1, w, N, hd);
      multi_axpy(c, V, N, j + 1, hd, w, N);
      multi_dot(c, V, N, j + 1, w, N, hd + (mr + 1));
      multi_axpy(c, V, N, j + 1, hd + (mr + 1), w, N);
      dot_dev(c, w, w, N, hd + 2 * (mr + 1));
      TT_CHECK_CUDA(cudaMemcpyAsync(hp, hd, sizeof(double) * (2 * (mr + 1) + 1), cudaMemcpyDeviceToHost,
                                    c->stream));
      c->sync();
      const double hn = std::sqrt(std::max(hp[2 * (mr + 1)], 0.0));
      double *Hc = &G.H[0];
      for (int i = 0; i <= j; ++i) Hc[(size_t)i * mr + j] = hp[i] + hp[(mr + 1) + i];
      Hc[(size_t)(j + 1) * mr + j] = hn;
      if (!std::isfinite(hn)) throw Error(TT_ENONFINITE, "gmres: non-finite Krylov vector");
      // apply previous rotations
      for (int i = 0; i < j; ++i) {
        const double a = Hc[(size_t)i * mr + j], bb = Hc[(size_t)(i + 1) * mr + j];
        Hc[(size_t)i * mr + j] = G.cs[i] * a + G.sn[i] * bb;
        Hc[(size_t)(i + 1) * mr + j] = -G.sn[i] * a + G.cs[i] * bb;
      }
      const double a = Hc[(size_t)j * mr + j], bb = Hc[(size_t)(j + 1) * mr + j];
      const double den = std::hypot(a, bb);
      G.cs[j] = den == 0.0 ? 1.0 : a / den;
      G.sn[j] = den == 0.0 ? 0.0 : bb / den;
      Hc[(size_t)j * mr + j] = den;
      Hc[(size_t)(j + 1) * mr + j] = 0.0;
      G.g[j + 1] = -G.sn[j] * G.g[j];
      G.g[j] = G.cs[j] * G.g[j];
      res = std::fabs(G.g[j + 1]);
      jend = j;
      const bool breakdown = hn <= 1e-300;
      if (!breakdown) scale(c, w, N, 1.0 / hn);
      if (res <= tol * nb || it >= G.maxit || breakdown) break;
    }
    // back substitution H y = g
    const int kk = jend + 1;
    std::vector<double> yv(kk, 0.0);
    for (int i = kk - 1; i >= 0; --i) {
      double s = G.g[i];
      for (int l = i + 1; l < kk; ++l) s -= G.H[(size_t)i * mr + l] * yv[l];
      const double dgl = G.H[(size_t)i * mr + i];
      yv[i] = dgl != 0.0 ? s / dgl : 0.0;
    }
    for (int i = 0; i < kk; ++i) hp[i] = -yv[i];
    TT_CHECK_CUDA(cudaMemcpyAsync(G.y.p(), hp, sizeof(double) * kk, cudaMemcpyHostToDevice, c->stream));
    multi_axpy(c, V, N, kk, G.y.p(), x, N);  // x += V y
    c->sync();
    if (res <= tol * nb || it >= G.maxit) {
      return it;
    }
  }
}

// FP32 GMRES for the correction equation of the iterative refinement:
// M d = b with ||b|| = 1, d starts at zero.  Same algorithm as gmres().
struct Gmres32 {
  int restart = 30;
  int maxit = 300;
  DBuf V, r, dev;
  std::vector<cudaEvent_t> ev;
  Gmres32() = default;
  Gmres32(const Gmres32 &) = delete;
  Gmres32 &operator=(const Gmres32 &) = delete;
  ~Gmres32() {
    for (auto e : ev) cudaEventDestroy(e);
  }
};

// Restarted GMRES in FP32 (classical Gram-Schmidt applied twice) for the
// correction equation of the iterative refinement.  The Arnoldi state (H,
// Givens rotations, residual estimate) lives on the device; the host queues
// step j + 1 before it waits for the residual of step j, so the device runs
// the steps back to back.  A step queued after convergence is discarded
// (only columns up to the converged one enter the solution).  Returns the
// number of steps run.
template <class MV>
int gmres32(Ctx *c, Gmres32 &G, MV &&mv, const float *b, float *x, size_t N, double tol) {
  const int mr = G.restart;
  TT_REQUIRE(mr + 1 <= KRY_MAX_VECS && 2 * mr + 2 <= 1024, "gmres32: restart too long");
  G.V.ensure(c, ((size_t)(mr + 1) * N + 1) / 2);
  G.r.ensure(c, (N + 1) / 2);
  // device state: H, cs, sn, g, y, st, inv, h1, h2, part1, part2, npart
  const size_t oH = 0, ocs = oH + (size_t)(mr + 1) * mr, osn = ocs + mr, og = osn + mr, oy = og + mr + 1,
               ost = oy + mr + 1, oinv = ost + 2 * mr + 2, oh1 = oinv + 1, oh2 = oh1 + mr + 1, op1 = oh2 + mr + 1,
               op2 = op1 + (size_t)(mr + 1) * KRY_MAX_SPLIT, onp = op2 + (size_t)(mr + 1) * KRY_MAX_SPLIT,
               total = onp + (size_t)c->sm_count * 4 + 1;
  G.dev.ensure(c, total);
  while ((int)G.ev.size() < mr) {
    cudaEvent_t e;
    TT_CHECK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    G.ev.push_back(e);
  }
  double *D = G.dev.p();
  double *H = D + oH, *cs = D + ocs, *sn = D + osn, *g = D + og, *y = D + oy, *st = D + ost, *inv = D + oinv,
         *h1 = D + oh1, *h2 = D + oh2, *p1 = D + op1, *p2 = D + op2, *np = D + onp;
  float *V = reinterpret_cast<float *>(G.V.p());
  float *r = reinterpret_cast<float *>(G.r.p());
  double *hp = c->h_pinned + 2048;  // landing area of the per-step status (2 mr + 2 doubles)
  int it = 0;
  TT_CHECK_CUDA(cudaMemsetAsync(x, 0, N * sizeof(float), c->stream));
  auto step = [&](int j) {
    float *w = V + (size_t)(j + 1) * N;
    mv(V + (size_t)j * N, w);
    int S = kry_mdot(c, V, N, j + 1, w, N, p1);
    kry_maxpy(c, V, N, j + 1, p1, S, w, N, h1, nullptr);
    S = kry_mdot(c, V, N, j + 1, w, N, p2);
    const int nb = kry_maxpy(c, V, N, j + 1, p2, S, w, N, h2, np);
    kry_arnoldi(c, j, mr, h1, h2, np, nb, H, cs, sn, g, st, inv);
    kry_scale(c, w, w, N, inv);
    TT_CHECK_CUDA(cudaMemcpyAsync(hp + 2 * j, st + 2 * j, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    TT_CHECK_CUDA(cudaEventRecord(G.ev[j], c->stream));
  };
  // true when step j ended the cycle (converged or broke down)
  auto finished = [&](int j) {
    TT_CHECK_CUDA(cudaEventSynchronize(G.ev[j]));
    const double res = hp[2 * j], hn = hp[2 * j + 1];
    if (!std::isfinite(hn) || !std::isfinite(res)) throw Error(TT_ENONFINITE, "gmres32: non-finite Krylov vector");
    return res <= tol || hn <= 1e-30;
  };
  while (true) {
    // r = b - M x ; beta = ||r||
    mv(x, r);
    axpby_f(c, N, 1.f, b, -1.f, r);
    const int nb = kry_sumsq(c, r, N, np);
    kry_start(c, np, nb, mr, g, st, inv);
    TT_CHECK_CUDA(cudaMemcpyAsync(hp + 2 * mr, st, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    c->sync();
    const double beta = hp[2 * mr];
    if (!std::isfinite(beta)) throw Error(TT_ENONFINITE, "gmres32: non-finite residual");
    if (!(beta > tol) || it >= G.maxit) return it;
    kry_scale(c, r, V, N, inv);
    int jend = 0;
    bool done = false;
    step(0);
    ++it;
    for (int j = 0; j < mr; ++j) {
      const bool more = j + 1 < mr && it < G.maxit;
      if (more) {
        step(j + 1);
        ++it;
      }
      const bool fin = finished(j);
      if (fin || !more) {
        jend = j;
        done = fin || it >= G.maxit;
        break;
      }
    }
    // x += V y,  y = H^-1 g over the columns 0..jend
    kry_trisolve(c, jend + 1, mr, H, g, y);
    multi_axpy_f(c, V, N, jend + 1, y, x, N);
    if (done) {
      c->sync();
      return it;
    }
  }
}

// The local system of one core (or of a merged pair of cores): Galerkin
// projection (Phi_L, A, Phi_R) with square ranks r0 x m x r1, solved to the
// relative residual tol from the initial guess in sol.  FP64 GMRES, or FP32
// Krylov corrections inside FP64 iterative refinement (TT_FP32_REFINED: SIMT
// contractions, one persistent GMRES kernel per correction when it fits;
// TT_TF32_SPLIT / TT_BF16_SPLIT: tcgen05 contractions).  A32: FP32 copy of the
// operator core (a_ajib layout) for the mixed precisions.
struct LocalSolver {
  Gmres G;
  Gmres32 G32;
  PGWork PGW;
  DBuf PL32, PR32, r32, d32, r64, T1, T2;

  long long solve(Ctx *c, int prec, const double *PL, const double *A, const float *A32, const double *PR, int r0,
                  int R1, int m, int R2, int r1, const double *rhs, double *sol, double tol) {
    const size_t N = (size_t)r0 * m * r1;
    auto mv = [&](const double *in, double *out) {
      local_matvec(c, PL, A, PR, in, r0, R1, r0, m, m, R2, r1, r1, out, T1, T2);
    };
    const bool use_tc = prec == TT_TF32_SPLIT || prec == TT_BF16_SPLIT;
    const int tc_kind = prec == TT_BF16_SPLIT ? 2 : (use_tc ? 1 : 0);
    if (prec == TT_FP64) {
      PhaseTimer pt(c, "solve.gmres");
      return gmres(c, G, mv, rhs, sol, N, tol);
    }
    // iterative refinement: FP64 residual, FP32 GMRES for the correction
    PhaseTimer pt(c, "solve.gmres_mixed");
    long long git = 0;
    const size_t nl = (size_t)r0 * R1 * r0, nr = (size_t)r1 * R2 * r1;
    PL32.ensure(c, (nl + 1) / 2);
    PR32.ensure(c, (nr + 1) / 2);
    float *pl32 = reinterpret_cast<float *>(PL32.p()), *pr32 = reinterpret_cast<float *>(PR32.p());
    d2f(c, PL, pl32, nl);
    d2f(c, PR, pr32, nr);
    auto mv32 = [&](const float *in, float *out) {
      local_matvec32(c, pl32, A32, pr32, in, r0, R1, r0, m, m, R2, r1, r1, out, T1, T2, tc_kind);
    };
    r32.ensure(c, (N + 1) / 2);
    d32.ensure(c, (N + 1) / 2);
    r64.ensure(c, N);
    float *r32p = reinterpret_cast<float *>(r32.p()), *d32p = reinterpret_cast<float *>(d32.p());
    const double nb = nrm2(c, rhs, N);
    for (int ref = 0; ref < 6 && nb > 0; ++ref) {
      mv(sol, r64.p());
      axpby(c, N, 1.0, rhs, -1.0, r64.p());
      const double nrr = nrm2(c, r64.p(), N);
      if (!(nrr > tol * nb)) break;
      d2f(c, r64.p(), r32p, N, 1.0 / nrr);
      // inner tolerance: the product's own accuracy bounds what the FP32 Krylov can reach
      const double tol_in = std::max(0.3 * tol * nb / nrr, prec == TT_BF16_SPLIT ? 3e-5 : 2e-6);
      if (!use_tc && c->persistent_gmres && pgmres32_fits(c, (int)N, G32.restart))
        git += pgmres32(c, pl32, A32, pr32, r0, R1, m, R2, r1, r32p, d32p, tol_in, G32.restart, G32.maxit, PGW);
      else
        git += gmres32(c, G32, mv32, r32p, d32p, N, tol_in);
      f2d_axpy(c, d32p, sol, N, nrr);
    }
    return git;
  }
};

struct Iface {
  std::vector<DBuf> L, R;
  void init(Ctx *c, int d) {
    L.clear();
    R.clear();
    L.resize(d + 1);
    R.resize(d + 1);
    L[0].alloc(c, 1);
    fill(c, L[0].p(), 1, 1.0);
    R[d].alloc(c, 1);
    fill(c, R[d].p(), 1, 1.0);
  }
};

// residual-enrichment split of a local solution (left-to-right sweep):
// sol (r0 n x r1) -> truncated u v, enriched with crz (r0 n x rz) and
// orthonormalised; x_k <- Q, x_{k+1} <- (R [v; 0]) x_{k+1}.
void split_enrich(Ctx *c, TT &x, int k, const SVD &s, int rk, const double *crz, int rz) {
  const int r0 = x.r[k], n = x.n[k], r1 = x.r[k + 1];
  const int rows = r0 * n;
  // ukT = [Ut[:rk]; crz^T]  ((rk + rz) x rows) = column-major (rows x (rk+rz))
  const int cols = rk + rz;
  DBuf ukT(c, (size_t)cols * rows);
  copy(c, ukT.p(), s.Ut.p(), (size_t)rk * rows);
  if (rz > 0) transpose(c, crz, ukT.p() + (size_t)rk * rows, rows, rz);
  DBuf Q, R;
  int kk;
  qr_rm_from_t(c, ukT.p(), rows, cols, Q, R, kk);
  // v = S Vt[:rk]  (rk x r1)
  DBuf v(c, (size_t)rk * r1);
  copy(c, v.p(), s.Vt.p(), (size_t)rk * r1);
  scale_rows(c, v.p(), rk, r1, s.S.p());
  // vnew = R[:, :rk] v   (kk x r1);  R row-major kk x cols
  DBuf vnew(c, (size_t)kk * r1);
  gemm(c, false, false, kk, r1, rk, 1.0, R.p(), cols, 0, v.p(), r1, 0, 0.0, vnew.p(), r1, 0);
  const int ncols = x.n[k + 1] * x.r[k + 2];
  DBuf nxt(c, (size_t)kk * ncols);
  gemm(c, false, false, kk, ncols, r1, 1.0, vnew.p(), r1, 0, x.core[k + 1].p(), ncols, 0, 0.0, nxt.p(), ncols, 0);
  Q.set_size((size_t)rows * kk);
  x.core[k] = std::move(Q);
  x.core[k + 1] = std::move(nxt);
  x.r[k + 1] = kk;
}

// QR-orthonormalise a (r0 n x r1) core block in place keeping its column count
void orth_core_cols(Ctx *c, TT &z, int k, const double *blk) {
  const int r0 = z.r[k], n = z.n[k], r1 = z.r[k + 1];
  const int rows = r0 * n;
  DBuf At(c, (size_t)rows * r1);
  transpose(c, blk, At.p(), rows, r1);
  DBuf Q, R;
  int kk;
  qr_rm_from_t(c, At.p(), rows, r1, Q, R, kk);
  DBuf out(c, (size_t)rows * r1);
  fill(c, out.p(), (size_t)rows * r1, 0.0);
  copy2d(c, out.p(), r1, Q.p(), kk, rows, kk);
  z.core[k] = std::move(out);
}

}  // namespace

void amen_solve(Ctx *c, TTOp &Aop, const TT &b, TT &x, double eps, int rmax, int nswp, int kick, uint64_t seed,
                SolveStats *st, int prec, TTOp *rhs_op) {
  TT &A = Aop.t;
  Aop.prepare(c);
  if (rhs_op) rhs_op->prepare(c);
  const bool use_tc = prec == TT_TF32_SPLIT || prec == TT_BF16_SPLIT;
  const bool mixed = prec == TT_FP32_REFINED || use_tc;
  if (mixed) Aop.prepare32(c);
  if (use_tc) TT_CHECK_CUDA(cudaMemsetAsync(c->d_scalar + 8, 0, sizeof(int), c->stream));
  const int d = A.d;
  TT_REQUIRE(b.d == d && x.d == d, "amen_solve: dimension mismatch");
  for (int k = 0; k < d; ++k)
    TT_REQUIRE(A.mo[k] == A.mi[k] && A.mi[k] == x.n[k] && b.n[k] == x.n[k], "amen_solve: mode mismatch");
  if (rhs_op)
    for (int k = 0; k < d; ++k)
      TT_REQUIRE(rhs_op->t.d == d && rhs_op->t.mo[k] == x.n[k] && rhs_op->t.mi[k] == b.n[k],
                 "amen_solve: rhs operator mode mismatch");
  DBuf T1, T2, T3;
  // Right-hand-side pieces through the frames y (x or z): plain b (interfaces
  // y'b, (r_y, r_b)) or rhs_op b (interfaces y' rhs_op b, (r_y, R, r_b)).
  auto rhs_local = [&](int k, const double *L, const double *R, int ry0, int ry1, double *out) {
    if (!rhs_op)
      vlocal(c, L, b.core[k].p(), R, ry0, b.r[k], b.n[k], b.r[k + 1], ry1, out, T3);
    else
      local_matvec(c, L, rhs_op->a_ajib[k].p(), R, b.core[k].p(), ry0, rhs_op->t.r[k], b.r[k], x.n[k], b.n[k],
                   rhs_op->t.r[k + 1], ry1, b.r[k + 1], out, T1, T2);
  };
  auto rhs_left = [&](int k, const double *L, const double *y, int ry0, int ry1, DBuf &out) {
    if (!rhs_op)
      vleft_update(c, L, y, b.core[k].p(), ry0, b.r[k], x.n[k], ry1, b.r[k + 1], out, T3);
    else
      left_update(c, L, y, rhs_op->a_ajib[k].p(), b.core[k].p(), ry0, rhs_op->t.r[k], b.r[k], x.n[k], b.n[k],
                  rhs_op->t.r[k + 1], ry1, b.r[k + 1], out, T1, T2);
  };
  auto rhs_right = [&](int k, const double *R, const double *y, int ry0, int ry1, DBuf &out) {
    if (!rhs_op)
      vright_update(c, R, y, b.core[k].p(), ry0, b.r[k], x.n[k], ry1, b.r[k + 1], out, T3);
    else
      right_update(c, R, y, rhs_op->a_jbai[k].p(), b.core[k].p(), ry0, rhs_op->t.r[k], b.r[k], x.n[k], b.n[k],
                   rhs_op->t.r[k + 1], ry1, b.r[k + 1], out, T1, T2);
  };
  const double loc_eps = eps / std::sqrt((double)d);
  TT z = tt_random(c, x.n, std::max(kick, 1), seed);
  orth_right(c, x, 0);
  orth_right(c, z, 0);
  Iface PX, QX, PZ, QZ;  // x'Ax, x'b, z'Ax, z'b
  PX.init(c, d);
  QX.init(c, d);
  PZ.init(c, d);
  QZ.init(c, d);
  auto right_all = [&]() {
    for (int k = d - 1; k >= 1; --k) {
      const int m = x.n[k], R1 = A.r[k], R2 = A.r[k + 1];
      right_update(c, PX.R[k + 1].p(), x.core[k].p(), Aop.a_jbai[k].p(), x.core[k].p(), x.r[k], R1, x.r[k], m, m,
                   R2, x.r[k + 1], x.r[k + 1], PX.R[k], T1, T2);
      rhs_right(k, QX.R[k + 1].p(), x.core[k].p(), x.r[k], x.r[k + 1], QX.R[k]);
      right_update(c, PZ.R[k + 1].p(), z.core[k].p(), Aop.a_jbai[k].p(), x.core[k].p(), z.r[k], R1, x.r[k], m, m,
                   R2, z.r[k + 1], x.r[k + 1], PZ.R[k], T1, T2);
      rhs_right(k, QZ.R[k + 1].p(), z.core[k].p(), z.r[k], z.r[k + 1], QZ.R[k]);
    }
  };
  right_all();
  LocalSolver LS;
  DBuf rhs, sol, solt, crz, czz, tmp;
  double maxdx = 0.0;
  int swp = 0;
  long long git = 0;
  for (swp = 0; swp < nswp; ++swp) {
    maxdx = 0.0;
    for (int k = 0; k < d; ++k) {
      const int m = x.n[k], R1 = A.r[k], R2 = A.r[k + 1];
      const int r0 = x.r[k], r1 = x.r[k + 1];
      const size_t N = (size_t)r0 * m * r1;
      rhs.ensure(c, N);
      rhs_local(k, QX.L[k].p(), QX.R[k + 1].p(), r0, r1, rhs.p());
      sol.ensure(c, N);
      copy(c, sol.p(), x.core[k].p(), N);
      git += LS.solve(c, prec, PX.L[k].p(), Aop.a_ajib[k].p(),
                      mixed ? reinterpret_cast<const float *>(Aop.a_ajib32[k].p()) : nullptr, PX.R[k + 1].p(), r0,
                      R1, m, R2, r1, rhs.p(), sol.p(), loc_eps);
      // relative change of the local solution
      tmp.ensure(c, N);
      copy(c, tmp.p(), sol.p(), N);
      axpby(c, N, -1.0, x.core[k].p(), 1.0, tmp.p());
      const double ns = nrm2(c, sol.p(), N);
      const double dx = ns > 0 ? nrm2(c, tmp.p(), N) / ns : 0.0;
      if (!std::isfinite(dx)) throw Error(TT_ENONFINITE, "amen_solve: non-finite local solution");
      maxdx = std::max(maxdx, dx);
      if (k == d - 1) {
        copy(c, x.core[k].p(), sol.p(), N);
        break;
      }
      SVD s;
      {
        PhaseTimer pt(c, "amen.svd");
        svd_rm(c, sol.p(), r0 * m, r1, s, SVD_ORTH_ANY);
      }
      double sn2 = 0;
      for (double v : s.Sh) sn2 += v * v;
      const int rk = trunc_rank(s.Sh, loc_eps * std::sqrt(sn2), rmax);
      // truncated solution solt = U[:, :rk] S Vt[:rk] = Ut[:rk]^T (S Vt[:rk])
      DBuf v(c, (size_t)rk * r1);
      copy(c, v.p(), s.Vt.p(), (size_t)rk * r1);
      scale_rows(c, v.p(), rk, r1, s.S.p());
      solt.ensure(c, N);
      gemm(c, true, false, r0 * m, r1, rk, 1.0, s.Ut.p(), r0 * m, 0, v.p(), r1, 0, 0.0, solt.p(), r1, 0);
      const int rz0 = z.r[k], rz1 = z.r[k + 1];
      if (kick <= 0) {
        // one-site ALS: no residual enrichment, the truncated solution alone
        split_enrich(c, x, k, s, rk, nullptr, 0);
        const int nr1 = x.r[k + 1];
        left_update(c, PX.L[k].p(), x.core[k].p(), Aop.a_ajib[k].p(), x.core[k].p(), r0, R1, r0, m, m, R2, nr1, nr1,
                    PX.L[k + 1], T1, T2);
        rhs_left(k, QX.L[k].p(), x.core[k].p(), r0, nr1, QX.L[k + 1]);
        left_update(c, PZ.L[k].p(), z.core[k].p(), Aop.a_ajib[k].p(), x.core[k].p(), rz0, R1, r0, m, m, R2, rz1, nr1,
                    PZ.L[k + 1], T1, T2);
        rhs_left(k, QZ.L[k].p(), z.core[k].p(), rz0, rz1, QZ.L[k + 1]);
        continue;
      }
      PhaseTimer pt_res(c, "amen.residual");
      // crz = x'b z - x'Ax z . solt     (r0, m, rz1)
      crz.ensure(c, (size_t)r0 * m * rz1);
      rhs_local(k, QX.L[k].p(), QZ.R[k + 1].p(), r0, rz1, crz.p());
      tmp.ensure(c, (size_t)r0 * m * rz1);
      local_matvec(c, PX.L[k].p(), Aop.a_ajib[k].p(), PZ.R[k + 1].p(), solt.p(), r0, R1, r0, m, m, R2, rz1, r1,
                   tmp.p(), T1, T2);
      axpby(c, (size_t)r0 * m * rz1, -1.0, tmp.p(), 1.0, crz.p());
      // czz = z'b z - z'Ax z . solt     (rz0, m, rz1)
      czz.ensure(c, (size_t)rz0 * m * rz1);
      rhs_local(k, QZ.L[k].p(), QZ.R[k + 1].p(), rz0, rz1, czz.p());
      tmp.ensure(c, (size_t)rz0 * m * rz1);
      local_matvec(c, PZ.L[k].p(), Aop.a_ajib[k].p(), PZ.R[k + 1].p(), solt.p(), rz0, R1, r0, m, m, R2, rz1, r1,
                   tmp.p(), T1, T2);
      axpby(c, (size_t)rz0 * m * rz1, -1.0, tmp.p(), 1.0, czz.p());
      {
        PhaseTimer pt(c, "amen.enrich_qr");
        orth_core_cols(c, z, k, czz.p());
        split_enrich(c, x, k, s, rk, crz.p(), rz1);
      }
      const int nr1 = x.r[k + 1];
      PhaseTimer pt_if(c, "amen.iface");
      left_update(c, PX.L[k].p(), x.core[k].p(), Aop.a_ajib[k].p(), x.core[k].p(), r0, R1, r0, m, m, R2, nr1, nr1,
                  PX.L[k + 1], T1, T2);
      rhs_left(k, QX.L[k].p(), x.core[k].p(), r0, nr1, QX.L[k + 1]);
      left_update(c, PZ.L[k].p(), z.core[k].p(), Aop.a_ajib[k].p(), x.core[k].p(), rz0, R1, r0, m, m, R2, rz1, nr1,
                  PZ.L[k + 1], T1, T2);
      rhs_left(k, QZ.L[k].p(), z.core[k].p(), rz0, rz1, QZ.L[k + 1]);
    }
    if (maxdx < eps) {
      ++swp;
      break;
    }
    if (swp + 1 < nswp) {
      PhaseTimer pt(c, "amen.reorth_ifaces");
      orth_right(c, x, 0);
      orth_right(c, z, 0);
      right_all();
    }
  }
  if (use_tc && tc_error_flag(c))
    throw Error(TT_ETIMEOUT, "amen_solve: a tensor-core GEMM gave up waiting for its MMAs");
  if (st) {
    st->sweeps = std::min(swp, nswp);
    st->max_dx = maxdx;
    st->gmres_iters = git;
  }
}

void amen_mv(Ctx *c, TTOp &Aop, const TT &xin, TT &y, double eps, int rmax, int nswp, int kick, uint64_t seed,
             SolveStats *st) {
  TT &A = Aop.t;
  Aop.prepare(c);
  const int d = A.d;
  TT_REQUIRE(xin.d == d && y.d == d, "amen_mv: dimension mismatch");
  for (int k = 0; k < d; ++k)
    TT_REQUIRE(A.mi[k] == xin.n[k] && A.mo[k] == y.n[k], "amen_mv: mode mismatch");
  const double loc_eps = eps / std::sqrt((double)d);
  TT z = tt_random(c, y.n, std::max(kick, 1), seed);
  orth_right(c, y, 0);
  orth_right(c, z, 0);
  Iface PY, PZ, YZ, ZY;  // y'Ax, z'Ax, (y,z) right, (z,y) left
  PY.init(c, d);
  PZ.init(c, d);
  YZ.init(c, d);
  ZY.init(c, d);
  DBuf T1, T2, T3;
  auto right_all = [&]() {
    for (int k = d - 1; k >= 1; --k) {
      const int m = A.mo[k], n = A.mi[k], R1 = A.r[k], R2 = A.r[k + 1];
      right_update(c, PY.R[k + 1].p(), y.core[k].p(), Aop.a_jbai[k].p(), xin.core[k].p(), y.r[k], R1, xin.r[k], m,
                   n, R2, y.r[k + 1], xin.r[k + 1], PY.R[k], T1, T2);
      right_update(c, PZ.R[k + 1].p(), z.core[k].p(), Aop.a_jbai[k].p(), xin.core[k].p(), z.r[k], R1, xin.r[k], m,
                   n, R2, z.r[k + 1], xin.r[k + 1], PZ.R[k], T1, T2);
      vright_update(c, YZ.R[k + 1].p(), y.core[k].p(), z.core[k].p(), y.r[k], z.r[k], m, y.r[k + 1], z.r[k + 1],
                    YZ.R[k], T3);
    }
  };
  right_all();
  DBuf sol, solt, crz, czz, tmp, tmp2;
  double maxdx = 0.0;
  int swp = 0;
  for (swp = 0; swp < nswp; ++swp) {
    maxdx = 0.0;
    for (int k = 0; k < d; ++k) {
      const int m = A.mo[k], n = A.mi[k], R1 = A.r[k], R2 = A.r[k + 1];
      const int r0 = y.r[k], r1 = y.r[k + 1], q0 = xin.r[k], q1 = xin.r[k + 1];
      const size_t N = (size_t)r0 * m * r1;
      sol.ensure(c, N);
      local_matvec(c, PY.L[k].p(), Aop.a_ajib[k].p(), PY.R[k + 1].p(), xin.core[k].p(), r0, R1, q0, m, n, R2, r1,
                   q1, sol.p(), T1, T2);
      tmp.ensure(c, N);
      copy(c, tmp.p(), sol.p(), N);
      axpby(c, N, -1.0, y.core[k].p(), 1.0, tmp.p());
      const double ns = nrm2(c, sol.p(), N);
      const double dx = ns > 0 ? nrm2(c, tmp.p(), N) / ns : 0.0;
      if (!std::isfinite(dx)) throw Error(TT_ENONFINITE, "amen_mv: non-finite local product");
      maxdx = std::max(maxdx, dx);
      if (k == d - 1) {
        copy(c, y.core[k].p(), sol.p(), N);
        break;
      }
      SVD s;
      {
        PhaseTimer pt(c, "amen.svd");
        svd_rm(c, sol.p(), r0 * m, r1, s, SVD_ORTH_ANY);
      }
      double sn2 = 0;
      for (double v : s.Sh) sn2 += v * v;
      const int rk = trunc_rank(s.Sh, loc_eps * std::sqrt(sn2), rmax);
      DBuf v(c, (size_t)rk * r1);
      copy(c, v.p(), s.Vt.p(), (size_t)rk * r1);
      scale_rows(c, v.p(), rk, r1, s.S.p());
      solt.ensure(c, N);
      gemm(c, true, false, r0 * m, r1, rk, 1.0, s.Ut.p(), r0 * m, 0, v.p(), r1, 0, 0.0, solt.p(), r1, 0);
      const int rz0 = z.r[k], rz1 = z.r[k + 1];
      // crz = y'Ax z - solt . YZ_R   (r0, m, rz1)
      crz.ensure(c, (size_t)r0 * m * rz1);
      local_matvec(c, PY.L[k].p(), Aop.a_ajib[k].p(), PZ.R[k + 1].p(), xin.core[k].p(), r0, R1, q0, m, n, R2, rz1,
                   q1, crz.p(), T1, T2);
      gemm(c, false, false, r0 * m, rz1, r1, -1.0, solt.p(), r1, 0, YZ.R[k + 1].p(), rz1, 0, 1.0, crz.p(), rz1, 0);
      // czz = z'Ax z - ZY_L . solt . YZ_R   (rz0, m, rz1)
      czz.ensure(c, (size_t)rz0 * m * rz1);
      local_matvec(c, PZ.L[k].p(), Aop.a_ajib[k].p(), PZ.R[k + 1].p(), xin.core[k].p(), rz0, R1, q0, m, n, R2,
                   rz1, q1, czz.p(), T1, T2);
      tmp.ensure(c, (size_t)rz0 * m * r1);
      gemm(c, false, false, rz0, m * r1, r0, 1.0, ZY.L[k].p(), r0, 0, solt.p(), m * r1, 0, 0.0, tmp.p(), m * r1, 0);
      gemm(c, false, false, rz0 * m, rz1, r1, -1.0, tmp.p(), r1, 0, YZ.R[k + 1].p(), rz1, 0, 1.0, czz.p(), rz1, 0);
      {
        PhaseTimer pt(c, "amen.enrich_qr");
        orth_core_cols(c, z, k, czz.p());
        split_enrich(c, y, k, s, rk, crz.p(), rz1);
      }
      const int nr1 = y.r[k + 1];
      left_update(c, PY.L[k].p(), y.core[k].p(), Aop.a_ajib[k].p(), xin.core[k].p(), r0, R1, q0, m, n, R2, nr1, q1,
                  PY.L[k + 1], T1, T2);
      left_update(c, PZ.L[k].p(), z.core[k].p(), Aop.a_ajib[k].p(), xin.core[k].p(), rz0, R1, q0, m, n, R2, rz1, q1,
                  PZ.L[k + 1], T1, T2);
      vleft_update(c, ZY.L[k].p(), z.core[k].p(), y.core[k].p(), rz0, r0, m, rz1, nr1, ZY.L[k + 1], T3);
    }
    if (maxdx < eps) {
      ++swp;
      break;
    }
    if (swp + 1 < nswp) {
      PhaseTimer pt(c, "amen.reorth_ifaces");
      orth_right(c, y, 0);
      orth_right(c, z, 0);
      right_all();
    }
  }
  if (st) {
    st->sweeps = std::min(swp, nswp);
    st->max_dx = maxdx;
  }
}

// Two-site DMRG solve of A x = b (the two-site member of the alternating
// family Sec. 3.5 names: "fix all cores but two"): for each bond k the local
// system of the merged supercore X_k X_{k+1} (modes n_k n_{k+1}) is projected
// with the interfaces of the cores outside the pair (Galerkin, as the
// one-site solve), solved by the same local solver, and split back by a
// truncated SVD (threshold eps/sqrt(d), cap rmax), so ranks adapt without
// residual enrichment.  The merged operator core (R_k, n n', n n', R_{k+2})
// is formed per pair: meant for moderate mode sizes.
void dmrg_solve(Ctx *c, TTOp &Aop, const TT &b, TT &x, double eps, int rmax, int nswp, SolveStats *st, int prec) {
  TT &A = Aop.t;
  Aop.prepare(c);
  const int d = A.d;
  TT_REQUIRE(d >= 2 && b.d == d && x.d == d, "dmrg_solve: need d >= 2 and matching dimensions");
  for (int k = 0; k < d; ++k)
    TT_REQUIRE(A.mo[k] == A.mi[k] && A.mi[k] == x.n[k] && b.n[k] == x.n[k], "dmrg_solve: mode mismatch");
  const bool mixed = prec != TT_FP64;
  const double loc_eps = eps / std::sqrt((double)d);
  orth_right(c, x, 0);
  Iface PX, QX;
  PX.init(c, d);
  QX.init(c, d);
  DBuf T1, T2, T3, W, Wt, W32, bm, rhs, sol, old;
  auto right_all = [&]() {
    for (int k = d - 1; k >= 2; --k) {
      const int m = x.n[k];
      right_update(c, PX.R[k + 1].p(), x.core[k].p(), Aop.a_jbai[k].p(), x.core[k].p(), x.r[k], A.r[k], x.r[k], m, m,
                   A.r[k + 1], x.r[k + 1], x.r[k + 1], PX.R[k], T1, T2);
      vright_update(c, QX.R[k + 1].p(), x.core[k].p(), b.core[k].p(), x.r[k], b.r[k], m, x.r[k + 1], b.r[k + 1],
                    QX.R[k], T3);
    }
  };
  right_all();
  LocalSolver LS;
  double maxdx = 0.0;
  long long git = 0;
  int swp = 0;
  for (swp = 0; swp < nswp; ++swp) {
    maxdx = 0.0;
    for (int k = 0; k + 1 < d; ++k) {
      const int n1 = x.n[k], n2 = x.n[k + 1], nn = n1 * n2;
      const int r0 = x.r[k], r1 = x.r[k + 1], r2 = x.r[k + 2];
      const int R0 = A.r[k], R1 = A.r[k + 1], R2 = A.r[k + 2];
      // merged operator core in the local-matvec layout (R0, in, out, R2):
      // W[a, (i1 i2), (o1 o2), c] = sum_b A_k[a, i1, o1, b] A_{k+1}[b, i2, o2, c]
      Wt.ensure(c, (size_t)R0 * n1 * n1 * n2 * n2 * R2);
      gemm(c, false, false, R0 * n1 * n1, n2 * n2 * R2, R1, 1.0, Aop.a_ajib[k].p(), R1, 0, Aop.a_ajib[k + 1].p(),
           n2 * n2 * R2, 0, 0.0, Wt.p(), n2 * n2 * R2, 0);
      W.ensure(c, (size_t)R0 * nn * nn * R2);
      {
        const int shape[6] = {R0, n1, n1, n2, n2, R2};
        const int perm[6] = {0, 1, 3, 2, 4, 5};
        permute(c, Wt.p(), W.p(), 6, shape, perm);
      }
      if (mixed) {
        W32.ensure(c, ((size_t)R0 * nn * nn * R2 + 1) / 2);
        d2f(c, W.p(), reinterpret_cast<float *>(W32.p()), (size_t)R0 * nn * nn * R2);
      }
      // merged right-hand side and initial guess
      bm.ensure(c, (size_t)b.r[k] * nn * b.r[k + 2]);
      gemm(c, false, false, b.r[k] * n1, n2 * b.r[k + 2], b.r[k + 1], 1.0, b.core[k].p(), b.r[k + 1], 0,
           b.core[k + 1].p(), n2 * b.r[k + 2], 0, 0.0, bm.p(), n2 * b.r[k + 2], 0);
      const size_t N = (size_t)r0 * nn * r2;
      rhs.ensure(c, N);
      vlocal(c, QX.L[k].p(), bm.p(), QX.R[k + 2].p(), r0, b.r[k], nn, b.r[k + 2], r2, rhs.p(), T3);
      sol.ensure(c, N);
      gemm(c, false, false, r0 * n1, n2 * r2, r1, 1.0, x.core[k].p(), r1, 0, x.core[k + 1].p(), n2 * r2, 0, 0.0,
           sol.p(), n2 * r2, 0);
      old.ensure(c, N);
      copy(c, old.p(), sol.p(), N);
      git += LS.solve(c, prec, PX.L[k].p(), W.p(), mixed ? reinterpret_cast<const float *>(W32.p()) : nullptr,
                      PX.R[k + 2].p(), r0, R0, nn, R2, r2, rhs.p(), sol.p(), loc_eps);
      axpby(c, N, 1.0, sol.p(), -1.0, old.p());
      const double ns = nrm2(c, sol.p(), N);
      const double dx = ns > 0 ? nrm2(c, old.p(), N) / ns : 0.0;
      if (!std::isfinite(dx)) throw Error(TT_ENONFINITE, "dmrg_solve: non-finite local solution");
      maxdx = std::max(maxdx, dx);
      // split the supercore: X_k = U (left-orthogonal), X_{k+1} = S V^T
      SVD sv;
      svd_rm(c, sol.p(), r0 * n1, n2 * r2, sv, SVD_ORTH_U);
      double sn2 = 0;
      for (double v : sv.Sh) sn2 += v * v;
      const int rk = trunc_rank(sv.Sh, loc_eps * std::sqrt(sn2), rmax);
      DBuf xk(c, (size_t)r0 * n1 * rk), xk1(c, (size_t)rk * n2 * r2);
      transpose(c, sv.Ut.p(), xk.p(), rk, r0 * n1);
      copy(c, xk1.p(), sv.Vt.p(), (size_t)rk * n2 * r2);
      scale_rows(c, xk1.p(), rk, n2 * r2, sv.S.p());
      x.core[k] = std::move(xk);
      x.core[k + 1] = std::move(xk1);
      x.r[k + 1] = rk;
      if (k + 2 < d) {
        left_update(c, PX.L[k].p(), x.core[k].p(), Aop.a_ajib[k].p(), x.core[k].p(), r0, R0, r0, n1, n1, R1, rk, rk,
                    PX.L[k + 1], T1, T2);
        vleft_update(c, QX.L[k].p(), x.core[k].p(), b.core[k].p(), r0, b.r[k], n1, rk, b.r[k + 1], QX.L[k + 1], T3);
      }
    }
    if (maxdx < eps) {
      ++swp;
      break;
    }
    if (swp + 1 < nswp) {
      orth_right(c, x, 0);
      right_all();
    }
  }
  if (st) {
    st->sweeps = std::min(swp, nswp);
    st->max_dx = maxdx;
    st->gmres_iters = git;
  }
}

}  // namespace tt
