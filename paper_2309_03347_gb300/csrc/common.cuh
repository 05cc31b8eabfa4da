// Internal declarations shared by the translation units of libkeig_tt.
// Everything here is FP64; all device work runs on the context stream.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "../../include/keig.h"

namespace tt {

// ----------------------------------------------------------------- errors
struct Error : public std::runtime_error {
  int code;
  Error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

#define TT_CHECK_CUDA(call)                                                                  \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      throw ::tt::Error(e_ == cudaErrorMemoryAllocation ? TT_ENOMEM : TT_ECUDA,              \
                        std::string(#call) + ": " + cudaGetErrorString(e_) + " at " +        \
                            __FILE__ + ":" + std::to_string(__LINE__));                      \
  } while (0)

#define TT_REQUIRE(cond, msg)                                   \
  do {                                                          \
    if (!(cond)) throw ::tt::Error(TT_EINVAL, std::string(msg)); \
  } while (0)

struct Ctx;

// ----------------------------------------------------------------- device buffer
// Owning device allocation from the stream-ordered pool of the context stream.
class DBuf {
 public:
  DBuf() = default;
  DBuf(Ctx *c, size_t n) { alloc(c, n); }
  ~DBuf() { release(); }
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  DBuf(DBuf &&o) noexcept { swap(o); }
  DBuf &operator=(DBuf &&o) noexcept {
    if (this != &o) {
      release();
      swap(o);
    }
    return *this;
  }
  void alloc(Ctx *c, size_t n);
  // grow (contents not kept) so that at least n doubles fit
  void ensure(Ctx *c, size_t n) {
    if (n > cap_) alloc(c, n);
  }
  void release();
  double *p() const { return p_; }
  size_t size() const { return n_; }
  void set_size(size_t n) { n_ = n; }
  void swap(DBuf &o) noexcept {
    std::swap(ctx_, o.ctx_);
    std::swap(p_, o.p_);
    std::swap(n_, o.n_);
    std::swap(cap_, o.cap_);
  }

 private:
  Ctx *ctx_ = nullptr;
  double *p_ = nullptr;
  size_t n_ = 0, cap_ = 0;
};

// ----------------------------------------------------------------- context
struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  // caller-supplied device allocator (tt_ctx_create); null: the stream-ordered pool
  tt_alloc_fn alloc_fn = nullptr;
  tt_free_fn free_fn = nullptr;
  void *alloc_user = nullptr;
  std::string err;
  int64_t launches = 0;
  double flops = 0.0;    // algorithmic contraction flops (FP64)
  double flops32 = 0.0;  // algorithmic contraction flops run in FP32
  int sm_count = 152;
  // spin limit of the bounded device waits (grid barriers); < 0: the kernels' defaults
  long long wait_limit = -1;
  // set while the context solves one of several batched problems: its
  // persistent-GMRES systems join grouped launches
  struct PGGroup *group = nullptr;
  // grid-size tuner of the persistent GMRES: per shape class, the measured
  // time per Arnoldi step of each candidate grid (all SMs, 1/2, 1/4, 1/8),
  // then the fastest (KEIG_PGMRES_TUNE=0 keeps one CTA per SM)
  bool pg_tune = true;
  std::map<uint64_t, int> pg_tuned;
  std::map<uint64_t, std::vector<std::pair<int, double>>> pg_trials;
  cudaEvent_t tune_ev[2] = {nullptr, nullptr};
  // scratch buffers reused across calls (grown on demand)
  DBuf ws_gemm;    // split-K partial sums (FP64)
  DBuf ws_gemm32;  // split-K partial sums (FP32, stored in a double-typed buffer)
  DBuf scratch[8];
  DBuf scalar_buf;             // owns d_scalar
  double *d_scalar = nullptr;  // small device area for reductions (64 doubles)
  // optional per-launch timing of the contraction GEMMs (CUDA events)
  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
  size_t ev_used = 0;
  std::vector<int> ev_tag;  // 0: FP64 GEMM, 1: FP32 GEMM, 2: tcgen05 TF32 GEMM
  double gemm_flops = 0.0, gemm32_flops = 0.0, gemmtc_flops = 0.0, pg_flops = 0.0;
  int64_t gemm_launches = 0, gemm32_launches = 0, gemmtc_launches = 0, pg_launches = 0;
  double gemm_ms_done = 0.0, gemm32_ms_done = 0.0, gemmtc_ms_done = 0.0, pg_ms_done = 0.0;  // folded-in event times
  DBuf ws_tc;  // split-K partial sums of the tensor-core GEMM
  void prof_begin(cudaEvent_t *b, cudaEvent_t *e, int tag = 0);
  void prof_fold();
  double *h_pinned = nullptr;  // pinned host staging (4096 doubles)
  void sync() { TT_CHECK_CUDA(cudaStreamSynchronize(stream)); }
  // host-side phase timers (enabled by the KEIG_PHASE_TIMES environment variable)
  bool phase_timing = false;
  bool mixed_svd = true;  // KEIG_FP64_SVD disables the FP32-preconditioned Jacobi
  bool persistent_gmres = true;  // KEIG_LAUNCHED_GMRES selects the per-step-launch FP32 GMRES
  struct Phase {
    std::string name;
    double ms;
    long long calls;
  };
  std::vector<Phase> phase_ms;
  void phase_add(const char *name, double ms) {
    for (auto &p : phase_ms)
      if (p.name == name) {
        p.ms += ms;
        ++p.calls;
        return;
      }
    phase_ms.push_back({name, ms, 1});
  }
  void count(int n = 1) { launches += n; }
};

// Scoped phase timer: synchronises the stream at both ends when enabled.
struct PhaseTimer {
  Ctx *c;
  const char *name;
  double t0 = 0;
  PhaseTimer(Ctx *cc, const char *n);
  ~PhaseTimer();
};

// ----------------------------------------------------------------- kernels (kernels.cu)
// C[b] = alpha op(A[b]) op(B[b]) + beta C[b], row-major, op = transpose when t* != 0.
void gemm(Ctx *c, bool ta, bool tb, int M, int N, int K, double alpha, const double *A, int lda,
          long long sA, const double *B, int ldb, long long sB, double beta, double *C, int ldc,
          long long sC, int batch = 1);
// out = permutation of a row-major tensor: out.shape[i] = in.shape[perm[i]]
void permute(Ctx *c, const double *in, double *out, int ndim, const int *shape, const int *perm);
// row-major rows x cols -> cols x rows
void transpose(Ctx *c, const double *in, double *out, int rows, int cols);
void fill(Ctx *c, double *p, size_t n, double v);
void copy(Ctx *c, double *dst, const double *src, size_t n);
void scale(Ctx *c, double *p, size_t n, double a);
void axpby(Ctx *c, size_t n, double a, const double *x, double b, double *y);  // y = a x + b y
// 2-D strided block copy: dst[i*ldd + j] = alpha * src[i*lds + j], i < rows, j < cols
void copy2d(Ctx *c, double *dst, int ldd, const double *src, int lds, int rows, int cols,
            double alpha = 1.0);
// row-major rows x cols: scale row i by s[i] (device vector)
void scale_rows(Ctx *c, double *a, int rows, int cols, const double *s);
// deterministic reductions; result left in device memory out[0]
void dot_dev(Ctx *c, const double *x, const double *y, size_t n, double *out);
double dot(Ctx *c, const double *x, const double *y, size_t n);
double nrm2(Ctx *c, const double *x, size_t n);
// GMRES helpers: h[j] = <V_j, w> for j < nv (V rows of length n), and w -= V^T h
void multi_dot(Ctx *c, const double *V, size_t ldv, int nv, const double *w, size_t n, double *h);
void multi_axpy(Ctx *c, const double *V, size_t ldv, int nv, const double *h, double *w, size_t n);
// any non-finite entry? (result to host)
bool has_nonfinite(Ctx *c, const double *x, size_t n);

// FP32 counterparts used by the mixed-precision local solves
void gemm_f32(Ctx *c, bool ta, bool tb, int M, int N, int K, float alpha, const float *A, int lda, long long sA,
              const float *B, int ldb, long long sB, float beta, float *C, int ldc, long long sC, int batch = 1);
// the same product on the tcgen05 tensor cores with the three-term split
// (tc_gemm.cu): kind::tf32, or kind::f16 with BF16 operands when bf16
void gemm_f32_tc(Ctx *c, bool ta, bool tb, int M, int N, int K, float alpha, const float *A, int lda, long long sA,
                 const float *B, int ldb, long long sB, float beta, float *C, int ldc, long long sC, int batch = 1,
                 bool bf16 = false);
// nonzero when a tensor-core GEMM gave up a bounded wait (reads device memory)
int tc_error_flag(Ctx *c);
void d2f(Ctx *c, const double *x, float *y, size_t n, double s = 1.0);
void f2d_axpy(Ctx *c, const float *x, double *y, size_t n, double a);
void axpby_f(Ctx *c, size_t n, float a, const float *x, float b, float *y);
void multi_dot_f(Ctx *c, const float *V, size_t ldv, int nv, const float *w, size_t n, double *h);
void multi_axpy_f(Ctx *c, const float *V, size_t ldv, int nv, const double *h, float *w, size_t n);
void dot_f_dev(Ctx *c, const float *x, const float *y, size_t n, double *out);

// Device-resident steps of the FP32 GMRES (krylov.cu).  Vectors are FP32
// columns of V with stride ldv; reductions accumulate in FP64.
constexpr int KRY_MAX_VECS = 64;   // basis vectors per Gram-Schmidt product
constexpr int KRY_MAX_SPLIT = 32;  // CTAs per vector in kry_mdot
// part[j S + s] = partial V_j . w; returns S (part holds nv * S doubles)
int kry_mdot(Ctx *c, const float *V, size_t ldv, int nv, const float *w, size_t n, double *part);
// w -= sum_j h_j V_j with h_j = sum_s part[j S + s]; hout (nv) = h if given;
// npart (returned count) = per-CTA sums of the new w^2 if given
int kry_maxpy(Ctx *c, const float *V, size_t ldv, int nv, const double *part, int S, float *w, size_t n,
              double *hout, double *npart);
// per-CTA partial sums of x^2; returns their count (<= 4 x SMs)
int kry_sumsq(Ctx *c, const float *x, size_t n, double *npart);
// Arnoldi step j of a cycle with restart mr (see krylov.cu)
void kry_arnoldi(Ctx *c, int j, int mr, const double *h1, const double *h2, const double *npart, int nb, double *H,
                 double *cs, double *sn, double *g, double *st, double *inv);
void kry_start(Ctx *c, const double *npart, int nb, int mr, double *g, double *st, double *inv);
void kry_trisolve(Ctx *c, int kk, int mr, const double *H, const double *g, double *y);
// y = s[0] x (s on the device; x == y allowed)
void kry_scale(Ctx *c, const float *x, float *y, size_t n, const double *s);

// Restarted FP32 GMRES of the local system Phi_L A Phi_R (FP32 operands,
// square: row and column ranks r0, r1, mode m) as one persistent cooperative
// kernel (pgmres.cu); x = solution from x0 = 0.  Returns the Arnoldi steps.
struct PGWork {
  DBuf V, T1, T2, ws, D, st;
};
bool pgmres32_fits(Ctx *c, int N, int restart);
// Grouped launches of the persistent GMRES across contexts (batched problems)
struct PGGroup;
PGGroup *pg_group_create(int device, int sm_count);
void pg_group_destroy(PGGroup *g);
void pg_group_set_active(PGGroup *g, int n);  // workers that will submit
void pg_group_join(PGGroup *g);               // a worker starts a problem
void pg_group_leave(PGGroup *g);              // ... and has finished it
void pg_group_stats(PGGroup *g, long long *launches, long long *systems);
int pgmres32(Ctx *c, const float *PL, const float *A32, const float *PR, int r0, int R1, int m, int R2, int r1,
             const float *b, float *x, double tol, int restart, int maxit, PGWork &W);

// Householder QR of column-major A (m x n, lda = m), overwritten by the
// reflectors; Q (m x k, k = min(m,n)) and R (k x n) written column-major.
void qr_colmajor(Ctx *c, double *A, int m, int n, double *Q, double *R);
// One-sided Jacobi SVD of a column-major square n x n matrix (destroyed):
// U (n x n), V (n x n) column-major and S (n) sorted by decreasing value.
void jacobi_svd(Ctx *c, double *B, int n, double *U, double *S, double *V);
// Same product B = U S V^T with rotations found in FP32 and refined by FP64
// matrix products (svd_mixed.cu): V orthonormal to FP64 rounding (U when
// exact_u), the other factor up to the cosines between near pairs.
bool jacobi_svd_mixed_fits(int n);
void jacobi_svd_mixed(Ctx *c, double *B, int n, double *U, double *S, double *V, bool exact_u);

// Kronecker core product of the exact TT matvec:
// Y[(a,b), i, (c,e)] = sum_j A[a,i,j,c] X[b,j,e]
void kron_core(Ctx *c, const double *A, int R0, int m, int n, int R1, const double *X, int r0,
               int r1, double *Y);
// out[a, b] = sum_i w[i] G[a, i, b]  (G: r0 x n x r1), w on device
void contract_mode(Ctx *c, const double *G, int r0, int n, int r1, const double *w, double *out);

}  // namespace tt
