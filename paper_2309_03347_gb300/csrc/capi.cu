// extern "C" boundary of libkeig_tt (declared in include/keig.h) and the
// k-eigenvalue fixed point of Eq. (TT_k_eff_fixed_points).
#include <atomic>
#include <chrono>
#include <thread>

#include "tt.cuh"

struct tt_ctx {
  tt::Ctx c;
};

// grouped persistent-GMRES launches of the last keig_batch call
static std::atomic<long long> g_batch_group_launches{0}, g_batch_group_systems{0};
struct tt_vec {
  tt::Ctx *owner;
  tt::TT t;
};
struct tt_op {
  tt::Ctx *owner;
  tt::TTOp op;
};

namespace {

template <class F>
int guarded(tt_ctx *ctx, F &&f) {
  if (!ctx) return TT_EINVAL;
  try {
    f();
    ctx->c.err.clear();
    return TT_OK;
  } catch (const tt::Error &e) {
    ctx->c.err = e.what();
    return e.code;
  } catch (const std::bad_alloc &) {
    ctx->c.err = "host allocation failed";
    return TT_ENOMEM;
  } catch (const std::exception &e) {
    ctx->c.err = e.what();
    return TT_EINVAL;
  }
}

std::vector<int> to_vec(const int *p, int n) { return std::vector<int>(p, p + n); }

void check_finite_host(const double *p, size_t n, const char *what) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) throw tt::Error(TT_EINVAL, std::string("non-finite value in ") + what);
}

tt::TT make_tt(tt::Ctx *c, int d, const int *n, const int *r, const double *cores, int on_dev) {
  TT_REQUIRE(d >= 1 && d <= 256 && n && r, "tt: bad shape arguments");
  std::vector<int> nv = to_vec(n, d), rv = to_vec(r, d + 1);
  TT_REQUIRE(rv[0] == 1 && rv[d] == 1, "tt: r[0] and r[d] must be 1");
  for (int k = 0; k < d; ++k) TT_REQUIRE(nv[k] >= 1 && rv[k] >= 1 && rv[k] <= 4096, "tt: bad mode or rank");
  tt::TT x = tt::tt_zeros(c, nv, rv);
  if (cores) {
    size_t off = 0;
    for (int k = 0; k < d; ++k) {
      const size_t sz = x.csize(k);
      if (!on_dev) check_finite_host(cores + off, sz, "TT cores");
      TT_CHECK_CUDA(cudaMemcpyAsync(x.core[k].p(), cores + off, sz * sizeof(double),
                                    on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
      off += sz;
    }
    c->sync();
  }
  return x;
}

void get_cores(tt::Ctx *c, const tt::TT &x, double *dst, int on_dev) {
  TT_REQUIRE(dst, "null destination");
  size_t off = 0;
  for (int k = 0; k < x.d; ++k) {
    const size_t sz = x.csize(k);
    TT_CHECK_CUDA(cudaMemcpyAsync(dst + off, x.core[k].p(), sz * sizeof(double),
                                  on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    off += sz;
  }
  c->sync();
}

void validate_problem(const tt_problem *p) {
  TT_REQUIRE(p, "null problem");
  TT_REQUIRE(p->l >= 1 && p->l <= 10, "problem: l must be in [1, 10]");
  TT_REQUIRE(p->G >= 1 && p->G <= 4096, "problem: bad G");
  TT_REQUIRE(p->n_mat >= 1 && p->n_mat <= 255, "problem: bad n_mat");
  TT_REQUIRE(p->n_dir >= 1 && p->n_dir <= 4096, "problem: bad n_dir");
  TT_REQUIRE(p->sig_t && p->sig_s && p->nu_sig_f && p->chi && p->mat && p->amu && p->aeta && p->axi && p->w,
             "problem: null table");
  for (int f = 0; f < 6; ++f) TT_REQUIRE(p->bc[f] == 0, "problem: only vacuum faces (bc = 0) are supported");
  for (int a = 0; a < 3; ++a) TT_REQUIRE(p->side[a] > 0 && std::isfinite(p->side[a]), "problem: bad side");
  const size_t G = p->G, nm = p->n_mat, nd = p->n_dir;
  check_finite_host(p->sig_t, nm * G, "sig_t");
  check_finite_host(p->sig_s, nm * G * G, "sig_s");
  check_finite_host(p->nu_sig_f, nm * G, "nu_sig_f");
  check_finite_host(p->chi, nm * G, "chi");
  check_finite_host(p->amu, nd, "amu");
  check_finite_host(p->aeta, nd, "aeta");
  check_finite_host(p->axi, nd, "axi");
  check_finite_host(p->w, nd, "w");
  if (p->sig_s1) check_finite_host(p->sig_s1, nm * G * G, "sig_s1");
  if (p->sig_s2) check_finite_host(p->sig_s2, nm * G * G, "sig_s2");
  if (p->sig_s3) check_finite_host(p->sig_s3, nm * G * G, "sig_s3");
  const size_t nc = ((size_t)1 << p->l) - 1;
  for (size_t i = 0; i < nc * nc * nc; ++i)
    TT_REQUIRE(p->mat[i] < p->n_mat, "problem: material index out of range");
}

}  // namespace

extern "C" {

const char *tt_version(void) { return "keig-tt 0.1 (sm_103a, FP64)"; }

int tt_ctx_create(tt_ctx **out, void *stream, tt_alloc_fn alloc_fn, tt_free_fn free_fn, void *user) {
  if (!out) return TT_EINVAL;
  *out = nullptr;
  if ((alloc_fn == nullptr) != (free_fn == nullptr)) return TT_EINVAL;
  tt_ctx *ctx = new (std::nothrow) tt_ctx();
  if (!ctx) return TT_ENOMEM;
  int rc = guarded(ctx, [&] {
    int ndev = 0;
    TT_CHECK_CUDA(cudaGetDeviceCount(&ndev));
    TT_REQUIRE(ndev > 0, "no CUDA device");
    TT_CHECK_CUDA(cudaGetDevice(&ctx->c.device));
    cudaDeviceProp prop;
    TT_CHECK_CUDA(cudaGetDeviceProperties(&prop, ctx->c.device));
    ctx->c.sm_count = prop.multiProcessorCount;
    ctx->c.stream = (cudaStream_t)stream;
    ctx->c.alloc_fn = alloc_fn;
    ctx->c.free_fn = free_fn;
    ctx->c.alloc_user = user;
    ctx->c.phase_timing = getenv("KEIG_PHASE_TIMES") != nullptr;
    ctx->c.mixed_svd = getenv("KEIG_FP64_SVD") == nullptr;
    ctx->c.persistent_gmres = getenv("KEIG_LAUNCHED_GMRES") == nullptr;
    {
      const char *t = getenv("KEIG_PGMRES_TUNE");
      ctx->c.pg_tune = !(t && t[0] == '0');
    }
    TT_CHECK_CUDA(cudaEventCreate(&ctx->c.tune_ev[0]));
    TT_CHECK_CUDA(cudaEventCreate(&ctx->c.tune_ev[1]));
    // keep freed blocks in the stream-ordered pool
    cudaMemPool_t pool;
    TT_CHECK_CUDA(cudaDeviceGetDefaultMemPool(&pool, ctx->c.device));
    uint64_t thr = UINT64_MAX;
    TT_CHECK_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    ctx->c.scalar_buf.alloc(&ctx->c, 64);
    ctx->c.d_scalar = ctx->c.scalar_buf.p();
    TT_CHECK_CUDA(cudaMemsetAsync(ctx->c.d_scalar, 0, 64 * sizeof(double), ctx->c.stream));
    TT_CHECK_CUDA(cudaMallocHost(&ctx->c.h_pinned, 4096 * sizeof(double)));
  });
  if (rc != TT_OK) {
    delete ctx;
    return rc == TT_EINVAL ? TT_ECUDA : rc;
  }
  *out = ctx;
  return TT_OK;
}

int tt_ctx_destroy(tt_ctx *ctx) {
  if (!ctx) return TT_EINVAL;
  cudaStreamSynchronize(ctx->c.stream);
  ctx->c.ws_gemm.release();
  ctx->c.ws_gemm32.release();
  ctx->c.ws_tc.release();
  for (auto &s : ctx->c.scratch) s.release();
  cudaStreamSynchronize(ctx->c.stream);
  ctx->c.scalar_buf.release();
  cudaStreamSynchronize(ctx->c.stream);
  if (ctx->c.h_pinned) cudaFreeHost(ctx->c.h_pinned);
  for (auto e : ctx->c.tune_ev)
    if (e) cudaEventDestroy(e);
  for (auto &e : ctx->c.ev_pool) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  delete ctx;
  return TT_OK;
}

const char *tt_last_error(const tt_ctx *ctx) { return ctx ? ctx->c.err.c_str() : "null context"; }

int tt_ctx_counters(tt_ctx *ctx, int64_t *launches, double *flops) {
  if (!ctx) return TT_EINVAL;
  if (launches) *launches = ctx->c.launches;
  if (flops) *flops = ctx->c.flops + ctx->c.flops32;
  return TT_OK;
}

int tt_gemm_f32(tt_ctx *ctx, int kind, int ta, int tb, int M, int N, int K, float alpha, const float *A, int lda,
                long long sA, const float *B, int ldb, long long sB, float beta, float *C, int ldc, long long sC,
                int batch) {
  return guarded(ctx, [&] {
    tt::Ctx *c = &ctx->c;
    TT_REQUIRE(kind >= 0 && kind <= 2, "tt_gemm_f32: kind must be 0, 1 or 2");
    TT_REQUIRE(A && B && C && M >= 0 && N >= 0 && K >= 0 && batch >= 1, "tt_gemm_f32: bad arguments");
    TT_REQUIRE(lda >= (ta ? M : K) && ldb >= (tb ? K : N) && ldc >= N, "tt_gemm_f32: leading dimension too small");
    if (kind == 0) {
      tt::gemm_f32(c, ta != 0, tb != 0, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch);
      return;
    }
    TT_CHECK_CUDA(cudaMemsetAsync(c->d_scalar + 8, 0, sizeof(int), c->stream));
    tt::gemm_f32_tc(c, ta != 0, tb != 0, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, kind == 2);
    if (tt::tc_error_flag(c)) throw tt::Error(TT_ETIMEOUT, "tt_gemm_f32: a tensor-core GEMM gave up waiting");
  });
}

int tt_ctx_set_wait_limit(tt_ctx *ctx, long long spins) {
  if (!ctx) return TT_EINVAL;
  ctx->c.wait_limit = spins < 0 ? -1 : spins;
  return TT_OK;
}

int tt_ctx_reset_counters(tt_ctx *ctx) {
  if (!ctx) return TT_EINVAL;
  ctx->c.launches = 0;
  ctx->c.flops = 0.0;
  ctx->c.flops32 = 0.0;
  return TT_OK;
}

int tt_ctx_set_profiling(tt_ctx *ctx, int on) {
  return guarded(ctx, [&] {
    ctx->c.prof_fold();
    ctx->c.profiling = on != 0;
    ctx->c.gemm_flops = ctx->c.gemm32_flops = ctx->c.gemmtc_flops = ctx->c.pg_flops = 0.0;
    ctx->c.gemm_launches = ctx->c.gemm32_launches = ctx->c.gemmtc_launches = ctx->c.pg_launches = 0;
    ctx->c.gemm_ms_done = ctx->c.gemm32_ms_done = ctx->c.gemmtc_ms_done = ctx->c.pg_ms_done = 0.0;
  });
}

int tt_ctx_gemm_stats(tt_ctx *ctx, int64_t *launches, double *ms, double *flops) {
  return guarded(ctx, [&] {
    ctx->c.prof_fold();
    if (launches) *launches = ctx->c.gemm_launches;
    if (ms) *ms = ctx->c.gemm_ms_done;
    if (flops) *flops = ctx->c.gemm_flops;
  });
}

int tt_ctx_gmres_stats(tt_ctx *ctx, int64_t *launches, double *ms, double *flops) {
  return guarded(ctx, [&] {
    ctx->c.prof_fold();
    if (launches) *launches = ctx->c.pg_launches;
    if (ms) *ms = ctx->c.pg_ms_done;
    if (flops) *flops = ctx->c.pg_flops;
  });
}

int tt_ctx_gemmtc_stats(tt_ctx *ctx, int64_t *launches, double *ms, double *flops) {
  return guarded(ctx, [&] {
    ctx->c.prof_fold();
    if (launches) *launches = ctx->c.gemmtc_launches;
    if (ms) *ms = ctx->c.gemmtc_ms_done;
    if (flops) *flops = ctx->c.gemmtc_flops;
  });
}

int tt_ctx_gemm32_stats(tt_ctx *ctx, int64_t *launches, double *ms, double *flops) {
  return guarded(ctx, [&] {
    ctx->c.prof_fold();
    if (launches) *launches = ctx->c.gemm32_launches;
    if (ms) *ms = ctx->c.gemm32_ms_done;
    if (flops) *flops = ctx->c.gemm32_flops;
  });
}

// ---------------------------------------------------------------- vectors
int tt_vec_create(tt_ctx *ctx, int d, const int *n, const int *r, const double *cores, int on_dev, tt_vec **out) {
  return guarded(ctx, [&] {
    TT_REQUIRE(out, "null out");
    tt::TT x = make_tt(&ctx->c, d, n, r, cores, on_dev);
    *out = new tt_vec{&ctx->c, std::move(x)};
  });
}

int tt_vec_destroy(tt_vec *x) {
  if (!x) return TT_EINVAL;
  delete x;
  return TT_OK;
}

int tt_vec_shape(const tt_vec *x, int *d, int *n, int *r) {
  if (!x || !d) return TT_EINVAL;
  *d = x->t.d;
  if (n)
    for (int k = 0; k < x->t.d; ++k) n[k] = x->t.n[k];
  if (r)
    for (int k = 0; k <= x->t.d; ++k) r[k] = x->t.r[k];
  return TT_OK;
}

int tt_vec_numel(const tt_vec *x, size_t *count) {
  if (!x || !count) return TT_EINVAL;
  *count = x->t.numel();
  return TT_OK;
}

int tt_vec_get_cores(tt_ctx *ctx, const tt_vec *x, double *dst, int on_dev) {
  return guarded(ctx, [&] {
    TT_REQUIRE(x, "null vector");
    get_cores(&ctx->c, x->t, dst, on_dev);
  });
}

int tt_vec_to_dense(tt_ctx *ctx, const tt_vec *x, double *dst, size_t len) {
  return guarded(ctx, [&] {
    TT_REQUIRE(x && dst, "null argument");
    tt::to_dense(&ctx->c, x->t, dst, len);
    ctx->c.sync();
  });
}

int tt_vec_axpby(tt_ctx *ctx, double a, const tt_vec *x, double b, tt_vec *y) {
  return guarded(ctx, [&] {
    TT_REQUIRE(x && y, "null vector");
    y->t = tt::add(&ctx->c, a, x->t, b, y->t);
  });
}

int tt_vec_scale(tt_ctx *ctx, tt_vec *x, double a) {
  return guarded(ctx, [&] {
    TT_REQUIRE(x, "null vector");
    tt::scale(&ctx->c, x->t, a);
  });
}

int tt_vec_dot(tt_ctx *ctx, const tt_vec *x, const tt_vec *y, double *out) {
  return guarded(ctx, [&] {
    TT_REQUIRE(x && y && out, "null argument");
    *out = tt::dot(&ctx->c, x->t, y->t);
  });
}

int tt_vec_norm(tt_ctx *ctx, const tt_vec *x, double *out) {
  return guarded(ctx, [&] {
    TT_REQUIRE(x && out, "null argument");
    *out = tt::norm(&ctx->c, x->t);
  });
}

int tt_vec_sum(tt_ctx *ctx, const tt_vec *x, double *out) {
  return guarded(ctx, [&] {
    TT_REQUIRE(x && out, "null argument");
    *out = tt::sum(&ctx->c, x->t);
  });
}

int tt_round(tt_ctx *ctx, tt_vec *x, double eps, int rmax) {
  return guarded(ctx, [&] {
    TT_REQUIRE(x, "null vector");
    TT_REQUIRE(eps >= 0 && std::isfinite(eps), "tt_round: eps must be finite and >= 0");
    TT_REQUIRE(x->t.max_rank() <= 512, "tt_round: rank above 512");
    tt::round(&ctx->c, x->t, eps, rmax);
  });
}

// ---------------------------------------------------------------- operators
int tt_op_create(tt_ctx *ctx, int d, const int *m, const int *n, const int *R, const double *cores, int on_dev,
                 tt_op **out) {
  return guarded(ctx, [&] {
    TT_REQUIRE(out && m && n, "null argument");
    std::vector<int> mn(d);
    for (int k = 0; k < d; ++k) {
      TT_REQUIRE(m[k] >= 1 && n[k] >= 1, "tt_op: bad mode");
      mn[k] = m[k] * n[k];
    }
    tt::TT x = make_tt(&ctx->c, d, mn.data(), R, cores, on_dev);
    x.mo = to_vec(m, d);
    x.mi = to_vec(n, d);
    tt_op *A = new tt_op{&ctx->c, {}};
    A->op.t = std::move(x);
    *out = A;
  });
}

int tt_op_destroy(tt_op *A) {
  if (!A) return TT_EINVAL;
  delete A;
  return TT_OK;
}

int tt_op_shape(const tt_op *A, int *d, int *m, int *n, int *R) {
  if (!A || !d) return TT_EINVAL;
  const tt::TT &t = A->op.t;
  *d = t.d;
  for (int k = 0; k < t.d; ++k) {
    if (m) m[k] = t.mo[k];
    if (n) n[k] = t.mi[k];
  }
  if (R)
    for (int k = 0; k <= t.d; ++k) R[k] = t.r[k];
  return TT_OK;
}

int tt_op_numel(const tt_op *A, size_t *count) {
  if (!A || !count) return TT_EINVAL;
  *count = A->op.t.numel();
  return TT_OK;
}

int tt_op_get_cores(tt_ctx *ctx, const tt_op *A, double *dst, int on_dev) {
  return guarded(ctx, [&] {
    TT_REQUIRE(A, "null operator");
    get_cores(&ctx->c, A->op.t, dst, on_dev);
  });
}

int tt_op_axpby(tt_ctx *ctx, double a, const tt_op *A, double b, const tt_op *B, double eps, int rmax,
                tt_op **out) {
  return guarded(ctx, [&] {
    TT_REQUIRE(A && B && out, "null argument");
    for (int k = 0; k < A->op.t.d; ++k)
      TT_REQUIRE(A->op.t.mo[k] == B->op.t.mo[k] && A->op.t.mi[k] == B->op.t.mi[k], "tt_op_axpby: modes differ");
    tt::TT s = tt::add(&ctx->c, a, A->op.t, b, B->op.t);
    if (eps >= 0) tt::round(&ctx->c, s, eps, rmax);
    tt_op *C = new tt_op{&ctx->c, {}};
    C->op.t = std::move(s);
    *out = C;
  });
}

int tt_build_operator(tt_ctx *ctx, const tt_problem *prob, tt_op_kind kind, double eps_op, tt_op **out) {
  return guarded(ctx, [&] {
    TT_REQUIRE(out, "null out");
    validate_problem(prob);
    TT_REQUIRE(kind == TT_OP_H || kind == TT_OP_S || kind == TT_OP_F, "tt_build_operator: bad kind");
    TT_REQUIRE(eps_op >= 0 && eps_op < 1, "tt_build_operator: bad eps_op");
    tt_op *A = new tt_op{&ctx->c, {}};
    try {
      A->op.t = tt::build_operator(&ctx->c, prob, (int)kind, eps_op);
    } catch (...) {
      delete A;
      throw;
    }
    *out = A;
  });
}

// ---------------------------------------------------------------- products and solves
int tt_matvec(tt_ctx *ctx, const tt_op *A, const tt_vec *x, double scale, int method, double eps, int rmax,
              int max_sweeps, tt_prec prec, tt_vec **y) {
  return guarded(ctx, [&] {
    TT_REQUIRE(A && x && y, "null argument");
    TT_REQUIRE(prec == TT_FP64, "tt_matvec: only TT_FP64 is built");
    TT_REQUIRE(std::isfinite(scale), "tt_matvec: non-finite scale");
    tt::Ctx *c = &ctx->c;
    if (method == TT_MV_EXACT) {
      tt::TT r = tt::matvec_exact(c, A->op.t, x->t);
      if (eps >= 0) {
        TT_REQUIRE(r.max_rank() <= 512, "tt_matvec: product rank above 512, use TT_MV_AMEN");
        tt::round(c, r, eps, rmax);
      }
      tt::scale(c, r, scale);
      *y = new tt_vec{c, std::move(r)};
    } else if (method == TT_MV_AMEN) {
      TT_REQUIRE(eps > 0, "tt_matvec: AMEn needs eps > 0");
      tt_op *Am = const_cast<tt_op *>(A);
      std::vector<int> outn(A->op.t.d);
      for (int k = 0; k < A->op.t.d; ++k) outn[k] = A->op.t.mo[k];
      tt::TT yy = tt::tt_ones(c, outn);
      tt::amen_mv(c, Am->op, x->t, yy, eps, rmax, std::max(1, max_sweeps), 4, 12345, nullptr);
      tt::scale(c, yy, scale);
      *y = new tt_vec{c, std::move(yy)};
    } else {
      throw tt::Error(TT_EINVAL, "tt_matvec: unknown method");
    }
  });
}

int tt_solve_local(tt_ctx *ctx, const tt_op *A, const tt_vec *b, tt_vec *x, double eps, int rmax, int max_sweeps,
                   int kick, tt_prec prec, int *sweeps_done, double *rel_change) {
  int conv = 1;
  int rc = guarded(ctx, [&] {
    TT_REQUIRE(A && b && x, "null argument");
    TT_REQUIRE(prec == TT_FP64 || prec == TT_FP32_REFINED || prec == TT_TF32_SPLIT || prec == TT_BF16_SPLIT,
               "tt_solve_local: prec must be TT_FP64, TT_FP32_REFINED, TT_TF32_SPLIT or TT_BF16_SPLIT");
    TT_REQUIRE(eps > 0 && eps < 1, "tt_solve_local: eps in (0, 1)");
    TT_REQUIRE(max_sweeps >= 1 && kick >= 0, "tt_solve_local: bad sweeps/kick");
    tt_op *Am = const_cast<tt_op *>(A);
    tt::SolveStats st;
    tt::amen_solve(&ctx->c, Am->op, b->t, x->t, eps, rmax, max_sweeps, kick, 4242, &st, (int)prec);
    if (sweeps_done) *sweeps_done = st.sweeps;
    if (rel_change) *rel_change = st.max_dx;
    conv = st.max_dx < eps;
  });
  if (rc == TT_OK && !conv) {
    ctx->c.err = "tt_solve_local: sweep limit reached before the local changes fell below eps";
    return TT_ENOCONV;
  }
  return rc;
}

int tt_solve_dmrg(tt_ctx *ctx, const tt_op *A, const tt_vec *b, tt_vec *x, double eps, int rmax, int max_sweeps,
                  tt_prec prec, int *sweeps_done, double *rel_change) {
  return guarded(ctx, [&] {
    TT_REQUIRE(A && b && x, "null argument");
    TT_REQUIRE(eps > 0 && eps < 1 && max_sweeps >= 1, "tt_solve_dmrg: bad eps or max_sweeps");
    TT_REQUIRE(prec == TT_FP64 || prec == TT_FP32_REFINED || prec == TT_TF32_SPLIT || prec == TT_BF16_SPLIT,
               "tt_solve_dmrg: prec must be TT_FP64, TT_FP32_REFINED, TT_TF32_SPLIT or TT_BF16_SPLIT");
    tt_op *Am = const_cast<tt_op *>(A);
    tt::SolveStats st;
    tt::dmrg_solve(&ctx->c, Am->op, b->t, x->t, eps, rmax, max_sweeps, &st, (int)prec);
    if (sweeps_done) *sweeps_done = st.sweeps;
    if (rel_change) *rel_change = st.max_dx;
    if (st.max_dx >= eps) throw tt::Error(TT_ENOCONV, "tt_solve_dmrg: max_sweeps reached");
  });
}

int tt_scalar_flux(tt_ctx *ctx, const tt_vec *psi, const double *w_host, int n_dir, tt_vec **phi) {
  return guarded(ctx, [&] {
    TT_REQUIRE(psi && w_host && phi, "null argument");
    const tt::TT &x = psi->t;
    TT_REQUIRE(x.d >= 4 && (x.n[1] == 8 || x.n[1] == 2) && x.n[2] == n_dir,
               "tt_scalar_flux: expected cores [G][8 or 2][n_dir][...]");
    tt::Ctx *c = &ctx->c;
    std::vector<double> ones(8, 1.0);
    tt::DBuf d1(c, 8), dw(c, n_dir);
    TT_CHECK_CUDA(cudaMemcpyAsync(d1.p(), ones.data(), 8 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    TT_CHECK_CUDA(cudaMemcpyAsync(dw.p(), w_host, n_dir * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    const int r1 = x.r[1], r2 = x.r[2], r3 = x.r[3];
    tt::DBuf A(c, (size_t)r1 * r2), B(c, (size_t)r2 * r3), W(c, (size_t)r1 * r3);
    tt::contract_mode(c, x.core[1].p(), r1, x.n[1], r2, d1.p(), A.p());
    tt::contract_mode(c, x.core[2].p(), r2, n_dir, r3, dw.p(), B.p());
    tt::gemm(c, false, false, r1, r3, r2, 1.0, A.p(), r2, 0, B.p(), r3, 0, 0.0, W.p(), r3, 0);
    tt::TT y;
    y.d = x.d - 2;
    y.n.push_back(x.n[0]);
    y.r.push_back(1);
    y.r.push_back(r3);
    y.core.resize(y.d);
    y.core[0].alloc(c, (size_t)x.n[0] * r3);
    tt::gemm(c, false, false, x.n[0], r3, r1, 1.0, x.core[0].p(), r1, 0, W.p(), r3, 0, 0.0, y.core[0].p(), r3, 0);
    for (int k = 3; k < x.d; ++k) {
      y.n.push_back(x.n[k]);
      y.r.push_back(x.r[k + 1]);
      y.core[k - 2].alloc(c, x.csize(k));
      tt::copy(c, y.core[k - 2].p(), x.core[k].p(), x.csize(k));
    }
    c->sync();
    *phi = new tt_vec{c, std::move(y)};
  });
}

int keig_default_opts(keig_opts *o) {
  if (!o) return TT_EINVAL;
  o->eps = 1e-7;
  o->rmax = 64;
  o->tol_k = 1e-9;
  o->tol_psi = 1e-5;
  o->max_iter = 400;
  o->solve_sweeps = 2;
  o->mv_sweeps = 2;
  o->kick = 4;
  o->scheme = 0;
  o->prec = TT_FP64;
  o->eps_op = 1e-12;
  o->psi0_cores = nullptr;
  o->mv_kind = 0;
  o->local_form = 0;
  o->solve_method = 0;
  return TT_OK;
}

}  // extern "C"

namespace {

using clk = std::chrono::steady_clock;

void check_opts(const keig_opts *opts) {
  TT_REQUIRE(opts, "null options");
  TT_REQUIRE(opts->prec == TT_FP64 || opts->prec == TT_FP32_REFINED || opts->prec == TT_TF32_SPLIT ||
                 opts->prec == TT_BF16_SPLIT,
             "keig: prec must be TT_FP64, TT_FP32_REFINED, TT_TF32_SPLIT or TT_BF16_SPLIT");
  TT_REQUIRE(opts->eps > 0 && opts->eps < 1 && opts->max_iter >= 1, "keig: bad eps/max_iter");
  TT_REQUIRE(opts->scheme == 0 || opts->scheme == 1, "keig: scheme must be 0 or 1");
  TT_REQUIRE(opts->mv_kind == 0 || opts->mv_kind == 1, "keig: mv_kind must be 0 or 1");
  TT_REQUIRE(opts->local_form == 0 || opts->local_form == 1, "keig: local_form must be 0 or 1");
  TT_REQUIRE(opts->solve_method == 0 || opts->solve_method == 2,
             "keig: solve_method must be 0 (AMEn) or 2 (two-site DMRG); one-site ALS (tt_solve_local with "
             "kick 0) keeps the ranks of its initial guess and does not converge inside the fixed point");
  TT_REQUIRE(!(opts->solve_method == 2 && opts->local_form == 1),
             "keig: the two-site DMRG solve uses Galerkin local systems (local_form 0)");
}

// The operators of one problem, forward or transposed (adjoint).
struct KeigOps {
  tt::TTOp LHS, RHS;  // scheme 0: H and S (+) F; scheme 1: H - S and F
  tt::TT f;           // sum(F Psi) = <f, Psi>
  int rS = 0;         // columns of the first RHS core that belong to S (scheme 0)
  bool ls = false;    // least-squares local systems: solve N Psi' = M^T B
  tt::TTOp N, MT;     // N = M^T M and M^T for the system matrix M (= LHS)
};

// N = M^T M for M = sum_b M_b whose row blocks M_b have disjoint rows
// (so M^T M = sum_b M_b^T M_b): each product is rounded before it is added.
tt::TT normal_operator(tt::Ctx *c, const std::vector<tt::TT> &blocks, double eps_op) {
  tt::TT N;
  for (size_t b = 0; b < blocks.size(); ++b) {
    for (int k = 1; k < blocks[b].d; ++k)
      TT_REQUIRE((long long)blocks[b].r[k] * blocks[b].r[k] <= 512,
                 "least-squares local systems: an operator block's rank is above 22");
    tt::TT P = tt::op_matmul_tn(c, blocks[b], blocks[b]);
    tt::round(c, P, eps_op, 0);
    if (b == 0) {
      N = std::move(P);
    } else {
      N = tt::add(c, 1.0, N, 1.0, P);
      tt::round(c, N, eps_op, 0);
    }
  }
  return N;
}

// The least-squares form of the linear solve (Eq. (linear_system_obj):
// minimise ||M Psi' - B||): its local systems are the projections of
// N = M^T M with right-hand side M^T B.  blocks: row blocks of M (empty: M
// itself as one block).
void make_ls(tt::Ctx *c, KeigOps &o, std::vector<tt::TT> blocks, const keig_opts *opts) {
  if (blocks.empty()) blocks.push_back(tt::tt_clone(c, o.LHS.t));
  o.N.t = normal_operator(c, blocks, opts->eps_op);
  o.MT.t = tt::transpose_op(c, o.LHS.t);
  o.ls = true;
}

KeigOps make_ops(tt::Ctx *c, tt::TT H, tt::TT S, tt::TT F, const keig_opts *opts) {
  KeigOps o;
  tt::TT ones = tt::tt_ones(c, F.mi);
  tt::TT FT = tt::transpose_op(c, F);
  o.f = tt::matvec_exact(c, FT, ones);
  tt::round(c, o.f, 1e-13, 0);
  o.rS = S.r[1];
  if (opts->scheme == 0) {
    o.RHS.t = tt::add(c, 1.0, S, 1.0, F);
    o.LHS.t = std::move(H);
  } else {
    o.RHS.t = std::move(F);
    o.LHS.t = tt::add(c, 1.0, H, -1.0, S);
    tt::round(c, o.LHS.t, opts->eps_op, 0);
  }
  return o;
}

// Eq. (TT_k_eff_fixed_points) on prepared operators; returns convergence.
bool run_fixed_point(tt::Ctx *c, KeigOps &ops, const keig_opts *opts, keig_result *out, tt::TT &psi,
                     clk::time_point t0, uint64_t seed) {
  auto ms = [&] { return std::chrono::duration<double, std::milli>(clk::now() - t0).count(); };
  const int d = ops.LHS.t.d;
  std::vector<int> modes = ops.LHS.t.mi;
  psi = tt::tt_ones(c, modes);
  if (opts->psi0_cores) {
    size_t off = 0;
    for (int k = 0; k < d; ++k) {
      check_finite_host(opts->psi0_cores + off, modes[k], "psi0");
      TT_CHECK_CUDA(cudaMemcpyAsync(psi.core[k].p(), opts->psi0_cores + off, modes[k] * sizeof(double),
                                    cudaMemcpyHostToDevice, c->stream));
      off += modes[k];
    }
  }
  double s = tt::dot(c, ops.f, psi);
  TT_REQUIRE(s != 0.0 && std::isfinite(s), "keig: initial guess has zero production");
  tt::scale(c, psi, 1.0 / s);
  double k = 1.0;
  double k_in_op = 1.0;  // 1/k_in_op is the scale of the F block stored in RHS
  tt::TT B = tt::tt_clone(c, psi);
  int it = 0;
  double dk = 1e300;
  bool conv = false;
  for (it = 0; it < opts->max_iter; ++it) {
    const double fac = k_in_op / k;  // rescale the F part from 1/k_in_op to 1/k
    if (opts->scheme == 0) {
      // F's first core occupies columns [rS, rS + rF) of the (1, G*G, rS + rF) first core
      const int rtot = ops.RHS.t.r[1], rF = rtot - ops.rS, ncol = ops.RHS.t.n[0];
      tt::copy2d(c, ops.RHS.t.core[0].p() + ops.rS, rtot, ops.RHS.t.core[0].p() + ops.rS, rtot, ncol, rF, fac);
    } else {
      tt::scale(c, ops.RHS.t.core[0].p(), ops.RHS.t.csize(0), fac);
    }
    ops.RHS.invalidate();
    k_in_op = k;
    tt::SolveStats mst, sst;
    if (opts->mv_kind == 1) {
      tt::PhaseTimer pt(c, "keig.mv_exact");
      B = tt::matvec_exact(c, ops.RHS.t, psi);
      tt::round(c, B, opts->eps, opts->rmax);
    } else {
      tt::PhaseTimer pt(c, "keig.mv");
      tt::amen_mv(c, ops.RHS, psi, B, opts->eps, opts->rmax, opts->mv_sweeps, opts->kick, seed + 1000 + it, &mst);
    }
    tt::TT psi_new = tt::tt_clone(c, psi);
    {
      tt::PhaseTimer pt(c, "keig.solve");
      const int kick = opts->kick;
      if (opts->solve_method == 2)
        tt::dmrg_solve(c, ops.LHS, B, psi_new, opts->eps, opts->rmax, opts->solve_sweeps, &sst, (int)opts->prec);
      else if (ops.ls)
        tt::amen_solve(c, ops.N, B, psi_new, opts->eps, opts->rmax, opts->solve_sweeps, kick, seed + 5000 + it,
                       &sst, (int)opts->prec, &ops.MT);
      else
        tt::amen_solve(c, ops.LHS, B, psi_new, opts->eps, opts->rmax, opts->solve_sweeps, kick, seed + 5000 + it,
                       &sst, (int)opts->prec);
    }
    if (c->phase_timing)
      fprintf(stderr, "keig it %d k %.12f mv_sweeps %d mv_dx %.2e solve_sweeps %d solve_dx %.2e gmres %lld ranks B %d psi %d\n",
              it, k, mst.sweeps, mst.max_dx, sst.sweeps, sst.max_dx, sst.gmres_iters, B.max_rank(), psi_new.max_rank());
    const double sn = tt::dot(c, ops.f, psi_new);
    if (!std::isfinite(sn) || sn == 0.0) throw tt::Error(TT_ENONFINITE, "keig: production became zero or non-finite");
    const double kn = k * sn;
    tt::scale(c, psi_new, 1.0 / sn);
    // relative change of Psi: ||a - b||^2 = <a,a> + <b,b> - 2<a,b>
    const double aa = tt::dot(c, psi_new, psi_new), bb = tt::dot(c, psi, psi), ab = tt::dot(c, psi_new, psi);
    const double dpsi = std::sqrt(std::max(aa + bb - 2 * ab, 0.0) / std::max(aa, 1e-300));
    dk = std::fabs(kn - k) / std::fabs(kn);
    k = kn;
    psi = std::move(psi_new);
    if (it < 512) {
      out->k_hist[it] = k;
      out->t_hist[it] = ms();
    }
    if (dk < opts->tol_k && dpsi < opts->tol_psi) {
      ++it;
      conv = true;
      break;
    }
  }
  if (c->phase_timing) {
    for (auto &p : c->phase_ms)
      fprintf(stderr, "phase %-22s %10.1f ms %8lld calls\n", p.name.c_str(), p.ms, p.calls);
    c->phase_ms.clear();
  }
  out->k = k;
  out->iters = std::min(it, opts->max_iter);
  out->dk_last = dk;
  out->max_rank = psi.max_rank();
  return conv;
}

// <y, A x> by the left-interface chain over all cores
double bilinear(tt::Ctx *c, tt::TTOp &A, const tt::TT &y, const tt::TT &x) {
  A.prepare(c);
  const tt::TT &a = A.t;
  tt::DBuf phi(c, 1), nxt, T1, T2;
  tt::fill(c, phi.p(), 1, 1.0);
  for (int k = 0; k < a.d; ++k) {
    tt::left_update(c, phi.p(), y.core[k].p(), A.a_ajib[k].p(), x.core[k].p(), y.r[k], a.r[k], x.r[k], a.mo[k],
                    a.mi[k], a.r[k + 1], y.r[k + 1], x.r[k + 1], nxt, T1, T2);
    phi.swap(nxt);
  }
  TT_CHECK_CUDA(cudaMemcpyAsync(c->h_pinned, phi.p(), sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  c->sync();
  return c->h_pinned[0];
}

// W[g, g'] = <y, (e_g e_g'^T (x) B) x> for an operator B over the cores after
// the group core: the right-interface chain of (y, B, x) over cores 1..d-1,
// then the open contraction with the first cores of y and x.
std::vector<double> open_bilinear(tt::Ctx *c, tt::TTOp &B, const tt::TT &y, const tt::TT &x) {
  B.prepare(c);
  const tt::TT &b = B.t;
  TT_REQUIRE(b.d == y.d - 1 && b.d == x.d - 1, "open_bilinear: dimension mismatch");
  tt::DBuf phi(c, 1), nxt, T1, T2;
  tt::fill(c, phi.p(), 1, 1.0);
  for (int k = y.d - 1; k >= 1; --k) {
    const int q = k - 1;  // core index in B
    tt::right_update(c, phi.p(), y.core[k].p(), B.a_jbai[q].p(), x.core[k].p(), y.r[k], b.r[q], x.r[k], b.mo[q],
                     b.mi[q], b.r[q + 1], y.r[k + 1], x.r[k + 1], nxt, T1, T2);
    phi.swap(nxt);
  }
  // phi: (ry1, 1, rx1);  W = y0 (G x ry1) phi x0^T (rx1 x G)
  const int G = y.n[0], ry1 = y.r[1], rx1 = x.r[1];
  tt::DBuf t(c, (size_t)G * rx1), W(c, (size_t)G * G);
  tt::gemm(c, false, false, G, rx1, ry1, 1.0, y.core[0].p(), ry1, 0, phi.p(), rx1, 0, 0.0, t.p(), rx1, 0);
  tt::gemm(c, false, true, G, G, rx1, 1.0, t.p(), rx1, 0, x.core[0].p(), rx1, 0, 0.0, W.p(), G, 0);
  std::vector<double> w((size_t)G * G);
  TT_CHECK_CUDA(cudaMemcpyAsync(w.data(), W.p(), w.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  c->sync();
  return w;
}

}  // namespace

extern "C" {

int keig_fixed_point(tt_ctx *ctx, const tt_problem *prob, const keig_opts *opts, keig_result *out,
                     tt_vec **psi_out, double *phi_out) {
  int conv = 0;
  int rc = guarded(ctx, [&] {
    TT_REQUIRE(out, "null argument");
    validate_problem(prob);
    check_opts(opts);
    const auto t0 = clk::now();
    tt::Ctx *c = &ctx->c;
    memset(out, 0, sizeof(*out));
    // operators (Sec. 3.2-3.3)
    tt::TT H, S, F;
    std::vector<tt::TT> blocks;  // octant row blocks of the system matrix (least-squares form)
    {
      tt::PhaseTimer pt(c, "keig.build_ops");
      tt::OpFactors fac = tt::make_factors(c, prob);
      H = tt::assemble_operator(c, prob, fac, TT_OP_H, -1, opts->eps_op);
      S = tt::assemble_operator(c, prob, fac, TT_OP_S, -1, opts->eps_op);
      F = tt::assemble_operator(c, prob, fac, TT_OP_F, -1, opts->eps_op);
      if (opts->local_form == 1)
        for (int o = 0; o < 8; ++o) {
          tt::TT Ho = tt::assemble_operator(c, prob, fac, TT_OP_H, -1, opts->eps_op, o);
          if (opts->scheme == 1) {
            tt::TT So = tt::assemble_operator(c, prob, fac, TT_OP_S, -1, opts->eps_op, o);
            Ho = tt::add(c, 1.0, Ho, -1.0, So);
            tt::round(c, Ho, opts->eps_op, 0);
          }
          blocks.push_back(std::move(Ho));
        }
    }
    KeigOps ops = make_ops(c, std::move(H), std::move(S), std::move(F), opts);
    if (opts->local_form == 1) {
      tt::PhaseTimer pt(c, "keig.build_normal");
      make_ls(c, ops, std::move(blocks), opts);
    }
    tt::TT psi;
    conv = run_fixed_point(c, ops, opts, out, psi, t0, 0);
    if (phi_out) {
      // scalar flux on the vertices, dense
      const int n = 1 << prob->l;
      tt_vec tmp{c, std::move(psi)};
      tt_vec *phi = nullptr;
      int r2 = tt_scalar_flux(ctx, &tmp, prob->w, prob->n_dir, &phi);
      if (r2 != TT_OK) throw tt::Error(r2, ctx->c.err);
      const size_t len = (size_t)prob->G * n * n * n;
      tt::DBuf dst(c, len);
      tt::to_dense(c, phi->t, dst.p(), len);
      TT_CHECK_CUDA(cudaMemcpyAsync(phi_out, dst.p(), len * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      c->sync();
      tt_vec_destroy(phi);
      psi = std::move(tmp.t);
    }
    if (psi_out) *psi_out = new tt_vec{c, std::move(psi)};
    c->sync();
    out->wall_ms = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
  });
  if (rc == TT_OK && !conv) {
    ctx->c.err = "keig_fixed_point: max_iter reached";
    return TT_ENOCONV;
  }
  return rc;
}

int keig_sensitivities(tt_ctx *ctx, const tt_problem *prob, const keig_opts *opts, double *dk_dsig_t,
                       double *dk_dsig_s, double *dk_dnu_sig_f, double *dk_dchi, keig_sens_info *info) {
  int conv = 0;
  int rc = guarded(ctx, [&] {
    validate_problem(prob);
    check_opts(opts);
    TT_REQUIRE(dk_dsig_t && dk_dsig_s && dk_dnu_sig_f && dk_dchi, "keig_sensitivities: null output");
    const auto t0 = clk::now();
    tt::Ctx *c = &ctx->c;
    const int G = prob->G, nm = prob->n_mat;
    tt::OpFactors fac = tt::make_factors(c, prob);
    tt::TT H = tt::assemble_operator(c, prob, fac, TT_OP_H, -1, opts->eps_op);
    tt::TT S = tt::assemble_operator(c, prob, fac, TT_OP_S, -1, opts->eps_op);
    tt::TT F = tt::assemble_operator(c, prob, fac, TT_OP_F, -1, opts->eps_op);
    // forward and adjoint fixed points (the adjoint uses the transposed
    // operators; it has the same eigenvalue)
    keig_result fwd, adj;
    memset(&fwd, 0, sizeof(fwd));
    memset(&adj, 0, sizeof(adj));
    tt::TTOp Fop;
    Fop.t = tt::tt_clone(c, F);
    KeigOps opsT = make_ops(c, tt::transpose_op(c, H), tt::transpose_op(c, S), tt::transpose_op(c, F), opts);
    KeigOps ops = make_ops(c, std::move(H), std::move(S), std::move(F), opts);
    tt::TT psi, psa;
    const bool c1 = run_fixed_point(c, ops, opts, &fwd, psi, t0, 0);
    const bool c2 = run_fixed_point(c, opsT, opts, &adj, psa, t0, 77);
    conv = c1 && c2;
    const double k = fwd.k;
    // <Psi^dagger, F Psi>
    const double P = bilinear(c, Fop, psa, psi);
    TT_REQUIRE(std::isfinite(P) && P != 0.0, "keig_sensitivities: <Psi^dagger, F Psi> vanished");
    // dk = -k^2 <Psi^dagger, (dH - dS - dF/k) Psi> / <Psi^dagger, F Psi>
    for (int m = 0; m < nm; ++m) {
      tt::TTOp Bc, Bs;
      Bc.t = tt::assemble_operator(c, prob, fac, tt::KIND_COLLISION, m, opts->eps_op);
      Bs.t = tt::assemble_operator(c, prob, fac, tt::KIND_SOURCE, m, opts->eps_op);
      const std::vector<double> Wc = open_bilinear(c, Bc, psa, psi);
      const std::vector<double> Ws = open_bilinear(c, Bs, psa, psi);
      const double *chi = prob->chi + (size_t)m * G, *nsf = prob->nu_sig_f + (size_t)m * G;
      for (int g = 0; g < G; ++g) {
        dk_dsig_t[(size_t)m * G + g] = -k * k * Wc[(size_t)g * G + g] / P;
        double a = 0.0, b = 0.0;
        for (int h = 0; h < G; ++h) {
          dk_dsig_s[((size_t)m * G + g) * G + h] = k * k * Ws[(size_t)g * G + h] / P;
          a += chi[h] * Ws[(size_t)h * G + g];  // d/d nsf_g: sum over destination groups h
          b += Ws[(size_t)g * G + h] * nsf[h];  // d/d chi_g: sum over source groups h
        }
        dk_dnu_sig_f[(size_t)m * G + g] = k * a / P;
        dk_dchi[(size_t)m * G + g] = k * b / P;
      }
    }
    if (info) {
      info->k = fwd.k;
      info->k_adjoint = adj.k;
      info->iters = fwd.iters;
      info->iters_adjoint = adj.iters;
      info->adjoint_production = P;
      info->wall_ms = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    }
  });
  if (rc == TT_OK && !conv) {
    ctx->c.err = "keig_sensitivities: a fixed point reached max_iter";
    return TT_ENOCONV;
  }
  return rc;
}

int keig_slab_fixed_point(tt_ctx *ctx, const tt_slab *slab, const keig_opts *opts, keig_result *out,
                          double *phi_out) {
  int conv = 0;
  int rc = guarded(ctx, [&] {
    TT_REQUIRE(slab && out, "keig_slab_fixed_point: null argument");
    check_opts(opts);
    TT_REQUIRE(slab->l >= 1 && slab->l <= 24, "slab: l out of range");
    TT_REQUIRE(slab->G >= 1 && slab->G <= 4096 && slab->n_mat >= 1 && slab->n_mat <= 255, "slab: bad G or n_mat");
    TT_REQUIRE(slab->n_dir >= 1 && slab->n_dir <= 4096, "slab: bad n_dir");
    TT_REQUIRE(std::isfinite(slab->width) && slab->width > 0, "slab: bad width");
    TT_REQUIRE(slab->sig_t && slab->sig_s && slab->nu_sig_f && slab->chi && slab->mat && slab->amu && slab->w,
               "slab: null table");
    const size_t G = slab->G, nm = slab->n_mat, nd = slab->n_dir, n = (size_t)1 << slab->l;
    check_finite_host(slab->sig_t, nm * G, "sig_t");
    check_finite_host(slab->sig_s, nm * G * G, "sig_s");
    check_finite_host(slab->nu_sig_f, nm * G, "nu_sig_f");
    check_finite_host(slab->chi, nm * G, "chi");
    check_finite_host(slab->amu, nd, "amu");
    check_finite_host(slab->w, nd, "w");
    for (size_t i = 0; i + 1 < n; ++i) TT_REQUIRE(slab->mat[i] < nm, "slab: material index out of range");
    for (size_t i = 0; i < nd; ++i) TT_REQUIRE(slab->amu[i] > 0, "slab: amu must be positive");
    const auto t0 = clk::now();
    tt::Ctx *c = &ctx->c;
    memset(out, 0, sizeof(*out));
    tt::TT H, S, F;
    {
      tt::PhaseTimer pt(c, "keig.build_ops");
      H = tt::assemble_slab_operator(c, slab, TT_OP_H, opts->eps_op);
      S = tt::assemble_slab_operator(c, slab, TT_OP_S, opts->eps_op);
      F = tt::assemble_slab_operator(c, slab, TT_OP_F, opts->eps_op);
    }
    KeigOps ops = make_ops(c, std::move(H), std::move(S), std::move(F), opts);
    tt::TT psi;
    conv = run_fixed_point(c, ops, opts, out, psi, t0, 0);
    if (phi_out) {
      tt_vec tmp{c, std::move(psi)};
      tt_vec *phi = nullptr;
      const int r2 = tt_scalar_flux(ctx, &tmp, slab->w, slab->n_dir, &phi);
      if (r2 != TT_OK) throw tt::Error(r2, ctx->c.err);
      const size_t len = G * n;
      tt::DBuf dst(c, len);
      tt::to_dense(c, phi->t, dst.p(), len);
      TT_CHECK_CUDA(cudaMemcpyAsync(phi_out, dst.p(), len * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      c->sync();
      tt_vec_destroy(phi);
    }
    c->sync();
    out->wall_ms = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
  });
  if (rc == TT_OK && !conv) {
    ctx->c.err = "keig_slab_fixed_point: max_iter reached";
    return TT_ENOCONV;
  }
  return rc;
}

int keig_gpt(tt_ctx *ctx, const tt_problem *prob, const keig_opts *opts, const double *resp_g,
             const double *resp_v, double tol_gpt, int max_gpt, double *dJ_dsig_t, double *dJ_dsig_s,
             double *dJ_dnu_sig_f, double *dJ_dchi, keig_gpt_info *info) {
  int conv = 0;
  const char *stage = "setup";
  int rc = guarded(ctx, [&] {
   try {
    validate_problem(prob);
    check_opts(opts);
    TT_REQUIRE(resp_g && resp_v, "keig_gpt: null response");
    TT_REQUIRE(dJ_dsig_t && dJ_dsig_s && dJ_dnu_sig_f && dJ_dchi, "keig_gpt: null output");
    TT_REQUIRE(tol_gpt > 0 && max_gpt >= 1 && max_gpt <= 10000, "keig_gpt: bad tolerance or step limit");
    const int G = prob->G, nm = prob->n_mat, l = prob->l;
    const size_t nv = (size_t)1 << (3 * l);
    check_finite_host(resp_g, G, "resp_g");
    check_finite_host(resp_v, nv, "resp_v");
    const auto t0 = clk::now();
    tt::Ctx *c = &ctx->c;
    tt::OpFactors fac = tt::make_factors(c, prob);
    tt::TT H = tt::assemble_operator(c, prob, fac, TT_OP_H, -1, opts->eps_op);
    tt::TT S = tt::assemble_operator(c, prob, fac, TT_OP_S, -1, opts->eps_op);
    tt::TT F = tt::assemble_operator(c, prob, fac, TT_OP_F, -1, opts->eps_op);
    tt::TT HT = tt::transpose_op(c, H), ST = tt::transpose_op(c, S), FT = tt::transpose_op(c, F);
    tt::TTOp Fop;
    Fop.t = tt::tt_clone(c, F);
    KeigOps opsT = make_ops(c, tt::tt_clone(c, HT), tt::tt_clone(c, ST), tt::tt_clone(c, FT), opts);
    KeigOps ops = make_ops(c, std::move(H), std::move(S), std::move(F), opts);
    keig_result fwd, adj;
    memset(&fwd, 0, sizeof(fwd));
    memset(&adj, 0, sizeof(adj));
    tt::TT psi, psa;
    stage = "fixed points";
    const bool c1 = run_fixed_point(c, ops, opts, &fwd, psi, t0, 0);
    const bool c2 = run_fixed_point(c, opsT, opts, &adj, psa, t0, 77);
    const double k = fwd.k;
    const double P = bilinear(c, Fop, psa, psi);  // <Psi^dagger, F Psi>
    TT_REQUIRE(std::isfinite(P) && P != 0.0, "keig_gpt: <Psi^dagger, F Psi> vanished");
    stage = "F Psi";
    tt::TT Fpsi = tt::matvec_exact(c, Fop.t, psi);
    tt::round(c, Fpsi, 1e-13, 0);
    // j = resp_g (x) (1_8 (x) w) (x) resp_v as a TT with the core order of Psi:
    // the quadrature is octant-symmetric (w holds one octant's weights), so
    // the angular factor has rank one; the vertex field is TT-SVD compressed
    stage = "response TT";
    tt::TT j;
    {
      const int npo = prob->n_dir;
      tt::DBuf dv(c, nv);
      TT_CHECK_CUDA(cudaMemcpyAsync(dv.p(), resp_v, nv * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      tt::TT jv = tt::tt_svd_dense(c, dv.p(), std::vector<int>(3 * l, 2), 1e-15, 0);
      j.d = 3 + jv.d;
      j.n = {G, 8, npo};
      j.r = {1, 1, 1};
      j.core.resize(j.d);
      j.core[0].alloc(c, (size_t)G);
      j.core[1].alloc(c, 8);
      j.core[2].alloc(c, (size_t)npo);
      TT_CHECK_CUDA(cudaMemcpyAsync(j.core[0].p(), resp_g, (size_t)G * sizeof(double), cudaMemcpyHostToDevice,
                                    c->stream));
      tt::fill(c, j.core[1].p(), 8, 1.0);
      TT_CHECK_CUDA(cudaMemcpyAsync(j.core[2].p(), prob->w, (size_t)npo * sizeof(double), cudaMemcpyHostToDevice,
                                    c->stream));
      for (int i = 0; i < jv.d; ++i) {
        j.n.push_back(jv.n[i]);
        j.r.push_back(jv.r[i]);
        j.core[3 + i] = std::move(jv.core[i]);
      }
      j.r.push_back(1);
      c->sync();  // the host staging above must outlive its copies
    }
    TT_REQUIRE(j.d == psi.d, "keig_gpt: response layout does not match the flux");
    stage = "functional and GPT source";
    const double J = tt::dot(c, j, psi);
    // s = j - J f
    tt::TT src = tt::add(c, 1.0, j, -J, ops.f);
    tt::round(c, src, 1e-14, 0);
    // H^T Gamma' = (S^T + F^T/k) Gamma + s, fundamental adjoint mode removed
    tt::TTOp LT, RT;
    LT.t = std::move(HT);
    RT.t = tt::add(c, 1.0, ST, 1.0 / k, FT);
    tt::TT gam = tt::tt_clone(c, src), B = tt::tt_clone(c, src);
    double change = 1e300;
    int it = 0;
    bool c3 = false;
    stage = "GPT iteration";
    for (it = 0; it < max_gpt; ++it) {
      tt::SolveStats mst, sst;
      tt::amen_mv(c, RT, gam, B, opts->eps, opts->rmax, opts->mv_sweeps, opts->kick, 9000 + it, &mst);
      tt::TT rhs = tt::add(c, 1.0, B, 1.0, src);
      tt::round(c, rhs, opts->eps, opts->rmax);
      tt::TT gnew = tt::tt_clone(c, gam);
      tt::amen_solve(c, LT, rhs, gnew, opts->eps, opts->rmax, opts->solve_sweeps, opts->kick, 19000 + it, &sst,
                     (int)opts->prec);
      const double cdef = tt::dot(c, gnew, Fpsi) / P;
      tt::TT g2 = tt::add(c, 1.0, gnew, -cdef, psa);
      tt::round(c, g2, opts->eps, opts->rmax);
      const double aa = tt::dot(c, g2, g2), bb = tt::dot(c, gam, gam), ab = tt::dot(c, g2, gam);
      if (!std::isfinite(aa) || !std::isfinite(ab)) throw tt::Error(TT_ENONFINITE, "keig_gpt: non-finite adjoint");
      change = std::sqrt(std::max(aa + bb - 2 * ab, 0.0) / std::max(aa, 1e-300));
      gam = std::move(g2);
      if (change < tol_gpt) {
        ++it;
        c3 = true;
        break;
      }
    }
    conv = c1 && c2 && c3;
    // dJ/dp = -<Gamma, (dH - dS - dF/k) Psi> - J sum(dF Psi), per material through
    // the open contractions (the sum is the contraction with the all-ones TT)
    stage = "derivative contractions";
    tt::TT ones = tt::tt_ones(c, psi.n);
    for (int m = 0; m < nm; ++m) {
      tt::TTOp Bc, Bs;
      Bc.t = tt::assemble_operator(c, prob, fac, tt::KIND_COLLISION, m, opts->eps_op);
      Bs.t = tt::assemble_operator(c, prob, fac, tt::KIND_SOURCE, m, opts->eps_op);
      const std::vector<double> Wc = open_bilinear(c, Bc, gam, psi);
      const std::vector<double> Ws = open_bilinear(c, Bs, gam, psi);
      const std::vector<double> W1 = open_bilinear(c, Bs, ones, psi);
      const double *chi = prob->chi + (size_t)m * G, *nsf = prob->nu_sig_f + (size_t)m * G;
      for (int g = 0; g < G; ++g) {
        dJ_dsig_t[(size_t)m * G + g] = -Wc[(size_t)g * G + g];
        double a = 0.0, b = 0.0;
        for (int h = 0; h < G; ++h) {
          dJ_dsig_s[((size_t)m * G + g) * G + h] = Ws[(size_t)g * G + h];
          a += chi[h] * (Ws[(size_t)h * G + g] / k - J * W1[(size_t)h * G + g]);  // d/d nsf_g
          b += (Ws[(size_t)g * G + h] / k - J * W1[(size_t)g * G + h]) * nsf[h];  // d/d chi_g
        }
        dJ_dnu_sig_f[(size_t)m * G + g] = a;
        dJ_dchi[(size_t)m * G + g] = b;
      }
    }
    if (info) {
      info->J = J;
      info->k = k;
      info->iters = fwd.iters;
      info->iters_adjoint = adj.iters;
      info->iters_gpt = it;
      info->gpt_change = change;
      info->wall_ms = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    }
   } catch (const tt::Error &e) {
    throw tt::Error(e.code, std::string("keig_gpt (") + stage + "): " + e.what());
   }
  });
  if (rc == TT_OK && !conv) {
    ctx->c.err = "keig_gpt: a fixed point or the GPT iteration reached its limit";
    return TT_ENOCONV;
  }
  return rc;
}

int keig_alpha(tt_ctx *ctx, const tt_problem *prob, const keig_opts *opts, double tol_k1, int max_steps,
               keig_alpha_result *out) {
  int conv = 0;
  int rc = guarded(ctx, [&] {
    validate_problem(prob);
    check_opts(opts);
    TT_REQUIRE(out, "keig_alpha: null result");
    TT_REQUIRE(prob->inv_v, "keig_alpha: the problem needs inv_v");
    check_finite_host(prob->inv_v, prob->G, "inv_v");
    TT_REQUIRE(tol_k1 > 0 && max_steps >= 1 && max_steps <= 64, "keig_alpha: bad tolerance or step limit");
    const auto t0 = clk::now();
    memset(out, 0, sizeof(*out));
    const int G = prob->G, nm = prob->n_mat;
    std::vector<double> st((size_t)nm * G);
    tt_problem q = *prob;
    int n = 0;
    // k(alpha): the k-eigenvalue of (H + alpha V^{-1}) Psi = (S + F/k) Psi.  V^{-1}
    // has the structure of the collision term, so H + alpha V^{-1} is H with
    // sigma_t + alpha / v.
    auto k_of = [&](double a) {
      for (int m = 0; m < nm; ++m)
        for (int g = 0; g < G; ++g) st[(size_t)m * G + g] = prob->sig_t[(size_t)m * G + g] + a * prob->inv_v[g];
      q.sig_t = st.data();
      keig_result r;
      const int rr = keig_fixed_point(ctx, &q, opts, &r, nullptr, nullptr);
      if (rr != TT_OK && rr != TT_ENOCONV) throw tt::Error(rr, ctx->c.err);
      out->outer_iters += r.iters;
      if (n < 64) {
        out->alpha_hist[n] = a;
        out->k_hist[n] = r.k;
      }
      ++n;
      return r.k;
    };
    // Eq. (alpha_eig_fixed_points): alpha^0 = 0, alpha^1 = 0.01, then the
    // secant step on k(alpha) = 1
    double a0 = 0.0, a1 = 0.01;
    double k0 = k_of(a0), k1 = k_of(a1);
    for (int s = 0; s < max_steps && std::fabs(k1 - 1.0) >= tol_k1; ++s) {
      TT_REQUIRE(k1 != k0, "keig_alpha: k(alpha) did not change between secant points");
      const double a2 = a0 + (1.0 - k0) * (a1 - a0) / (k1 - k0);
      a0 = a1;
      k0 = k1;
      a1 = a2;
      k1 = k_of(a1);
    }
    conv = std::fabs(k1 - 1.0) < tol_k1;
    out->alpha = a1;
    out->k = k1;
    out->steps = n;
    out->wall_ms = std::chrono::duration<double, std::milli>(clk::now() - t0).count();
  });
  if (rc == TT_OK && !conv) {
    ctx->c.err = "keig_alpha: secant step limit reached";
    return TT_ENOCONV;
  }
  return rc;
}

int keig_batch(tt_ctx *const *ctxs, int n_ctx, const tt_problem *probs, const keig_opts *opts, int n_prob,
               keig_result *out, int *status) {
  if (!ctxs || n_ctx < 1 || n_ctx > 1024 || !probs || !opts || !out || !status || n_prob < 0) return TT_EINVAL;
  for (int w = 0; w < n_ctx; ++w)
    if (!ctxs[w] || ctxs[w]->c.device != ctxs[0]->c.device || ctxs[w]->c.group) return TT_EINVAL;
  // the workers' persistent-GMRES systems share grouped launches
  tt::PGGroup *group = nullptr;
  if (n_ctx > 1 && getenv("KEIG_BATCH_UNGROUPED") == nullptr) {
    cudaSetDevice(ctxs[0]->c.device);
    try {
      group = tt::pg_group_create(ctxs[0]->c.device, ctxs[0]->c.sm_count);
    } catch (const tt::Error &e) {
      return e.code;
    }
    tt::pg_group_set_active(group, 0);
  }
  std::atomic<int> next{0};
  auto worker = [&](int w) {
    cudaSetDevice(ctxs[w]->c.device);
    ctxs[w]->c.group = group;
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= n_prob) break;
      if (group) tt::pg_group_join(group);
      status[i] = keig_fixed_point(ctxs[w], &probs[i], &opts[i], &out[i], nullptr, nullptr);
      if (group) tt::pg_group_leave(group);
    }
    ctxs[w]->c.group = nullptr;
  };
  std::vector<std::thread> th;
  th.reserve(n_ctx);
  for (int w = 0; w < n_ctx; ++w) th.emplace_back(worker, w);
  for (auto &t : th) t.join();
  if (group) {
    long long l = 0, s = 0;
    tt::pg_group_stats(group, &l, &s);
    g_batch_group_launches = l;
    g_batch_group_systems = s;
    tt::pg_group_destroy(group);
  } else {
    g_batch_group_launches = g_batch_group_systems = 0;
  }
  int rc = TT_OK;
  for (int i = 0; i < n_prob && rc == TT_OK; ++i)
    if (status[i] != TT_OK) rc = status[i];
  return rc;
}

int keig_batch_stats(long long *group_launches, long long *group_systems) {
  if (!group_launches || !group_systems) return TT_EINVAL;
  *group_launches = g_batch_group_launches;
  *group_systems = g_batch_group_systems;
  return TT_OK;
}

}  // extern "C"
