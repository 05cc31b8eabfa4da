/*
 * keig.h — C-ABI of the GB300 tensor-train k-eigenvalue library.
 *
 * Method: arXiv 2309.03347 ("Tensor networks for solving realistic
 * time-independent Boltzmann neutron transport equation").  The discretised
 * k-eigenvalue problem H Psi = (S + F/k) Psi (Eq. (OpFormkNTE)) is solved in a
 * mixed TT/QTT format (Sec. 3.2-3.4): every operator is a sum of tensor
 * products of one-dimensional factors (Sec. 3.2.1-3.2.2), turned into QTT by
 * Algorithm 1, and the fixed point of Eq. (TT_k_eff_fixed_points) runs on TT
 * vectors with TT linear algebra (Sec. 3.5).
 *
 * Conventions for every entry point:
 *  - Return value: TT_OK (0) or a negative status below.  The message of the
 *    last failure of a context is returned by tt_last_error() (string owned by
 *    the context, valid until its next call).
 *  - All device work is enqueued on the context's CUDA stream; calls that
 *    return host data (sizes, scalars, copies to host) synchronise it.
 *  - Handles (tt_ctx, tt_vec, tt_op) are opaque, owned by the caller from
 *    creation to the matching *_destroy call.  Input arrays are copied; the
 *    library never keeps a caller pointer after a call returns.
 *  - Floating point is FP64 unless a tt_prec argument says otherwise.
 *  - No CPU fallback: without a usable CUDA device every call that needs one
 *    fails with TT_ECUDA.
 *
 * Layouts (all row-major, the first index slowest):
 *  - TT vector core k: (r_{k-1}, n_k, r_k), r_0 = r_d = 1 (Eq. (TT_def_element)).
 *    Cores are exchanged as one array, core 0 first.
 *  - TT matrix core k: (R_{k-1}, m_k, n_k, R_k), output index m (i_k), input
 *    index n (j_k) (Eq. (TT-matrix-componentwise)).
 *  - Angular flux Psi: (G, L, n, n, n), x fastest (Appendix A.3, Eq. (aflux)).
 *    Its TT form has cores [g:G][octant:8][direction:L/8][z bits][y bits]
 *    [x bits], bits most-significant first, so row-major flattening of the
 *    dense TT equals that layout.
 */
#ifndef KEIG_H
#define KEIG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  TT_OK = 0,
  TT_EINVAL = -1,     /* bad argument (sizes, pointers, non-finite input) */
  TT_ENOMEM = -2,     /* device allocation failed */
  TT_ECUDA = -3,      /* CUDA runtime error (message holds the CUDA string) */
  TT_ENOCONV = -4,    /* iteration limit reached; best iterate returned */
  TT_ETIMEOUT = -5,   /* a bounded device wait gave up */
  TT_ENONFINITE = -6  /* a NaN/Inf appeared during the computation */
};

typedef struct tt_ctx tt_ctx;
typedef struct tt_vec tt_vec;
typedef struct tt_op tt_op;

/* ---------------------------------------------------------------- context */

/* Device allocator supplied by the caller (e.g. a framework's caching
 * allocator): alloc returns `bytes` of device memory usable on `cuda_stream`
 * (aligned to at least 256 bytes) or NULL when it cannot; free returns a
 * block obtained from alloc once the library's work on `cuda_stream` that
 * uses it has been enqueued (stream-ordered reuse).  `user` is passed back
 * unchanged.  Both are called only from the host thread that calls the
 * library. */
typedef void *(*tt_alloc_fn)(size_t bytes, void *cuda_stream, void *user);
typedef void (*tt_free_fn)(void *ptr, void *cuda_stream, void *user);

/* Create a context bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  alloc_fn / free_fn:
 * the device allocator for every buffer the context makes (both NULL: the
 * device's stream-ordered pool, with freed blocks kept in the pool; exactly
 * one NULL is TT_EINVAL).  When alloc_fn returns NULL the running call fails
 * with TT_ENOMEM, frees what it allocated, and the context stays usable.
 * out: new handle. */
int tt_ctx_create(tt_ctx **out, void *cuda_stream, tt_alloc_fn alloc_fn, tt_free_fn free_fn, void *user);
int tt_ctx_destroy(tt_ctx *ctx);
const char *tt_last_error(const tt_ctx *ctx);
/* Library version string (static storage). */
const char *tt_version(void);
/* Counters since creation or the last reset: kernel launches issued by the
 * library and algorithmic flops of the core contractions (the operator-core
 * x vector-core products: exact matvec, local-system matvecs and interface
 * updates), in FP64 and, for the mixed-precision solves, FP32 together. */
int tt_ctx_counters(tt_ctx *ctx, int64_t *launches, double *contraction_flops);
int tt_ctx_reset_counters(tt_ctx *ctx);
/* Spin limit of the library's bounded device waits (the grid barriers of the
 * persistent GMRES kernel): a CTA that has waited `spins` polls gives up,
 * records TT_ETIMEOUT and returns, every other CTA of the launch returns at
 * its next barrier, and the call fails with TT_ETIMEOUT; the context stays
 * usable.  spins < 0 restores the default (2^24 polls of about 40 ns).  Small
 * values make the waits run out: that is how the failure path is tested. */
int tt_ctx_set_wait_limit(tt_ctx *ctx, long long spins);
/* Per-launch timing of the dense contraction kernel (the FP64 GEMM that all
 * core contractions run on): when enabled, every launch is bracketed by CUDA
 * events on the context stream.  tt_ctx_gemm_stats synchronises and returns
 * the launches, their summed device time (ms) and their algorithmic flops
 * (2 M N K per product) since profiling was enabled. */
int tt_ctx_set_profiling(tt_ctx *ctx, int on);
int tt_ctx_gemm_stats(tt_ctx *ctx, int64_t *launches, double *ms, double *flops);
/* The same for the FP32 GEMM that carries the contractions of the
 * mixed-precision (TT_FP32_REFINED) local solves. */
int tt_ctx_gemm32_stats(tt_ctx *ctx, int64_t *launches, double *ms, double *flops);
/* The same for the tcgen05 TF32 three-term GEMM of TT_TF32_SPLIT (flops
 * counted algorithmically, 2 M N K per product, not per MMA pass). */
int tt_ctx_gemmtc_stats(tt_ctx *ctx, int64_t *launches, double *ms, double *flops);
/* The same for the persistent FP32 GMRES kernel of the TT_FP32_REFINED local
 * solves (one launch per correction solve); flops = the local matvecs at
 * 2 n r0 r1 (r0 R1 + n R1 R2 + r1 R2) each plus the Gram-Schmidt passes. */
int tt_ctx_gmres_stats(tt_ctx *ctx, int64_t *launches, double *ms, double *flops);

/* The FP32 contraction GEMM of the mixed-precision local solves, exposed so
 * that it can be checked directly: C[b] = alpha op(A[b]) op(B[b]) + beta C[b]
 * for b < batch, row-major, op = transpose when ta / tb != 0, device
 * pointers, batch strides sA, sB, sC (elements).  kind: 0 the FP32 SIMT GEMM
 * (TT_FP32_REFINED), 1 the tcgen05 TF32 three-term split (TT_TF32_SPLIT),
 * 2 the tcgen05 BF16 three-term split (TT_BF16_SPLIT).  Enqueued on the
 * context stream; kinds 1 and 2 synchronise to read the bounded-wait flag
 * (TT_ETIMEOUT if an MMA wait gave up). */
int tt_gemm_f32(tt_ctx *ctx, int kind, int ta, int tb, int M, int N, int K, float alpha, const float *A, int lda,
                long long sA, const float *B, int ldb, long long sB, float beta, float *C, int ldc, long long sC,
                int batch);

/* Peak fused-multiply-add rate of the current device in flop/s (FP64 when
 * fp64 != 0, else FP32): four CTAs of 256 threads per SM each run eight
 * independent FMA chains for 16 x iters rounds; the best of `reps` timed
 * launches (CUDA events on cuda_stream) after one warm-up.  The roofline
 * denominator of the FP64 and FP32 SIMT kernels; the paper has no
 * counterpart. */
int tt_measure_fma_peak(void *cuda_stream, int fp64, int iters, int reps, double *flops_per_s);

/* ---------------------------------------------------------------- TT vectors */

/* New TT vector with d cores of modes n[0..d-1] and bond ranks r[0..d]
 * (r[0] = r[d] = 1).  cores == NULL gives zeros; else `cores` holds all core
 * entries back to back (sum_k r_k n_k r_{k+1} doubles), on the device if
 * cores_on_device != 0, else on the host. */
int tt_vec_create(tt_ctx *ctx, int d, const int *n, const int *r, const double *cores,
                  int cores_on_device, tt_vec **out);
int tt_vec_destroy(tt_vec *x);
/* d of x; with n (d ints) and r (d+1 ints) non-NULL also the modes and ranks. */
int tt_vec_shape(const tt_vec *x, int *d, int *n, int *r);
/* Number of stored doubles (sum over cores). */
int tt_vec_numel(const tt_vec *x, size_t *count);
/* Copy all cores to `dst` (numel doubles), device or host memory. */
int tt_vec_get_cores(tt_ctx *ctx, const tt_vec *x, double *dst, int dst_on_device);
/* Dense tensor (prod n_k doubles, row-major) into device memory `dst`
 * (a test helper for small tensors; TT_EINVAL above 2^28 entries). */
int tt_vec_to_dense(tt_ctx *ctx, const tt_vec *x, double *dst_device, size_t len);
/* y = alpha x + beta y in TT form (block concatenation, ranks add), no
 * rounding: Sec. 2.2 ("the sum of tensors in TT format is itself a tensor in
 * TT format").  Result replaces *y's cores. */
int tt_vec_axpby(tt_ctx *ctx, double alpha, const tt_vec *x, double beta, tt_vec *y);
/* x *= alpha (scales the first core). */
int tt_vec_scale(tt_ctx *ctx, tt_vec *x, double alpha);
/* <x, y> and ||x||_F by core-wise contraction (Appendix B.3, the
 * contraction of a tensor with a vector, applied core by core). */
int tt_vec_dot(tt_ctx *ctx, const tt_vec *x, const tt_vec *y, double *out);
int tt_vec_norm(tt_ctx *ctx, const tt_vec *x, double *out);
/* Sum of all entries (contraction of every core with a vector of ones). */
int tt_vec_sum(tt_ctx *ctx, const tt_vec *x, double *out);

/* TT rounding in place: left-to-right Householder QR sweep, then a
 * right-to-left truncated-SVD sweep keeping per bond the fewest singular
 * values whose discarded tail has norm <= eps ||x||_F / sqrt(d-1), and at
 * most rmax (rmax <= 0: no cap).  Rounding after TT sums is what Sec. 2.2
 * and Sec. 3.3 call for ("a rank reduction step could be necessary").
 * Limits: every bond rank before truncation must be <= 512. */
int tt_round(tt_ctx *ctx, tt_vec *x, double eps, int rmax);

/* ---------------------------------------------------------------- TT matrices */

int tt_op_create(tt_ctx *ctx, int d, const int *m, const int *n, const int *R, const double *cores,
                 int cores_on_device, tt_op **out);
int tt_op_destroy(tt_op *A);
int tt_op_shape(const tt_op *A, int *d, int *m, int *n, int *R);
int tt_op_numel(const tt_op *A, size_t *count);
int tt_op_get_cores(tt_ctx *ctx, const tt_op *A, double *dst, int dst_on_device);
/* C = alpha A + beta B (new operator, ranks add), then rounded with
 * (eps, rmax) when eps >= 0.  out: new handle. */
int tt_op_axpby(tt_ctx *ctx, double alpha, const tt_op *A, double beta, const tt_op *B, double eps,
                int rmax, tt_op **out);

/* ---------------------------------------------------------------- the problem */

/* The k-eigenvalue problem of Sec. 2.1 as the paper states it: a cube of
 * n = 2^l vertices per axis with cell-constant multigroup cross sections,
 * discrete ordinates ordered octant-major (Appendix A.2, Eq. (hat-mu)),
 * vacuum faces (Eq. (BCS)).  Host arrays, copied by the library. */
typedef struct {
  int l;                    /* 2^l grid points per axis, 1 <= l <= 10 */
  double side[3];           /* domain lengths x, y, z; Delta = side/(2^l - 1) */
  int G;                    /* energy groups */
  int n_mat;                /* materials, 1..255 */
  const double *sig_t;      /* [n_mat][G] total cross section */
  const double *sig_s;      /* [n_mat][G_to][G_from] scattering g_from -> g_to */
  const double *nu_sig_f;   /* [n_mat][G] nu * fission cross section */
  const double *chi;        /* [n_mat][G] fission spectrum */
  const double *inv_v;      /* [G] 1/v (alpha problem; unused, may be NULL) */
  const uint8_t *mat;       /* [(2^l-1)^3] cell materials, z-major, x fastest */
  int n_dir;                /* directions per octant (L/8) */
  const double *amu, *aeta, *axi; /* [n_dir] absolute direction cosines */
  const double *w;          /* [n_dir] weights of one octant, 8*sum(w) = 1 */
  int bc[6];                /* x-,x+,y-,y+,z-,z+; only 0 (vacuum) is accepted */
  const double *sig_s1;     /* [n_mat][G_to][G_from] P1 scattering moments (linearly anisotropic
                               scattering, N_s = 1 of the moment operators L^N, L^{N,+} of
                               Appendix A.2 with weights summing to 1: direction l's source gains
                               3 sum_a Omega_a(l) sum_l' w_l' Omega_a(l') (sig_s1 psi_l')), or NULL
                               (isotropic, the paper's case).  Enters S only; the derivative
                               outputs of keig_sensitivities / keig_gpt cover sig_s (P0) */
  const double *sig_s2;     /* [n_mat][G_to][G_from] P2 moments, or NULL; order n adds to the source of
                               direction l: sum_m Y_nm(Omega_l) sum_l' w_l' Y_nm(Omega_l') (sig_sn psi_l'),
                               Y_nm the real spherical harmonics with unit mean square over the sphere */
  const double *sig_s3;     /* [n_mat][G_to][G_from] P3 moments, or NULL */
} tt_problem;

typedef enum {
  TT_OP_H = 0, /* streaming + collision, Sec. 3.2.1 */
  TT_OP_S = 1, /* scattering, Sec. 3.2.2 */
  TT_OP_F = 2  /* fission, Sec. 3.2.2 */
} tt_op_kind;

typedef enum {
  TT_FP64 = 0,        /* every contraction in FP64 */
  TT_TF32_SPLIT = 1,  /* linear solves: as TT_FP32_REFINED, with the Krylov contractions on the tcgen05
                         tensor cores (kind::tf32, FP32 accumulation in tensor memory) with the
                         three-term split A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi */
  TT_BF16_SPLIT = 2,  /* linear solves: as TT_TF32_SPLIT with BF16 operands (tcgen05 kind::f16, FP32
                         accumulation in tensor memory): x = hi + lo with hi = bf16(x), lo = bf16(x - hi),
                         A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi (about 16 significant bits per product);
                         the FP32 correction solves stop at 3e-5 and the FP64 refinement finishes */
  TT_FP32_REFINED = 3 /* linear solves: Krylov iterations of each local system with FP32 contractions,
                         wrapped in FP64 iterative refinement (FP64 residual, FP32 correction solve,
                         one persistent GMRES kernel per correction) until the FP64 residual meets
                         the tolerance; products, QR, k and all interfaces stay FP64.  (In every
                         precision the SVDs of the truncations find their rotations in FP32 and
                         refine them by FP64 products; the truncation error stays exact.) */
} tt_prec;

/* Build H, S or F as a TT matrix with cores over the modes
 * [G][8][L/8][2 x 3l]: each rank-1 term of Sec. 3.2 (per octant: the x, y, z
 * streaming terms and one collision term per material, or one S/F term per
 * material) is a tensor product of the 1-D factors D+/-, Ip+/-, Ip+/-_noBC,
 * diagonal angular matrices, octant selectors and group matrices; each
 * spatial factor is converted to QTT by Algorithm 1 (reshape, index-pair
 * permutation, TT-SVD) on the device, the heterogeneous material masks are
 * QTT-compressed the same way, and the terms are summed and rounded with
 * eps_op (Sec. 3.3, "the QTT format of the operator is the sum over all
 * boundary conditions").  out: new handle. */
int tt_build_operator(tt_ctx *ctx, const tt_problem *prob, tt_op_kind kind, double eps_op, tt_op **out);

/* ---------------------------------------------------------------- products and solves */

enum { TT_MV_EXACT = 0, TT_MV_AMEN = 1 };

/* y = scale * A x.  method TT_MV_EXACT: core-wise Kronecker products
 * (ranks multiply, Sec. 3.5: the "explicit and exact algorithm") followed by
 * tt_round(eps, rmax) when eps >= 0.  TT_MV_AMEN: the optimisation form of
 * Eq. (mv_obj) solved core by core with residual enrichment, to relative
 * accuracy eps and ranks <= rmax, at most max_sweeps sweeps (the paper's
 * choice, "amen_mv").  *y: new handle. */
int tt_matvec(tt_ctx *ctx, const tt_op *A, const tt_vec *x, double scale, int method, double eps,
              int rmax, int max_sweeps, tt_prec prec, tt_vec **y);

/* Solve A x = b by alternating local solves over the cores with residual
 * enrichment (Sec. 3.5, Eq. (linear_system_obj) and the AMEn method it
 * names): the local systems are Galerkin projections onto the current
 * interfaces, solved by restarted GMRES to eps/sqrt(d); the local solution is
 * split by a truncated SVD (threshold eps/sqrt(d), cap rmax) and enriched
 * with a rank-`kick` residual direction (kick = 0: one-site ALS, no
 * enrichment).  x: initial guess on entry, solution
 * on return.  sweeps_done / rel_change (may be NULL): sweeps run and the
 * largest relative change of a local solution in the last sweep.
 * TT_ENOCONV when max_sweeps ran out (x still holds the last iterate). */
int tt_solve_local(tt_ctx *ctx, const tt_op *A, const tt_vec *b, tt_vec *x, double eps, int rmax,
                   int max_sweeps, int kick, tt_prec prec, int *sweeps_done, double *rel_change);

/* Solve A x = b by two-site DMRG sweeps (the two-site member of the
 * alternating family of Sec. 3.5: all cores fixed but a neighbouring pair):
 * for each bond the Galerkin local system of the merged supercore (modes
 * n_k n_{k+1}) is solved by the local solver of tt_solve_local (GMRES in FP64
 * or the FP32-refined / tensor-core forms of prec) and split back by a
 * truncated SVD (threshold eps/sqrt(d), cap rmax), which adapts the ranks
 * without enrichment.  The merged operator core holds R_k (n_k n_{k+1})^2
 * R_{k+2} doubles, so the method suits moderate mode sizes.  x: initial guess
 * on entry, solution on return.  TT_ENOCONV when the largest relative change
 * of a supercore is still >= eps after max_sweeps sweeps. */
int tt_solve_dmrg(tt_ctx *ctx, const tt_op *A, const tt_vec *b, tt_vec *x, double eps, int rmax, int max_sweeps,
                  tt_prec prec, int *sweeps_done, double *rel_change);

/* ---------------------------------------------------------------- the eigen loop */

typedef struct {
  double eps;        /* TT truncation tolerance of products and solves */
  int rmax;          /* TT rank cap of the flux */
  double tol_k;      /* stop when |k' - k| / k < tol_k ... */
  double tol_psi;    /* ... and the relative change of Psi is < tol_psi */
  int max_iter;      /* outer iterations */
  int solve_sweeps;  /* AMEn sweeps per linear solve */
  int mv_sweeps;     /* AMEn sweeps per product */
  int kick;          /* enrichment rank */
  int scheme;        /* 0: paper, H Psi' = (S + F/k) Psi; 1: (H - S) Psi' = F Psi / k */
  tt_prec prec;
  double eps_op;     /* operator rounding tolerance */
  const double *psi0_cores; /* optional host TT initial guess (rank-1 cores), NULL = ones */
  int mv_kind;       /* product B = (S + F/k) Psi: 0 the AMEn product (the paper's choice),
                        1 the exact TT product (core-wise Kronecker) rounded at eps / rmax */
  int local_form;    /* local systems of the linear solve M Psi' = B (M = H, or H - S with scheme 1):
                        0 Galerkin projections of M (what AMEn does);
                        1 least squares, the functional ||M Psi' - B||^2 of Eq. (linear_system_obj):
                          projections of N = M^T M (built once per problem as the sum over
                          octant row blocks of M_o^T M_o, rounded at eps_op) with right-hand side
                          M^T B.  The symmetric part of the vertex diamond-difference H is
                          indefinite, so a Galerkin projection of H onto rank-capped frames can
                          be singular; N's projections are symmetric positive definite.
                        Applies to keig_fixed_point (other entry points use 0). */
  int solve_method;  /* the alternating method of the linear solve (Sec. 3.5, "ALS, DMRG, AMEn"):
                        0 AMEn (one site, residual enrichment of rank kick); 2 two-site DMRG
                        (tt_solve_dmrg; Galerkin local systems only).  One-site ALS (tt_solve_local
                        with kick = 0) keeps the ranks of its initial guess, so it is not offered
                        inside the fixed point (TT_EINVAL for 1) */
} keig_opts;

typedef struct {
  double k;          /* final eigenvalue */
  int iters;         /* outer iterations run */
  double dk_last;    /* |k' - k| / k of the last iteration */
  double wall_ms;    /* time from entry to return */
  int max_rank;      /* largest bond rank of the final Psi */
  double k_hist[512];/* k after each outer iteration (first 512) */
  double t_hist[512];/* ms since entry at the end of each outer iteration */
} keig_result;

/* Fill opts with defaults (eps 1e-7, rmax 64, tol_k 1e-9, tol_psi 1e-5,
 * max_iter 400, solve_sweeps 2, mv_sweeps 2, kick 4, scheme 0, FP64,
 * eps_op 1e-12, AMEn product, Galerkin local systems, AMEn solve). */
int keig_default_opts(keig_opts *opts);

/* The QTT fixed point of Eq. (TT_k_eff_fixed_points):
 *   B = (S + F/k) Psi;  H Psi' = B;  k' = k sum(F Psi') / sum(F Psi),
 * with Psi normalised each iteration so that sum(F Psi) = 1.  The sum of all
 * entries of F Psi is the dot product of Psi with the TT vector F^T 1, built
 * once.  Builds H, S, F from `prob` (included in wall_ms).
 * psi_out (may be NULL): new handle with the final flux.
 * phi_out (may be NULL): host buffer of G*n^3 doubles receiving the scalar
 * flux phi[g][k][j][i] = sum_l w_l psi (dense; small grids only). */
int keig_fixed_point(tt_ctx *ctx, const tt_problem *prob, const keig_opts *opts, keig_result *out,
                     tt_vec **psi_out, double *phi_out);

/* The alpha-eigenvalue problem (alpha V^{-1} + H) Psi = (S + F) Psi
 * (Eq. (OpFormAlphaNTE)) by the paper's procedure (Eq.
 * (alpha_eig_fixed_points)): k-eigenvalue fixed points of
 * (H + alpha V^{-1}) Psi = (S + F/k) Psi at alpha = 0 and alpha = 0.01, then
 * secant steps alpha' = alpha_{-1} + (1 - k_{-1})(alpha - alpha_{-1}) /
 * (k - k_{-1}) (the printed update is dimensionally garbled; this is the
 * secant reading) until |k - 1| < tol_k1 or max_steps (<= 64) further
 * solves.  V^{-1} = diag(1/v) (x) (octant selector (x) I) (x) Ip^3 has the
 * structure of the collision term, so each solve is keig_fixed_point with
 * sigma_t + alpha / v.  prob->inv_v ([G]) is required. */
typedef struct {
  double alpha;          /* the alpha eigenvalue */
  double k;              /* k at the final alpha (1 within tol_k1) */
  int steps;             /* k-eigenvalue solves run */
  int outer_iters;       /* their outer iterations in total */
  double wall_ms;
  double alpha_hist[64]; /* alpha of each solve */
  double k_hist[64];     /* k of each solve */
} keig_alpha_result;
int keig_alpha(tt_ctx *ctx, const tt_problem *prob, const keig_opts *opts, double tol_k1, int max_steps,
               keig_alpha_result *out);

/* Many independent problems at once (batching).  One problem's sweep is a
 * chain of small contractions that occupies a few SMs at a time, so problems
 * are solved side by side: n_ctx worker threads, each driving its own context
 * (create each on its own CUDA stream), take problems from a shared counter
 * and run keig_fixed_point on them.  probs, opts, out and status are arrays
 * of n_prob entries (host); status[i] receives problem i's return code.
 * Returns TT_OK when every problem returned TT_OK, else the first failing
 * code in problem order.  Contexts must not be used elsewhere meanwhile. */
int keig_batch(tt_ctx *const *ctxs, int n_ctx, const tt_problem *probs, const keig_opts *opts, int n_prob,
               keig_result *out, int *status);
/* With more than one context (all on one device), keig_batch gathers the
 * workers' local systems that run in the persistent FP32 GMRES kernel
 * (TT_FP32_REFINED) into grouped cooperative launches: a worker submits its
 * system and waits; the first waiting worker leads, waits until every worker
 * that is solving a problem has submitted or 300 us have passed, gives each
 * gathered system a range of CTAs in proportion to its size, launches them
 * all in one kernel (each system with its own grid barrier over its CTAs) and
 * hands back the statuses.  Without grouping, each system's launch occupies
 * every SM and the workers' launches run one after another.  keig_batch_stats
 * returns the grouped launches and the systems they carried in the last
 * keig_batch call. */
int keig_batch_stats(long long *group_launches, long long *group_systems);

/* Sensitivities of k to every cross-section entry by the adjoint method.
 * Differentiating H Psi = (S + F/k) Psi and testing with the adjoint
 * eigenvector Psi^dagger of the transposed problem
 * H^T Psi^dagger = (S^T + F^T/k) Psi^dagger gives
 *   dk/dp = -k^2 <Psi^dagger, (dH/dp - dS/dp - (dF/dp)/k) Psi> / <Psi^dagger, F Psi>.
 * The paper has no adjoint; it follows from Eq. (OpFormkNTE).  Both fixed
 * points run the QTT iteration of Eq. (TT_k_eff_fixed_points) (the adjoint
 * one on the transposed TT operators, cores with i_k and j_k swapped).  H, S
 * and F are linear in the tables and the group matrix enters only through the
 * first TT core, so per material one open contraction gives the G x G matrix
 * W[g][g'] = <Psi^dagger, (e_g e_g'^T (x) B) Psi> for the collision and the
 * source structure B, from which all derivatives follow.
 * Outputs (host arrays, caller-owned): dk_dsig_t [n_mat][G],
 * dk_dsig_s [n_mat][G_to][G_from], dk_dnu_sig_f [n_mat][G], dk_dchi [n_mat][G].
 * TT_ENOCONV if either fixed point reached max_iter (outputs still written). */
typedef struct {
  double k;                  /* eigenvalue of the forward fixed point */
  double k_adjoint;          /* eigenvalue of the adjoint fixed point */
  int iters, iters_adjoint;  /* outer iterations of each */
  double adjoint_production; /* <Psi^dagger, F Psi> with sum(F Psi) = sum(F^T Psi^dagger) = 1 */
  double wall_ms;
} keig_sens_info;
int keig_sensitivities(tt_ctx *ctx, const tt_problem *prob, const keig_opts *opts, double *dk_dsig_t,
                       double *dk_dsig_s, double *dk_dnu_sig_f, double *dk_dchi, keig_sens_info *info);

/* ---------------------------------------------------------------- 1-D slab */

/* The 1-D slab problem of the paper's 1-D case study (Sec. 4.1): the same
 * vertex diamond-difference operators restricted to x, 2^l points across a
 * slab of the given width, vacuum on both faces.  Directions: a half-range
 * set amu[d] > 0 used for both signs of mu with weights w[d]
 * (2 * sum(w) = 1).  Tables as in tt_problem; mat[c] gives the material of
 * cell c (2^l - 1 cells).  Host arrays, copied by the library. */
typedef struct {
  int l;                    /* 2^l points, 1 <= l <= 24 */
  double width;             /* slab width; Delta = width / (2^l - 1) */
  int G, n_mat;
  const double *sig_t;      /* [n_mat][G] */
  const double *sig_s;      /* [n_mat][G_to][G_from] */
  const double *nu_sig_f;   /* [n_mat][G] */
  const double *chi;        /* [n_mat][G] */
  const uint8_t *mat;       /* [2^l - 1] */
  int n_dir;                /* directions per half range */
  const double *amu;        /* [n_dir] mu > 0 */
  const double *w;          /* [n_dir] weights of one half range */
} tt_slab;

/* The k fixed point of Eq. (TT_k_eff_fixed_points) on the slab operators,
 * TT cores [G][2 (mu < 0, mu > 0)][n_dir][x bits] (the paper's ISTT), with
 * the options and result of keig_fixed_point (opts->prec as there).
 * phi_out: NULL or host [G][2^l], the scalar flux sum over both half ranges
 * of w[d] psi, normalised so that sum(F Psi) = 1.  TT_ENOCONV at max_iter. */
int keig_slab_fixed_point(tt_ctx *ctx, const tt_slab *slab, const keig_opts *opts, keig_result *out,
                          double *phi_out);

/* Gradient of a flux functional by generalised perturbation theory (GPT).
 * The functional is J = sum_g sum_v resp_g[g] resp_v[v] phi[g, v] of the
 * scalar flux phi = sum_l w_l Psi[g, l, v] of the eigenvector normalised so
 * that sum(F Psi) = <f, Psi> = 1 (f = F^T 1).  With A = H - S - F/k,
 * differentiating A Psi = 0, the normalisation and J, and introducing the
 * generalised adjoint Gamma with
 *   A^T Gamma = j - J f,   <Gamma, F Psi> = 0     (j = resp_g (x) w (x) resp_v),
 * gives  dJ/dp = -<Gamma, (dH/dp - dS/dp - (dF/dp)/k) Psi> - J sum((dF/dp) Psi).
 * The paper has no adjoint; this follows from Eq. (OpFormkNTE).  Gamma comes
 * from the fixed-source iteration H^T Gamma' = (S^T + F^T/k) Gamma + (j - J f)
 * on the transposed TT operators (AMEn product and solve as in the k fixed
 * point), with the fundamental adjoint mode removed after every step
 * (Gamma' -= <Gamma', F Psi> / <Psi^dagger, F Psi> Psi^dagger); it converges at
 * the dominance ratio.  The derivatives then use the same per-material open
 * contractions as keig_sensitivities.
 * resp_g: [G] host; resp_v: [(2^l)^3] host, vertex order z, y, x (x fastest),
 * the order of phi_out of keig_fixed_point; the angular weights are those of
 * prob (octant-symmetric: phi = sum over octants and prob->w).  tol_gpt: stop when the relative
 * change of Gamma falls below it; max_gpt: step limit (1..10000).
 * Outputs as keig_sensitivities (dJ instead of dk).  TT_ENOCONV if a fixed
 * point or the GPT iteration reached its limit (outputs still written). */
typedef struct {
  double J;               /* the functional of the production-normalised eigenvector */
  double k;               /* forward eigenvalue */
  int iters, iters_adjoint, iters_gpt;
  double gpt_change;      /* relative change of Gamma at the last GPT step */
  double wall_ms;
} keig_gpt_info;
int keig_gpt(tt_ctx *ctx, const tt_problem *prob, const keig_opts *opts, const double *resp_g,
             const double *resp_v, double tol_gpt, int max_gpt, double *dJ_dsig_t, double *dJ_dsig_s,
             double *dJ_dnu_sig_f, double *dJ_dchi, keig_gpt_info *info);

/* Scalar flux of a flux TT (contract the octant and direction cores with the
 * quadrature weights, Appendix B.4) as a TT with cores [G][2 x 3l]; for a
 * slab flux (cores [G][2][n_dir][x bits]) the hemisphere core takes the place
 * of the octant core and the result has cores [G][2 x l]. */
int tt_scalar_flux(tt_ctx *ctx, const tt_vec *psi, const double *w_host, int n_dir, tt_vec **phi);

/* ---------------------------------------------------------------- allocation-free inner product */

/* <x, y> of two TT vectors without allocating device memory.  The paper has
 * no counterpart: this is a service for callers that cannot allocate at the
 * point of use (a host that gives the library a fixed memory budget, or a
 * real-time loop where cudaMalloc/cudaFree would stall or serialise the
 * device).
 *
 * x_cores, y_cores: device pointers to all cores of x and y back to back,
 * core 0 first, each core (r_k, n_k, r_{k+1}) row-major (the layout of
 * tt_vec_get_cores).  rx, ry: host arrays of d+1 bond ranks (first and last
 * 1), each at most 128.  n: host array of d mode sizes, each at most 64.
 * out: device pointer receiving one double.  cuda_stream: the cudaStream_t
 * the work is enqueued on (the call does not synchronise it).  err/err_len:
 * optional caller buffer for a message on failure.
 *
 * Scratch lives in one fixed 8.25 MiB device array that every GPU loading the
 * library holds until the process exits; the call never allocates.  The first
 * call on each device looks up that array's device address (no allocation)
 * and keeps it for the process, so make that first call before any stream
 * capture; a cudaDeviceReset() invalidates the kept address.  All calls
 * share the array: calls that overlap on the GPU race and must be serialised
 * by the caller (one stream, or events).  Sizes above the limits return
 * TT_EINVAL before any work is enqueued. */
int tt_dot_noalloc(const double *x_cores, const int *rx, const double *y_cores, const int *ry, int d,
                   const int *n, double *out, void *cuda_stream, char *err, size_t err_len);

#ifdef __cplusplus
}
#endif
#endif /* KEIG_H */
