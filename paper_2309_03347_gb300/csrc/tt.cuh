// Tensor-train containers and algorithms (device-resident cores, host-side
// rank bookkeeping).
#pragma once
#include "common.cuh"

namespace tt {

// TT vector (or TT matrix with mode n[k] = mo[k] * mi[k]); cores row-major
// (r[k], n[k], r[k+1]), matrices (R[k], mo[k], mi[k], R[k+1]).
struct TT {
  int d = 0;
  std::vector<int> n, r;
  std::vector<int> mo, mi;  // matrices only (output / input mode sizes)
  std::vector<DBuf> core;
  bool is_matrix() const { return !mo.empty(); }
  size_t csize(int k) const { return (size_t)r[k] * n[k] * r[k + 1]; }
  size_t numel() const {
    size_t s = 0;
    for (int k = 0; k < d; ++k) s += csize(k);
    return s;
  }
  int max_rank() const {
    int m = 1;
    for (int v : r) m = std::max(m, v);
    return m;
  }
};

// An operator with the permuted core layouts the contractions use.
struct TTOp {
  TT t;
  std::vector<DBuf> a_ajib;  // (R0, n_in, n_out, R1)  : local matvec / left interface
  std::vector<DBuf> a_jbai;  // (n_in, R1, R0, n_out)  : right interface
  std::vector<DBuf> a_ajib32;  // FP32 copy of a_ajib (mixed-precision local solves)
  void prepare(Ctx *c);
  void prepare32(Ctx *c);
  bool prepared = false;
  bool prepared32 = false;
  void invalidate() {
    prepared = prepared32 = false;
    a_ajib.clear();
    a_jbai.clear();
    a_ajib32.clear();
  }
};

TT tt_zeros(Ctx *c, const std::vector<int> &n, const std::vector<int> &r);
TT tt_clone(Ctx *c, const TT &x);
TT tt_ones(Ctx *c, const std::vector<int> &n);
TT tt_random(Ctx *c, const std::vector<int> &n, int rank, uint64_t seed);
void tt_check(const TT &x);

// SVD of a row-major m x n device matrix A (not modified).  k = min(m, n).
// Ut: k x m (rows = left singular vectors), Vt: k x n, S: k (device and host),
// all sorted by decreasing singular value; A = Ut^T S Vt to FP64 rounding.
// orth names the factor that must be orthonormal to FP64 rounding
// (SVD_ORTH_U: Ut, SVD_ORTH_V: Vt); with the mixed-precision small SVD the
// other factor is orthonormal only up to the cosines left between columns of
// nearly equal singular values, which leaves the truncation error (the norm
// of the dropped part) exact.
struct SVD {
  int m = 0, n = 0, k = 0;
  DBuf Ut, Vt, S;
  std::vector<double> Sh;
};
enum { SVD_ORTH_U = 1, SVD_ORTH_V = 2, SVD_ORTH_ANY = 3 };
void svd_rm(Ctx *c, const double *A, int m, int n, SVD &out, int orth);
int trunc_rank(const std::vector<double> &s, double delta, int rmax);

// QR of a row-major m x n matrix A given as its transpose At (n x m
// row-major = A column-major, destroyed).  Q: m x k row-major, R: k x n
// row-major, k = min(m, n).
void qr_rm_from_t(Ctx *c, double *At, int m, int n, DBuf &Q, DBuf &R, int &k);

void orth_left(Ctx *c, TT &x, int upto);   // cores 0..upto-1 left-orthogonal
void orth_right(Ctx *c, TT &x, int downto);  // cores downto+1..d-1 right-orthogonal
void round(Ctx *c, TT &x, double eps, int rmax);

double dot(Ctx *c, const TT &x, const TT &y);
double norm(Ctx *c, const TT &x);
double sum(Ctx *c, const TT &x);
void scale(Ctx *c, TT &x, double a);
TT add(Ctx *c, double a, const TT &x, double b, const TT &y);
TT matvec_exact(Ctx *c, const TT &A, const TT &x);
TT transpose_op(Ctx *c, const TT &A);
TT op_matmul_tn(Ctx *c, const TT &A, const TT &B);  // A^T B, ranks multiply
void to_dense(Ctx *c, const TT &x, double *dst, size_t len);
TT tt_svd_dense(Ctx *c, const double *a, const std::vector<int> &modes, double eps, int rmax);

// AMEn (amen.cu)
struct SolveStats {
  int sweeps = 0;
  double max_dx = 0.0;
  long long gmres_iters = 0;
};
// A x = b by AMEn with Galerkin local systems; with rhs_op the right-hand side
// is rhs_op b (projected through operator interfaces), which with A = M^T M and
// rhs_op = M^T gives the least-squares local systems of min ||M x - b||
void amen_solve(Ctx *c, TTOp &A, const TT &b, TT &x, double eps, int rmax, int nswp, int kick,
                uint64_t seed, SolveStats *st, int prec = TT_FP64, TTOp *rhs_op = nullptr);
// two-site DMRG (merged pairs of cores, SVD split); Galerkin local systems
void dmrg_solve(Ctx *c, TTOp &A, const TT &b, TT &x, double eps, int rmax, int nswp, SolveStats *st,
                int prec = TT_FP64);
void amen_mv(Ctx *c, TTOp &A, const TT &x, TT &y, double eps, int rmax, int nswp, int kick,
             uint64_t seed, SolveStats *st);
// interface updates (amen.cu); operator cores in the permuted layouts of TTOp
void left_update(Ctx *c, const double *PhiL, const double *y, const double *Aajib, const double *x, int ry1,
                 int R1, int rx1, int m, int n, int R2, int ry2, int rx2, DBuf &out, DBuf &T1, DBuf &T2);
void right_update(Ctx *c, const double *PhiR, const double *y, const double *Ajbai, const double *x, int ry1,
                  int R1, int rx1, int m, int n, int R2, int ry2, int rx2, DBuf &out, DBuf &T1, DBuf &T2);

// operator construction (build_op.cu)
// QTT factors and material masks of one problem, shared by every operator built from it
struct OpFactors {
  std::vector<std::vector<DBuf>> qf;
  std::vector<std::vector<int>> qr;
  int iD[3][2], iIp[2], iIpN[2];
  std::vector<TT> masks;
  std::vector<int> mask_index;
};
// operator kinds beyond tt_op_kind: the collision term and the S/F source
// structure without their group core (derivatives w.r.t. the group matrices)
enum { KIND_COLLISION = 10, KIND_SOURCE = 11 };
OpFactors make_factors(Ctx *c, const tt_problem *p);
// only_oct >= 0: the rows of that octant only (every term of H, S and F has
// its rows in one octant, so the operator is the sum of its octant row blocks)
TT assemble_operator(Ctx *c, const tt_problem *p, const OpFactors &F, int kind, int only_mat, double eps_op,
                     int only_oct = -1);
TT build_operator(Ctx *c, const tt_problem *p, int kind, double eps_op);
// H, S or F of a 1-D slab over the modes [G][2][n_dir][x bits]
TT assemble_slab_operator(Ctx *c, const tt_slab *s, int kind, double eps_op);

}  // namespace tt
