/*
 * ORACLE (test infrastructure only).  Plain, slow FP64 full-grid transport
 * code used to check the GPU tensor-train path; nothing in the product path
 * may call it.
 *
 * What it computes (arXiv 2309.03347):
 *   - the vertex-form diamond-difference cell balance, Eq. (Discretized_kNTE)
 *     of Sec. 2.1.4: for cell c and direction l,
 *       sum_a |Omega_a|/(4 Delta_a) * sum_{4 edges || a}(psi_down - psi_up)
 *       + sigma_t(c)/8 * sum_{8 corners} psi  =  b
 *     written at the cell's downstream corner (the matrix form of Sec. 2.1.5
 *     and Appendix A.3 places the equation of the cell upstream of each
 *     vertex in that vertex's row);
 *   - the transport operator H is block lower-triangular per (g, l): applying
 *     H^{-1} is one sweep in downstream order ("forward substitution",
 *     Sec. 3.4.2).  Rows on the inflow faces of a direction are the same
 *     balance for a ghost cell whose outer corners are zero, which is what
 *     the boundary rows of the matrices D+/-, Ip+/- of Sec. 3.2.1 give;
 *   - the scattering and fission operators S, F (Sec. 3.2.2) applied to the
 *     scalar flux phi = sum_l w_l psi_l, averaged over the 8 corners of the
 *     upstream cell, zero on inflow-face rows (the "noBC" interpolation);
 *   - optional linearly anisotropic scattering (N_s = 1 of the moment
 *     operators L^N, L^{N,+} of Appendix A.2, quadrature weights summing to
 *     1): the source of direction l gains
 *       3 sum_a Omega_a(l) sum_g' sig_s1[g][g'] Jbar_a(g', c),
 *     J_a = sum_l w_l Omega_a(l) psi_l (signed cosines), averaged over the
 *     8 corners of the upstream cell like phi;
 *   - the k fixed point of Eq. (k_eff_fixed_points):
 *       Psi' = H^{-1}(S + F/k) Psi,  k' = k * sum(F Psi') / sum(F Psi).
 *
 * Layout: psi[g][l][k][j][i] with i (x) fastest, n = 2^l points per axis
 * (Appendix A.3, Eq. (aflux)).  Octant o of direction l = o*(L/8) + d has
 * sign bits x = o&1, y = o&2, z = o&4 (set = positive cosine).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int l;             /* n = 2^l vertices per axis */
  double dx, dy, dz; /* cell sizes */
  int G, n_mat;
  const double *sig_t;    /* [n_mat][G] */
  const double *sig_s;    /* [n_mat][G_to][G_from] */
  const double *nu_sig_f; /* [n_mat][G] */
  const double *chi;      /* [n_mat][G] */
  const uint8_t *mat;     /* [(n-1)^3] cells, x fastest */
  int L;                  /* directions, octant-major */
  const double *amu, *aeta, *axi; /* [L/8] absolute cosines */
  const double *w8;               /* [L/8] weights (sum over all L = 1) */
  int bc[6];                      /* x-,x+,y-,y+,z-,z+ : must be 0 (vacuum) */
  int threads;                    /* <= 0: library default */
  const double *sig_s1;           /* [n_mat][G_to][G_from] P1 scattering moments, or NULL */
} oracle_problem;

static inline int sgn_bit(int o, int axis) { return (o >> axis) & 1; }

/* upstream cell index along one axis for vertex coordinate v (clamped) */
static inline int row_cell(int v, int pos, int n) {
  int c = pos ? v - 1 : v;
  if (c < 0) c = 0;
  if (c > n - 2) c = n - 2;
  return c;
}

static inline int on_inflow(int v, int pos, int n) { return pos ? (v == 0) : (v == n - 1); }

/* Solve H_{g,l} psi = b for one (g, l) by a downstream sweep.
 * fixed != NULL: vertices with fixed_mask set take fixed[] (Dirichlet) instead
 * of their row equation (the inflow faces in the power iteration). */
static void sweep_one(const oracle_problem *p, int g, int ell, const double *b,
                      const uint8_t *fixed_mask, const double *fixed, double *psi) {
  const int n = 1 << p->l;
  const int m8 = p->L / 8;
  const int o = ell / m8, d = ell % m8;
  const int px = sgn_bit(o, 0), py = sgn_bit(o, 1), pz = sgn_bit(o, 2);
  const double cx = p->amu[d] / (4.0 * p->dx);
  const double cy = p->aeta[d] / (4.0 * p->dy);
  const double cz = p->axi[d] / (4.0 * p->dz);
  const int nc = n - 1;
  for (int kk = 0; kk < n; ++kk) {
    const int k = pz ? kk : n - 1 - kk;
    const int ku = pz ? k - 1 : k + 1;
    const int ck = row_cell(k, pz, n);
    for (int jj = 0; jj < n; ++jj) {
      const int j = py ? jj : n - 1 - jj;
      const int ju = py ? j - 1 : j + 1;
      const int cj = row_cell(j, py, n);
      for (int ii = 0; ii < n; ++ii) {
        const int i = px ? ii : n - 1 - ii;
        const int iu = px ? i - 1 : i + 1;
        const size_t v = ((size_t)k * n + j) * n + i;
        if (fixed_mask && fixed_mask[v]) {
          psi[v] = fixed[v];
          continue;
        }
        const int ci = row_cell(i, px, n);
        const int m = p->mat[((size_t)ck * nc + cj) * nc + ci];
        const double st = p->sig_t[m * p->G + g];
        /* the 8 corners of the upstream cell; out-of-range corners are 0 */
        double c[2][2][2]; /* [dk][dj][di]: 0 = this vertex's plane, 1 = upstream */
        for (int a = 0; a < 2; ++a)
          for (int bb = 0; bb < 2; ++bb)
            for (int e = 0; e < 2; ++e) {
              int K = a ? ku : k, J = bb ? ju : j, I = e ? iu : i;
              if (K < 0 || K >= n || J < 0 || J >= n || I < 0 || I >= n)
                c[a][bb][e] = 0.0;
              else if (a == 0 && bb == 0 && e == 0)
                c[a][bb][e] = 0.0; /* the unknown */
              else
                c[a][bb][e] = psi[((size_t)K * n + J) * n + I];
            }
        /* balance with the unknown psi_v set to zero */
        double rest = 0.0;
        for (int a = 0; a < 2; ++a)
          for (int bb = 0; bb < 2; ++bb) rest += cx * (c[a][bb][0] - c[a][bb][1]);
        for (int a = 0; a < 2; ++a)
          for (int e = 0; e < 2; ++e) rest += cy * (c[a][0][e] - c[a][1][e]);
        for (int bb = 0; bb < 2; ++bb)
          for (int e = 0; e < 2; ++e) rest += cz * (c[0][bb][e] - c[1][bb][e]);
        double s8 = 0.0;
        for (int a = 0; a < 2; ++a)
          for (int bb = 0; bb < 2; ++bb)
            for (int e = 0; e < 2; ++e) s8 += c[a][bb][e];
        rest += st / 8.0 * s8;
        const double diag = cx + cy + cz + st / 8.0;
        psi[v] = (b[v] - rest) / diag;
      }
    }
  }
}

/* out = H psi for all (g, l), by the same balance (ghost corners are zero). */
void oracle_apply_H(const oracle_problem *p, const double *psi, double *out) {
  const int n = 1 << p->l, nc = n - 1;
  const size_t n3 = (size_t)n * n * n;
  const int m8 = p->L / 8;
  for (int g = 0; g < p->G; ++g)
    for (int ell = 0; ell < p->L; ++ell) {
      const int o = ell / m8, d = ell % m8;
      const int px = sgn_bit(o, 0), py = sgn_bit(o, 1), pz = sgn_bit(o, 2);
      const double cx = p->amu[d] / (4.0 * p->dx);
      const double cy = p->aeta[d] / (4.0 * p->dy);
      const double cz = p->axi[d] / (4.0 * p->dz);
      const double *ps = psi + ((size_t)g * p->L + ell) * n3;
      double *ou = out + ((size_t)g * p->L + ell) * n3;
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            const int ku = pz ? k - 1 : k + 1, ju = py ? j - 1 : j + 1, iu = px ? i - 1 : i + 1;
            const int m = p->mat[((size_t)row_cell(k, pz, n) * nc + row_cell(j, py, n)) * nc +
                                 row_cell(i, px, n)];
            const double st = p->sig_t[m * p->G + g];
            double c[2][2][2];
            for (int a = 0; a < 2; ++a)
              for (int bb = 0; bb < 2; ++bb)
                for (int e = 0; e < 2; ++e) {
                  int K = a ? ku : k, J = bb ? ju : j, I = e ? iu : i;
                  c[a][bb][e] = (K < 0 || K >= n || J < 0 || J >= n || I < 0 || I >= n)
                                    ? 0.0
                                    : ps[((size_t)K * n + J) * n + I];
                }
            double r = 0.0, s8 = 0.0;
            for (int a = 0; a < 2; ++a)
              for (int bb = 0; bb < 2; ++bb) r += cx * (c[a][bb][0] - c[a][bb][1]);
            for (int a = 0; a < 2; ++a)
              for (int e = 0; e < 2; ++e) r += cy * (c[a][0][e] - c[a][1][e]);
            for (int bb = 0; bb < 2; ++bb)
              for (int e = 0; e < 2; ++e) r += cz * (c[0][bb][e] - c[1][bb][e]);
            for (int a = 0; a < 2; ++a)
              for (int bb = 0; bb < 2; ++bb)
                for (int e = 0; e < 2; ++e) s8 += c[a][bb][e];
            ou[((size_t)k * n + j) * n + i] = r + st / 8.0 * s8;
          }
    }
}

/* psi = H^{-1} b for all (g, l) (vacuum semantics of the matrix H). */
void oracle_sweep(const oracle_problem *p, const double *b, double *psi) {
  const int n = 1 << p->l;
  const size_t n3 = (size_t)n * n * n;
  const int GL = p->G * p->L;
#pragma omp parallel for schedule(static) num_threads(p->threads > 0 ? p->threads : omp_get_max_threads())
  for (int q = 0; q < GL; ++q) {
    const int g = q / p->L, ell = q % p->L;
    sweep_one(p, g, ell, b + (size_t)q * n3, NULL, NULL, psi + (size_t)q * n3);
  }
}

/* scalar flux phi[g][v] = sum_l w_l psi[g][l][v] */
static void scalar_flux(const oracle_problem *p, const double *psi, double *phi) {
  const int n = 1 << p->l;
  const size_t n3 = (size_t)n * n * n;
  const int m8 = p->L / 8;
  memset(phi, 0, sizeof(double) * p->G * n3);
  for (int g = 0; g < p->G; ++g)
    for (int ell = 0; ell < p->L; ++ell) {
      const double w = p->w8[ell % m8];
      const double *ps = psi + ((size_t)g * p->L + ell) * n3;
      double *ph = phi + (size_t)g * n3;
      for (size_t v = 0; v < n3; ++v) ph[v] += w * ps[v];
    }
}

/* cell average of phi over the 8 corners: pbar[g][c] */
static void cell_average(const oracle_problem *p, const double *phi, double *pbar) {
  const int n = 1 << p->l, nc = n - 1;
  const size_t n3 = (size_t)n * n * n, c3 = (size_t)nc * nc * nc;
  for (int g = 0; g < p->G; ++g)
    for (int k = 0; k < nc; ++k)
      for (int j = 0; j < nc; ++j)
        for (int i = 0; i < nc; ++i) {
          double s = 0.0;
          for (int a = 0; a < 2; ++a)
            for (int bb = 0; bb < 2; ++bb)
              for (int e = 0; e < 2; ++e)
                s += phi[(size_t)g * n3 + ((size_t)(k + a) * n + (j + bb)) * n + (i + e)];
          pbar[(size_t)g * c3 + ((size_t)k * nc + j) * nc + i] = s / 8.0;
        }
}

/* Per-cell group sources:
 *   qs[g][c] = sum_g' sig_s[m][g][g'] pbar[g'][c]
 *   qf[g][c] = chi[m][g] * sum_g' nu_sig_f[m][g'] pbar[g'][c]              */
static void cell_sources(const oracle_problem *p, const double *pbar, double *qs, double *qf) {
  const int n = 1 << p->l, nc = n - 1, G = p->G;
  const size_t c3 = (size_t)nc * nc * nc;
  for (size_t c = 0; c < c3; ++c) {
    const int m = p->mat[c];
    double prod = 0.0;
    for (int gp = 0; gp < G; ++gp) prod += p->nu_sig_f[m * G + gp] * pbar[(size_t)gp * c3 + c];
    for (int g = 0; g < G; ++g) {
      double s = 0.0;
      for (int gp = 0; gp < G; ++gp)
        s += p->sig_s[((size_t)m * G + g) * G + gp] * pbar[(size_t)gp * c3 + c];
      qs[(size_t)g * c3 + c] = s;
      qf[(size_t)g * c3 + c] = p->chi[m * G + g] * prod;
    }
  }
}

/* signed cosine of direction l = o*(L/8) + d along axis a (0 x, 1 y, 2 z) */
static inline double cosine(const oracle_problem *p, int ell, int a) {
  const int m8 = p->L / 8, o = ell / m8, d = ell % m8;
  const double c = a == 0 ? p->amu[d] : a == 1 ? p->aeta[d] : p->axi[d];
  return sgn_bit(o, a) ? c : -c;
}

/* first angular moments J[a][g][v] = sum_l w_l Omega_a(l) psi[g][l][v] */
static void current(const oracle_problem *p, const double *psi, double *J) {
  const int n = 1 << p->l;
  const size_t n3 = (size_t)n * n * n;
  const int m8 = p->L / 8, G = p->G;
  memset(J, 0, sizeof(double) * 3 * G * n3);
  for (int a = 0; a < 3; ++a)
    for (int g = 0; g < G; ++g)
      for (int ell = 0; ell < p->L; ++ell) {
        const double w = p->w8[ell % m8] * cosine(p, ell, a);
        const double *ps = psi + ((size_t)g * p->L + ell) * n3;
        double *jj = J + ((size_t)a * G + g) * n3;
        for (size_t v = 0; v < n3; ++v) jj[v] += w * ps[v];
      }
}

/* P1 cell sources q1[a][g][c] = sum_g' sig_s1[m][g][g'] Jbar[a][g'][c] */
static void p1_sources(const oracle_problem *p, const double *Jbar, double *q1) {
  const int n = 1 << p->l, nc = n - 1, G = p->G;
  const size_t c3 = (size_t)nc * nc * nc;
  for (int a = 0; a < 3; ++a)
    for (size_t c = 0; c < c3; ++c) {
      const int m = p->mat[c];
      for (int g = 0; g < G; ++g) {
        double s = 0.0;
        for (int gp = 0; gp < G; ++gp)
          s += p->sig_s1[((size_t)m * G + g) * G + gp] * Jbar[((size_t)a * G + gp) * c3 + c];
        q1[((size_t)a * G + g) * c3 + c] = s;
      }
    }
}

/* per-cell scattering source of direction l: q0[c] + 3 sum_a Omega_a(l) q1[a][g][c] */
static void direction_source(const oracle_problem *p, int g, int ell, const double *q0, const double *q1,
                             double *out) {
  const int n = 1 << p->l, nc = n - 1, G = p->G;
  const size_t c3 = (size_t)nc * nc * nc;
  const double ox = 3.0 * cosine(p, ell, 0), oy = 3.0 * cosine(p, ell, 1), oz = 3.0 * cosine(p, ell, 2);
  const double *qx = q1 + ((size_t)0 * G + g) * c3, *qy = q1 + ((size_t)1 * G + g) * c3,
               *qz = q1 + ((size_t)2 * G + g) * c3;
  for (size_t c = 0; c < c3; ++c) out[c] = q0[c] + ox * qx[c] + oy * qy[c] + oz * qz[c];
}

/* Spread a per-cell source onto the rows of direction l (octant o): row v
 * takes the value of its upstream cell, inflow-face rows are zero. */
static void rows_from_cells(const oracle_problem *p, int o, const double *qc, double *rows) {
  const int n = 1 << p->l, nc = n - 1;
  const int px = sgn_bit(o, 0), py = sgn_bit(o, 1), pz = sgn_bit(o, 2);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        const size_t v = ((size_t)k * n + j) * n + i;
        if (on_inflow(k, pz, n) || on_inflow(j, py, n) || on_inflow(i, px, n)) {
          rows[v] = 0.0;
          continue;
        }
        rows[v] = qc[((size_t)row_cell(k, pz, n) * nc + row_cell(j, py, n)) * nc + row_cell(i, px, n)];
      }
}

/* out_s = S psi, out_f = F psi (full vectors) */
void oracle_apply_SF(const oracle_problem *p, const double *psi, double *out_s, double *out_f) {
  const int n = 1 << p->l, nc = n - 1;
  const size_t n3 = (size_t)n * n * n, c3 = (size_t)nc * nc * nc;
  const int m8 = p->L / 8;
  double *phi = (double *)malloc(sizeof(double) * p->G * n3);
  double *pbar = (double *)malloc(sizeof(double) * p->G * c3);
  double *qs = (double *)malloc(sizeof(double) * p->G * c3);
  double *qf = (double *)malloc(sizeof(double) * p->G * c3);
  scalar_flux(p, psi, phi);
  cell_average(p, phi, pbar);
  cell_sources(p, pbar, qs, qf);
  double *J = NULL, *Jbar = NULL, *q1 = NULL, *qd = NULL;
  if (p->sig_s1) {
    J = (double *)malloc(sizeof(double) * 3 * p->G * n3);
    Jbar = (double *)malloc(sizeof(double) * 3 * p->G * c3);
    q1 = (double *)malloc(sizeof(double) * 3 * p->G * c3);
    qd = (double *)malloc(sizeof(double) * c3);
    current(p, psi, J);
    for (int a = 0; a < 3; ++a) cell_average(p, J + (size_t)a * p->G * n3, Jbar + (size_t)a * p->G * c3);
    p1_sources(p, Jbar, q1);
  }
  for (int g = 0; g < p->G; ++g)
    for (int ell = 0; ell < p->L; ++ell) {
      const size_t off = ((size_t)g * p->L + ell) * n3;
      if (out_s) {
        if (p->sig_s1) {
          direction_source(p, g, ell, qs + (size_t)g * c3, q1, qd);
          rows_from_cells(p, ell / m8, qd, out_s + off);
        } else {
          rows_from_cells(p, ell / m8, qs + (size_t)g * c3, out_s + off);
        }
      }
      if (out_f) rows_from_cells(p, ell / m8, qf + (size_t)g * c3, out_f + off);
    }
  free(J);
  free(Jbar);
  free(q1);
  free(qd);
  free(phi);
  free(pbar);
  free(qs);
  free(qf);
}

/* sum of all entries of F psi, evaluated row by row from the per-cell fission
 * source: every direction of octant o contributes its non-inflow rows. */
static double production(const oracle_problem *p, const double *pbar) {
  const int n = 1 << p->l, nc = n - 1, G = p->G;
  const size_t c3 = (size_t)nc * nc * nc;
  const int m8 = p->L / 8;
  double *qs = (double *)malloc(sizeof(double) * G * c3);
  double *qf = (double *)malloc(sizeof(double) * G * c3);
  cell_sources(p, pbar, qs, qf);
  double tot = 0.0;
  for (int o = 0; o < 8; ++o) {
    const int px = sgn_bit(o, 0), py = sgn_bit(o, 1), pz = sgn_bit(o, 2);
    double so = 0.0;
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          if (on_inflow(k, pz, n) || on_inflow(j, py, n) || on_inflow(i, px, n)) continue;
          const size_t c = ((size_t)row_cell(k, pz, n) * nc + row_cell(j, py, n)) * nc + row_cell(i, px, n);
          for (int g = 0; g < G; ++g) so += qf[(size_t)g * c3 + c];
        }
    tot += (double)m8 * so;
  }
  free(qs);
  free(qf);
  return tot;
}

typedef struct {
  double tol_k;     /* stop when |k' - k| < tol_k */
  int max_iter;
  double k0;        /* initial k */
  int store_psi;    /* keep the full angular flux */
} oracle_keig_opts;

typedef struct {
  double k;
  int iters;
  double dk_last;
} oracle_keig_result;

/* Power iteration of Eq. (k_eff_fixed_points).  psi0 (full vector, may be
 * NULL when store_psi == 0 and phi0 given) is the initial guess.  On return
 * phi_out[g][v] holds the scalar flux normalised so that sum(F Psi) = 1 and,
 * if psi_out != NULL, the angular flux with the same normalisation.
 * k_hist (may be NULL) receives k after each iteration (max_iter entries). */
int oracle_keig(const oracle_problem *p, const oracle_keig_opts *opt, const double *psi0,
                const double *phi0, double *phi_out, double *psi_out, double *k_hist,
                oracle_keig_result *res) {
  const int n = 1 << p->l, nc = n - 1, G = p->G, L = p->L, m8 = L / 8;
  const size_t n3 = (size_t)n * n * n, c3 = (size_t)nc * nc * nc;
  for (int f = 0; f < 6; ++f)
    if (p->bc[f]) return -1; /* vacuum faces only (Eq. (BCS)) */
  const int keep_psi = opt->store_psi || psi_out != NULL;
  double *psi = keep_psi ? (double *)malloc(sizeof(double) * G * L * n3) : NULL;
  double *psi_new = keep_psi ? (double *)malloc(sizeof(double) * G * L * n3) : NULL;
  double *phi = (double *)malloc(sizeof(double) * G * n3);
  double *pbar = (double *)malloc(sizeof(double) * G * c3);
  double *qs = (double *)malloc(sizeof(double) * G * c3);
  double *qf = (double *)malloc(sizeof(double) * G * c3);
  const int nthr = p->threads > 0 ? p->threads : omp_get_max_threads();
  double *acc = (double *)malloc(sizeof(double) * nthr * n3);
  double *work = (double *)malloc(sizeof(double) * nthr * 3 * n3);
  uint8_t *fmask = (uint8_t *)malloc(8 * n3);
  /* linearly anisotropic scattering: first moments and their sources */
  const int p1 = p->sig_s1 != NULL;
  double *J = p1 ? (double *)calloc((size_t)3 * G * n3, sizeof(double)) : NULL;
  double *Jbar = p1 ? (double *)calloc((size_t)3 * G * c3, sizeof(double)) : NULL;
  double *q1 = p1 ? (double *)malloc(sizeof(double) * 3 * G * c3) : NULL;
  double *accJ = p1 ? (double *)malloc(sizeof(double) * nthr * 3 * n3) : NULL;
  double *qd = p1 ? (double *)malloc(sizeof(double) * nthr * c3) : NULL;

  /* inflow Dirichlet masks per octant (all inflow-face vertices) */
  for (int o = 0; o < 8; ++o) {
    const int px = sgn_bit(o, 0), py = sgn_bit(o, 1), pz = sgn_bit(o, 2);
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
          fmask[o * n3 + ((size_t)k * n + j) * n + i] =
              on_inflow(k, pz, n) || on_inflow(j, py, n) || on_inflow(i, px, n);
  }

  if (psi0) {
    if (keep_psi) memcpy(psi, psi0, sizeof(double) * G * L * n3);
    scalar_flux(p, psi0, phi);
    if (p1) current(p, psi0, J);
  } else {
    memcpy(phi, phi0, sizeof(double) * G * n3);
  }
  cell_average(p, phi, pbar);
  double P = production(p, pbar);
  double k = opt->k0;
  /* normalise so that sum(F Psi) = 1 */
  for (size_t v = 0; v < (size_t)G * n3; ++v) phi[v] /= P;
  for (size_t v = 0; v < (size_t)G * c3; ++v) pbar[v] /= P;
  if (p1) {
    for (size_t v = 0; v < (size_t)3 * G * n3; ++v) J[v] /= P;
    for (int a = 0; a < 3; ++a) cell_average(p, J + (size_t)a * G * n3, Jbar + (size_t)a * G * c3);
  }
  if (keep_psi)
    for (size_t v = 0; v < (size_t)G * L * n3; ++v) psi[v] /= P;

  int it = 0;
  double dk = 1e300;
  for (it = 0; it < opt->max_iter; ++it) {
    cell_sources(p, pbar, qs, qf);
    for (size_t v = 0; v < (size_t)G * c3; ++v) qs[v] += qf[v] / k;
    if (p1) p1_sources(p, Jbar, q1);
    double *phin = (double *)calloc((size_t)G * n3, sizeof(double));
    double *Jn = p1 ? (double *)calloc((size_t)3 * G * n3, sizeof(double)) : NULL;
    for (int g = 0; g < G; ++g) {
      memset(acc, 0, sizeof(double) * nthr * n3);
      if (p1) memset(accJ, 0, sizeof(double) * nthr * 3 * n3);
#pragma omp parallel num_threads(nthr)
      {
        const int t = omp_get_thread_num();
        double *rows = work + (size_t)t * 3 * n3;
        double *fixv = rows + n3;
        double *out = rows + 2 * n3;
#pragma omp for schedule(static)
        for (int ell = 0; ell < L; ++ell) {
          const int o = ell / m8, d = ell % m8;
          if (p1) {
            double *qt = qd + (size_t)t * c3;
            direction_source(p, g, ell, qs + (size_t)g * c3, q1, qt);
            rows_from_cells(p, o, qt, rows);
          } else {
            rows_from_cells(p, o, qs + (size_t)g * c3, rows);
          }
          /* vacuum inflow faces: psi = 0 there (the face rows of H form a
           * homogeneous triangular system with positive diagonal) */
          for (size_t v = 0; v < n3; ++v) fixv[v] = 0.0;
          sweep_one(p, g, ell, rows, fmask + o * n3, fixv, out);
          double *a = acc + (size_t)t * n3;
          const double w = p->w8[d];
          for (size_t v = 0; v < n3; ++v) a[v] += w * out[v];
          if (p1)
            for (int ax = 0; ax < 3; ++ax) {
              double *aj = accJ + ((size_t)t * 3 + ax) * n3;
              const double wc = w * cosine(p, ell, ax);
              for (size_t v = 0; v < n3; ++v) aj[v] += wc * out[v];
            }
          if (keep_psi) memcpy(psi_new + ((size_t)g * L + ell) * n3, out, sizeof(double) * n3);
        }
      }
      for (int t = 0; t < nthr; ++t)
        for (size_t v = 0; v < n3; ++v) phin[(size_t)g * n3 + v] += acc[(size_t)t * n3 + v];
      if (p1)
        for (int ax = 0; ax < 3; ++ax)
          for (int t = 0; t < nthr; ++t)
            for (size_t v = 0; v < n3; ++v)
              Jn[((size_t)ax * G + g) * n3 + v] += accJ[((size_t)t * 3 + ax) * n3 + v];
    }
    memcpy(phi, phin, sizeof(double) * G * n3);
    free(phin);
    if (p1) {
      memcpy(J, Jn, sizeof(double) * 3 * G * n3);
      free(Jn);
    }
    cell_average(p, phi, pbar);
    const double Pn = production(p, pbar); /* previous iterate had P = 1 */
    const double kn = k * Pn;
    dk = fabs(kn - k);
    k = kn;
    for (size_t v = 0; v < (size_t)G * n3; ++v) phi[v] /= Pn;
    for (size_t v = 0; v < (size_t)G * c3; ++v) pbar[v] /= Pn;
    if (p1) {
      for (size_t v = 0; v < (size_t)3 * G * n3; ++v) J[v] /= Pn;
      for (int a = 0; a < 3; ++a) cell_average(p, J + (size_t)a * G * n3, Jbar + (size_t)a * G * c3);
    }
    if (keep_psi) {
      for (size_t v = 0; v < (size_t)G * L * n3; ++v) psi_new[v] /= Pn;
      double *t = psi;
      psi = psi_new;
      psi_new = t;
    }
    if (k_hist) k_hist[it] = k;
    if (dk < opt->tol_k) {
      ++it;
      break;
    }
  }
  if (phi_out) memcpy(phi_out, phi, sizeof(double) * G * n3);
  if (psi_out && keep_psi) memcpy(psi_out, psi, sizeof(double) * G * L * n3);
  res->k = k;
  res->iters = it;
  res->dk_last = dk;
  free(psi);
  free(psi_new);
  free(phi);
  free(pbar);
  free(qs);
  free(qf);
  free(acc);
  free(work);
  free(fmask);
  free(J);
  free(Jbar);
  free(q1);
  free(accJ);
  free(qd);
  return dk < opt->tol_k ? 0 : 1;
}

/* leakage, absorption and production of a (normalised) solution, for the
 * global balance check: each cell balance weighted by w and summed over
 * cells, directions and groups telescopes the streaming terms to the faces. */
void oracle_balance(const oracle_problem *p, const double *psi, double *leak, double *absorb,
                    double *scat_out, double *scat_in, double *prod) {
  const int n = 1 << p->l, nc = n - 1, G = p->G, L = p->L, m8 = L / 8;
  const size_t n3 = (size_t)n * n * n, c3 = (size_t)nc * nc * nc;
  double *phi = (double *)malloc(sizeof(double) * G * n3);
  double *pbar = (double *)malloc(sizeof(double) * G * c3);
  double *qs = (double *)malloc(sizeof(double) * G * c3);
  double *qf = (double *)malloc(sizeof(double) * G * c3);
  scalar_flux(p, psi, phi);
  cell_average(p, phi, pbar);
  cell_sources(p, pbar, qs, qf);
  double A = 0, Si = 0, So = 0, Pr = 0, Lk = 0;
  const double vol = p->dx * p->dy * p->dz;
  for (size_t c = 0; c < c3; ++c) {
    const int m = p->mat[c];
    for (int g = 0; g < G; ++g) {
      A += vol * p->sig_t[m * G + g] * pbar[(size_t)g * c3 + c];
      Si += vol * qs[(size_t)g * c3 + c];
      Pr += vol * qf[(size_t)g * c3 + c];
    }
  }
  /* net outflow through the six faces: face-averaged psi times the cosine */
  for (int g = 0; g < G; ++g)
    for (int ell = 0; ell < L; ++ell) {
      const int o = ell / m8, d = ell % m8;
      const double w = p->w8[d];
      const double *ps = psi + ((size_t)g * L + ell) * n3;
      const double sc[3] = {(o & 1) ? p->amu[d] : -p->amu[d], (o & 2) ? p->aeta[d] : -p->aeta[d],
                            (o & 4) ? p->axi[d] : -p->axi[d]};
      for (int axis = 0; axis < 3; ++axis)
        for (int side = 0; side < 2; ++side) {
          /* outward normal sign: side 0 -> -, side 1 -> + */
          const double nrm = side ? 1.0 : -1.0;
          const int fix = side ? n - 1 : 0;
          double area = axis == 0 ? p->dy * p->dz : axis == 1 ? p->dx * p->dz : p->dx * p->dy;
          double s = 0.0;
          for (int a = 0; a < nc; ++a)
            for (int bq = 0; bq < nc; ++bq) {
              double f = 0.0;
              for (int u = 0; u < 2; ++u)
                for (int t = 0; t < 2; ++t) {
                  int i, j, k;
                  if (axis == 0) { i = fix; j = a + u; k = bq + t; }
                  else if (axis == 1) { j = fix; i = a + u; k = bq + t; }
                  else { k = fix; i = a + u; j = bq + t; }
                  f += ps[((size_t)k * n + j) * n + i];
                }
              s += f / 4.0;
            }
          Lk += w * nrm * sc[axis] * area * s;
        }
    }
  (void)So;
  *leak = Lk;
  *absorb = A;
  *scat_out = 0.0;
  *scat_in = Si;
  *prod = Pr;
  free(phi);
  free(pbar);
  free(qs);
  free(qf);
}
