// Construction of the transport operators H, S, F as TT matrices over the
// modes [G][8][L/8][z bits][y bits][x bits] (Sec. 3.2-3.3 and Algorithm 1).
//
// Each operator is a sum of rank-1 terms (tensor products of univariate
// factors).  Per octant o with cosine signs (sx, sy, sz) (bit set =
// positive, octant order of Eq. (hat-mu)):
//   H: I_G (x) E_o (x) diag|mu|  (x) Ip_z (x) Ip_y (x) Dt_x
//      I_G (x) E_o (x) diag|eta| (x) Ip_z (x) Dt_y (x) Ip_x
//      I_G (x) E_o (x) diag|xi|  (x) Dt_z (x) Ip_y (x) Ip_x
//      sum_m diag(sig_t(m)) (x) E_o (x) I (x) M_m^o (Ip_z (x) Ip_y (x) Ip_x)
//   S: sum_m Sig_s(m)        (x) e_o 1^T (x) 1 w^T (x) M_m^o (Ip_z,noBC (x) Ip_y,noBC (x) Ip_x,noBC)
//   F: sum_m chi(m) nsf(m)^T (x) e_o 1^T (x) 1 w^T (x) M_m^o (same)
// with Dt+ = D+, Dt- = -D- (so that mu D^{sign mu} = |mu| Dt), E_o = e_o e_o^T,
// and M_m^o the diagonal mask of the rows whose upstream cell (cell i-1 along
// a positive cosine, cell i along a negative one, clamped) is material m.
// Every n x n spatial factor goes to QTT by Algorithm 1 (reshape, pair the
// (i_k, j_k) indices, TT-SVD) on the device; the masks are QTT-compressed by
// TT-SVD of their n^3 values; terms are added and rounded.
#include <algorithm>

#include "tt.cuh"

namespace tt {

namespace {

std::vector<double> factor_D(int n, double delta, bool pos) {
  std::vector<double> a((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    a[(size_t)i * n + i] = 1.0 / delta;
    if (pos && i > 0) a[(size_t)i * n + i - 1] = -1.0 / delta;
    if (!pos && i + 1 < n) a[(size_t)i * n + i + 1] = -1.0 / delta;
  }
  return a;
}

std::vector<double> factor_Ip(int n, bool pos, bool no_bc) {
  std::vector<double> a((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    a[(size_t)i * n + i] = 0.5;
    if (pos && i > 0) a[(size_t)i * n + i - 1] = 0.5;
    if (!pos && i + 1 < n) a[(size_t)i * n + i + 1] = 0.5;
  }
  if (no_bc) {
    const int row = pos ? 0 : n - 1;
    for (int j = 0; j < n; ++j) a[(size_t)row * n + j] = 0.0;
  }
  return a;
}

// Real spherical harmonic Y_nm (m > 0 cosine type, m < 0 sine type) with
// unit mean square over the sphere, at the unit direction (x, y, z), z the
// polar axis: sqrt((2n+1)(2 - delta_m0)(n-|m|)!/(n+|m|)!) P_n^|m|(z) trig(|m| phi),
// P_n^m by the standard three-term recurrence in n (no Condon-Shortley phase).
double real_sh(int n, int m, double x, double y, double z) {
  const int am = m < 0 ? -m : m;
  const double st = std::sqrt(std::max(0.0, 1.0 - z * z));
  double pmm = 1.0;
  for (int i = 1; i <= am; ++i) pmm *= (2.0 * i - 1.0) * st;
  double P = pmm;
  if (n > am) {
    double a = pmm, b = z * (2.0 * am + 1.0) * pmm;
    for (int ll = am + 2; ll <= n; ++ll) {
      const double cnew = (z * (2.0 * ll - 1.0) * b - (ll + am - 1.0) * a) / (ll - am);
      a = b;
      b = cnew;
    }
    P = b;
  }
  double ratio = 1.0;  // (n-|m|)! / (n+|m|)!
  for (int i = n - am + 1; i <= n + am; ++i) ratio /= i;
  const double norm = std::sqrt((2.0 * n + 1.0) * (am == 0 ? 1.0 : 2.0) * ratio);
  const double phi = std::atan2(y, x);
  return norm * P * (m >= 0 ? std::cos(am * phi) : std::sin(am * phi));
}

// Parity of Y_nm in (x, y, z): Y(s_x x, s_y y, s_z z) = s_x^px s_y^py s_z^pz Y(x, y, z)
void sh_parity(int n, int m, int &px, int &py, int &pz) {
  const int am = m < 0 ? -m : m;
  pz = (n - am) & 1;
  px = m >= 0 ? (am & 1) : ((am - 1) & 1);
  py = m >= 0 ? 0 : 1;
}

int row_cell(int v, bool pos, int n) {
  int c = pos ? v - 1 : v;
  return std::max(0, std::min(c, n - 2));
}

DBuf upload(Ctx *c, const std::vector<double> &h) {
  DBuf b(c, h.size());
  TT_CHECK_CUDA(cudaMemcpyAsync(b.p(), h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  return b;
}

// Algorithm 1 for one 2^l x 2^l factor: QTT-matrix cores (r, 2, 2, r).
std::vector<DBuf> qtt_factor(Ctx *c, const std::vector<double> &mat, int l, std::vector<int> &ranks) {
  const int n = 1 << l;
  DBuf dm = upload(c, mat);
  DBuf perm(c, (size_t)n * n);
  std::vector<int> shape(2 * l, 2), p(2 * l);
  for (int k = 0; k < l; ++k) {
    p[2 * k] = k;          // i_k
    p[2 * k + 1] = l + k;  // j_k
  }
  permute(c, dm.p(), perm.p(), 2 * l, shape.data(), p.data());
  std::vector<int> modes(l, 4);
  TT t = tt_svd_dense(c, perm.p(), modes, 1e-14, 0);
  ranks = t.r;
  return std::move(t.core);
}

__global__ void diag_times_op_kernel(const double *__restrict__ mk, int rc0, int rc1,
                                     const double *__restrict__ S, int Rs0, int Rs1, double *__restrict__ out) {
  // out[(a,al), i, j, (b,be)] = mk[a, i, b] * S[al, i, j, be]
  const long long tot = (long long)rc0 * Rs0 * 4 * rc1 * Rs1;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    long long rem = e;
    const int be = (int)(rem % Rs1);
    rem /= Rs1;
    const int b = (int)(rem % rc1);
    rem /= rc1;
    const int j = (int)(rem % 2);
    rem /= 2;
    const int i = (int)(rem % 2);
    rem /= 2;
    const int al = (int)(rem % Rs0);
    const int a = (int)(rem / Rs0);
    out[e] = mk[((long long)a * 2 + i) * rc1 + b] * S[(((long long)al * 2 + i) * 2 + j) * Rs1 + be];
  }
}

struct Term {
  std::vector<std::vector<double>> head;  // G x G, (8 or 2) x (8 or 2), nd x nd factors
  std::vector<int> f;                     // per spatial axis (outermost first): index into the QTT factor list
  int mask;                               // -1 or index into the mask list
};

// Sum of rank-1 terms as one TT matrix: head cores h0.. of each term, then
// the QTT cores of its spatial factors axis by axis (l bits each), each term
// optionally multiplied row-wise by a diagonal mask TT; partial sums rounded
// every few terms and at the end at eps_op.
TT assemble_terms(Ctx *c, const std::vector<Term> &terms, int h0, const std::vector<int> &hsz, int naxes, int l,
                  const std::vector<std::vector<DBuf>> &qf, const std::vector<std::vector<int>> &qr,
                  const std::vector<TT> &masks, double eps_op) {
  const int nh = (int)hsz.size() - h0;  // head cores kept
  const int d = nh + naxes * l;
  const int sp0 = nh;  // index of the first spatial core
  std::vector<int> mo(d), mi(d);
  for (int k = 0; k < sp0; ++k) mo[k] = mi[k] = hsz[k + h0];
  for (int k = sp0; k < d; ++k) mo[k] = mi[k] = 2;
  TT acc;
  bool have = false;
  int pending = 0;
  for (const Term &t : terms) {
    TT x;
    x.d = d;
    x.mo = mo;
    x.mi = mi;
    x.n.resize(d);
    for (int k = 0; k < d; ++k) x.n[k] = mo[k] * mi[k];
    x.r.assign(d + 1, 1);
    x.core.resize(d);
    for (int k = 0; k < sp0; ++k) x.core[k] = upload(c, t.head[k + h0]);
    for (int a = 0; a < naxes; ++a)
      for (int b = 0; b < l; ++b) {
        const int k = sp0 + a * l + b;
        x.r[k] = qr[t.f[a]][b];
        x.r[k + 1] = qr[t.f[a]][b + 1];
        x.core[k].alloc(c, x.csize(k));
        copy(c, x.core[k].p(), qf[t.f[a]][b].p(), x.csize(k));
      }
    if (t.mask >= 0) {
      // M (Ip (x) ... (x) Ip): core-wise product with the diagonal mask TT
      const TT &mk = masks[t.mask];
      for (int q = 0; q < naxes * l; ++q) {
        const int k = sp0 + q;
        const int rc0 = mk.r[q], rc1 = mk.r[q + 1], Rs0 = x.r[k], Rs1 = x.r[k + 1];
        DBuf out(c, (size_t)rc0 * Rs0 * 4 * rc1 * Rs1);
        const long long tot = (long long)rc0 * Rs0 * 4 * rc1 * Rs1;
        diag_times_op_kernel<<<(unsigned)std::min<long long>((tot + 255) / 256, 4096), 256, 0, c->stream>>>(
            mk.core[q].p(), rc0, rc1, x.core[k].p(), Rs0, Rs1, out.p());
        c->count();
        TT_CHECK_CUDA(cudaGetLastError());
        x.core[k] = std::move(out);
      }
      for (int q = 1; q < naxes * l; ++q) x.r[sp0 + q] *= mk.r[q];
      round(c, x, 1e-14, 0);
    }
    if (!have) {
      acc = std::move(x);
      have = true;
    } else {
      acc = add(c, 1.0, acc, 1.0, x);
      if (++pending >= 4) {
        round(c, acc, eps_op, 0);
        pending = 0;
      }
    }
  }
  TT_REQUIRE(have, "build_operator: operator has no terms");
  round(c, acc, eps_op, 0);
  return acc;
}

}  // namespace

OpFactors make_factors(Ctx *c, const tt_problem *p) {
  OpFactors F;
  const int l = p->l, n = 1 << l, nm = p->n_mat;
  const double del[3] = {p->side[0] / (n - 1), p->side[1] / (n - 1), p->side[2] / (n - 1)};
  auto add_factor = [&](std::vector<double> f) {
    std::vector<int> rk;
    F.qf.push_back(qtt_factor(c, f, l, rk));
    F.qr.push_back(rk);
    return (int)F.qf.size() - 1;
  };
  for (int pos = 0; pos < 2; ++pos) {
    F.iIp[pos] = add_factor(factor_Ip(n, pos, false));
    F.iIpN[pos] = add_factor(factor_Ip(n, pos, true));
    for (int a = 0; a < 3; ++a) F.iD[a][pos] = add_factor(factor_D(n, del[a], pos));
  }
  // material masks per (octant, material) in QTT (only when heterogeneous)
  F.mask_index.assign((size_t)8 * nm, -1);
  if (nm > 1) {
    const int nc = n - 1;
    std::vector<double> mv((size_t)n * n * n);
    std::vector<int> mode3(3 * l, 2);
    for (int o = 0; o < 8; ++o) {
      const bool px = o & 1, py = o & 2, pz = o & 4;
      for (int m = 0; m < nm; ++m) {
        size_t cnt = 0;
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
              const int mat = p->mat[((size_t)row_cell(k, pz, n) * nc + row_cell(j, py, n)) * nc + row_cell(i, px, n)];
              mv[((size_t)k * n + j) * n + i] = (mat == m) ? 1.0 : 0.0;
              cnt += (mat == m);
            }
        if (!cnt) continue;
        DBuf dmv = upload(c, mv);
        F.masks.push_back(tt_svd_dense(c, dmv.p(), mode3, 1e-14, 0));
        F.mask_index[(size_t)o * nm + m] = (int)F.masks.size() - 1;
      }
    }
  }
  return F;
}

TT assemble_operator(Ctx *c, const tt_problem *p, const OpFactors &F, int kind, int only_mat, double eps_op,
                     int only_oct) {
  const int l = p->l, G = p->G, nd = p->n_dir, nm = p->n_mat;
  // derivative kinds omit the group core (the operator is linear in the group matrix)
  const bool group_core = !(kind == KIND_COLLISION || kind == KIND_SOURCE);
  const int h0 = group_core ? 0 : 1;  // first head factor used
  std::vector<Term> terms;
  auto eye = [](int k) {
    std::vector<double> a((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i) a[(size_t)i * k + i] = 1.0;
    return a;
  };
  auto diag = [](const double *v, int k) {
    std::vector<double> a((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i) a[(size_t)i * k + i] = v[i];
    return a;
  };
  std::vector<double> dirm((size_t)nd * nd);
  for (int a = 0; a < nd; ++a)
    for (int b = 0; b < nd; ++b) dirm[(size_t)a * nd + b] = p->w[b];
  for (int o = 0; o < 8; ++o) {
    if (only_oct >= 0 && o != only_oct) continue;  // the rows of one octant only
    const int px = (o & 1) ? 1 : 0, py = (o & 2) ? 1 : 0, pz = (o & 4) ? 1 : 0;
    std::vector<double> E(64, 0.0), Intg(64, 0.0);
    E[o * 8 + o] = 1.0;
    for (int j = 0; j < 8; ++j) Intg[o * 8 + j] = 1.0;
    if (kind == TT_OP_H) {
      terms.push_back({{eye(G), E, diag(p->amu, nd)}, {F.iIp[pz], F.iIp[py], F.iD[0][px]}, -1});
      terms.push_back({{eye(G), E, diag(p->aeta, nd)}, {F.iIp[pz], F.iD[1][py], F.iIp[px]}, -1});
      terms.push_back({{eye(G), E, diag(p->axi, nd)}, {F.iD[2][pz], F.iIp[py], F.iIp[px]}, -1});
    }
    for (int m = 0; m < nm; ++m) {
      if (only_mat >= 0 && m != only_mat) continue;
      const int mi = nm > 1 ? F.mask_index[(size_t)o * nm + m] : -1;
      if (nm > 1 && mi < 0) continue;
      if (kind == TT_OP_H || kind == KIND_COLLISION) {
        terms.push_back({{kind == TT_OP_H ? diag(p->sig_t + (size_t)m * G, G) : std::vector<double>(), E, eye(nd)},
                         {F.iIp[pz], F.iIp[py], F.iIp[px]}, mi});
      } else if (kind == KIND_SOURCE) {
        terms.push_back({{std::vector<double>(), Intg, dirm}, {F.iIpN[pz], F.iIpN[py], F.iIpN[px]}, mi});
      } else {
        std::vector<double> gm((size_t)G * G);
        bool nonzero = false;
        for (int a = 0; a < G; ++a)
          for (int b = 0; b < G; ++b) {
            const double v = kind == TT_OP_S ? p->sig_s[((size_t)m * G + a) * G + b]
                                             : p->chi[(size_t)m * G + a] * p->nu_sig_f[(size_t)m * G + b];
            gm[(size_t)a * G + b] = v;
            nonzero |= v != 0.0;
          }
        if (nonzero) terms.push_back({{gm, Intg, dirm}, {F.iIpN[pz], F.iIpN[py], F.iIpN[px]}, mi});
        if (kind == TT_OP_S && p->sig_s1) {
          // linear anisotropy: for each axis a, row (o, d) gains 3 Omega_a(o, d)
          // sum_{o', d'} w_d' Omega_a(o', d') (P1 group matrix): a rank-1 angular
          // factor (sign pattern over octants) (x) (|Omega_a| (|Omega_a| w)^T)
          std::vector<double> g1((size_t)G * G);
          bool nz1 = false;
          for (size_t e = 0; e < (size_t)G * G; ++e) {
            g1[e] = 3.0 * p->sig_s1[(size_t)m * G * G + e];
            nz1 |= g1[e] != 0.0;
          }
          const double *cosv[3] = {p->amu, p->aeta, p->axi};
          for (int a = 0; a < 3 && nz1; ++a) {
            std::vector<double> octm(64, 0.0), dirp((size_t)nd * nd);
            const double so = (o >> a) & 1 ? 1.0 : -1.0;
            for (int j = 0; j < 8; ++j) octm[o * 8 + j] = so * ((j >> a) & 1 ? 1.0 : -1.0);
            for (int x = 0; x < nd; ++x)
              for (int y = 0; y < nd; ++y) dirp[(size_t)x * nd + y] = cosv[a][x] * cosv[a][y] * p->w[y];
            terms.push_back({{g1, octm, dirp}, {F.iIpN[pz], F.iIpN[py], F.iIpN[px]}, mi});
          }
        }
        if (kind == TT_OP_S) {
          // orders 2 and 3: for each m, Y_nm factors into an octant sign pattern
          // (its parity) times its value at the first-octant direction, so the
          // angular factor (row octant o) is rank one:
          //   (sign(o) sign(o')) (x) (Y_nm(d) Y_nm(d') w_d')
          const double *sn_tab[2] = {p->sig_s2, p->sig_s3};
          for (int nn = 2; nn <= 3; ++nn) {
            const double *sn = sn_tab[nn - 2];
            if (!sn) continue;
            std::vector<double> gn((size_t)G * G);
            bool nzn = false;
            for (size_t e = 0; e < (size_t)G * G; ++e) {
              gn[e] = sn[(size_t)m * G * G + e];
              nzn |= gn[e] != 0.0;
            }
            if (!nzn) continue;
            for (int mm = -nn; mm <= nn; ++mm) {
              int qx, qy, qz;
              sh_parity(nn, mm, qx, qy, qz);
              auto sgn = [&](int oo) {
                double sv = 1.0;
                if (qx && !(oo & 1)) sv = -sv;
                if (qy && !(oo & 2)) sv = -sv;
                if (qz && !(oo & 4)) sv = -sv;
                return sv;
              };
              std::vector<double> octm(64, 0.0), dirp((size_t)nd * nd), v(nd);
              for (int j = 0; j < 8; ++j) octm[o * 8 + j] = sgn(o) * sgn(j);
              for (int dd = 0; dd < nd; ++dd) v[dd] = real_sh(nn, mm, p->amu[dd], p->aeta[dd], p->axi[dd]);
              for (int x = 0; x < nd; ++x)
                for (int y = 0; y < nd; ++y) dirp[(size_t)x * nd + y] = v[x] * v[y] * p->w[y];
              terms.push_back({{gn, octm, dirp}, {F.iIpN[pz], F.iIpN[py], F.iIpN[px]}, mi});
            }
          }
        }
      }
    }
  }
  return assemble_terms(c, terms, h0, {G, 8, nd}, 3, l, F.qf, F.qr, F.masks, eps_op);
}

// 1-D slab operators over the modes [G][2][n_dir][x bits]: the terms of the
// 3-D operators restricted to x, with a hemisphere core (0: mu < 0, 1: mu > 0)
// in place of the octant core:
//   H: I_G (x) E_h (x) diag|mu| (x) Dt_x  +  sum_m diag(sig_t(m)) (x) E_h (x) I (x) M_m^h Ip_x
//   S: sum_m Sig_s(m)          (x) e_h 1^T (x) 1 w^T (x) M_m^h Ip_x,noBC
//   F: sum_m chi(m) nsf(m)^T   (x) e_h 1^T (x) 1 w^T (x) M_m^h Ip_x,noBC
TT assemble_slab_operator(Ctx *c, const tt_slab *s, int kind, double eps_op) {
  const int l = s->l, n = 1 << l, G = s->G, nd = s->n_dir, nm = s->n_mat;
  const double del = s->width / (n - 1);
  std::vector<std::vector<DBuf>> qf;
  std::vector<std::vector<int>> qr;
  auto add_factor = [&](std::vector<double> f) {
    std::vector<int> rk;
    qf.push_back(qtt_factor(c, f, l, rk));
    qr.push_back(rk);
    return (int)qf.size() - 1;
  };
  int iD[2], iIp[2], iIpN[2];
  for (int pos = 0; pos < 2; ++pos) {
    iD[pos] = add_factor(factor_D(n, del, pos));
    iIp[pos] = add_factor(factor_Ip(n, pos, false));
    iIpN[pos] = add_factor(factor_Ip(n, pos, true));
  }
  // row masks per (hemisphere, material) when heterogeneous
  std::vector<TT> masks;
  std::vector<int> mask_index((size_t)2 * nm, -1);
  if (nm > 1) {
    std::vector<double> mv(n);
    for (int h = 0; h < 2; ++h)
      for (int m = 0; m < nm; ++m) {
        int cnt = 0;
        for (int i = 0; i < n; ++i) {
          const int mat = s->mat[row_cell(i, h == 1, n)];
          mv[i] = mat == m ? 1.0 : 0.0;
          cnt += mat == m;
        }
        if (!cnt) continue;
        DBuf dmv = upload(c, mv);
        masks.push_back(tt_svd_dense(c, dmv.p(), std::vector<int>(l, 2), 1e-14, 0));
        mask_index[(size_t)h * nm + m] = (int)masks.size() - 1;
      }
  }
  auto eye = [](int k) {
    std::vector<double> a((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i) a[(size_t)i * k + i] = 1.0;
    return a;
  };
  auto diag = [](const double *v, int k) {
    std::vector<double> a((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i) a[(size_t)i * k + i] = v[i];
    return a;
  };
  std::vector<double> dirm((size_t)nd * nd);
  for (int a = 0; a < nd; ++a)
    for (int b = 0; b < nd; ++b) dirm[(size_t)a * nd + b] = s->w[b];
  std::vector<Term> terms;
  for (int h = 0; h < 2; ++h) {
    std::vector<double> E(4, 0.0), Intg(4, 0.0);
    E[h * 2 + h] = 1.0;
    Intg[h * 2] = Intg[h * 2 + 1] = 1.0;
    if (kind == TT_OP_H) terms.push_back({{eye(G), E, diag(s->amu, nd)}, {iD[h]}, -1});
    for (int m = 0; m < nm; ++m) {
      const int mi = nm > 1 ? mask_index[(size_t)h * nm + m] : -1;
      if (nm > 1 && mi < 0) continue;
      if (kind == TT_OP_H) {
        terms.push_back({{diag(s->sig_t + (size_t)m * G, G), E, eye(nd)}, {iIp[h]}, mi});
      } else {
        std::vector<double> gm((size_t)G * G);
        bool nonzero = false;
        for (int a = 0; a < G; ++a)
          for (int b = 0; b < G; ++b) {
            const double v = kind == TT_OP_S ? s->sig_s[((size_t)m * G + a) * G + b]
                                             : s->chi[(size_t)m * G + a] * s->nu_sig_f[(size_t)m * G + b];
            gm[(size_t)a * G + b] = v;
            nonzero |= v != 0.0;
          }
        if (!nonzero) continue;
        terms.push_back({{gm, Intg, dirm}, {iIpN[h]}, mi});
      }
    }
  }
  return assemble_terms(c, terms, 0, {G, 2, nd}, 1, l, qf, qr, masks, eps_op);
}

TT build_operator(Ctx *c, const tt_problem *p, int kind, double eps_op) {
  OpFactors F = make_factors(c, p);
  return assemble_operator(c, p, F, kind, -1, eps_op);
}

}  // namespace tt
