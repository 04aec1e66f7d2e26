// Host-side setup of the radial operators (runs once per (N,K,M,m_p,alpha,Re,dt,c)).
//
// Paper section 2: radial points clustered like Chebyshev points, derivatives
// by 9-point finite differences (banded matrices), implicit viscous and
// pressure-Poisson solves by LU per Fourier mode (section 2.2), boundary
// conditions by the influence-matrix technique (section 2).  The stencil
// weights come from Fornberg's recursion; the LU is banded and pivot-free,
// each factor checked against its matrix before use.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>

#include "opf_internal.h"

namespace opf {

using cplx = std::complex<double>;

static inline int row_lo(int N, int n) { return std::min(std::max(n - 4, 0), N - 9); }
static inline int row_hi(int N, int n) { return std::min(n + 4, N - 1); }

bool make_plan(int n, FftPlan* p) {
  p->n = n;
  p->nst = 0;
  int m = n;
  const int order[4] = {4, 2, 3, 5};
  for (int R : order) {
    while (m % R == 0) {
      if (p->nst == kMaxRadix) return false;
      p->rad[p->nst++] = R;
      m /= R;
    }
  }
  return m == 1 && n >= 1;
}

// Fornberg (1988) recursion: weights c[t*(md+1)+d] of node x[t] for the
// d-th derivative at z, d = 0..md.
static void fornberg(double z, const double* x, int n, int md, double* c) {
  const int s = md + 1;
  for (int i = 0; i < n * s; ++i) c[i] = 0.0;
  double c1 = 1.0, c4 = x[0] - z;
  c[0] = 1.0;
  for (int i = 1; i < n; ++i) {
    const int mn = std::min(i, md);
    double c2 = 1.0;
    const double c5 = c4;
    c4 = x[i] - z;
    for (int j = 0; j < i; ++j) {
      const double c3 = x[i] - x[j];
      c2 *= c3;
      if (j == i - 1) {
        for (int k = mn; k >= 1; --k)
          c[i * s + k] = c1 * (k * c[(i - 1) * s + k - 1] - c5 * c[(i - 1) * s + k]) / c2;
        c[i * s] = -c1 * c5 * c[(i - 1) * s] / c2;
      }
      for (int k = mn; k >= 1; --k) c[j * s + k] = (c4 * c[j * s + k] - k * c[j * s + k - 1]) / c3;
      c[j * s] = c4 * c[j * s] / c3;
    }
    c1 = c2;
  }
}

// Extended point set {-r_N..-r_1, r_1..r_N}; index e -> value, folded column, is_ghost.
struct Ext {
  const std::vector<double>& r;
  int N;
  double x(int e) const { return e < N ? -r[N - 1 - e] : r[e - N]; }
  int col(int e) const { return e < N ? N - 1 - e : e - N; }
  bool ghost(int e) const { return e < N; }
  int first(int n) const {  // first extended index of row n's stencil
    int q = N + n;
    return (q + 4 > 2 * N - 1) ? 2 * N - 9 : q - 4;
  }
};

// 9-point D1, D2 rows for both parities, folded, stored [parity][n][9]
// against columns row_lo(n) + t.
static void build_stencils(Setup* s) {
  const int N = s->N;
  Ext ext{s->r, N};
  s->d1.assign(2 * N * kStencil, 0.0);
  s->d2.assign(2 * N * kStencil, 0.0);
  double x[kStencil], c[kStencil * 3];
  for (int n = 0; n < N; ++n) {
    const int e0 = ext.first(n);
    for (int t = 0; t < kStencil; ++t) x[t] = ext.x(e0 + t);
    fornberg(s->r[n], x, kStencil, 2, c);
    const int lo = row_lo(N, n);
    for (int par = 0; par < 2; ++par) {
      const double sg = par == 0 ? 1.0 : -1.0;
      for (int t = 0; t < kStencil; ++t) {
        const int e = e0 + t;
        const double f = ext.ghost(e) ? sg : 1.0;
        const int slot = ext.col(e) - lo;
        s->d1[(par * N + n) * kStencil + slot] += f * c[t * 3 + 1];
        s->d2[(par * N + n) * kStencil + slot] += f * c[t * 3 + 2];
      }
    }
  }
}

// Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on P_n.
static void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// w_n such that sum w_n f(r_n) integrates f(r) r over [0,1] for even f:
// over each [r_(n-1), r_n] (r_0 = 0) the 9-point interpolant of r f through
// row n's stencil is integrated exactly.
static void build_quadrature(Setup* s) {
  const int N = s->N;
  Ext ext{s->r, N};
  double gx[8], gw[8];
  gauss_legendre(8, gx, gw);
  s->wq.assign(N, 0.0);
  for (int n = 0; n < N; ++n) {
    const double a = n == 0 ? 0.0 : s->r[n - 1], b = s->r[n];
    const int e0 = ext.first(n);
    double nodes[kStencil];
    for (int t = 0; t < kStencil; ++t) nodes[t] = ext.x(e0 + t);
    for (int t = 0; t < kStencil; ++t) {
      double integral = 0.0;
      for (int g = 0; g < 8; ++g) {
        const double xg = 0.5 * (b - a) * gx[g] + 0.5 * (a + b);
        double l = 1.0;
        for (int u = 0; u < kStencil; ++u)
          if (u != t) l *= (xg - nodes[u]) / (nodes[t] - nodes[u]);
        integral += 0.5 * (b - a) * gw[g] * l;
      }
      s->wq[ext.col(e0 + t)] += integral * nodes[t];
    }
  }
}

// Dense work matrix for one operator; only the band is ever non-zero.
struct Op {
  int N;
  std::vector<double> a;  // row-major N x N
  double& at(int i, int j) { return a[(size_t)i * N + j]; }
};

// Rows n < N-1:  diag_n * I + coef2 * (D2 + D1 / r)  with D of parity par.
static void assemble(const Setup* s, int par, double coef2, const std::vector<double>& diag, Op* op) {
  const int N = s->N;
  op->N = N;
  op->a.assign((size_t)N * N, 0.0);
  for (int n = 0; n < N - 1; ++n) {
    const int lo = row_lo(N, n);
    for (int t = 0; t < kStencil; ++t) {
      const int j = lo + t;
      if (j >= N) break;
      op->at(n, j) += coef2 * (s->d2[(par * N + n) * kStencil + t] +
                               s->rinv[n] * s->d1[(par * N + n) * kStencil + t]);
    }
    op->at(n, n) += diag[n];
  }
}

static void wall_dirichlet(Op* op) {
  const int N = op->N;
  for (int j = 0; j < N; ++j) op->at(N - 1, j) = 0.0;
  op->at(N - 1, N - 1) = 1.0;
}

static void wall_neumann(const Setup* s, int par, Op* op) {
  const int N = op->N;
  for (int j = 0; j < N; ++j) op->at(N - 1, j) = 0.0;
  const int lo = row_lo(N, N - 1);
  for (int t = 0; t < kStencil; ++t) op->at(N - 1, lo + t) = s->d1[(par * N + N - 1) * kStencil + t];
}

// Pivot-free banded LU of op into 13-slot rows; checks the factor on a test
// right-hand side against the unfactored matrix.
// Solve with a factor stored by factor(): unit-lower L, then 1/U_ii, then the
// row-scaled unit-upper U (the same order as the GPU substitution).
static void lu_solve(const double* f, int N, double* x) {
  for (int i = 0; i < N; ++i)
    for (int t = 0; t < 8; ++t)
      if (i - 8 + t >= 0) x[i] -= f[(size_t)i * kLuSlots + t] * x[i - 8 + t];
  for (int i = 0; i < N; ++i) x[i] *= f[(size_t)i * kLuSlots + 8];
  for (int i = N - 1; i >= 0; --i)
    for (int t = 1; t <= 4; ++t)
      if (i + t < N) x[i] -= f[(size_t)i * kLuSlots + 8 + t] * x[i + t];
}

static bool factor(Op* op, double* out, std::string* err, const char* what) {
  const int N = op->N;
  const std::vector<double> orig = op->a;
  for (int k = 0; k < N - 1; ++k) {
    const double piv = op->at(k, k);
    if (piv == 0.0 || !std::isfinite(piv)) {
      *err = std::string("zero pivot in banded LU of ") + what;
      return false;
    }
    const int hk = row_hi(N, k);
    for (int i = k + 1; i <= std::min(N - 1, k + 8); ++i) {
      if (op->at(i, k) == 0.0) continue;
      const double l = op->at(i, k) / piv;
      op->at(i, k) = l;
      for (int j = k + 1; j <= hk; ++j) op->at(i, j) -= l * op->at(k, j);
    }
  }
  for (int i = 0; i < N; ++i) {
    double* row = out + (size_t)i * kLuSlots;
    for (int t = 0; t < 8; ++t) {
      const int j = i - 8 + t;
      row[t] = (j >= 0) ? op->at(i, j) : 0.0;
    }
    row[8] = 1.0 / op->at(i, i);
    // U stored row-scaled by 1/U_ii (unit upper triangle), so the backward
    // recursion needs no division: x_i = y_i / U_ii - sum_t (U_i,i+t / U_ii) x_i+t
    for (int t = 1; t <= 4; ++t) row[8 + t] = (i + t < N) ? op->at(i, i + t) * row[8] : 0.0;
  }
  // self-check: solve A x = b and compare A x with b
  std::vector<double> b(N), x(N);
  for (int i = 0; i < N; ++i) b[i] = std::sin(1.0 + i) + 0.5;
  x = b;
  lu_solve(out, N, x.data());
  double res = 0.0, anorm = 0.0, xnorm = 0.0;
  for (int i = 0; i < N; ++i) {
    double acc = 0.0, rs = 0.0;
    for (int j = 0; j < N; ++j) {
      acc += orig[(size_t)i * N + j] * x[j];
      rs += std::fabs(orig[(size_t)i * N + j]);
    }
    res = std::max(res, std::fabs(acc - b[i]));
    anorm = std::max(anorm, rs);
    xnorm = std::max(xnorm, std::fabs(x[i]));
  }
  if (!(res <= 1e-12 * anorm * xnorm)) {
    char buf[200];
    std::snprintf(buf, sizeof buf, "pivot-free LU of %s inaccurate (residual %.3e)", what,
                  res / (anorm * xnorm));
    *err = buf;
    return false;
  }
  return true;
}

// Device order of a factor (13 N values, like the row slots): per column c,
// [N][4] L(c+1+t, c), [N][4] L(c+5+t, c) (the wall rows' wider band),
// [N] 1/U_ii, [N][4] U~(c-1-t, c), t = 0..3.  The substitution's four lanes
// of a chain read the entries of one column at a time, so a warp's loads come
// in 32-byte runs instead of one 104-byte row per lane.  Applied after every
// host use of the row form.
static void to_columns(double* f, int N) {
  std::vector<double> g((size_t)kLuSlots * N, 0.0);
  for (int c = 0; c < N; ++c)
    for (int t = 0; t < 4; ++t) {
      const int r = c + 1 + t, rw = c + 5 + t, ru = c - 1 - t;
      g[(size_t)c * 4 + t] = r < N ? f[(size_t)r * kLuSlots + 7 - t] : 0.0;
      g[(size_t)4 * N + c * 4 + t] = rw < N ? f[(size_t)rw * kLuSlots + 3 - t] : 0.0;
      g[(size_t)9 * N + c * 4 + t] = ru >= 0 ? f[(size_t)ru * kLuSlots + 9 + t] : 0.0;
    }
  for (int i = 0; i < N; ++i) g[(size_t)8 * N + i] = f[(size_t)i * kLuSlots + 8];
  std::copy(g.begin(), g.end(), f);
}

// Two-partition (SPIKE) form of an operator, for the latency-bound solves:
// rows split at k = N/2 into a top block T and a bottom block B, each
// factored on its own (13-slot rows, local indices), so the two halves are
// substituted at the same time.  The blocks couple only through the upper
// band of T's last four rows (columns k..k+3) and the lower band of B's first
// four rows (columns k-4..k-1):
//   x_T = y_T - S_T x_B[0:4],    S_T = T^{-1} H(0:k, k:k+4)      (k x 4)
//   x_B = y_B - S_B x_T[k-4:k],  S_B = B^{-1} H(k:N, k-4:k)  ((N-k) x 4)
// with y = the block solves of the right-hand side; the interface values
// z = (x_T[k-4:k], x_B[0:4]) solve G z = (y_T[k-4:k], y_B[0:4]),
// G = [I, S_T[k-4:k]; S_B[0:4], I], whose inverse R (8 x 8) is stored.
// out_lu: N rows of 13 slots (T's rows, then B's); out_spk: N rows of 4
// (S_T, then S_B); out_r: 64 (R row-major).  Checked against the unfactored
// matrix on a test right-hand side.
static bool inv_dense(int n, std::vector<double> a, std::vector<double>* out) {
  std::vector<double> x((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) x[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int i = c + 1; i < n; ++i)
      if (std::fabs(a[(size_t)i * n + c]) > std::fabs(a[(size_t)p * n + c])) p = i;
    if (a[(size_t)p * n + c] == 0.0) return false;
    for (int j = 0; j < n; ++j) {
      std::swap(a[(size_t)c * n + j], a[(size_t)p * n + j]);
      std::swap(x[(size_t)c * n + j], x[(size_t)p * n + j]);
    }
    const double inv = 1.0 / a[(size_t)c * n + c];
    for (int j = 0; j < n; ++j) {
      a[(size_t)c * n + j] *= inv;
      x[(size_t)c * n + j] *= inv;
    }
    for (int i = 0; i < n; ++i) {
      if (i == c) continue;
      const double f = a[(size_t)i * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        a[(size_t)i * n + j] -= f * a[(size_t)c * n + j];
        x[(size_t)i * n + j] -= f * x[(size_t)c * n + j];
      }
    }
  }
  *out = x;
  return true;
}

static bool factor_split(const Op& full, double* out_lu, double* out_spk, double* out_r, std::string* err,
                         const char* what) {
  const int N = full.N, k = N / 2, nb = N - k;
  Op top, bot;
  top.N = k;
  top.a.assign((size_t)k * k, 0.0);
  bot.N = nb;
  bot.a.assign((size_t)nb * nb, 0.0);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) top.at(i, j) = full.a[(size_t)i * N + j];
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j) bot.at(i, j) = full.a[(size_t)(k + i) * N + k + j];
  // the coupling must lie within the four columns / rows the device uses
  for (int i = 0; i < k; ++i)
    for (int j = k + 4; j < N; ++j)
      if (full.a[(size_t)i * N + j] != 0.0) {
        *err = std::string("split solve: upper coupling wider than 4 in ") + what;
        return false;
      }
  for (int i = k; i < N; ++i)
    for (int j = 0; j < k - 4; ++j)
      if (full.a[(size_t)i * N + j] != 0.0) {
        *err = std::string("split solve: lower coupling wider than 4 in ") + what;
        return false;
      }
  std::string e2;
  if (!factor(&top, out_lu, err, what) || !factor(&bot, out_lu + (size_t)k * kLuSlots, err, what)) return false;
  std::vector<double> v(N);
  for (int c = 0; c < 4; ++c) {
    for (int i = 0; i < k; ++i) v[i] = full.a[(size_t)i * N + k + c];
    lu_solve(out_lu, k, v.data());
    for (int i = 0; i < k; ++i) out_spk[(size_t)i * 4 + c] = v[i];
    for (int i = 0; i < nb; ++i) v[i] = full.a[(size_t)(k + i) * N + k - 4 + c];
    lu_solve(out_lu + (size_t)k * kLuSlots, nb, v.data());
    for (int i = 0; i < nb; ++i) out_spk[(size_t)(k + i) * 4 + c] = v[i];
  }
  std::vector<double> G(64, 0.0), R;
  for (int a = 0; a < 8; ++a) G[(size_t)a * 8 + a] = 1.0;
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 4; ++c) {
      G[(size_t)a * 8 + 4 + c] = out_spk[(size_t)(k - 4 + a) * 4 + c];  // S_T rows k-4..k-1
      G[(size_t)(4 + a) * 8 + c] = out_spk[(size_t)(k + a) * 4 + c];    // S_B rows 0..3
    }
  if (!inv_dense(8, G, &R)) {
    *err = std::string("split solve: singular interface in ") + what;
    return false;
  }
  std::copy(R.begin(), R.end(), out_r);
  // self-check of the whole split solve against the unfactored matrix
  std::vector<double> b(N), x(N), z(8);
  for (int i = 0; i < N; ++i) b[i] = std::cos(0.7 * i) + 0.3;
  x = b;
  lu_solve(out_lu, k, x.data());
  lu_solve(out_lu + (size_t)k * kLuSlots, nb, x.data() + k);
  double y[8];
  for (int a = 0; a < 4; ++a) y[a] = x[k - 4 + a], y[4 + a] = x[k + a];
  for (int a = 0; a < 8; ++a) {
    z[a] = 0.0;
    for (int c = 0; c < 8; ++c) z[a] += out_r[a * 8 + c] * y[c];
  }
  for (int i = 0; i < k; ++i)
    for (int c = 0; c < 4; ++c) x[i] -= out_spk[(size_t)i * 4 + c] * z[4 + c];
  for (int i = 0; i < nb; ++i)
    for (int c = 0; c < 4; ++c) x[k + i] -= out_spk[(size_t)(k + i) * 4 + c] * z[c];
  double res = 0.0, anorm = 0.0, xnorm = 0.0;
  for (int i = 0; i < N; ++i) {
    double acc = 0.0, rs = 0.0;
    for (int j = 0; j < N; ++j) {
      acc += full.a[(size_t)i * N + j] * x[j];
      rs += std::fabs(full.a[(size_t)i * N + j]);
    }
    res = std::max(res, std::fabs(acc - b[i]));
    anorm = std::max(anorm, rs);
    xnorm = std::max(xnorm, std::fabs(x[i]));
  }
  if (!(res <= 1e-12 * anorm * xnorm)) {
    char buf[200];
    std::snprintf(buf, sizeof buf, "split solve of %s inaccurate (residual %.3e)", what, res / (anorm * xnorm));
    *err = buf;
    return false;
  }
  return true;
}

// Banded LU solve with the 13-slot factor (same arithmetic as the device).

static void d1_apply(const Setup* s, int par, const double* v, double* out) {
  const int N = s->N;
  for (int n = 0; n < N; ++n) {
    const int lo = row_lo(N, n);
    double acc = 0.0;
    for (int t = 0; t < kStencil; ++t)
      if (lo + t < N) acc += s->d1[(par * N + n) * kStencil + t] * v[lo + t];
    out[n] = acc;
  }
}

// 4x4 complex inverse by Gauss-Jordan with partial pivoting.
static bool inv4(cplx A[4][4], cplx X[4][4]) {
  cplx a[4][8];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 8; ++j) a[i][j] = j < 4 ? A[i][j] : cplx(j - 4 == i ? 1.0 : 0.0, 0.0);
  for (int c = 0; c < 4; ++c) {
    int p = c;
    for (int i = c + 1; i < 4; ++i)
      if (std::abs(a[i][c]) > std::abs(a[p][c])) p = i;
    if (std::abs(a[p][c]) == 0.0) return false;
    for (int j = 0; j < 8; ++j) std::swap(a[c][j], a[p][j]);
    const cplx inv = 1.0 / a[c][c];
    for (int j = 0; j < 8; ++j) a[c][j] *= inv;
    for (int i = 0; i < 4; ++i) {
      if (i == c) continue;
      const cplx f = a[i][c];
      for (int j = 0; j < 8; ++j) a[i][j] -= f * a[c][j];
    }
  }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) X[i][j] = a[i][j + 4];
  return true;
}

bool build_setup(Setup* s, std::string* err) {
  const int N = s->N, K = s->K, M = s->M, mp = s->m_p;
  const int nk = 2 * K - 1;
  s->r.resize(N);
  s->rinv.resize(N);
  if (!s->r_user.empty()) {  // section 2: the points may also come from the user
    if ((int)s->r_user.size() != N) {
      *err = "user mesh: need N points";
      return false;
    }
    for (int n = 0; n < N; ++n) {
      const double x = s->r_user[n];
      if (!(x > 0.0 && x <= 1.0) || (n > 0 && !(x > s->r_user[n - 1]))) {
        *err = "user mesh: points must increase strictly within (0, 1]";
        return false;
      }
    }
    if (s->r_user[N - 1] != 1.0) {
      *err = "user mesh: the last point must be the wall r = 1";
      return false;
    }
    for (int n = 0; n < N; ++n) {
      s->r[n] = s->r_user[n];
      s->rinv[n] = 1.0 / s->r[n];
    }
  } else {
    for (int n = 0; n < N; ++n) {  // section 2: points bunched towards the wall
      s->r[n] = std::cos(M_PI * (double)(N - 1 - n) / (2.0 * N - 1.0));
      s->rinv[n] = 1.0 / s->r[n];
    }
    s->r[N - 1] = 1.0;
    s->rinv[N - 1] = 1.0;
  }
  build_stencils(s);
  build_quadrature(s);

  // Helmholtz operators exist per (|k|, |j|), |j| in {|m~-1|, m~, m~+1}.
  const int jmax = mp * (M - 1) + 1;
  s->jidx.assign(jmax + 1, -1);
  s->hop.assign(3 * M, 0);
  for (int m = 0; m < M; ++m) {
    const int mt = mp * m;
    const int js[3] = {mt + 1, std::abs(mt - 1), mt};
    for (int f = 0; f < 3; ++f) s->jidx[js[f]] = 0;
  }
  s->nJ = 0;
  for (int j = 0; j <= jmax; ++j)
    if (s->jidx[j] == 0) s->jidx[j] = s->nJ++;
    else s->jidx[j] = -1;
  for (int m = 0; m < M; ++m) {
    const int mt = mp * m;
    s->hop[3 * m + 0] = s->jidx[mt + 1];
    s->hop[3 * m + 1] = s->jidx[std::abs(mt - 1)];
    s->hop[3 * m + 2] = s->jidx[mt];
  }
  std::vector<int> jval(s->nJ);
  for (int j = 0; j <= jmax; ++j)
    if (s->jidx[j] >= 0) jval[s->jidx[j]] = j;

  const double nu = 1.0 / s->Re, c = s->c, idt = 1.0 / s->dt;
  const size_t opsz = (size_t)N * kLuSlots;
  s->luH.assign((size_t)K * s->nJ * opsz, 0.0);
  s->luP.assign((size_t)(K * M + 1) * opsz, 0.0);
  if (s->spike && (N % 2 || N < 26)) {
    *err = "split solve needs an even N >= 26";
    return false;
  }
  const size_t nH = s->spike ? (size_t)K * s->nJ : 0, nP = s->spike ? (size_t)(K * M + 1) : 0;
  s->luH2.assign(nH * opsz, 0.0);
  s->luP2.assign(nP * opsz, 0.0);
  s->spkH.assign(nH * N * 4, 0.0);
  s->spkP.assign(nP * N * 4, 0.0);
  s->rH.assign(nH * 64, 0.0);
  s->rP.assign(nP * 64, 0.0);
  Op op;
  std::vector<double> diag(N);
  char what[96];
  for (int ik = 0; ik < K; ++ik) {
    const double ak2 = std::pow(s->alpha * ik, 2);
    for (int q = 0; q < s->nJ; ++q) {  // H_j = 1/dt - c nu (D2 + D1/r - j^2/r^2 - ak^2)
      const int j = jval[q];
      for (int n = 0; n < N; ++n) diag[n] = idt + c * nu * (j * j * s->rinv[n] * s->rinv[n] + ak2);
      assemble(s, j & 1, -c * nu, diag, &op);
      wall_dirichlet(&op);
      std::snprintf(what, sizeof what, "Helmholtz |k|=%d |j|=%d", ik, j);
      const size_t o = (size_t)ik * s->nJ + q;
      if (s->spike && !factor_split(op, &s->luH2[o * opsz], &s->spkH[o * N * 4], &s->rH[o * 64], err, what))
        return false;
      if (!factor(&op, &s->luH[o * opsz], err, what)) return false;
    }
    for (int m = 0; m < M; ++m) {  // P = D2 + D1/r - m~^2/r^2 - ak^2, Neumann wall row
      const int mt = mp * m;
      for (int n = 0; n < N; ++n) diag[n] = -(mt * mt * s->rinv[n] * s->rinv[n] + ak2);
      assemble(s, mt & 1, 1.0, diag, &op);
      if (ik == 0 && m == 0) {  // pure Neumann is singular here: gauge p(1) = 0
        wall_dirichlet(&op);
        const size_t o = (size_t)K * M;
        if (s->spike &&
            !factor_split(op, &s->luP2[o * opsz], &s->spkP[o * N * 4], &s->rP[o * 64], err, "Poisson (0,0)"))
          return false;
        if (!factor(&op, &s->luP[o * opsz], err, "Poisson (0,0)")) return false;
        continue;
      }
      wall_neumann(s, mt & 1, &op);
      std::snprintf(what, sizeof what, "Poisson |k|=%d m=%d", ik, m);
      const size_t o = (size_t)ik * M + m;
      if (s->spike && !factor_split(op, &s->luP2[o * opsz], &s->spkP[o * N * 4], &s->rP[o * 64], err, what))
        return false;
      if (!factor(&op, &s->luP[o * opsz], err, what)) return false;
    }
  }

  // Influence-matrix responses per (|k|, m) and inverse 4x4 matrices per (k, m).
  s->basis.assign((size_t)K * M * 6 * N, 0.0);
  s->ainv.assign((size_t)M * nk * 32, 0.0);
  std::vector<double> p1(N), dp(N), v(N);
  for (int ik = 0; ik < K; ++ik) {
    for (int m = 0; m < M; ++m) {
      if (ik == 0 && m == 0) continue;
      const int mt = mp * m;
      const int ps = mt & 1;
      const double ak = s->alpha * ik;
      double* B = &s->basis[(((size_t)ik * M + m) * 6) * N];
      const double* Pf = &s->luP[((size_t)ik * M + m) * opsz];
      const double* Hp = &s->luH[((size_t)ik * s->nJ + s->hop[3 * m + 0]) * opsz];
      const double* Hm = &s->luH[((size_t)ik * s->nJ + s->hop[3 * m + 1]) * opsz];
      const double* Hz = &s->luH[((size_t)ik * s->nJ + s->hop[3 * m + 2]) * opsz];
      std::fill(p1.begin(), p1.end(), 0.0);
      p1[N - 1] = 1.0;  // unit wall derivative of p, lap p = 0 inside
      lu_solve(Pf, N, p1.data());
      d1_apply(s, ps, p1.data(), dp.data());
      for (int n = 0; n < N; ++n) B[0 * N + n] = -(dp[n] - mt * s->rinv[n] * p1[n]);
      for (int n = 0; n < N; ++n) B[1 * N + n] = -(dp[n] + mt * s->rinv[n] * p1[n]);
      for (int n = 0; n < N; ++n) B[2 * N + n] = -ak * p1[n];  // u_z response = i * this (k > 0)
      B[0 * N + N - 1] = B[1 * N + N - 1] = B[2 * N + N - 1] = 0.0;
      lu_solve(Hp, N, B + 0 * N);
      lu_solve(Hm, N, B + 1 * N);
      lu_solve(Hz, N, B + 2 * N);
      for (int f = 0; f < 3; ++f) {
        double* e = B + (3 + f) * N;
        std::fill(e, e + N, 0.0);
        e[N - 1] = 1.0;
        lu_solve(f == 0 ? Hp : (f == 1 ? Hm : Hz), N, e);
      }
      const double* w = &s->d1[((ps ^ 1) * N + N - 1) * kStencil];
      const int lo = row_lo(N, N - 1);
      for (int sgn = -1; sgn <= 1; sgn += 2) {
        if (ik == 0 && sgn < 0) continue;
        const int k = sgn * ik;
        const int kk = k + K - 1;
        const double akk = s->alpha * k;
        // g(u) = (u+(1), u-(1), u_z(1), div u(1)), div in +- form
        auto g4 = [&](const cplx* up, const cplx* um, cplx uz_wall) {
          cplx acc = 0.0;
          for (int t = 0; t < kStencil; ++t) acc += w[t] * (up[lo + t] + um[lo + t]);
          return 0.5 * acc +
                 0.5 * ((1.0 + mt) * up[N - 1] + (1.0 - mt) * um[N - 1]) * s->rinv[N - 1] +
                 cplx(0, akk) * uz_wall;
        };
        std::vector<cplx> up(N), um(N), zero(N, 0.0);
        cplx A[4][4], X[4][4];
        for (int n = 0; n < N; ++n) {
          up[n] = B[0 * N + n];
          um[n] = B[1 * N + n];
        }
        const cplx uz1 = cplx(0, (double)sgn) * B[2 * N + N - 1];
        A[0][0] = up[N - 1];
        A[1][0] = um[N - 1];
        A[2][0] = uz1;
        A[3][0] = g4(up.data(), um.data(), uz1);
        for (int n = 0; n < N; ++n) up[n] = B[3 * N + n];
        A[0][1] = up[N - 1];
        A[1][1] = 0.0;
        A[2][1] = 0.0;
        A[3][1] = g4(up.data(), zero.data(), 0.0);
        for (int n = 0; n < N; ++n) um[n] = B[4 * N + n];
        A[0][2] = 0.0;
        A[1][2] = um[N - 1];
        A[2][2] = 0.0;
        A[3][2] = g4(zero.data(), um.data(), 0.0);
        A[0][3] = 0.0;
        A[1][3] = 0.0;
        A[2][3] = B[5 * N + N - 1];
        A[3][3] = g4(zero.data(), zero.data(), B[5 * N + N - 1]);
        if (!inv4(A, X)) {
          char buf[96];
          std::snprintf(buf, sizeof buf, "singular influence matrix at k=%d m=%d", k, m);
          *err = buf;
          return false;
        }
        double* o = &s->ainv[((size_t)m * nk + kk) * 32];
        for (int i = 0; i < 4; ++i)
          for (int j = 0; j < 4; ++j) {
            o[(i * 4 + j) * 2 + 0] = X[i][j].real();
            o[(i * 4 + j) * 2 + 1] = X[i][j].imag();
          }
      }
    }
  }

  // Fixed flux: response G of the (0,0) axial mode to a unit uniform forcing.
  s->G.assign(N, 1.0);
  s->G[N - 1] = 0.0;
  lu_solve(&s->luH[((size_t)0 * s->nJ + s->hop[2]) * opsz], N, s->G.data());
  double fg = 0.0;
  for (int n = 0; n < N; ++n) fg += s->wq[n] * s->G[n];
  s->flux_G = fg;
  // the factors in the order the device reads them (the split forms: each
  // half as an operator of its own size)
  for (size_t o = 0; o * opsz < s->luH.size(); ++o) to_columns(&s->luH[o * opsz], N);
  for (size_t o = 0; o * opsz < s->luP.size(); ++o) to_columns(&s->luP[o * opsz], N);
  const int kh = N / 2;
  for (std::vector<double>* v : {&s->luH2, &s->luP2})
    for (size_t o = 0; o * opsz < v->size(); ++o) {
      to_columns(&(*v)[o * opsz], kh);
      to_columns(&(*v)[o * opsz + (size_t)kh * kLuSlots], N - kh);
    }
  return true;
}

}  // namespace opf

// ---- resolution change (the paper: initial conditions of another resolution
// are truncated or interpolated automatically).  Fourier modes: copied where
// both resolutions have them, zero otherwise.  Radial profiles: the 9-point
// Lagrange interpolant through the source mesh extended to negative r by the
// field's axis parity ((-1)^(m_p m) for u_z, (-1)^(m_p m + 1) for u_r and
// u_theta), nodes nearest the target point, shifted inward at the ends.
extern "C" int opf_change_resolution(int N1, int K1, int M1, const double* in, int N2, int K2, int M2, int m_p,
                                     double* out) {
  if (N1 < 9 || N2 < 1 || K1 < 1 || K2 < 1 || M1 < 1 || M2 < 1 || m_p < 1 || !in || !out) {
    opf::set_last_error("opf_change_resolution: sizes must be positive and the source N >= 9");
    return OPF_EINVAL;
  }
  auto mesh = [](int N) {
    std::vector<double> r(N);
    for (int n = 0; n < N; ++n) r[n] = std::cos(M_PI * (double)(N - 1 - n) / (2.0 * N - 1.0));
    return r;
  };
  const std::vector<double> r1 = mesh(N1), r2 = mesh(N2);
  // extended source nodes: e < N1 -> -r1[N1-1-e] (ghost), else r1[e-N1]
  auto ext_x = [&](int e) { return e < N1 ? -r1[N1 - 1 - e] : r1[e - N1]; };
  std::vector<int> first(N2);
  std::vector<double> w((size_t)N2 * 9);
  for (int n = 0; n < N2; ++n) {
    const double z = r2[n];
    int q = N1;  // nearest extended node
    for (int e = 0; e < 2 * N1; ++e)
      if (std::fabs(ext_x(e) - z) < std::fabs(ext_x(q) - z)) q = e;
    const int f = std::min(std::max(q - 4, 0), 2 * N1 - 9);
    first[n] = f;
    double x[9], c[9];
    for (int t = 0; t < 9; ++t) x[t] = ext_x(f + t);
    opf::fornberg(z, x, 9, 0, c);
    for (int t = 0; t < 9; ++t) w[(size_t)n * 9 + t] = c[t];
    if (ext_x(q) == z)  // a target on a source node takes its value exactly
      for (int t = 0; t < 9; ++t) w[(size_t)n * 9 + t] = (f + t == q) ? 1.0 : 0.0;
  }
  const int nk1 = 2 * K1 - 1, nk2 = 2 * K2 - 1;
  for (int c = 0; c < 3; ++c)
    for (int m = 0; m < M2; ++m)
      for (int kk2 = 0; kk2 < nk2; ++kk2) {
        const int k = kk2 - (K2 - 1), kk1 = k + (K1 - 1);
        double* o = out + 2 * ((((size_t)c * M2 + m) * nk2 + kk2) * N2);
        if (m >= M1 || kk1 < 0 || kk1 >= nk1) {
          for (int n = 0; n < 2 * N2; ++n) o[n] = 0.0;
          continue;
        }
        const double* s = in + 2 * ((((size_t)c * M1 + m) * nk1 + kk1) * N1);
        const int mt = m_p * m;
        const double par = ((c == 2 ? mt : mt + 1) % 2 == 0) ? 1.0 : -1.0;
        for (int n = 0; n < N2; ++n) {
          double re = 0.0, im = 0.0;
          for (int t = 0; t < 9; ++t) {
            const int e = first[n] + t;
            const int col = e < N1 ? N1 - 1 - e : e - N1;
            const double sg = e < N1 ? par : 1.0;
            re += w[(size_t)n * 9 + t] * sg * s[2 * col];
            im += w[(size_t)n * 9 + t] * sg * s[2 * col + 1];
          }
          o[2 * n] = re;
          o[2 * n + 1] = im;
        }
      }
  return OPF_OK;
}
