// Newton-Krylov-trust-region ("hookstep") solver for F(x) = 0 (paper
// section 2: the Newton utility calls a combined Krylov / trust-region method
// for invariant solutions).  count independent problems of size n advance in
// lockstep so that each Jacobian-vector product of all of them is one
// batched call (for the pipe flow: one batched GPU time integration).
//
// Per Newton iteration and problem:
//   * GMRES (Arnoldi with modified Gram-Schmidt, applied twice, FP64) builds
//     V_{k+1}, H (k+1 x k) with J V_k = V_{k+1} H, v_1 = F / |F|;
//   * hookstep: with H = U S W^T (thin SVD, one-sided Jacobi) and
//     p = U^T (|F| e_1), minimise |p + S z| subject to |z| <= Delta:
//     z_i = -p_i s_i / (s_i^2 + mu), mu >= 0 the smallest value meeting the
//     radius; the step is dx = V_k W z;
//   * the trial F(x + dx) is accepted when the actual reduction of |F|^2 is
//     at least 1 % of the predicted one; Delta halves on rejection and
//     doubles after a good step that hit the radius.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "opf_internal.h"

namespace {

double dot(const double* a, const double* b, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

// One-sided Jacobi SVD of the m x k matrix A (column-major, m >= k):
// A = U diag(s) W^T with U m x k (columns orthonormal), W k x k orthogonal.
void jacobi_svd(int m, int k, const std::vector<double>& A, std::vector<double>& U,
                std::vector<double>& s, std::vector<double>& W) {
  U = A;
  W.assign((size_t)k * k, 0.0);
  for (int i = 0; i < k; ++i) W[(size_t)i * k + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < k - 1; ++p)
      for (int q = p + 1; q < k; ++q) {
        double* up = &U[(size_t)p * m];
        double* uq = &U[(size_t)q * m];
        const double a = dot(up, up, m), b = dot(uq, uq, m), c = dot(up, uq, m);
        if (std::fabs(c) <= 1e-15 * std::sqrt(a * b) || c == 0.0) continue;
        off = std::max(off, std::fabs(c) / std::sqrt(a * b));
        const double zeta = (b - a) / (2.0 * c);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = cs * t;
        for (int i = 0; i < m; ++i) {
          const double x = up[i], y = uq[i];
          up[i] = cs * x - sn * y;
          uq[i] = sn * x + cs * y;
        }
        double* wp = &W[(size_t)p * k];
        double* wq = &W[(size_t)q * k];
        for (int i = 0; i < k; ++i) {
          const double x = wp[i], y = wq[i];
          wp[i] = cs * x - sn * y;
          wq[i] = sn * x + cs * y;
        }
      }
    if (off < 1e-15) break;
  }
  s.assign(k, 0.0);
  for (int j = 0; j < k; ++j) {
    double* u = &U[(size_t)j * m];
    s[j] = std::sqrt(dot(u, u, m));
    if (s[j] > 0)
      for (int i = 0; i < m; ++i) u[i] /= s[j];
  }
}

struct Problem {
  std::vector<double> x, f;  // current point and residual
  double fnorm = 0.0, delta = 0.0;
  bool done = false;
  int iters = 0;
  // Krylov data of the current Newton iteration
  std::vector<std::vector<double>> V;
  std::vector<double> H;  // (kmax + 1) x kmax, column-major
  int k = 0;
  bool krylov_done = false;
  double beta = 0.0;
  // hookstep data
  std::vector<double> U, s, W, p;
  double rperp2 = 0.0;
};

// least-squares residual of min |beta e1 + H y| over the first k columns
double lsq_residual(const Problem& P, int k, int ld) {
  std::vector<double> A((size_t)(k + 1) * k);
  for (int j = 0; j < k; ++j)
    for (int i = 0; i <= k; ++i) A[(size_t)j * (k + 1) + i] = P.H[(size_t)j * ld + i];
  std::vector<double> U, s, W;
  jacobi_svd(k + 1, k, A, U, s, W);
  double pp = 0.0;
  for (int j = 0; j < k; ++j) {
    const double pj = P.beta * U[(size_t)j * (k + 1)];
    pp += pj * pj;
  }
  return std::sqrt(std::max(0.0, P.beta * P.beta - pp));
}

// z(mu) and its norm for the hookstep
double hook_norm(const Problem& P, double mu, std::vector<double>* z) {
  double n2 = 0.0;
  for (size_t i = 0; i < P.s.size(); ++i) {
    const double zi = P.s[i] > 0 ? -P.p[i] * P.s[i] / (P.s[i] * P.s[i] + mu) : 0.0;
    if (z) (*z)[i] = zi;
    n2 += zi * zi;
  }
  return std::sqrt(n2);
}

}  // namespace

extern "C" int opf_nk_core(int n, int count, double* x, const double* scale, opf_nk_residual F,
                           opf_nk_jv JV, void* ctx, const opf_nk_opts* o, double* res_out,
                           int* iters_out) {
  if (n < 1 || count < 1 || !x || !F || !JV || !o) return OPF_EINVAL;
  const int kmax = std::max(1, o->max_krylov);
  std::vector<Problem> P(count);
  std::vector<double*> xp(count), fp(count), vp(count), jp(count);
  std::vector<std::vector<double>> tmpx(count, std::vector<double>(n)), tmpf(count, std::vector<double>(n));
  for (int i = 0; i < count; ++i) {
    P[i].x.assign(x + (size_t)i * n, x + (size_t)(i + 1) * n);
    P[i].f.assign(n, 0.0);
    xp[i] = P[i].x.data();
    fp[i] = P[i].f.data();
  }
  std::vector<int> all(count);
  for (int i = 0; i < count; ++i) all[i] = i;
  int rc = F(ctx, count, all.data(), xp.data(), fp.data(), 1);
  if (rc) return rc;
  for (int i = 0; i < count; ++i) {
    P[i].fnorm = std::sqrt(dot(P[i].f.data(), P[i].f.data(), n));
    const double xn = std::sqrt(dot(P[i].x.data(), P[i].x.data(), n));
    P[i].delta = o->delta0 > 0 ? o->delta0 : 0.1 * std::max(xn, 1e-12);
  }
  for (int it = 0; it < o->max_newton; ++it) {
    int active = 0;
    for (int i = 0; i < count; ++i) {
      P[i].done = P[i].done || P[i].fnorm <= o->tol * (scale ? scale[i] : 1.0);
      if (!P[i].done) ++active;
    }
    if (!active) break;
    // ---- GMRES (lockstep Arnoldi)
    for (int i = 0; i < count; ++i) {
      Problem& Q = P[i];
      Q.k = 0;
      Q.krylov_done = Q.done;
      Q.beta = Q.fnorm;
      Q.V.assign(1, std::vector<double>(n));
      Q.H.assign((size_t)(kmax + 1) * kmax, 0.0);
      if (!Q.done)
        for (int j = 0; j < n; ++j) Q.V[0][j] = Q.f[j] / Q.beta;
    }
    for (int j = 0; j < kmax; ++j) {
      std::vector<int> who;
      for (int i = 0; i < count; ++i)
        if (!P[i].krylov_done) who.push_back(i);
      if (who.empty()) break;
      std::vector<double*> xs, vs, js;
      for (int i : who) {
        xs.push_back(P[i].x.data());
        vs.push_back(P[i].V[j].data());
        js.push_back(tmpf[i].data());
      }
      rc = JV(ctx, (int)who.size(), who.data(), xs.data(), vs.data(), js.data());
      if (rc) return rc;
      for (int i : who) {
        Problem& Q = P[i];
        std::vector<double>& w = tmpf[i];
        for (int pass = 0; pass < 2; ++pass)  // modified Gram-Schmidt, twice
          for (int l = 0; l <= j; ++l) {
            const double h = dot(w.data(), Q.V[l].data(), n);
            Q.H[(size_t)j * (kmax + 1) + l] += h;
            for (int t = 0; t < n; ++t) w[t] -= h * Q.V[l][t];
          }
        const double hn = std::sqrt(dot(w.data(), w.data(), n));
        Q.H[(size_t)j * (kmax + 1) + j + 1] = hn;
        Q.k = j + 1;
        Q.V.emplace_back(n);
        if (hn > 0)
          for (int t = 0; t < n; ++t) Q.V[j + 1][t] = w[t] / hn;
        const double r = lsq_residual(Q, Q.k, kmax + 1);
        if (r <= o->gmres_tol * Q.beta || hn <= 1e-14 * Q.beta) Q.krylov_done = true;
      }
    }
    // ---- SVD of each Hessenberg
    for (int i = 0; i < count; ++i) {
      Problem& Q = P[i];
      if (Q.done) continue;
      const int k = Q.k, m = k + 1;
      std::vector<double> A((size_t)m * k);
      for (int j = 0; j < k; ++j)
        for (int r = 0; r < m; ++r) A[(size_t)j * m + r] = Q.H[(size_t)j * (kmax + 1) + r];
      jacobi_svd(m, k, A, Q.U, Q.s, Q.W);
      Q.p.assign(k, 0.0);
      double pp = 0.0;
      for (int j = 0; j < k; ++j) {
        Q.p[j] = Q.beta * Q.U[(size_t)j * m];  // U^T (beta e1)
        pp += Q.p[j] * Q.p[j];
      }
      Q.rperp2 = std::max(0.0, Q.beta * Q.beta - pp);
    }
    // ---- hooksteps with trust-region acceptance (lockstep trials)
    std::vector<char> settled(count, 0);
    std::vector<double> pred(count, 0.0);
    for (int trial = 0; trial < o->max_hook; ++trial) {
      std::vector<int> who;
      for (int i = 0; i < count; ++i) {
        Problem& Q = P[i];
        if (Q.done || settled[i]) continue;
        const int k = Q.k;
        std::vector<double> z(k);
        double nz = hook_norm(Q, 0.0, &z);
        if (nz > Q.delta) {  // smallest mu with |z(mu)| = delta (bisection on log mu)
          double lo = 0.0, hi = 1.0;
          while (hook_norm(Q, hi, nullptr) > Q.delta) hi *= 4.0;
          for (int b = 0; b < 100; ++b) {
            const double mid = 0.5 * (lo + hi);
            if (hook_norm(Q, mid, nullptr) > Q.delta) lo = mid;
            else hi = mid;
          }
          nz = hook_norm(Q, hi, &z);
        }
        // predicted residual |p + S z|^2 + rperp^2
        double r2 = Q.rperp2;
        for (int j = 0; j < k; ++j) {
          const double e = Q.p[j] + Q.s[j] * z[j];
          r2 += e * e;
        }
        pred[i] = r2;
        // dx = V_k W z
        std::vector<double> y(k, 0.0);
        for (int a = 0; a < k; ++a)
          for (int b = 0; b < k; ++b) y[a] += Q.W[(size_t)b * k + a] * z[b];
        std::vector<double>& xt = tmpx[i];
        xt = Q.x;
        for (int a = 0; a < k; ++a)
          for (int t = 0; t < n; ++t) xt[t] += y[a] * Q.V[a][t];
        who.push_back(i);
      }
      if (who.empty()) break;
      std::vector<double*> xs, fs;
      for (int i : who) {
        xs.push_back(tmpx[i].data());
        fs.push_back(tmpf[i].data());
      }
      rc = F(ctx, (int)who.size(), who.data(), xs.data(), fs.data(), 0);
      if (rc) return rc;
      for (size_t w = 0; w < who.size(); ++w) {
        const int i = who[w];
        Problem& Q = P[i];
        const double fn = std::sqrt(dot(tmpf[i].data(), tmpf[i].data(), n));
        const double actual = Q.fnorm * Q.fnorm - fn * fn;
        const double predicted = Q.fnorm * Q.fnorm - pred[i];
        const double rho = predicted > 0 ? actual / predicted : -1.0;
        if (std::isfinite(fn) && rho >= 0.01) {
          double step2 = 0.0;
          for (int t = 0; t < n; ++t) step2 += (tmpx[i][t] - Q.x[t]) * (tmpx[i][t] - Q.x[t]);
          Q.x = tmpx[i];
          Q.f = tmpf[i];
          Q.fnorm = fn;
          if (rho > 0.75 && std::sqrt(step2) >= 0.99 * Q.delta) Q.delta *= 2.0;
          settled[i] = 1;
          ++Q.iters;
        } else {
          Q.delta *= 0.5;
        }
      }
    }
    // the accepted points are the new Newton points: refresh their cached data
    std::vector<double*> xs, fs;
    std::vector<int> who;
    for (int i = 0; i < count; ++i)
      if (settled[i]) {
        who.push_back(i);
        xs.push_back(P[i].x.data());
        fs.push_back(P[i].f.data());
      }
    if (!xs.empty()) {
      rc = F(ctx, (int)xs.size(), who.data(), xs.data(), fs.data(), 1);
      if (rc) return rc;
    }
    for (int i = 0; i < count; ++i)
      if (settled[i]) P[i].fnorm = std::sqrt(dot(P[i].f.data(), P[i].f.data(), n));
    bool any_progress = false;
    for (int i = 0; i < count; ++i) any_progress = any_progress || settled[i] || P[i].done;
    if (!any_progress) break;
  }
  for (int i = 0; i < count; ++i) {
    std::memcpy(x + (size_t)i * n, P[i].x.data(), (size_t)n * sizeof(double));
    if (res_out) res_out[i] = P[i].fnorm / (scale ? scale[i] : 1.0);
    if (iters_out) iters_out[i] = P[i].iters;
  }
  return OPF_OK;
}
