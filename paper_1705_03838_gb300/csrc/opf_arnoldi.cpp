// Arnoldi iteration for the leading eigenvalues of linear maps (the stability
// of invariant solutions: the paper's Newton utility finds travelling waves
// and periodic orbits, and section 3.2 reports the leading eigenvalue of one).
//
// count independent maps of size n advance in lockstep, so each Krylov step
// applies all of them in one call (for the pipe flow: one batched time
// integration).  Orthogonalisation: modified Gram-Schmidt applied twice, FP64.
// Ritz values: eigenvalues of the k x k upper Hessenberg matrix by the
// implicit double-shift (Francis) QR iteration of Golub & Van Loan (Matrix
// Computations, section 7.5); residual estimates |h_{k+1,k}| |e_k^T y| with y
// the unit eigenvector of H, found by inverse iteration in complex arithmetic.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "opf_internal.h"

namespace {

using cplx = std::complex<double>;

double dot(const double* a, const double* b, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

// Householder vector v (v[0] = 1) and beta with (I - beta v v^T) x = -+|x| e_1
void house(const double* x, int m, double* v, double* beta) {
  double sigma = 0.0;
  for (int i = 1; i < m; ++i) sigma += x[i] * x[i];
  v[0] = 1.0;
  for (int i = 1; i < m; ++i) v[i] = x[i];
  if (sigma == 0.0) {
    *beta = 0.0;
    return;
  }
  const double mu = std::sqrt(x[0] * x[0] + sigma);
  const double v0 = x[0] <= 0.0 ? x[0] - mu : -sigma / (x[0] + mu);
  *beta = 2.0 * v0 * v0 / (sigma + v0 * v0);
  for (int i = 1; i < m; ++i) v[i] /= v0;
}

// Eigenvalues of the real upper Hessenberg matrix H (k x k, row-major,
// overwritten).  Returns false if the iteration does not converge.
bool hessenberg_eigenvalues(std::vector<double>& H, int k, std::vector<cplx>& ev) {
  auto h = [&](int i, int j) -> double& { return H[(size_t)i * k + j]; };
  ev.clear();
  double norm = 0.0;
  for (int i = 0; i < k; ++i)
    for (int j = std::max(0, i - 1); j < k; ++j) norm = std::max(norm, std::fabs(h(i, j)));
  const double eps = 2.220446049250313e-16;
  int hi = k - 1, iter = 0, total = 0;
  while (hi >= 0) {
    // lowest row lo of the unreduced block ending at hi
    int lo = hi;
    while (lo > 0) {
      const double s = std::fabs(h(lo - 1, lo - 1)) + std::fabs(h(lo, lo));
      if (std::fabs(h(lo, lo - 1)) <= eps * (s > 0.0 ? s : norm)) {
        h(lo, lo - 1) = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {  // 1 x 1 block
      ev.push_back(cplx(h(hi, hi), 0.0));
      --hi;
      iter = 0;
      continue;
    }
    if (lo == hi - 1) {  // 2 x 2 block
      const double a = h(hi - 1, hi - 1), b = h(hi - 1, hi), c = h(hi, hi - 1), d = h(hi, hi);
      const double p = 0.5 * (a - d), disc = p * p + b * c, mid = 0.5 * (a + d);
      if (disc >= 0.0) {  // real pair mid +- r: the larger in modulus first, the other from the determinant
        const double r = std::sqrt(disc), big = mid + (mid >= 0.0 ? r : -r);
        const double det = a * d - b * c;
        ev.push_back(cplx(big, 0.0));
        ev.push_back(cplx(big != 0.0 ? det / big : 0.0, 0.0));
      } else {
        const double r = std::sqrt(-disc);
        ev.push_back(cplx(mid, r));
        ev.push_back(cplx(mid, -r));
      }
      hi -= 2;
      iter = 0;
      continue;
    }
    if (++total > 100 * k) return false;
    // Francis double-shift step on rows/columns lo..hi
    double s, t;
    if (++iter % 11 == 10) {  // exceptional shift after a run without deflation
      const double w = std::fabs(h(hi, hi - 1)) + std::fabs(h(hi - 1, hi - 2));
      s = 1.5 * w;
      t = w * w;
    } else {
      s = h(hi - 1, hi - 1) + h(hi, hi);
      t = h(hi - 1, hi - 1) * h(hi, hi) - h(hi - 1, hi) * h(hi, hi - 1);
    }
    double x = h(lo, lo) * h(lo, lo) + h(lo, lo + 1) * h(lo + 1, lo) - s * h(lo, lo) + t;
    double y = h(lo + 1, lo) * (h(lo, lo) + h(lo + 1, lo + 1) - s);
    double z = h(lo + 1, lo) * h(lo + 2, lo + 1);
    for (int q = lo; q <= hi - 2; ++q) {
      double v[3], beta;
      const double xv[3] = {x, y, z};
      house(xv, 3, v, &beta);
      const int c0 = std::max(lo, q - 1);
      for (int j = c0; j < k; ++j) {  // rows q..q+2 from the left
        const double w = beta * (v[0] * h(q, j) + v[1] * h(q + 1, j) + v[2] * h(q + 2, j));
        h(q, j) -= w * v[0];
        h(q + 1, j) -= w * v[1];
        h(q + 2, j) -= w * v[2];
      }
      const int r1 = std::min(q + 3, hi);
      for (int i = 0; i <= r1; ++i) {  // columns q..q+2 from the right
        const double w = beta * (h(i, q) * v[0] + h(i, q + 1) * v[1] + h(i, q + 2) * v[2]);
        h(i, q) -= w * v[0];
        h(i, q + 1) -= w * v[1];
        h(i, q + 2) -= w * v[2];
      }
      x = h(q + 1, q);
      y = h(q + 2, q);
      if (q < hi - 2) z = h(q + 3, q);
    }
    double v[2], beta;
    const double xv[2] = {x, y};
    house(xv, 2, v, &beta);
    for (int j = std::max(lo, hi - 2); j < k; ++j) {
      const double w = beta * (v[0] * h(hi - 1, j) + v[1] * h(hi, j));
      h(hi - 1, j) -= w * v[0];
      h(hi, j) -= w * v[1];
    }
    for (int i = 0; i <= hi; ++i) {
      const double w = beta * (h(i, hi - 1) * v[0] + h(i, hi) * v[1]);
      h(i, hi - 1) -= w * v[0];
      h(i, hi) -= w * v[1];
    }
    // the step keeps H Hessenberg: clear round-off below the subdiagonal
    for (int i = lo + 2; i <= hi; ++i)
      for (int j = lo; j < i - 1; ++j) h(i, j) = 0.0;
  }
  return true;
}

// |e_{k-1}^T y| for the unit solution of (H - theta I) y = y0 by two steps of
// inverse iteration (complex Gaussian elimination with partial pivoting)
double ritz_tail(const std::vector<double>& H, int k, cplx theta) {
  std::vector<cplx> y(k, cplx(1.0, 0.0));
  const double shift_eps = 1e-14 * (1.0 + std::abs(theta));
  for (int rep = 0; rep < 2; ++rep) {
    std::vector<cplx> A((size_t)k * k);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) A[(size_t)i * k + j] = cplx(H[(size_t)i * k + j], 0.0);
    for (int i = 0; i < k; ++i) A[(size_t)i * k + i] -= theta + cplx(shift_eps, 0.0);
    std::vector<cplx> b = y;
    for (int c = 0; c < k; ++c) {
      int p = c;
      for (int i = c + 1; i < k; ++i)
        if (std::abs(A[(size_t)i * k + c]) > std::abs(A[(size_t)p * k + c])) p = i;
      if (p != c) {
        for (int j = 0; j < k; ++j) std::swap(A[(size_t)p * k + j], A[(size_t)c * k + j]);
        std::swap(b[p], b[c]);
      }
      const cplx piv = A[(size_t)c * k + c];
      if (std::abs(piv) == 0.0) continue;
      for (int i = c + 1; i < k; ++i) {
        const cplx f = A[(size_t)i * k + c] / piv;
        if (f == cplx(0.0, 0.0)) continue;
        for (int j = c; j < k; ++j) A[(size_t)i * k + j] -= f * A[(size_t)c * k + j];
        b[i] -= f * b[c];
      }
    }
    for (int i = k - 1; i >= 0; --i) {
      cplx acc = b[i];
      for (int j = i + 1; j < k; ++j) acc -= A[(size_t)i * k + j] * y[j];
      const cplx d = A[(size_t)i * k + i];
      y[i] = std::abs(d) > 0.0 ? acc / d : acc / cplx(shift_eps, 0.0);
    }
    double nrm = 0.0;
    for (const cplx& v : y) nrm += std::norm(v);
    nrm = std::sqrt(nrm);
    if (nrm == 0.0 || !std::isfinite(nrm)) return 1.0;
    for (cplx& v : y) v /= nrm;
  }
  return std::abs(y[k - 1]);
}

}  // namespace

extern "C" int opf_arnoldi_core(int n, int count, const double* v0, int kdim, int nev, opf_linear_map A, void* ctx,
                                double* eig_re, double* eig_im, double* resid, int* kused) {
  if (n < 1 || count < 1 || !v0 || kdim < 1 || nev < 1 || nev > kdim || !A || !eig_re || !eig_im)
    return OPF_EINVAL;
  kdim = std::min(kdim, n);
  // V[i]: (kdim + 1) basis vectors of problem i; H[i]: (kdim + 1) x kdim, row-major
  std::vector<std::vector<double>> V(count), H(count);
  std::vector<int> k_done(count, 0);
  std::vector<char> active(count, 1);
  for (int i = 0; i < count; ++i) {
    V[i].assign((size_t)(kdim + 1) * n, 0.0);
    H[i].assign((size_t)(kdim + 1) * kdim, 0.0);
    const double* s = v0 + (size_t)i * n;
    const double nrm = std::sqrt(dot(s, s, n));
    if (!(nrm > 0.0)) return OPF_EINVAL;
    for (int t = 0; t < n; ++t) V[i][t] = s[t] / nrm;
  }
  std::vector<double> hnorm(count, 0.0);
  for (int j = 0; j < kdim; ++j) {
    std::vector<int> idx;
    std::vector<double*> in, out;
    for (int i = 0; i < count; ++i)
      if (active[i]) {
        idx.push_back(i);
        in.push_back(&V[i][(size_t)j * n]);
        out.push_back(&V[i][(size_t)(j + 1) * n]);
      }
    if (idx.empty()) break;
    int rc = A(ctx, (int)idx.size(), idx.data(), in.data(), out.data());
    if (rc) return rc;
    for (size_t q = 0; q < idx.size(); ++q) {
      const int i = idx[q];
      double* w = out[q];
      auto hij = [&](int r, int c) -> double& { return H[i][(size_t)r * kdim + c]; };
      for (int pass = 0; pass < 2; ++pass)
        for (int r = 0; r <= j; ++r) {
          const double* vr = &V[i][(size_t)r * n];
          const double c = dot(vr, w, n);
          hij(r, j) += c;
          for (int t = 0; t < n; ++t) w[t] -= c * vr[t];
        }
      const double beta = std::sqrt(dot(w, w, n));
      hij(j + 1, j) = beta;
      for (int r = 0; r <= j + 1; ++r) hnorm[i] = std::max(hnorm[i], std::fabs(hij(r, j)));
      k_done[i] = j + 1;
      if (beta <= 1e-13 * hnorm[i]) {  // invariant subspace found
        active[i] = 0;
        continue;
      }
      for (int t = 0; t < n; ++t) w[t] /= beta;
    }
  }
  for (int i = 0; i < count; ++i) {
    const int k = k_done[i];
    if (kused) kused[i] = k;
    std::vector<double> Hk((size_t)k * k);
    for (int r = 0; r < k; ++r)
      for (int c = 0; c < k; ++c) Hk[(size_t)r * k + c] = H[i][(size_t)r * kdim + c];
    std::vector<double> work = Hk;
    std::vector<cplx> ev;
    if (!hessenberg_eigenvalues(work, k, ev)) {
      opf::set_last_error("opf_arnoldi_core: Hessenberg QR iteration did not converge");
      return OPF_ECUDA;
    }
    std::stable_sort(ev.begin(), ev.end(), [](const cplx& a, const cplx& b) { return std::abs(a) > std::abs(b); });
    const double hk = H[i][(size_t)k * kdim + (k - 1)];
    for (int e = 0; e < nev; ++e) {
      const cplx th = e < (int)ev.size() ? ev[e] : cplx(0.0, 0.0);
      eig_re[(size_t)i * nev + e] = th.real();
      eig_im[(size_t)i * nev + e] = th.imag();
      if (resid) resid[(size_t)i * nev + e] = e < (int)ev.size() ? std::fabs(hk) * ritz_tail(Hk, k, th) : 0.0;
    }
  }
  return OPF_OK;
}
