// Small dense linear algebra for the GCRO-DR cycle end (matrices of order <= restart + 1,
// complex128, column-major, on the host): LU solve with partial pivoting, thin
// Householder QR, inverse of an upper-triangular matrix, and the eigenvalues and right
// eigenvectors of a general matrix by the shifted QR algorithm.
#include "small_la.h"

#include <cmath>
#include <cstring>

namespace hz_small {

bool lu_solve(int n, std::vector<cplx> A, std::vector<cplx>& B, int nrhs) {
  for (int k = 0; k < n; k++) {
    int p = k;
    double best = std::abs(A[size_t(k) * n + k]);
    for (int i = k + 1; i < n; i++)
      if (std::abs(A[size_t(k) * n + i]) > best) { best = std::abs(A[size_t(k) * n + i]); p = i; }
    if (!(best > 0.0) || !std::isfinite(best)) return false;
    if (p != k) {
      for (int j = 0; j < n; j++) std::swap(A[size_t(j) * n + k], A[size_t(j) * n + p]);
      for (int j = 0; j < nrhs; j++) std::swap(B[size_t(j) * n + k], B[size_t(j) * n + p]);
    }
    const cplx d = A[size_t(k) * n + k];
    for (int i = k + 1; i < n; i++) {
      const cplx l = A[size_t(k) * n + i] / d;
      A[size_t(k) * n + i] = l;
      for (int j = k + 1; j < n; j++) A[size_t(j) * n + i] -= l * A[size_t(j) * n + k];
      for (int j = 0; j < nrhs; j++) B[size_t(j) * n + i] -= l * B[size_t(j) * n + k];
    }
  }
  for (int j = 0; j < nrhs; j++)
    for (int i = n - 1; i >= 0; i--) {
      cplx s = B[size_t(j) * n + i];
      for (int q = i + 1; q < n; q++) s -= A[size_t(q) * n + i] * B[size_t(j) * n + q];
      B[size_t(j) * n + i] = s / A[size_t(i) * n + i];
    }
  return true;
}

void qr_thin(int rows, int cols, const std::vector<cplx>& A, std::vector<cplx>& Q, std::vector<cplx>& R) {
  std::vector<cplx> W(A);
  std::vector<std::vector<cplx>> vs(static_cast<size_t>(cols));
  for (int j = 0; j < cols; j++) {
    double nx = 0;
    for (int i = j; i < rows; i++) nx += std::norm(W[size_t(j) * rows + i]);
    nx = std::sqrt(nx);
    const cplx x0 = W[size_t(j) * rows + j];
    const cplx ph = std::abs(x0) > 0 ? x0 / std::abs(x0) : cplx(1.0, 0.0);
    const cplx alpha = -ph * nx;
    std::vector<cplx> v(size_t(rows - j));
    for (int i = j; i < rows; i++) v[size_t(i - j)] = W[size_t(j) * rows + i];
    v[0] -= alpha;
    double nv = 0;
    for (const cplx& e : v) nv += std::norm(e);
    nv = std::sqrt(nv);
    if (nv > 0)
      for (cplx& e : v) e /= nv;
    for (int c = j; c < cols; c++) {                     // W <- (I - 2 v v^H) W
      cplx s = 0;
      for (int i = j; i < rows; i++) s += std::conj(v[size_t(i - j)]) * W[size_t(c) * rows + i];
      for (int i = j; i < rows; i++) W[size_t(c) * rows + i] -= 2.0 * v[size_t(i - j)] * s;
    }
    vs[size_t(j)].swap(v);
  }
  R.assign(size_t(cols) * cols, 0.0);
  for (int c = 0; c < cols; c++)
    for (int i = 0; i <= c; i++) R[size_t(c) * cols + i] = W[size_t(c) * rows + i];
  Q.assign(size_t(rows) * cols, 0.0);
  for (int c = 0; c < cols; c++) Q[size_t(c) * rows + c] = 1.0;
  for (int j = cols - 1; j >= 0; j--) {                  // Q = H_0 ... H_{cols-1} I
    const std::vector<cplx>& v = vs[size_t(j)];
    for (int c = 0; c < cols; c++) {
      cplx s = 0;
      for (int i = j; i < rows; i++) s += std::conj(v[size_t(i - j)]) * Q[size_t(c) * rows + i];
      for (int i = j; i < rows; i++) Q[size_t(c) * rows + i] -= 2.0 * v[size_t(i - j)] * s;
    }
  }
}

bool tri_inv_upper(int k, std::vector<cplx>& R) {
  std::vector<cplx> X(size_t(k) * k, 0.0);
  for (int c = 0; c < k; c++) {
    for (int i = c; i >= 0; i--) {
      cplx s = (i == c) ? cplx(1.0, 0.0) : cplx(0.0, 0.0);
      for (int q = i + 1; q <= c; q++) s -= R[size_t(q) * k + i] * X[size_t(c) * k + q];
      const cplx d = R[size_t(i) * k + i];
      if (!(std::abs(d) > 0.0)) return false;
      X[size_t(c) * k + i] = s / d;
    }
  }
  R.swap(X);
  return true;
}

// Complex Givens rotation [c, s; -conj(s), c] with [c, s; -conj(s), c] [a; b] = [r; 0].
static void rot(cplx a, cplx b, double& c, cplx& s) {
  const double aa = std::abs(a);
  if (aa == 0.0) {
    c = 0.0;
    s = cplx(1.0, 0.0);
    return;
  }
  const double rho = std::sqrt(aa * aa + std::norm(b));
  c = aa / rho;
  s = (a / aa) * std::conj(b) / rho;
}

bool eig(int n, const std::vector<cplx>& A, std::vector<cplx>& w, std::vector<cplx>& V, std::string& err) {
  auto at = [n](std::vector<cplx>& M, int i, int j) -> cplx& { return M[size_t(j) * n + i]; };
  std::vector<cplx> H(A), Q(size_t(n) * n, 0.0);
  for (int i = 0; i < n; i++) at(Q, i, i) = 1.0;
  for (const cplx& e : H)
    if (!std::isfinite(e.real()) || !std::isfinite(e.imag())) {
      err = "eig: non-finite input";
      return false;
    }
  // 1. Householder reduction to upper Hessenberg form, H = Q^H A Q
  std::vector<cplx> v(static_cast<size_t>(n));
  for (int k = 0; k + 2 < n; k++) {
    double nx = 0.0;
    for (int i = k + 1; i < n; i++) nx += std::norm(at(H, i, k));
    nx = std::sqrt(nx);
    if (nx == 0.0) continue;
    const cplx x0 = at(H, k + 1, k);
    const cplx ph = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : cplx(1.0, 0.0);
    for (int i = k + 1; i < n; i++) v[size_t(i)] = at(H, i, k);
    v[size_t(k + 1)] += ph * nx;                      // v = x + phase(x0) ||x|| e1
    double nv = 0.0;
    for (int i = k + 1; i < n; i++) nv += std::norm(v[size_t(i)]);
    nv = std::sqrt(nv);
    for (int i = k + 1; i < n; i++) v[size_t(i)] /= nv;
    for (int j = 0; j < n; j++) {                     // H <- (I - 2 v v^H) H
      cplx s = 0.0;
      for (int i = k + 1; i < n; i++) s += std::conj(v[size_t(i)]) * at(H, i, j);
      for (int i = k + 1; i < n; i++) at(H, i, j) -= 2.0 * v[size_t(i)] * s;
    }
    for (int i = 0; i < n; i++) {                     // H <- H (I - 2 v v^H), Q <- Q (I - 2 v v^H)
      cplx s = 0.0, t = 0.0;
      for (int j = k + 1; j < n; j++) {
        s += at(H, i, j) * v[size_t(j)];
        t += at(Q, i, j) * v[size_t(j)];
      }
      for (int j = k + 1; j < n; j++) {
        at(H, i, j) -= 2.0 * s * std::conj(v[size_t(j)]);
        at(Q, i, j) -= 2.0 * t * std::conj(v[size_t(j)]);
      }
    }
    for (int i = k + 2; i < n; i++) at(H, i, k) = 0.0;
  }
  // 2. shifted QR iteration (Wilkinson shift, bulge chased by Givens rotations) to the
  //    complex Schur form T = Q^H A Q, deflating negligible subdiagonal entries
  const double eps = 2.220446049250313e-16;
  double hnorm = 0.0;
  for (const cplx& e : H) hnorm = std::max(hnorm, std::abs(e));
  int hi = n - 1, iter = 0, total = 0;
  while (hi > 0) {
    int l = hi;
    while (l > 0) {
      const double scale = std::abs(at(H, l - 1, l - 1)) + std::abs(at(H, l, l));
      if (std::abs(at(H, l, l - 1)) <= eps * (scale > 0.0 ? scale : hnorm)) break;
      l--;
    }
    if (l > 0) at(H, l, l - 1) = 0.0;
    if (l == hi) {                                    // a 1 x 1 block has converged
      hi--;
      iter = 0;
      continue;
    }
    if (++total > 60 * n) {
      err = "eig: the QR iteration did not converge";
      return false;
    }
    cplx mu;
    if (iter > 0 && iter % 11 == 0) {                 // exceptional shift out of a cycle
      mu = at(H, hi, hi) + std::abs(at(H, hi, hi - 1));
    } else {                                          // eigenvalue of the trailing 2 x 2 closest to H[hi][hi]
      const cplx a = at(H, hi - 1, hi - 1), b = at(H, hi - 1, hi), c = at(H, hi, hi - 1), d = at(H, hi, hi);
      const cplx half = 0.5 * (a - d);
      const cplx disc = std::sqrt(half * half + b * c);
      const cplx m1 = 0.5 * (a + d) + disc, m2 = 0.5 * (a + d) - disc;
      mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
    }
    iter++;
    cplx x = at(H, l, l) - mu, y = at(H, l + 1, l);
    for (int k = l; k < hi; k++) {
      double cs;
      cplx sn;
      rot(x, y, cs, sn);
      for (int j = std::max(l, k - 1); j < n; j++) {  // rows k, k + 1
        const cplx hk = at(H, k, j), hk1 = at(H, k + 1, j);
        at(H, k, j) = cs * hk + sn * hk1;
        at(H, k + 1, j) = -std::conj(sn) * hk + cs * hk1;
      }
      const int rmax = std::min(k + 2, hi);
      for (int i = 0; i <= rmax; i++) {               // columns k, k + 1 (times the rotation's adjoint)
        const cplx hk = at(H, i, k), hk1 = at(H, i, k + 1);
        at(H, i, k) = cs * hk + std::conj(sn) * hk1;
        at(H, i, k + 1) = -sn * hk + cs * hk1;
      }
      for (int i = 0; i < n; i++) {
        const cplx qk = at(Q, i, k), qk1 = at(Q, i, k + 1);
        at(Q, i, k) = cs * qk + std::conj(sn) * qk1;
        at(Q, i, k + 1) = -sn * qk + cs * qk1;
      }
      if (k + 1 < hi) {
        x = at(H, k + 1, k);
        y = at(H, k + 2, k);
      }
    }
  }
  // 3. eigenvectors of the triangular T by back substitution, then V = Q X, unit columns
  w.resize(size_t(n));
  for (int i = 0; i < n; i++) w[size_t(i)] = at(H, i, i);
  double tnorm = 0.0;
  for (int j = 0; j < n; j++)
    for (int i = 0; i <= j; i++) tnorm = std::max(tnorm, std::abs(at(H, i, j)));
  const double tiny = eps * std::max(tnorm, 1e-300);
  std::vector<cplx> X(size_t(n) * n, 0.0);
  for (int k = 0; k < n; k++) {
    at(X, k, k) = 1.0;
    for (int i = k - 1; i >= 0; i--) {
      cplx s = 0.0;
      for (int j = i + 1; j <= k; j++) s += at(H, i, j) * at(X, j, k);
      cplx d = at(H, i, i) - w[size_t(k)];
      if (std::abs(d) < tiny) d = tiny;
      at(X, i, k) = -s / d;
    }
  }
  V.assign(size_t(n) * n, 0.0);
  for (int k = 0; k < n; k++) {
    double nrm = 0.0;
    for (int i = 0; i < n; i++) {
      cplx s = 0.0;
      for (int j = 0; j <= k; j++) s += at(Q, i, j) * at(X, j, k);
      at(V, i, k) = s;
      nrm += std::norm(s);
    }
    nrm = std::sqrt(nrm);
    for (int i = 0; i < n; i++) at(V, i, k) /= nrm;
  }
  return true;
}

}  // namespace hz_small
