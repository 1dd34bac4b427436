// Small dense linear algebra for the GCRO-DR cycle end (matrices of order <= restart + 1,
// complex128, column-major): LU solve with partial pivoting, thin Householder QR,
// inverse of an upper-triangular matrix, and the eigen-decomposition of a general
// matrix through cuSOLVER (cusolverDnXgeev, right eigenvectors).
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

EigSolver::~EigSolver() {
  if (dA) cudaFree(dA);
  if (dW) cudaFree(dW);
  if (dVR) cudaFree(dVR);
  if (dwork) cudaFree(dwork);
  if (dinfo) cudaFree(dinfo);
  if (params) cusolverDnDestroyParams(params);
  if (handle) cusolverDnDestroy(handle);
}

bool eig(EigSolver& E, cudaStream_t st, int n, const std::vector<cplx>& A, std::vector<cplx>& w,
         std::vector<cplx>& VR, std::string& err) {
  if (!E.handle) {
    if (cusolverDnCreate(&E.handle) != CUSOLVER_STATUS_SUCCESS || cusolverDnCreateParams(&E.params) !=
                                                                      CUSOLVER_STATUS_SUCCESS) {
      err = "cuSOLVER initialisation failed";
      return false;
    }
  }
  cusolverDnSetStream(E.handle, st);
  if (n > E.cap) {
    if (E.dA) cudaFree(E.dA);
    if (E.dW) cudaFree(E.dW);
    if (E.dVR) cudaFree(E.dVR);
    if (!E.dinfo && cudaMalloc(&E.dinfo, sizeof(int)) != cudaSuccess) { err = "eig: cudaMalloc"; return false; }
    if (cudaMalloc(&E.dA, size_t(n) * n * 16) != cudaSuccess || cudaMalloc(&E.dW, size_t(n) * 16) != cudaSuccess ||
        cudaMalloc(&E.dVR, size_t(n) * n * 16) != cudaSuccess) {
      cudaGetLastError();
      err = "eig: cudaMalloc";
      return false;
    }
    E.cap = n;
  }
  cudaMemcpyAsync(E.dA, A.data(), size_t(n) * n * 16, cudaMemcpyHostToDevice, st);
  size_t dbytes = 0, hbytes = 0;
  if (cusolverDnXgeev_bufferSize(E.handle, E.params, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR, n,
                                 CUDA_C_64F, E.dA, n, CUDA_C_64F, E.dW, CUDA_C_64F, nullptr, n, CUDA_C_64F, E.dVR,
                                 n, CUDA_C_64F, &dbytes, &hbytes) != CUSOLVER_STATUS_SUCCESS) {
    err = "cusolverDnXgeev_bufferSize failed";
    return false;
  }
  if (dbytes > E.dbytes) {
    if (E.dwork) cudaFree(E.dwork);
    if (cudaMalloc(&E.dwork, dbytes) != cudaSuccess) {
      cudaGetLastError();
      err = "eig: workspace cudaMalloc";
      return false;
    }
    E.dbytes = dbytes;
  }
  if (hbytes > E.hwork.size()) E.hwork.resize(hbytes);
  if (cusolverDnXgeev(E.handle, E.params, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR, n, CUDA_C_64F,
                      E.dA, n, CUDA_C_64F, E.dW, CUDA_C_64F, nullptr, n, CUDA_C_64F, E.dVR, n, CUDA_C_64F,
                      E.dwork, E.dbytes, E.hwork.empty() ? nullptr : E.hwork.data(), E.hwork.size(),
                      E.dinfo) != CUSOLVER_STATUS_SUCCESS) {
    err = "cusolverDnXgeev failed";
    return false;
  }
  int info = 0;
  w.resize(size_t(n));
  VR.resize(size_t(n) * n);
  cudaMemcpyAsync(w.data(), E.dW, size_t(n) * 16, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(VR.data(), E.dVR, size_t(n) * n * 16, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&info, E.dinfo, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    err = "eig: stream synchronise failed";
    return false;
  }
  if (info != 0) {
    err = "cusolverDnXgeev info " + std::to_string(info);
    return false;
  }
  return true;
}

}  // namespace hz_small
