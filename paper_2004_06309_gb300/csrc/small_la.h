// Small dense complex linear algebra used at the end of a GCRO-DR cycle (matrices of
// order <= restart + 1, column-major std::complex<double>).
#pragma once

#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <complex>
#include <string>
#include <vector>

namespace hz_small {

using cplx = std::complex<double>;

// B <- A^{-1} B (A n x n, B n x nrhs) by LU with partial pivoting; false if A is singular.
bool lu_solve(int n, std::vector<cplx> A, std::vector<cplx>& B, int nrhs);

// Thin QR of A (rows x cols, rows >= cols) by Householder reflections: Q rows x cols
// with orthonormal columns, R cols x cols upper triangular, A = Q R.
void qr_thin(int rows, int cols, const std::vector<cplx>& A, std::vector<cplx>& Q, std::vector<cplx>& R);

// R <- R^{-1} for an upper-triangular k x k R; false on a zero diagonal entry.
bool tri_inv_upper(int k, std::vector<cplx>& R);

// Eigenvalues w and right eigenvectors VR (columns) of a general n x n matrix, by
// cuSOLVER on `st`; device buffers are kept in the solver between calls.
struct EigSolver {
  cusolverDnHandle_t handle = nullptr;
  cusolverDnParams_t params = nullptr;
  void *dA = nullptr, *dW = nullptr, *dVR = nullptr, *dwork = nullptr;
  int* dinfo = nullptr;
  size_t dbytes = 0;
  std::vector<char> hwork;
  int cap = 0;
  ~EigSolver();
};
bool eig(EigSolver& E, cudaStream_t st, int n, const std::vector<cplx>& A, std::vector<cplx>& w,
         std::vector<cplx>& VR, std::string& err);

}  // namespace hz_small
