// Small dense complex linear algebra used at the end of a GCRO-DR cycle (matrices of
// order <= restart + 1, column-major std::complex<double>).
#pragma once

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

// Eigenvalues w and right eigenvectors V (unit columns) of a general complex n x n
// matrix A, on the host: Householder reduction to upper Hessenberg form, the shifted QR
// algorithm (Wilkinson shifts, bulge chased by Givens rotations, deflation of negligible
// subdiagonal entries, an exceptional shift every 11 steps without deflation) to the
// complex Schur form A = Q T Q^H, then the eigenvectors of T by back substitution and
// V = Q X (Golub and Van Loan, Matrix Computations, chapter 7).  False (with err) on a
// non-finite input or if the iteration does not converge within 60 n steps.
bool eig(int n, const std::vector<cplx>& A, std::vector<cplx>& w, std::vector<cplx>& V, std::string& err);

}  // namespace hz_small
