// Host FP64 dense helpers for the small projected problems at the end of each
// Lan-DR / MinRes-DR cycle (Sec. 1-2; row-major).
#pragma once

#include <complex>
#include <vector>

#include "../../include/dlz.h"

namespace dlz {

// Eigen-decomposition of symmetric A (n x n): w ascending, column j of Z the
// eigenvector of w[j] (Z may be null: eigenvalues only).  false if the QR
// iteration did not converge.
bool sym_eig(int n, const double *A, double *w, double *Z);
// Smallest and largest eigenvalue of symmetric A (n x n) by Householder reduction and
// Sturm bisection; false on non-finite input.
bool sym_extremes(int n, const double *A, double *lo, double *hi);
// y = argmin ||c - T y|| (rows > cols); q (optional, rows == cols + 1): unit
// vector orthogonal to range(T).
bool lstsq(int rows, int cols, const double *T, const double *c, double *y, double *q);
// A = L L^T (lower L); false if A is not positive definite.
bool cholesky(int n, const double *A, double *L);
// L x = b / L^T x = b in place; `first` (optional): the envelope of L from envelope()
void lower_solve(int n, const double *L, double *b, const int *first = nullptr);
void upper_t_solve(int n, const double *L, double *b, const int *first = nullptr);
void envelope(int n, const double *L, std::vector<int> &first);
// The same solves for nrhs right-hand sides at once: B (n x nrhs, row-major) is
// overwritten by L^-1 B / L^-T B (first: the envelope of L, required).
void lower_solve_rows(int n, const double *L, double *B, int nrhs, const int *first);
void upper_t_solve_rows(int n, const double *L, double *B, int nrhs, const int *first);
bool lu_factor(int n, double *A, int *piv);
void lu_solve(int n, const double *LU, const int *piv, double *b);
bool lu_factor(int n, std::complex<double> *A, int *piv);
void lu_solve(int n, const std::complex<double> *LU, const int *piv, std::complex<double> *b);
// Orthonormalise the columns of P (rows x cols) left to right, MGS twice.
bool mgs_columns(int rows, int cols, double *P);
// Complex helpers (small_dense_z.cpp).  zgeev: eigenvalues w[n] and unit eigenvectors
// (column j of Z, may be null) of a general complex A (n x n); false on non-finite input
// or no convergence.  zlstsq: y = argmin ||c - A y|| (rows > cols) and, if rows ==
// cols + 1 and q is not null, the unit vector q spanning range(A)^perp.  zmgs_columns:
// MGS twice on the columns of P (rows x cols); false on a zero column.
bool zgeev(int n, const std::complex<double> *A, std::complex<double> *w, std::complex<double> *Z);
bool zlstsq(int rows, int cols, const std::complex<double> *A, const std::complex<double> *c,
            std::complex<double> *y, std::complex<double> *q);
bool zmgs_columns(int rows, int cols, std::complex<double> *P);

}  // namespace dlz
