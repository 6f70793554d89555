// Host FP64 dense linear algebra used once at plan time (no LAPACK on either machine).
// All matrices are column-major.
#pragma once
#include <vector>

namespace m2l {

// R factor (n x n, upper triangular, column-major) of the tall matrix obtained by stacking
// `blocks` vertically; every block is column-major with n columns and blocks[i].size()/n rows.
// Tall-skinny QR: Householder QR of block pairs, reduced pairwise (OpenMP over pairs).
std::vector<double> stacked_r_factor(std::vector<std::vector<double>> blocks, int n);

// One-sided (Hestenes) Jacobi SVD of the m x n matrix A (m >= n): A = U diag(s) V^T with s
// descending; U is m x n, V is n x n. Columns of U for zero singular values are left zero.
void jacobi_svd(const std::vector<double> &A, int m, int n, std::vector<double> &U,
                std::vector<double> &s, std::vector<double> &V);

// Two passes of modified Gram-Schmidt over the first `cols` columns of the column-major
// rows x cols matrix M, in place and in column order. The right singular vectors that
// jacobi_svd accumulates from its rotations drift from orthogonality by about n * sweeps * eps
// (1.7e-13 measured at n = 152); a truncated product U_k U_k^T K built from them is off by as
// much. This restores orthonormality to rounding and moves each column by about that drift,
// leaving the spanned subspaces as they were.
void orthonormalize_columns(double *M, int rows, int cols);

}  // namespace m2l
