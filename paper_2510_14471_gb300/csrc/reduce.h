// Row reduction of the SUR model (Remark rem:reduction): an orthonormal
// basis Q of range(W), W = [X_1 ... X_G], by Cholesky QR twice, and the
// float64 products that move responses and gradients between the M rows of
// the model and the n rows of the reduced one.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace glmsur {

// C(i, j) = sum_p A(i, p) B(p, j) for i < m, j < n, p < kdim, float64, with
// A(i, p) at A[i * ars + p * acs], B(p, j) at B[p * brs + j * bcs] and C(i, j)
// at C[i * crs + j * ccs] (any layout: strides carry transposes).
// With a workspace ws of nz * m * n doubles and nz > 1 the depth is split in
// nz chunks (partial tiles into ws, then summed in a fixed order): the grid
// then fills the SMs when m x n has few tiles and the depth is long.
void launch_dgemm(int m, int n, int64_t kdim, const double* A, int64_t ars, int64_t acs, const double* B,
                  int64_t brs, int64_t bcs, double* C, int64_t crs, int64_t ccs, cudaStream_t s,
                  double* ws = nullptr, int nz = 1);
// Depth chunks for launch_dgemm on `sms` SMs (1: no split).
int dgemm_split(int m, int n, int64_t kdim, int sms);

// One float64 product C = A B of a batch (layout as launch_dgemm).
struct DgemmProblem {
  int m, n;
  int64_t kdim;
  const double* A;
  int64_t ars, acs;
  const double* B;
  int64_t brs, bcs;
  double* C;
  int64_t crs, ccs;
};
// Output tiles of an m x n product.
int dgemm_tiles(int m, int n);
// Every problem of `probs` (DEVICE array of count) in one launch; max_tiles =
// the largest dgemm_tiles of them.  The problems' outputs must not overlap.
void launch_dgemm_batched(const DgemmProblem* probs, int count, int max_tiles, cudaStream_t s);

// Linv = L^-1 for a row-major lower-triangular n x n L (its strict upper
// triangle is ignored); Linv row-major with zeros above the diagonal.
cudaError_t launch_tri_inverse(int n, const double* L, double* Linv, cudaStream_t s);

// Energy of the responses outside range(W), per right-hand side j:
// out[j] = max(0, sum_i s_i^2 (||y_ij||^2 - ||Q^T y_ij||^2)), y_ij = Y[j * ldy
// + i M ...] (M rows), Q^T y_ij = Yr[(j G + i) n ...] (n rows), s = isq or
// ones (the row scaling of a preconditioner block).  part: G x k workspace.
void launch_complement_energy(int G, int64_t M, int64_t n, int k, const double* Y, int64_t ldy, const double* Yr,
                              const double* isq, double* part, double* out, cudaStream_t s);

// Zero the strict upper triangle of a row-major n x n matrix.
void launch_zero_upper(int n, double* A, cudaStream_t s);

}  // namespace glmsur
