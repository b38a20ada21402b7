// Restricted multivariate GLM (Sec. "Multivariate linear models with
// parameters restrictions"): Y = Z0 B + U, rows of U iid (0, Omega0),
// restrictions C_i b_i = gamma_i on each column of B.  After the model
// reduction Z0 = Q0 R0 the solve is the SUR iteration on the G equations
// [R0; C_i] (padded with zero rows to N + kmax rows) with Sigma = Omega0 (x) I
// on the first N rows and 0 on the restriction rows; the setup QR of those
// blocks is the updating QRD [R0; C_i] = Qt_i R_i (eq. MvRGLMQRi).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace glmsur {

// Xt (column-major, leading dimension Mp = N + kmax, G N columns): block i,
// column c, row t = R0[t][c] (t < N; R0 row-major upper triangular),
// C[koff[i] + t - N, c] (N <= t < N + k_i; C column-major, leading dimension
// ldc), 0 below.
void launch_mv_build_x(int G, int N, int Mp, const double* R0, const double* C, int64_t ldc, const int* koff,
                       double* Xt, cudaStream_t s);
// yp (column-major, (G Mp) x k): equation i, row t of right-hand side j =
// Y0[t, i, j] (t < N; Y0 column-major N x (G k), column j G + i), gamma
// [koff[i] + t - N, j] (N <= t < N + k_i; column-major, leading dimension
// ldd; zero when gamma is null), 0 below.
void launch_mv_assemble(int G, int N, int Mp, int k, const double* Y0, const double* gamma, int64_t ldd,
                        const int* koff, double* yp, cudaStream_t s);

}  // namespace glmsur
