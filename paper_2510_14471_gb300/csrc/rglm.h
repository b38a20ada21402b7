// Linear restrictions folded into the augmented system (Sec. 4.1).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace glmsur {

// N = (+)R_i^T R_i + C^T C, its Cholesky factor (in N) and N^-1 (row-major n x n).
cudaError_t rglm_factor(const Geom& gm, const double* R, const double* C, int64_t ldc, int kc, const int* col_blk,
                        double* N, double* Minv, int* flag, cudaStream_t s);
// In-place Cholesky N = L L^T of a row-major SPD n x n matrix (one CTA;
// the strict upper triangle is left as it was); flag |= 1 on a pivot not
// above rel_tol times the largest diagonal entry.
cudaError_t cholesky_lower(int n, double* N, int* flag, double rel_tol, cudaStream_t s);
// a = [R_i^T e_i] + sign_d C^T d; c = N^-1 a; f_i = R_i c_i (or c -> b_out).
cudaError_t rglm_coef(const Geom& gm, int k, const double* e, const double* R, const double* Minv, const double* C,
                      int64_t ldc, int kc, const double* d, int64_t ldd, double sign_d, double* cbuf, double* fbuf,
                      double* b_out, int64_t ldb, cudaStream_t s);
// restriction rows of the projected residual and their partial sum of squares
cudaError_t rglm_gc(const Geom& gm, int k, int kc, const double* C, int64_t ldc, const double* cbuf, const double* d,
                    int64_t ldd, const double* lam, int mode, double* gC, double* cpart, int row, cudaStream_t s);

}  // namespace glmsur
