// Kernels of the adjoint solve (dL/dy, dL/dOmega for a loss L(b)).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace glmsur {

// C = padded [s_i R_i^-T g_i] (n' x k, element (col, j) at col * k + j); g is
// the caller's n x k column-major dL/db (leading dimension ldg), s_i =
// blk_scale[i] or 1.
void launch_adj_seed(const Geom& gm, int k, const double* R, const double* gb, int64_t ldg, double* C,
                     cudaStream_t s, const double* blk_scale = nullptr);
// Number of row chunks of the Omega-gradient reduction (its workspace holds
// chunks x G x G doubles).
int adj_omega_chunks(const Geom& gm, int k, int sms);
// out (G x G column-major, leading dimension ldo) = -diag(s) sym(sum_t,j Lam[t,:,j]^T W[t,:,j]) diag(s),
// s = blk_scale or ones
void launch_adj_omega(const Geom& gm, int k, const double* Lam, const double* W, double* part, int nch,
                      double* out, int64_t ldo, cudaStream_t s, const double* blk_scale = nullptr);

}  // namespace glmsur
