// Kernels of the adjoint solve (dL/dy, dL/dOmega for a loss L(b)).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace glmsur {

// C = padded [R_i^-T g_i] (n' x k, element (col, j) at col * k + j); g is the
// caller's n x k column-major dL/db (leading dimension ldg).
void launch_adj_seed(const Geom& gm, int k, const double* R, const double* gb, int64_t ldg, double* C,
                     cudaStream_t s);
// Number of row chunks of the Omega-gradient reduction (its workspace holds
// chunks x G x G doubles).
int adj_omega_chunks(const Geom& gm, int k, int sms);
// out (G x G column-major, leading dimension ldo) = -sym(sum_t,j Lam[t,:,j]^T W[t,:,j])
void launch_adj_omega(const Geom& gm, int k, const double* Lam, const double* W, double* part, int nch,
                      double* out, int64_t ldo, cudaStream_t s);

}  // namespace glmsur
