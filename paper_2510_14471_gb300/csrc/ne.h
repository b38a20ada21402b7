// PCG-NE: the conjugate gradient method (Algorithm pcg with K = I) on the
// normal equations (X^T Sigma^-1 X) beta = X^T Sigma^-1 y of the SUR model,
// the comparator of the Monte-Carlo study (Sec. "Statistical properties of
// the PCG-Aug estimator") and of the experiments (Sec. "Experimental Tests").
// X = (+) Q_i R_i is applied through the setup factors and Sigma^-1 =
// Omega^-1 (x) I_M row by row, so one step reads Q twice and never forms X.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace glmsur {

// Device state of k independent CG runs in the n coefficients (element
// (col, j) of an n x k array at col * k + j).
struct NeState {
  int k = 0;
  double tol = 0.0;
  int maxit = 0;
  double* beta = nullptr;    // iterate
  double* f = nullptr;       // gradient f = A beta - h (Algorithm pcg, f = G x - h)
  double* p = nullptr;       // search direction
  double* q = nullptr;       // A p
  double* c = nullptr;       // f^T f (k)
  double* c1 = nullptr;      // f_1^T f_1 (k)
  double* relres = nullptr;  // sqrt(c / c1) (k)
  int* active = nullptr;     // column still iterating (k)
  int* iters = nullptr;      // steps taken (k)
  int* status = nullptr;     // glm_sur_status, or kStatusRunning (k)
};

// cvec = padded [R_i p_i] (n' x k, element (padded col, j) at col * k + j;
// the pad columns are left as they are)
void launch_ne_rmul(const Geom& gm, int k, const double* R, const double* p, double* cvec, cudaStream_t s);
// With C = padded Q^T s for s = -Sigma^-1 (X p) (step) or s = -Sigma^-1 y
// (init): q = -[R_i^T C_i] = A p (or h); init sets beta = 0, f = p = -h,
// c = c1 = f^T f; a step takes lambda = c / p^T q, beta -= lambda p,
// f -= lambda q, c' = f^T f, the stopping tests and p = f + (c'/c) p.
void launch_ne_step(const Geom& gm, int k, const double* R, const double* C, const NeState& st, int init,
                    cudaStream_t s);
// b (n x k column-major, leading dimension ldb) = beta
void launch_ne_store(const Geom& gm, int k, const double* beta, double* b, int64_t ldb, cudaStream_t s);

}  // namespace glmsur
