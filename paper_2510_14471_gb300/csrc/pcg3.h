// Algorithm glmpcg3 (the alternative PCG-Aug) in float64: s_i in place of
// u_i and v_i, u_i = Pi s_i recomputed every step (Sec. 3.2).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace glmsur {

// Per-column state (device arrays of k) of the glmpcg3 iteration.
struct Pcg3State {
  int k = 0;
  double tol = 0.0;
  int maxit = 0;
  double *c = nullptr, *c1 = nullptr, *lam = nullptr, *mu = nullptr, *relres = nullptr;
  int *active = nullptr, *iters = nullptr, *status = nullptr;
  double* dpart = nullptr;   // nblk x k partial sums of d
  int nblk = 0;
  const double* c1_extra = nullptr;   // (nullable, k) added to the first c (reduced handles)
};

// Sm = -Sigma u (as the Sigma-residual kernel returns it for a zero right side).
// dpart[b][j] = sum over the rows of CTA b of u * Sigma u (column j); vectors (M, G, k) row-major.
void launch_pcg3_dot(int64_t M, int G, int k, const double* u, const double* Sm, const Pcg3State& st, cudaStream_t s);
// r = -y (r_1 = Sigma w_1 + X z_1 - y with w_1 = 0, z_1 = 0)
void launch_pcg3_neg(int64_t n_elem, const double* y, double* r, cudaStream_t s);
// d_j = sum_b dpart[b][j]; lambda_j = c_j / d_j; a non-positive or non-finite d stops column j (breakdown).
void launch_pcg3_lambda(const Pcg3State& st, cudaStream_t s);
// live columns: w -= lambda u;  r -= lambda (Sigma u + s - u)   (X X*^T s = s - Pi s for D = I)
void launch_pcg3_wr(int64_t n_elem, int k, const Pcg3State& st, const double* u, const double* Sm, const double* sv,
                    double* w, double* r, cudaStream_t s);
// c' = sum of the partials of (Pi r)^T (Pi r); init: c = c1 = c'; else the stop tests and mu = c' / c.
void launch_pcg3_after(const Pcg3State& st, const double* cpart, int ncpart, int init, cudaStream_t s);
// init: s = r; else live columns: s = r + mu s.
void launch_pcg3_s(int64_t n_elem, int k, const Pcg3State& st, const double* r, double* sv, int init, cudaStream_t s);

}  // namespace glmsur
