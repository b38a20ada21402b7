// Data movement of the restricted multivariate GLM: the regressor blocks
// [R0; C_i] and the responses [Q0^T y_i; gamma_i] of the reduced model.
#include <cuda_runtime.h>

#include "common.cuh"
#include "mvrglm.h"

namespace glmsur {

namespace {

__global__ void k_mv_build_x(int G, int N, int Mp, const double* __restrict__ R0, const double* __restrict__ C,
                             int64_t ldc, const int* __restrict__ koff, double* __restrict__ Xt) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t tot = (int64_t)Mp * G * N;
  if (id >= tot) return;
  const int t = (int)(id % Mp);
  const int64_t col = id / Mp;                 // global column i N + c
  const int i = (int)(col / N), c = (int)(col % N);
  const int ki = koff[i + 1] - koff[i];
  double v = 0.0;
  if (t < N) v = R0[(int64_t)t * N + c];
  else if (t < N + ki) v = C[(int64_t)(koff[i] + t - N) + (int64_t)c * ldc];
  Xt[id] = v;
}

__global__ void k_mv_assemble(int G, int N, int Mp, int k, const double* __restrict__ Y0,
                              const double* __restrict__ gamma, int64_t ldd, const int* __restrict__ koff,
                              double* __restrict__ yp) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t m = (int64_t)G * Mp;
  if (id >= m * k) return;
  const int j = (int)(id / m);
  const int64_t r = id % m;
  const int i = (int)(r / Mp), t = (int)(r % Mp);
  const int ki = koff[i + 1] - koff[i];
  double v = 0.0;
  if (t < N) v = Y0[(int64_t)t + ((int64_t)j * G + i) * N];
  else if (t < N + ki && gamma) v = gamma[(int64_t)(koff[i] + t - N) + (int64_t)j * ldd];
  yp[id] = v;
}

}  // namespace

void launch_mv_build_x(int G, int N, int Mp, const double* R0, const double* C, int64_t ldc, const int* koff,
                       double* Xt, cudaStream_t s) {
  const int64_t tot = (int64_t)Mp * G * N;
  k_mv_build_x<<<(unsigned)ceil_div(tot, 256), 256, 0, s>>>(G, N, Mp, R0, C, ldc, koff, Xt);
}

void launch_mv_assemble(int G, int N, int Mp, int k, const double* Y0, const double* gamma, int64_t ldd,
                        const int* koff, double* yp, cudaStream_t s) {
  const int64_t tot = (int64_t)G * Mp * k;
  k_mv_assemble<<<(unsigned)ceil_div(tot, 256), 256, 0, s>>>(G, N, Mp, k, Y0, gamma, ldd, koff, yp);
}

}  // namespace glmsur
