// Allocation-free entry point: the per-block least-squares estimate
// b_i = R_i^-1 Q_i^T y_i from the factors a handle already holds, with every
// intermediate kept in one fixed device array that is part of the library
// image (no cudaMalloc, cudaFree or allocating library call on this path).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "glm_sur.h"
#include "internal.h"
#include "noalloc.h"

namespace glmsur {

// Shared scratch of glm_sur_ols_static.  Every GPU that loads the library
// holds it until the process exits; every call uses it from the start, so
// calls that overlap on the GPU (different streams, no ordering) race.
// Nothing in it has to start at zero: each call writes every entry it reads.
static __device__ __align__(256) double g_ols_scratch[kOlsScratchDoubles];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device; the host-side symbol is only a stand-in, not a device address).
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_ols_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// part[rb][col][j] = sum over rows t of range rb of Q[t, col] * y_j[block(col)][t]
// grid (R, quad groups, k); thread = one column quad.  y is read in the
// caller's column-major vec layout (block i of column j at Y + j*ldy + i*M).
__global__ void __launch_bounds__(256)
k_ols_partial_static(int64_t M, int np, int nq, int k, const double* __restrict__ Q,
                     const double* __restrict__ Y, int64_t ldy, const int* __restrict__ quad_blk,
                     double* __restrict__ part) {
  const int j = blockIdx.z;
  const int qpg = (int)ceil_div(nq, gridDim.y);
  const int q = blockIdx.y * qpg + threadIdx.x;
  if (threadIdx.x >= qpg || q >= nq) return;
  const int64_t r0 = M * blockIdx.x / gridDim.x, r1 = M * (blockIdx.x + 1) / gridDim.x;
  const int blk = quad_blk[q];
  const double* yb = Y + (int64_t)j * ldy + (int64_t)blk * M;
  double acc[4] = {0, 0, 0, 0};
  for (int64_t t = r0; t < r1; ++t) {
    double qv[4];
    Vec4<double>::load(Q + t * np + 4 * q, qv);
    const double yv = yb[t];
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] += qv[c] * yv;
  }
  double* dst = part + ((int64_t)blockIdx.x * np + 4 * q) * k + j;
#pragma unroll
  for (int c = 0; c < 4; ++c) dst[(int64_t)c * k] = acc[c];
}

// C[col][j] = sum_rb part[rb][col][j] (fixed order)
__global__ void k_ols_reduce_static(int64_t nidx, int nrb, const double* __restrict__ part, double* __restrict__ C) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= nidx) return;
  double s = 0.0;
  for (int r = 0; r < nrb; ++r) s += part[(int64_t)r * nidx + idx];
  C[idx] = s;
}

// b_i = R_i^-1 C_i (back substitution; one thread per (block, column))
__global__ void k_ols_trisolve_static(int G, int k, const double* __restrict__ R, const int64_t* __restrict__ r_off,
                                      const int* __restrict__ n_i, const int* __restrict__ off,
                                      const int* __restrict__ poff, const double* __restrict__ C, double* b,
                                      int64_t ldb) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= G * k) return;
  const int i = id / k, j = id % k;
  const int ni = n_i[i];
  const double* Ri = R + r_off[i];
  double x[kMaxBlockCols];
  for (int r = ni - 1; r >= 0; --r) {
    double s = C[(int64_t)(poff[i] + r) * k + j];
    for (int c = r + 1; c < ni; ++c) s -= Ri[r * ni + c] * x[c];
    x[r] = s / Ri[r * ni + r];
  }
  for (int r = 0; r < ni; ++r) b[(int64_t)j * ldb + off[i] + r] = x[r];
}

}  // namespace

glm_sur_status ols_static(const Geom& gm, const double* Q64, const double* R, const double* Y, int64_t ldy, int k,
                          double* b, int64_t ldb, int sms, cudaStream_t s) {
  const int64_t cidx = (int64_t)gm.np * k;
  // row ranges: as many as the scratch holds next to C, at most 2 per SM
  const int64_t fit = (int64_t)kOlsScratchDoubles / cidx - 1;
  if (fit < 1) return GLM_SUR_INVALID_ARG;
  const int64_t lim = std::min<int64_t>(fit, std::min<int64_t>((int64_t)2 * sms, gm.M));
  const int R_rows = (int)std::max<int64_t>(1, lim);
  double* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    set_last_error(e, "cudaGetSymbolAddress(ols scratch)", __FILE__, __LINE__);
    return GLM_SUR_CUDA_ERROR;
  }
  double* part = scratch;
  double* C = scratch + (int64_t)R_rows * cidx;
  const int nqg = (int)std::max<int64_t>(1, ceil_div(gm.nq, 256));
  const int qpg = (int)ceil_div(gm.nq, nqg);
  const int threads = (int)std::min<int64_t>(256, ceil_div(qpg, 32) * 32);
  k_ols_partial_static<<<dim3(R_rows, nqg, k), threads, 0, s>>>(gm.M, gm.np, gm.nq, k, Q64, Y, ldy, gm.d_quad_blk,
                                                                 part);
  k_ols_reduce_static<<<(unsigned)ceil_div(cidx, 256), 256, 0, s>>>(cidx, R_rows, part, C);
  k_ols_trisolve_static<<<(unsigned)ceil_div((int64_t)gm.G * k, 128), 128, 0, s>>>(
      gm.G, k, R, gm.d_r_off, gm.d_n_i, gm.d_off, gm.d_poff, C, b, ldb);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(e, "ols static launch", __FILE__, __LINE__);
    return GLM_SUR_CUDA_ERROR;
  }
  return GLM_SUR_OK;
}

}  // namespace glmsur
