// Row reduction of the SUR model (Remark rem:reduction).  With W = [X_1 ...
// X_G] (M x n) = Q R_W, Q orthonormal (M x n), the rows of the model outside
// range(W) carry no regressor; Sigma = Omega (x) I_M acts on every row alike,
// so rotating the rows of each equation by [Q Q_perp] splits eq. (aug1) into
// the reduced model (X_i' = R_W[:, block i], y_i' = Q^T y_i, M' = n rows)
// and rows that do not touch b.  b of the reduced model is b of the model.
// Q comes from Cholesky QR twice: W^T W = L1 L1^T, Q1 = W L1^-T, then the same
// on Q1; R_W = L2^T L1^T.  The products below are float64 (the responses and
// the basis are float64 data).
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "reduce.h"

namespace glmsur {

namespace {

constexpr int kTM = 64, kTN = 64, kTK = 16;   // output tile and depth step of the float64 product

// One kTM x kTN output tile at (i0, j0): 256 threads, 4 x 4 outputs each; A
// and B tiles staged in shared memory.
__device__ __forceinline__ void dgemm_tile(int i0, int j0, int m, int n, int64_t kdim, const double* __restrict__ A,
                                           int64_t ars, int64_t acs, const double* __restrict__ B, int64_t brs,
                                           int64_t bcs, double* __restrict__ C, int64_t crs, int64_t ccs) {
  __shared__ double As[kTK][kTM + 1];
  __shared__ double Bs[kTK][kTN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int64_t p0 = 0; p0 < kdim; p0 += kTK) {
    // the depth index runs fastest across threads: unit-stride operands load coalesced
    for (int e = threadIdx.x; e < kTK * kTM; e += 256) {
      const int pp = e % kTK, ii = e / kTK;
      const int64_t p = p0 + pp;
      const int i = i0 + ii;
      As[pp][ii] = (i < m && p < kdim) ? A[(int64_t)i * ars + p * acs] : 0.0;
    }
    for (int e = threadIdx.x; e < kTK * kTN; e += 256) {
      const int pp = e % kTK, jj = e / kTK;
      const int64_t p = p0 + pp;
      const int j = j0 + jj;
      Bs[pp][jj] = (j < n && p < kdim) ? B[p * brs + (int64_t)j * bcs] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int pp = 0; pp < kTK; ++pp) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[pp][ty * 4 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[pp][tx * 4 + c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] += a[r] * b[c];
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty * 4 + r;
    if (i >= m) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx * 4 + c;
      if (j < n) C[(int64_t)i * crs + (int64_t)j * ccs] = acc[r][c];
    }
  }
}

__global__ void __launch_bounds__(256)
k_dgemm(int m, int n, int64_t kdim, const double* __restrict__ A, int64_t ars, int64_t acs,
        const double* __restrict__ B, int64_t brs, int64_t bcs, double* __restrict__ C, int64_t crs, int64_t ccs) {
  dgemm_tile(blockIdx.y * kTM, blockIdx.x * kTN, m, n, kdim, A, ars, acs, B, brs, bcs, C, crs, ccs);
}

// Depth-split product: CTA (x, y, z) computes tile (y, x) over depth chunk z
// into ws[z] (m x n row-major); the chunks are summed by k_dgemm_sum.
__global__ void __launch_bounds__(256)
k_dgemm_split(int m, int n, int64_t kdim, int64_t kc, const double* __restrict__ A, int64_t ars, int64_t acs,
              const double* __restrict__ B, int64_t brs, int64_t bcs, double* __restrict__ ws) {
  const int64_t p0 = (int64_t)blockIdx.z * kc;
  const int64_t len = kdim - p0 < kc ? kdim - p0 : kc;
  dgemm_tile(blockIdx.y * kTM, blockIdx.x * kTN, m, n, len, A + p0 * acs, ars, acs, B + p0 * brs, brs, bcs,
             ws + (int64_t)blockIdx.z * m * n, n, 1);
}

// C(i, j) = sum over the chunks z = 0, 1, ... of ws[z](i, j) (fixed order)
__global__ void k_dgemm_sum(int m, int n, int nz, const double* __restrict__ ws, double* __restrict__ C, int64_t crs,
                            int64_t ccs) {
  const int64_t mn = (int64_t)m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < mn; e += (int64_t)gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int z = 0; z < nz; ++z) t += ws[z * mn + e];
    const int64_t i = e / n, j = e - i * n;
    C[i * crs + j * ccs] = t;
  }
}

// grid (tiles, problems): CTA (t, q) computes tile t of problem q (row-major
// over its tiles), or nothing when problem q has fewer tiles
__global__ void __launch_bounds__(256) k_dgemm_batched(const DgemmProblem* __restrict__ probs) {
  const DgemmProblem pr = probs[blockIdx.y];
  const int tn = (int)ceil_div(pr.n, kTN), tm = (int)ceil_div(pr.m, kTM);
  const int t = blockIdx.x;
  if (pr.m < 1 || pr.n < 1 || t >= tm * tn) return;
  dgemm_tile((t / tn) * kTM, (t % tn) * kTN, pr.m, pr.n, pr.kdim, pr.A, pr.ars, pr.acs, pr.B, pr.brs, pr.bcs, pr.C,
             pr.crs, pr.ccs);
}

// Column j of L^-1 (forward substitution L y = e_j; one CTA per column).
__global__ void __launch_bounds__(256) k_tri_inverse_cols(int n, const double* __restrict__ L,
                                                          double* __restrict__ Linv) {
  extern __shared__ double y[];
  __shared__ double red[8];
  const int j = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = 0.0;
  __syncthreads();
  for (int i = j; i < n; ++i) {
    double part = 0.0;
    for (int s = j + threadIdx.x; s < i; s += blockDim.x) part += L[(int64_t)i * n + s] * y[s];
    part = warp_sum(part);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      y[i] = ((i == j ? 1.0 : 0.0) - t) / L[(int64_t)i * n + i];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) Linv[(int64_t)i * n + j] = y[i];
}

__global__ void k_zero_upper(int n, double* __restrict__ A) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  if (j > i) A[idx] = 0.0;
}

}  // namespace

int dgemm_split(int m, int n, int64_t kdim, int sms) {
  const int64_t tiles = ceil_div(m, kTM) * ceil_div(n, kTN);
  int64_t z = ceil_div((int64_t)16 * sms, tiles);   // about 16 CTAs per SM
  z = std::min<int64_t>(z, 32);
  z = std::min<int64_t>(z, kdim / 512);              // chunks of at least 512
  return (int)std::max<int64_t>(z, 1);
}

void launch_dgemm(int m, int n, int64_t kdim, const double* A, int64_t ars, int64_t acs, const double* B,
                  int64_t brs, int64_t bcs, double* C, int64_t crs, int64_t ccs, cudaStream_t s, double* ws,
                  int nz) {
  if (ws != nullptr && nz > 1) {
    const int64_t kc = ceil_div(ceil_div(kdim, nz), kTK) * kTK;
    const int z = (int)ceil_div(kdim, kc);
    k_dgemm_split<<<dim3((unsigned)ceil_div(n, kTN), (unsigned)ceil_div(m, kTM), (unsigned)z), 256, 0, s>>>(
        m, n, kdim, kc, A, ars, acs, B, brs, bcs, ws);
    const int64_t mn = (int64_t)m * n;
    k_dgemm_sum<<<(unsigned)std::min<int64_t>(ceil_div(mn, 256), 152 * 8), 256, 0, s>>>(m, n, z, ws, C, crs, ccs);
    return;
  }
  dim3 grid((unsigned)ceil_div(n, kTN), (unsigned)ceil_div(m, kTM));
  k_dgemm<<<grid, 256, 0, s>>>(m, n, kdim, A, ars, acs, B, brs, bcs, C, crs, ccs);
}

int dgemm_tiles(int m, int n) { return (int)(ceil_div(m, kTM) * ceil_div(n, kTN)); }

void launch_dgemm_batched(const DgemmProblem* probs, int count, int max_tiles, cudaStream_t s) {
  if (count < 1 || max_tiles < 1) return;
  k_dgemm_batched<<<dim3((unsigned)max_tiles, (unsigned)count), 256, 0, s>>>(probs);
}

cudaError_t launch_tri_inverse(int n, const double* L, double* Linv, cudaStream_t s) {
  const size_t smem = sizeof(double) * (size_t)n;
  cudaError_t e = cudaFuncSetAttribute(k_tri_inverse_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_tri_inverse_cols<<<n, 256, smem, s>>>(n, L, Linv);
  return cudaGetLastError();
}

void launch_zero_upper(int n, double* A, cudaStream_t s) {
  k_zero_upper<<<(unsigned)ceil_div((int64_t)n * n, 256), 256, 0, s>>>(n, A);
}


namespace {

// part[j G + i] = s_i^2 (||y_ij||^2 - ||Q^T y_ij||^2): one CTA per (equation, rhs)
__global__ void __launch_bounds__(256)
k_complement_energy(int G, int64_t M, int64_t n, const double* __restrict__ Y, int64_t ldy,
                    const double* __restrict__ Yr, const double* __restrict__ isq, double* __restrict__ part) {
  __shared__ double red[256];
  const int i = blockIdx.x, j = blockIdx.y;
  const double* y = Y + (int64_t)j * ldy + (int64_t)i * M;
  const double* yr = Yr + ((int64_t)j * G + i) * n;
  double a = 0.0;
  for (int64_t t = threadIdx.x; t < M; t += 256) a += y[t] * y[t];
  for (int64_t t = threadIdx.x; t < n; t += 256) a -= yr[t] * yr[t];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(int64_t)j * G + i] = isq ? red[0] * isq[i] * isq[i] : red[0];
}

__global__ void k_complement_sum(int G, int k, const double* __restrict__ part, double* __restrict__ out) {
  const int j = threadIdx.x;
  if (j >= k) return;
  double t = 0.0;
  for (int i = 0; i < G; ++i) t += part[(int64_t)j * G + i];
  out[j] = t > 0.0 ? t : 0.0;
}

}  // namespace

void launch_complement_energy(int G, int64_t M, int64_t n, int k, const double* Y, int64_t ldy, const double* Yr,
                              const double* isq, double* part, double* out, cudaStream_t s) {
  k_complement_energy<<<dim3((unsigned)G, (unsigned)k), 256, 0, s>>>(G, M, n, Y, ldy, Yr, isq, part);
  k_complement_sum<<<1, 64, 0, s>>>(G, k, part, out);
}

}  // namespace glmsur
