// Linear restrictions C b = d folded into the augmented system (Sec. 4.1):
// eq. (RGLM1setup) Sigma_aug = diag(Omega (x) I_M, 0), X_aug = [(+)X_i; C],
// y_aug = [y; d], preconditioner eq. (invprec) with D = I.  With X_i = Q_i R_i,
// X_aug^T X_aug = (+) R_i^T R_i + C^T C =: N, and (eq. rglm1m with D = I)
//   X*^T xi = N^-1 X_aug^T xi,   Pi xi = xi - X_aug N^-1 X_aug^T xi,
//   X_aug^T xi = [R_i^T Q_i^T xi_i] + C^T xi_C.
// N^-1 is formed once (Cholesky in float64, then its columns by two
// triangular solves); each PCG step then needs, after the usual reduction
// e = Q^T S, the coefficients c = N^-1 [R_i^T e_i], f_i = R_i c_i (so that
// the usual update t = S - Q f applies), and the restriction rows of the
// projected residual, g_C <- g_C + lambda C c.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "rglm.h"

namespace glmsur {

namespace {

// N[a][b] = [blk(a) == blk(b)] (R_i^T R_i)[ra][rb] + sum_c C[c][a] C[c][b]
// (N row-major n x n; C column-major kc x n with leading dimension ldc)
__global__ void k_rglm_normal(int n, int kc, const double* __restrict__ C, int64_t ldc,
                              const int* __restrict__ col_blk, const int* __restrict__ off,
                              const int* __restrict__ n_i, const double* __restrict__ R,
                              const int64_t* __restrict__ r_off, double* __restrict__ N) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  const int a = (int)(idx / n), b = (int)(idx % n);
  double s = 0.0;
  for (int c = 0; c < kc; ++c) s += C[(int64_t)a * ldc + c] * C[(int64_t)b * ldc + c];
  const int ia = col_blk[a];
  if (ia == col_blk[b]) {
    const int ni = n_i[ia], ra = a - off[ia], rb = b - off[ia];
    const double* Ri = R + r_off[ia];
    const int top = ra < rb ? ra : rb;
    for (int q = 0; q <= top; ++q) s += Ri[q * ni + ra] * Ri[q * ni + rb];
  }
  N[idx] = s;
}

// In-place Cholesky N = L L^T (lower triangle of the row-major N), one CTA.
// flag |= 1 when a pivot is not above rel_tol times the largest diagonal
// entry of N (N singular: C and the X_i do not determine b).
__global__ void __launch_bounds__(1024) k_rglm_cholesky(int n, double* __restrict__ N, int* flag, double rel_tol) {
  __shared__ double piv, floor_s;
  if (threadIdx.x == 0) {
    double dmax = 0.0;
    for (int j = 0; j < n; ++j) dmax = fmax(dmax, N[(int64_t)j * n + j]);
    floor_s = rel_tol * dmax;
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      const double v = N[(int64_t)j * n + j];
      piv = (v > floor_s && v > 0.0 && isfinite(v)) ? sqrt(v) : 0.0;
      if (piv == 0.0) atomicOr(flag, 1);
      N[(int64_t)j * n + j] = piv;
    }
    __syncthreads();
    const double p = piv;
    if (p == 0.0) return;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) N[(int64_t)i * n + j] /= p;
    __syncthreads();
    // trailing update of the lower triangle: N[a][b] -= L[a][j] L[b][j],
    // j < b <= a; one warp per row a, lanes over b
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int ga = j + 1 + warp; ga < n; ga += nw) {
      const double la = N[(int64_t)ga * n + j];
      for (int gb = j + 1 + lane; gb <= ga; gb += 32) N[(int64_t)ga * n + gb] -= la * N[(int64_t)gb * n + j];
    }
    __syncthreads();
  }
}

// Column j of N^-1 = L^-T L^-1 e_j (one CTA per column; x in shared memory)
__global__ void __launch_bounds__(256) k_rglm_inverse_cols(int n, const double* __restrict__ L,
                                                           double* __restrict__ Minv) {
  extern __shared__ double x[];
  __shared__ double red[8];
  __shared__ double xi_s;
  const int j = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // forward: L y = e_j  (y_i = 0 for i < j)
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = 0.0;
  __syncthreads();
  for (int i = j; i < n; ++i) {
    double part = 0.0;
    for (int s = j + threadIdx.x; s < i; s += blockDim.x) part += L[(int64_t)i * n + s] * x[s];
    part = warp_sum(part);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      xi_s = ((i == j ? 1.0 : 0.0) - t) / L[(int64_t)i * n + i];
      x[i] = xi_s;
    }
    __syncthreads();
  }
  // backward: L^T z = y
  for (int i = n - 1; i >= 0; --i) {
    double part = 0.0;
    for (int s = i + 1 + threadIdx.x; s < n; s += blockDim.x) part += L[(int64_t)s * n + i] * x[s];
    part = warp_sum(part);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      x[i] = (x[i] - t) / L[(int64_t)i * n + i];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) Minv[(int64_t)i * n + j] = x[i];
}

// Per step (and at the start and the recovery):
//   a = [R_i^T e_i] (+ sign_d C^T d),  c = N^-1 a,  f_i = R_i c_i.
// grid (G, k): CTA (i, j) recomputes a for column j (n values, shared memory),
// forms c over the rows of block i and f_i; writes c (n x k) and f (padded
// n' x k, the layout of the projection coefficients).  When b_out != null the
// CTA writes c to b_out (column-major n x k, ldb) instead (recovery).
__global__ void __launch_bounds__(256) k_rglm_coef(int G, int n, int k, const double* __restrict__ e,
                                                   const int* __restrict__ n_i, const int* __restrict__ off,
                                                   const int* __restrict__ poff, const double* __restrict__ R,
                                                   const int64_t* __restrict__ r_off,
                                                   const double* __restrict__ Minv, const double* __restrict__ Cm,
                                                   int64_t ldc, int kc, const double* __restrict__ d,
                                                   int64_t ldd, double sign_d, double* __restrict__ cbuf,
                                                   double* __restrict__ fbuf, double* __restrict__ b_out,
                                                   int64_t ldb) {
  extern __shared__ double a[];   // n values
  __shared__ double ci[kMaxBlockCols];
  const int i = blockIdx.x, j = blockIdx.y;
  // a = R^T e (+ sign_d C^T d) for column j
  for (int col = threadIdx.x; col < n; col += blockDim.x) a[col] = 0.0;
  __syncthreads();
  for (int bb = 0; bb < G; ++bb) {
    const int nb = n_i[bb], o = off[bb], po = poff[bb];
    const double* Rb = R + r_off[bb];
    for (int r = threadIdx.x; r < nb; r += blockDim.x) {
      double s = 0.0;
      for (int q = 0; q <= r; ++q) s += Rb[q * nb + r] * e[(int64_t)(po + q) * k + j];
      a[o + r] = s;
    }
  }
  __syncthreads();
  if (d != nullptr && kc > 0) {
    for (int col = threadIdx.x; col < n; col += blockDim.x) {
      double s = 0.0;
      for (int c = 0; c < kc; ++c) s += Cm[(int64_t)col * ldc + c] * d[(int64_t)j * ldd + c];
      a[col] += sign_d * s;
    }
    __syncthreads();
  }
  // c over the rows of block i: one warp per row, lanes over n
  const int ni = n_i[i], oi = off[i];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = warp; r < ni; r += nw) {
    const double* mrow = Minv + (int64_t)(oi + r) * n;
    double s = 0.0;
    for (int col = lane; col < n; col += 32) s += mrow[col] * a[col];
    s = warp_sum(s);
    if (lane == 0) ci[r] = s;
  }
  __syncthreads();
  if (b_out != nullptr) {
    for (int r = threadIdx.x; r < ni; r += blockDim.x) b_out[(int64_t)j * ldb + oi + r] = ci[r];
    return;
  }
  for (int r = threadIdx.x; r < ni; r += blockDim.x) cbuf[(int64_t)(oi + r) * k + j] = ci[r];
  const double* Ri = R + r_off[i];
  const int pi = poff[i], nq4 = poff[i + 1] - poff[i];
  for (int r = threadIdx.x; r < nq4; r += blockDim.x) {
    double s = 0.0;
    if (r < ni)
      for (int q = r; q < ni; ++q) s += Ri[r * ni + q] * ci[q];
    fbuf[(int64_t)(pi + r) * k + j] = s;   // padded rows get 0
  }
}

// Restriction rows of the projected residual, one CTA per column j:
//   mode 0 (step):  g_C += lambda_j C c
//   mode 1 (start): g_C  = C c - d
//   mode 2 (start, d = 0): g_C = C c
// and the partial sum ||g_C||^2 into cpart[row * k + j].
__global__ void __launch_bounds__(128) k_rglm_gc(int n, int k, int kc, const double* __restrict__ Cm, int64_t ldc,
                                                 const double* __restrict__ cbuf, const double* __restrict__ d,
                                                 int64_t ldd, const double* __restrict__ lam, int mode,
                                                 double* __restrict__ gC, double* __restrict__ cpart, int row) {
  __shared__ double red[4];
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int c = threadIdx.x; c < kc; c += blockDim.x) {
    double s = 0.0;
    for (int col = 0; col < n; ++col) s += Cm[(int64_t)col * ldc + c] * cbuf[(int64_t)col * k + j];
    double g;
    if (mode == 1) g = s - d[(int64_t)j * ldd + c];
    else if (mode == 2) g = s;
    else g = gC[(int64_t)j * kc + c] + lam[j] * s;
    gC[(int64_t)j * kc + c] = g;
    acc += g * g;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    cpart[(int64_t)row * k + j] = t;
  }
}

}  // namespace

cudaError_t rglm_factor(const Geom& gm, const double* R, const double* C, int64_t ldc, int kc, const int* col_blk,
                        double* N, double* Minv, int* flag, cudaStream_t s) {
  const int n = gm.n;
  k_rglm_normal<<<(unsigned)ceil_div((int64_t)n * n, 256), 256, 0, s>>>(n, kc, C, ldc, col_blk, gm.d_off, gm.d_n_i, R,
                                                                      gm.d_r_off, N);
  k_rglm_cholesky<<<1, 1024, 0, s>>>(n, N, flag, 0.0);
  const size_t smem = sizeof(double) * (size_t)n;
  cudaError_t e = cudaFuncSetAttribute(k_rglm_inverse_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // (set once here, outside any stream capture, for the per-step launches)
  e = cudaFuncSetAttribute(k_rglm_coef, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_rglm_inverse_cols<<<n, 256, smem, s>>>(n, N, Minv);
  return cudaGetLastError();
}

cudaError_t cholesky_lower(int n, double* N, int* flag, double rel_tol, cudaStream_t s) {
  k_rglm_cholesky<<<1, 1024, 0, s>>>(n, N, flag, rel_tol);
  return cudaGetLastError();
}

cudaError_t rglm_coef(const Geom& gm, int k, const double* e, const double* R, const double* Minv, const double* C,
                      int64_t ldc, int kc, const double* d, int64_t ldd, double sign_d, double* cbuf, double* fbuf,
                      double* b_out, int64_t ldb, cudaStream_t s) {
  const size_t smem = sizeof(double) * (size_t)gm.n;
  k_rglm_coef<<<dim3(gm.G, k), 256, smem, s>>>(gm.G, gm.n, k, e, gm.d_n_i, gm.d_off, gm.d_poff, R, gm.d_r_off, Minv,
                                               C, ldc, kc, d, ldd, sign_d, cbuf, fbuf, b_out, ldb);
  return cudaGetLastError();
}

cudaError_t rglm_gc(const Geom& gm, int k, int kc, const double* C, int64_t ldc, const double* cbuf, const double* d,
                    int64_t ldd, const double* lam, int mode, double* gC, double* cpart, int row, cudaStream_t s) {
  k_rglm_gc<<<k, 128, 0, s>>>(gm.n, k, kc, C, ldc, cbuf, d, ldd, lam, mode, gC, cpart, row);
  return cudaGetLastError();
}

}  // namespace glmsur
