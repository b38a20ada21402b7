// Adjoint of the augmented system (eq. (aug1)) for a loss L(b).
//
// K = [[Sigma, X], [X^T, 0]] is symmetric, so (lam; mu) = K^-1 (0; dL/db)
// gives dL/dy = lam and dL/dK = -(lam; mu)(w; b)^T.  lam is found with the
// forward machinery: lam_1 = Q_i R_i^-T (dL/db)_i satisfies X^T lam_1 = dL/db,
// and lam_2 = lam - lam_1 solves eq. (aug1) with y' = -Sigma lam_1 (w-part in
// null(X^T)), i.e. the same PCG-Aug iteration.  Sigma = Omega (x) I_M puts
// omega_ab on the diagonal of block (a, b), so
//   dL/domega_ab = -sum_t sum_j Lam[t, a, j] W[t, b, j],
// a G x G reduction over the M rows and k right-hand sides.
#include <cuda_runtime.h>

#include <algorithm>

#include "adjoint.h"
#include "common.cuh"

namespace glmsur {

namespace {

constexpr int kOmTile = 32;     // output tile of the Omega gradient (32 x 32)
constexpr int kOmPairs = 32;    // (row, rhs) pairs staged per pass

// z_i = s_i R_i^-T g_i (forward substitution, R_i row-major upper
// triangular; s_i = blk_scale[i], or 1 when blk_scale is null), written to
// the padded coefficient layout C[(poff_i + r) * k + j] with the pad columns
// of block i set to zero.  One thread per (block, rhs).
__global__ void k_adj_seed(int G, int k, const double* __restrict__ R, const int64_t* __restrict__ r_off,
                           const int* __restrict__ n_i, const int* __restrict__ off, const int* __restrict__ poff,
                           const double* __restrict__ gb, int64_t ldg, const double* __restrict__ blk_scale,
                           double* __restrict__ C) {
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= G * k) return;
  const int i = id / k, j = id % k;
  const int ni = n_i[i];
  const double* Ri = R + r_off[i];
  double z[kMaxBlockCols];
  for (int r = 0; r < ni; ++r) {
    double s = gb[(int64_t)j * ldg + off[i] + r];
    for (int c = 0; c < r; ++c) s -= Ri[c * ni + r] * z[c];
    z[r] = s / Ri[r * ni + r];
  }
  const double sc = blk_scale ? blk_scale[i] : 1.0;
  const int w = poff[i + 1] - poff[i];
  for (int r = 0; r < w; ++r) C[(int64_t)(poff[i] + r) * k + j] = r < ni ? sc * z[r] : 0.0;
}

// part[ch][a][b] = sum over the (t, j) pairs of chunk ch of Lam[t,a,j] W[t,b,j]
// grid (tiles of a, tiles of b, chunks); 256 threads, 4 outputs each.
__global__ void __launch_bounds__(256)
k_adj_omega_partial(int64_t M, int G, int k, int64_t chunk, const double* __restrict__ Lam,
                    const double* __restrict__ W, double* __restrict__ part) {
  __shared__ double Ls[kOmPairs][kOmTile + 1];
  __shared__ double Ws[kOmPairs][kOmTile + 1];
  const int a0 = blockIdx.x * kOmTile, b0 = blockIdx.y * kOmTile;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;   // ty: 8 row groups of 4
  const int64_t P = M * k;
  const int64_t p0 = (int64_t)blockIdx.z * chunk;
  const int64_t p1 = p0 + chunk < P ? p0 + chunk : P;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t pb = p0; pb < p1; pb += kOmPairs) {
    for (int e = tid; e < kOmPairs * kOmTile; e += 256) {
      const int pr = e / kOmTile, x = e % kOmTile;
      const int64_t p = pb + pr;
      double lv = 0.0, wv = 0.0;
      if (p < p1) {
        const int64_t t = p / k;
        const int j = (int)(p - t * k);
        if (a0 + x < G) lv = Lam[(t * G + a0 + x) * k + j];
        if (b0 + x < G) wv = W[(t * G + b0 + x) * k + j];
      }
      Ls[pr][x] = lv;
      Ws[pr][x] = wv;
    }
    __syncthreads();
#pragma unroll 8
    for (int pr = 0; pr < kOmPairs; ++pr) {
      const double wv = Ws[pr][tx];
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[r] += Ls[pr][ty * 4 + r] * wv;
    }
    __syncthreads();
  }
  const int b = b0 + tx;
  if (b < G) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int a = a0 + ty * 4 + r;
      if (a < G) part[((int64_t)blockIdx.z * G + a) * G + b] = acc[r];
    }
  }
}

// out[a + b * ldo] = -(1/2) s_a s_b sum_ch (part[ch][a][b] + part[ch][b][a])   (fixed order;
// s = blk_scale, or 1 when it is null)
__global__ void k_adj_omega_reduce(int G, int nch, const double* __restrict__ part, double* __restrict__ out,
                                   int64_t ldo, const double* __restrict__ blk_scale) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)G * G) return;
  const int a = (int)(idx % G), b = (int)(idx / G);
  const int64_t GG = (int64_t)G * G;
  double s = 0.0;
  for (int ch = 0; ch < nch; ++ch) s += part[ch * GG + (int64_t)a * G + b] + part[ch * GG + (int64_t)b * G + a];
  out[(int64_t)b * ldo + a] = blk_scale ? -0.5 * blk_scale[a] * blk_scale[b] * s : -0.5 * s;
}

}  // namespace

void launch_adj_seed(const Geom& gm, int k, const double* R, const double* gb, int64_t ldg, double* C,
                     cudaStream_t s, const double* blk_scale) {
  const int n = gm.G * k;
  k_adj_seed<<<(unsigned)ceil_div(n, 128), 128, 0, s>>>(gm.G, k, R, gm.d_r_off, gm.d_n_i, gm.d_off, gm.d_poff, gb,
                                                       ldg, blk_scale, C);
}

int adj_omega_chunks(const Geom& gm, int k, int sms) {
  const int64_t tiles = ceil_div(gm.G, kOmTile) * ceil_div(gm.G, kOmTile);
  const int64_t pairs = gm.M * k;
  // about two CTAs per SM, each chunk at least a few passes long
  const int64_t want = std::max<int64_t>(1, ceil_div((int64_t)2 * sms, tiles));
  const int64_t most = std::max<int64_t>(1, pairs / (4 * kOmPairs));
  return (int)std::min<int64_t>(want, most);
}

void launch_adj_omega(const Geom& gm, int k, const double* Lam, const double* W, double* part, int nch,
                      double* out, int64_t ldo, cudaStream_t s, const double* blk_scale) {
  const int64_t pairs = gm.M * k;
  const int64_t chunk = ceil_div(ceil_div(pairs, nch), kOmPairs) * kOmPairs;
  const unsigned tg = (unsigned)ceil_div(gm.G, kOmTile);
  k_adj_omega_partial<<<dim3(tg, tg, nch), 256, 0, s>>>(gm.M, gm.G, k, chunk, Lam, W, part);
  const int64_t gg = (int64_t)gm.G * gm.G;
  k_adj_omega_reduce<<<(unsigned)ceil_div(gg, 256), 256, 0, s>>>(gm.G, nch, part, out, ldo, blk_scale);
}

}  // namespace glmsur
