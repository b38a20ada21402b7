// Batched solves: many independent SUR instances of uneven G, M and n_i, each
// with K right-hand sides, in one persistent launch.  CTAs take instances
// from an atomic work counter; one CTA runs the whole estimate of one
// instance on its own (float32 PCG-Aug steps of Algorithm glmpcg2 inside a
// float64 iterative-refinement loop, then b = X*^T (y - Sigma w)), so every
// reduction of the method is a CTA-level reduction and no CTA ever waits for
// another.  The setup (TSQR of all blocks of all instances) reuses the
// single-instance kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "batch.h"
#include "common.cuh"
#include "internal.h"

namespace glmsur {

namespace {

constexpr int kBT = 256;          // threads per CTA
constexpr int kPairsPerThread = 4;

// Shared memory of one CTA (carved from dynamic shared memory; sizes follow
// the largest instance of the batch).
struct Smem {
  double* om64;    // G x Gq
  float* om32;
  int* n_i;        // G
  int* poff;       // G + 1
  int* r_loc;      // G
  double* red;     // (kBT / 32) * K
  double* colv;    // 4 * K
  double* tile64;  // kTR x G x K
  float* tile32;   // 2 x kTR x G x K
  double* e64;     // np x K
  float* e32;      // np x K
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline size_t smem_bytes(int K, int kTR, int maxG, int maxNp) {
  size_t b = 0;
  b += align16(sizeof(double) * maxG * ((maxG + 3) & ~3));
  b += align16(sizeof(float) * maxG * ((maxG + 3) & ~3));
  b += align16(sizeof(int) * maxG) * 2 + align16(sizeof(int) * (maxG + 1));
  b += align16(sizeof(double) * (kBT / 32) * K) + align16(sizeof(double) * 4 * K);
  b += align16(sizeof(double) * kTR * maxG * K) + align16(sizeof(float) * 2 * kTR * maxG * K);
  b += align16(sizeof(double) * maxNp * K) + align16(sizeof(float) * maxNp * K);
  return b;
}

__device__ inline Smem carve(unsigned char* base, int K, int kTR, int maxG, int maxNp) {
  Smem s;
  size_t o = 0;
  const int Gq = (maxG + 3) & ~3;
  s.om64 = reinterpret_cast<double*>(base + o); o += align16(sizeof(double) * maxG * Gq);
  s.om32 = reinterpret_cast<float*>(base + o); o += align16(sizeof(float) * maxG * Gq);
  s.n_i = reinterpret_cast<int*>(base + o); o += align16(sizeof(int) * maxG);
  s.r_loc = reinterpret_cast<int*>(base + o); o += align16(sizeof(int) * maxG);
  s.poff = reinterpret_cast<int*>(base + o); o += align16(sizeof(int) * (maxG + 1));
  s.red = reinterpret_cast<double*>(base + o); o += align16(sizeof(double) * (kBT / 32) * K);
  s.colv = reinterpret_cast<double*>(base + o); o += align16(sizeof(double) * 4 * K);
  s.tile64 = reinterpret_cast<double*>(base + o); o += align16(sizeof(double) * kTR * maxG * K);
  s.tile32 = reinterpret_cast<float*>(base + o); o += align16(sizeof(float) * 2 * kTR * maxG * K);
  s.e64 = reinterpret_cast<double*>(base + o); o += align16(sizeof(double) * maxNp * K);
  s.e32 = reinterpret_cast<float*>(base + o);
  return s;
}

// Deterministic CTA sum where thread t holds a value of column t % K (every
// loop below strides by kBT, a multiple of K, so a thread's column is fixed);
// out[j] for j < K, visible to all threads on return.
template <int K>
__device__ void cta_sum_strided(double v, double* red, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off >= K; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __syncthreads();
  if (lane < K) red[warp * K + lane] = v;
  __syncthreads();
  if (threadIdx.x < K) {
    double t = 0.0;
    for (int w = 0; w < kBT / 32; ++w) t += red[w * K + threadIdx.x];
    out[threadIdx.x] = t;
  }
  __syncthreads();
}

// One instance, K right-hand sides, by one CTA.
template <int K, int kTR>
struct Inst {
  const BatchInst& d;
  const Smem& sm;
  const BatchPools& P;

  __device__ int G() const { return d.G; }
  __device__ int64_t GK() const { return (int64_t)d.G * K; }

  // Accumulate acc(pair) += sum_{rows of tile} Q[t, 4q+c] * tile[r][blk(q)][j]
  // for the thread's (quad, column) pairs.
  template <typename TQ, typename TT, typename TA>
  __device__ void accumulate(const TQ* Q, const TT* tile, int64_t t0, int tr, TA (&acc)[kPairsPerThread][4]) const {
    const int npairs = d.nq * K;
#pragma unroll
    for (int a = 0; a < kPairsPerThread; ++a) {
      const int pr = threadIdx.x + a * kBT;
      if (pr < npairs) {
        const int q = pr / K, j = pr % K;
        const int blk = P.quad_blk[d.quad0 + q];
        for (int r = 0; r < tr; ++r) {
          const TQ* qp = Q + d.q_off + (t0 + r) * d.np + 4 * q;
          const TA sv = (TA)tile[((int64_t)r * d.G + blk) * K + j];
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[a][c] += (TA)qp[c] * sv;
        }
      }
    }
  }

  // Write the accumulators to e (np x K) in shared memory.
  template <typename TA, typename TE>
  __device__ void store_acc(TA (&acc)[kPairsPerThread][4], TE* e) const {
    const int npairs = d.nq * K;
#pragma unroll
    for (int a = 0; a < kPairsPerThread; ++a) {
      const int pr = threadIdx.x + a * kBT;
      if (pr < npairs) {
        const int q = pr / K, j = pr % K;
#pragma unroll
        for (int c = 0; c < 4; ++c) e[(4 * q + c) * K + j] = (TE)acc[a][c];
      }
    }
  }

  // (Q e)[t, i, j] = sum over block i's columns
  template <typename TQ, typename TE>
  __device__ TE qe(const TQ* Q, const TE* e, int64_t t, int i, int j) const {
    const TQ* qp = Q + d.q_off + t * d.np + sm.poff[i];
    const TE* ep = e + sm.poff[i] * K + j;
    TE s = 0;
    for (int c = 0; c < sm.n_i[i]; ++c) s += (TE)qp[c] * ep[c * K];
    return s;
  }
};

template <int K, int kTR>
__device__ void solve_instance(const BatchInst& dsc, const BatchPools& P, const BatchOpts& o, const Smem& sm) {
  Inst<K, kTR> I{dsc, sm, P};
  double* tile64 = sm.tile64;
  float* tile32 = sm.tile32;
  double* e64 = sm.e64;
  float* e32 = sm.e32;
  const int G = dsc.G, Gq = dsc.Gq;
  const int64_t M = dsc.M, GK = (int64_t)G * K;
  const int64_t nv = M * GK;
  const int tid = threadIdx.x;
  // instance constants in shared memory
  for (int e = tid; e < G * Gq; e += kBT) {
    sm.om64[e] = P.om64[dsc.om_off + e];
    sm.om32[e] = P.om32[dsc.om_off + e];
  }
  for (int i = tid; i < G; i += kBT) {
    sm.n_i[i] = P.n_i[dsc.blk0 + i];
    sm.poff[i] = P.poff[dsc.blk0 + i];
    sm.r_loc[i] = (int)(P.r_off[dsc.blk0 + i] - P.r_off[dsc.blk0]);
  }
  if (tid == 0) sm.poff[G] = dsc.np;
  double* w64 = P.w64 + dsc.v_off;
  double* E64 = P.E64 + dsc.v_off;
  double* d64 = P.d64 + dsc.v_off;
  float* g32 = P.g32 + dsc.v_off;
  float* u32 = P.u32 + dsc.v_off;
  float* w32 = P.w32 + dsc.v_off;
  float* wb32 = P.wb32 + dsc.v_off;   // best-iterate snapshots of the inner solves
  const double* Y = P.Y + dsc.y_off;   // column-major m x K, ld = m
  const int64_t m = M * G;
  for (int64_t e = tid; e < nv; e += kBT) w64[e] = 0.0;
  __shared__ double rho0[kBatchMaxK], prev[kBatchMaxK], rrout[kBatchMaxK];
  __shared__ int fin[kBatchMaxK], live[kBatchMaxK], revert[kBatchMaxK], iters_acc[kBatchMaxK];
  if (tid < K) { fin[tid] = kStatusRunning; iters_acc[tid] = 0; rrout[tid] = 1.0; }
  __syncthreads();

  for (int outer = 0;; ++outer) {
    // ---- float64 residual rho = P (y - Sigma w64): E = y - W Omega ; e = Q^T E ; rho = E - Q e
    double acc64[kPairsPerThread][4] = {};
    for (int64_t t0 = 0; t0 < M; t0 += kTR) {
      const int tr = (int)((M - t0) < kTR ? (M - t0) : kTR);
      for (int e = tid; e < tr * GK; e += kBT) {
        const int j = e % K, rest = e / K, h = rest % G, r = rest / G;
        const int64_t t = t0 + r;
        double s = 0.0;
        for (int gg = 0; gg < G; ++gg) s += w64[(t * G + gg) * K + j] * sm.om64[gg * Gq + h];
        const double ev = Y[(int64_t)j * m + (int64_t)h * M + t] - s;
        tile64[e] = ev;
        E64[t * GK + h * K + j] = ev;
      }
      __syncthreads();
      I.accumulate(P.q64, tile64, t0, tr, acc64);
      __syncthreads();
    }
    I.store_acc(acc64, e64);
    __syncthreads();
    double nrm = 0.0;
    for (int64_t e = tid; e < nv; e += kBT) {
      const int j = (int)(e % K), h = (int)((e / K) % G);
      const int64_t t = e / GK;
      const double rho = E64[e] - I.qe(P.q64, e64, t, h, j);
      nrm += rho * rho;
      g32[e] = (float)(-rho);
    }
    cta_sum_strided<K>(nrm, sm.red, sm.colv);
    // ---- per-column decisions (reference: the single-instance refinement loop)
    if (tid < K) {
      const int j = tid;
      const double cur = sqrt(sm.colv[j]);
      revert[j] = 0;
      if (outer == 0) rho0[j] = cur;
      if (fin[j] == kStatusRunning) {
        const double rr = rho0[j] > 0 ? cur / rho0[j] : 0.0;
        if (!isfinite(cur)) fin[j] = GLM_SUR_NONFINITE;
        else if (outer > 0 && cur >= prev[j]) {
          revert[j] = 1;
          fin[j] = (rrout[j] <= o.tol) ? GLM_SUR_OK : GLM_SUR_STAGNATED;
        } else {
          rrout[j] = rr;
          const bool floor = outer > 0 && cur > kRefineMinGain * prev[j];
          prev[j] = cur;
          if (rr <= o.tol) fin[j] = GLM_SUR_OK;
          else if (floor) fin[j] = GLM_SUR_STAGNATED;
          else if (outer >= o.max_refine) fin[j] = GLM_SUR_NOT_CONVERGED;
        }
      }
      live[j] = fin[j] == kStatusRunning;
    }
    __syncthreads();
    int any_live = 0, any_rev = 0;
    for (int j = 0; j < K; ++j) { any_live |= live[j]; any_rev |= revert[j]; }
    if (any_rev)
      for (int64_t e = tid; e < nv; e += kBT)
        if (revert[e % K]) w64[e] -= d64[e];
    __syncthreads();
    if (!any_live) break;
    // ---- inner float32 PCG on P Sigma delta = rho (live columns)
    for (int64_t e = tid; e < nv; e += kBT) {
      if (!live[e % K]) g32[e] = 0.f;
      u32[e] = 0.f;
      w32[e] = 0.f;
      wb32[e] = 0.f;
    }
    double c1[K], c[K], cbest[K], csnap[K], cstop[K];
    int ibest[K], act[K], it_done[K], snap[K], conv[K];
    {
      double cs = 0.0;
      __syncthreads();
      for (int64_t e = tid; e < nv; e += kBT) cs += (double)g32[e] * (double)g32[e];
      cta_sum_strided<K>(cs, sm.red, sm.colv + K);
#pragma unroll
      for (int j = 0; j < K; ++j) {
        c1[j] = c[j] = cbest[j] = csnap[j] = cstop[j] = sm.colv[K + j];
        ibest[j] = 0;
        act[j] = (c1[j] > 0.0) && isfinite(c1[j]);
        it_done[j] = 0;
        snap[j] = 0;
        conv[j] = 0;
      }
    }
    double mu[K] = {};
    for (int it = 1; it <= o.inner_maxit; ++it) {
      int anyact = 0;
#pragma unroll
      for (int j = 0; j < K; ++j) anyact |= act[j];
      if (!anyact) break;
      // pass A: u = g + mu u ; S = U Omega ; d = u.S ; e = Q^T S
      float acc32[kPairsPerThread][4] = {};
      double dd = 0.0;
      for (int64_t t0 = 0; t0 < M; t0 += kTR) {
        const int tr = (int)((M - t0) < kTR ? (M - t0) : kTR);
        for (int e = tid; e < tr * GK; e += kBT) {
          const int j = e % K;
          const int64_t gi = t0 * GK + e;
          float un = u32[gi];
          if (act[j]) {
            un = g32[gi] + (float)mu[j] * un;
            u32[gi] = un;
          }
          tile32[e] = un;     // u tile
        }
        __syncthreads();
        // S tile into the second half of tile32, d partials
        float* St = tile32 + kTR * GK;
        for (int e = tid; e < tr * GK; e += kBT) {
          const int j = e % K, rest = e / K, h = rest % G, r = rest / G;
          float s = 0.f;
          for (int gg = 0; gg < G; ++gg) s += tile32[(r * G + gg) * K + j] * sm.om32[gg * Gq + h];
          St[e] = s;
          dd += (double)(s * tile32[e]);
        }
        __syncthreads();
        I.accumulate(P.q32, St, t0, tr, acc32);
        __syncthreads();
      }
      I.store_acc(acc32, e32);
      cta_sum_strided<K>(dd, sm.red, sm.colv + 2 * K);
      double lam[K];
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const double dj = sm.colv[2 * K + j];
        lam[j] = 0.0;
        if (act[j]) {
          if (!(dj > 0.0) || !isfinite(dj)) act[j] = 0;
          else lam[j] = c[j] / dj;
        }
      }
      // pass B: t = S - Q e ; g -= lam t ; w -= lam u ; c' = g.g
      double cn = 0.0;
      for (int64_t t0 = 0; t0 < M; t0 += kTR) {
        const int tr = (int)((M - t0) < kTR ? (M - t0) : kTR);
        for (int e = tid; e < tr * GK; e += kBT) tile32[e] = u32[t0 * GK + e];
        __syncthreads();
        for (int e = tid; e < tr * GK; e += kBT) {
          const int j = e % K, rest = e / K, h = rest % G, r = rest / G;
          const int64_t gi = t0 * GK + e;
          float s = 0.f;
          for (int gg = 0; gg < G; ++gg) s += tile32[(r * G + gg) * K + j] * sm.om32[gg * Gq + h];
          const float tval = s - I.qe(P.q32, e32, t0 + r, h, j);
          const float gn = g32[gi] - (float)lam[j] * tval;
          g32[gi] = gn;
          const float wo = w32[gi];
          if (snap[j]) wb32[gi] = wo;   // the w whose c was a new quarter-low
          w32[gi] = wo - (float)lam[j] * tile32[e];
          cn += (double)(gn * gn);
        }
        __syncthreads();
      }
      cta_sum_strided<K>(cn, sm.red, sm.colv + 3 * K);
#pragma unroll
      for (int j = 0; j < K; ++j) {
        snap[j] = 0;
        if (!act[j]) { mu[j] = 0.0; continue; }
        const double cj = sm.colv[3 * K + j];
        it_done[j] = it;
        cstop[j] = cj;
        if (cj < cbest[j]) { cbest[j] = cj; ibest[j] = it; }
        const bool done_conv = isfinite(cj) && cj >= 0.0 && sqrt(cj / c1[j]) <= o.inner_tol;
        if (done_conv || !isfinite(cj) || cj < 0.0 || it - ibest[j] >= o.inner_window || it >= o.inner_maxit) {
          act[j] = 0;
          mu[j] = 0.0;
          conv[j] = done_conv;
        } else {
          if (cj < 0.25 * csnap[j]) { csnap[j] = cj; snap[j] = 1; }   // saved in the next pass B
          mu[j] = cj / c[j];
          c[j] = cj;
        }
      }
    }
    // columns that stopped without converging take their saved best w
    {
      int any_restore = 0;
#pragma unroll
      for (int j = 0; j < K; ++j) any_restore |= (!conv[j] && !(cstop[j] <= csnap[j]));
      if (any_restore) {
        for (int64_t e = tid; e < nv; e += kBT) {
          const int j = (int)(e % K);
          if (!conv[j] && !(cstop[j] <= csnap[j])) w32[e] = wb32[e];
        }
        __syncthreads();
      }
    }
    if (tid < K) iters_acc[tid] += it_done[tid];
    // ---- d = P (double) w32 ; w64 += d on the live columns
    double accp[kPairsPerThread][4] = {};
    for (int64_t t0 = 0; t0 < M; t0 += kTR) {
      const int tr = (int)((M - t0) < kTR ? (M - t0) : kTR);
      for (int e = tid; e < tr * GK; e += kBT) tile64[e] = (double)w32[t0 * GK + e];
      __syncthreads();
      I.accumulate(P.q64, tile64, t0, tr, accp);
      __syncthreads();
    }
    I.store_acc(accp, e64);
    __syncthreads();
    for (int64_t e = tid; e < nv; e += kBT) {
      const int j = (int)(e % K), h = (int)((e / K) % G);
      const int64_t t = e / GK;
      const double dv = live[j] ? (double)w32[e] - I.qe(P.q64, e64, t, h, j) : 0.0;
      d64[e] = dv;
      w64[e] += dv;
    }
    __syncthreads();
  }
  // ---- b = R^-1 Q^T (y - Sigma w64)
  double accb[kPairsPerThread][4] = {};
  for (int64_t t0 = 0; t0 < M; t0 += kTR) {
    const int tr = (int)((M - t0) < kTR ? (M - t0) : kTR);
    for (int e = tid; e < tr * GK; e += kBT) {
      const int j = e % K, rest = e / K, h = rest % G, r = rest / G;
      const int64_t t = t0 + r;
      double s = 0.0;
      for (int gg = 0; gg < G; ++gg) s += w64[(t * G + gg) * K + j] * sm.om64[gg * Gq + h];
      tile64[e] = Y[(int64_t)j * m + (int64_t)h * M + t] - s;
    }
    __syncthreads();
    I.accumulate(P.q64, tile64, t0, tr, accb);
    __syncthreads();
  }
  I.store_acc(accb, e64);
  __syncthreads();
  const double* Rb = P.R + P.r_off[dsc.blk0];
  for (int id = tid; id < G * K; id += kBT) {
    const int i = id / K, j = id % K;
    const int ni = sm.n_i[i];
    const double* Ri = Rb + sm.r_loc[i];
    double x[kBatchMaxCols];
    for (int r = ni - 1; r >= 0; --r) {
      double s = e64[(sm.poff[i] + r) * K + j];
      for (int cc = r + 1; cc < ni; ++cc) s -= Ri[r * ni + cc] * x[cc];
      x[r] = s / Ri[r * ni + r];
    }
    int offi = 0;
    for (int q = 0; q < i; ++q) offi += sm.n_i[q];
    for (int r = 0; r < ni; ++r) P.b[dsc.b_off + (int64_t)j * dsc.n + offi + r] = x[r];
  }
  if (tid < K) {
    P.status[(int64_t)dsc.index * K + tid] = fin[tid];
    P.iters[(int64_t)dsc.index * K + tid] = iters_acc[tid];
    P.relres[(int64_t)dsc.index * K + tid] = rrout[tid];
  }
  __syncthreads();
}

template <int K, int kTR>
__global__ void __launch_bounds__(kBT)
k_batch_solve(const BatchInst* __restrict__ insts, int count, BatchPools P, BatchOpts o, int* counter, int maxG,
              int maxNp) {
  extern __shared__ __align__(128) unsigned char smraw[];
  const Smem sm = carve(smraw, K, kTR, maxG, maxNp);
  __shared__ int next;
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(counter, 1);
    __syncthreads();
    const int idx = next;
    __syncthreads();
    if (idx >= count) return;
    const BatchInst d = insts[idx];
    solve_instance<K, kTR>(d, P, o, sm);
  }
}

}  // namespace

template <int K, int TR>
static cudaError_t launch_k(const BatchInst* insts, int count, const BatchPools& P, const BatchOpts& o, int* counter,
                            int grid, int maxG, int maxNp, cudaStream_t s) {
  const size_t smem = smem_bytes(K, TR, maxG, maxNp);
  k_batch_solve<K, TR><<<grid, kBT, smem, s>>>(insts, count, P, o, counter, maxG, maxNp);
  return cudaGetLastError();
}

template <int K, int TR>
static cudaError_t prep_k(int maxG, int maxNp, int* ctas) {
  const size_t smem = smem_bytes(K, TR, maxG, maxNp);
  cudaError_t e = cudaFuncSetAttribute(k_batch_solve<K, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_batch_solve<K, TR>, kBT, smem);
}

#define GS_BATCH_DISPATCH(K, TR, CALL)                          \
  switch (K * 100 + TR) {                                       \
    case 108: return CALL(1, 8);                                \
    case 116: return CALL(1, 16);                               \
    case 132: return CALL(1, 32);                               \
    case 208: return CALL(2, 8);                                \
    case 216: return CALL(2, 16);                               \
    case 232: return CALL(2, 32);                               \
    case 408: return CALL(4, 8);                                \
    case 416: return CALL(4, 16);                               \
    case 432: return CALL(4, 32);                               \
    case 808: return CALL(8, 8);                                \
    case 816: return CALL(8, 16);                               \
    case 832: return CALL(8, 32);                               \
    default: return cudaErrorInvalidValue;                      \
  }

cudaError_t batch_prepare(int K, int TR, int maxG, int maxNp, int* ctas_per_sm) {
#define C_(k, t) prep_k<k, t>(maxG, maxNp, ctas_per_sm)
  GS_BATCH_DISPATCH(K, TR, C_)
#undef C_
}

cudaError_t batch_solve_launch(int K, int TR, const BatchInst* insts, int count, const BatchPools& P,
                               const BatchOpts& o, int* counter, int grid, int maxG, int maxNp, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
#define C_(k, t) launch_k<k, t>(insts, count, P, o, counter, grid, maxG, maxNp, s)
  GS_BATCH_DISPATCH(K, TR, C_)
#undef C_
}

}  // namespace glmsur
