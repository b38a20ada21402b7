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
#include "tma.cuh"

namespace glmsur {

namespace {

constexpr int kBT = 512;          // threads per CTA (one CTA per SM: 16 warps)
constexpr int kPairsPerThread = 4;
static_assert(kPairsPerThread * kBT >= kBatchMaxPairs, "every (column quad, rhs) pair needs a thread slot");

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
  double* tile64;  // kTR x G x K           (float64 passes; shares space with ibuf)
  float* tile32;   // 2 x kTR x G x K
  float* ibuf;     // inner passes: 2 stages of [u | g | w | Q] row tiles
  double* e64;     // np x K
  float* e32;      // np x K
  void* qtile;     // kTR x np rows of Q (float64), staged per row tile (shares space with ibuf)
  int maxG, maxNp; // the batch's largest G and n' (the carve's dimensions)
};

// Floats of one inner-pipeline stage: u, g, w tiles (kTR x G x K) and Q rows (kTR x np).
__host__ __device__ inline size_t stage_floats(int K, int kTR, int maxG, int maxNp) {
  return (size_t)3 * kTR * maxG * K + (size_t)kTR * maxNp;
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline size_t smem_bytes(int K, int kTR, int maxG, int maxNp) {
  size_t b = 0;
  b += align16(sizeof(double) * maxG * ((maxG + 3) & ~3));
  b += align16(sizeof(float) * maxG * ((maxG + 3) & ~3));
  b += align16(sizeof(int) * maxG) * 2 + align16(sizeof(int) * (maxG + 1));
  b += align16(sizeof(double) * (kBT / 32) * K) + align16(sizeof(double) * 4 * K);
  b += align16(sizeof(float) * 2 * kTR * maxG * K);
  b += align16(sizeof(double) * maxNp * K) + align16(sizeof(float) * maxNp * K);
  const size_t f64 = align16(sizeof(double) * kTR * maxG * K) + align16(sizeof(double) * kTR * maxNp);
  const size_t pipe = sizeof(float) * 2 * stage_floats(K, kTR, maxG, maxNp);
  b += f64 > pipe ? f64 : pipe;
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
  s.tile32 = reinterpret_cast<float*>(base + o); o += align16(sizeof(float) * 2 * kTR * maxG * K);
  s.e64 = reinterpret_cast<double*>(base + o); o += align16(sizeof(double) * maxNp * K);
  s.e32 = reinterpret_cast<float*>(base + o); o += align16(sizeof(float) * maxNp * K);
  s.tile64 = reinterpret_cast<double*>(base + o);
  s.qtile = base + o + align16(sizeof(double) * kTR * maxG * K);
  s.ibuf = reinterpret_cast<float*>(base + o);
  s.maxG = maxG;
  s.maxNp = maxNp;
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

// Ampere-style asynchronous 16-byte copies global -> shared (no registers
// held while in flight), grouped and awaited with wait_group.
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Start copying n floats src -> dst (both 16-byte aligned, n a multiple of 4
// when vec4): asynchronously in 16-byte pieces, else as plain copies that are
// complete on return.
__device__ __forceinline__ void copy_async(const float* src, float* dst, int n, bool vec4) {
  if (vec4) {
    for (int e = 4 * threadIdx.x; e < n; e += 4 * kBT) cp_async16(dst + e, src + e);
  } else {
    for (int e = threadIdx.x; e < n; e += kBT) dst[e] = __ldcg(src + e);
  }
}

// dst[0..n) = src[0..n) (float32 row tile of a (M, G, K) vector; all
// threads, four vector loads per thread issued before their stores).  With
// K a multiple of 4 every row tile starts on a 16-byte boundary and moves as
// float4, else as scalars.
template <int K>
__device__ __forceinline__ void copy_tile(const float* __restrict__ src, float* __restrict__ dst, int n) {
  if constexpr (K % 4 == 0) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    const int n4 = n >> 2;
    int e = threadIdx.x;
    for (; e + 3 * kBT < n4; e += 4 * kBT) {
      const float4 a = __ldcg(s4 + e), b = __ldcg(s4 + e + kBT), c = __ldcg(s4 + e + 2 * kBT),
                   d = __ldcg(s4 + e + 3 * kBT);
      d4[e] = a; d4[e + kBT] = b; d4[e + 2 * kBT] = c; d4[e + 3 * kBT] = d;
    }
    for (; e < n4; e += kBT) d4[e] = __ldcg(s4 + e);
  } else {
    int e = threadIdx.x;
    for (; e + 3 * kBT < n; e += 4 * kBT) {
      const float a = __ldcg(src + e), b = __ldcg(src + e + kBT), c = __ldcg(src + e + 2 * kBT),
                  d = __ldcg(src + e + 3 * kBT);
      dst[e] = a; dst[e + kBT] = b; dst[e + 2 * kBT] = c; dst[e + 3 * kBT] = d;
    }
    for (; e < n; e += kBT) dst[e] = __ldcg(src + e);
  }
}

// S[e] = sum_g U[r, g, j] Omega[g, h] for the elements e = (r G + h) K + j
// of a row tile (tr rows), four elements per thread in flight; calls
// epi(e, r, h, j, S[e]) for each.  U and S may be float or double.
template <int K, typename T, typename Epi>
__device__ __forceinline__ void sigma_rows(const T* __restrict__ U, int tr, int G, int Gq, const T* __restrict__ om,
                                           Epi epi) {
  const int n = tr * G * K;
  for (int e0 = threadIdx.x; e0 < n; e0 += 4 * kBT) {
    int ub[4], hh[4];
    T sv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int e = e0 + a * kBT < n ? e0 + a * kBT : e0;
      const int j = e % K, rest = e / K, h = rest % G, r = rest / G;
      ub[a] = r * G * K + j;
      hh[a] = h;
      sv[a] = (T)0;
    }
    for (int g = 0; g < G; ++g) {
      const T* om_g = om + g * Gq;
#pragma unroll
      for (int a = 0; a < 4; ++a) sv[a] += U[ub[a] + g * K] * om_g[hh[a]];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int e = e0 + a * kBT;
      if (e < n) epi(e, ub[a] / (G * K), hh[a], ub[a] % K, sv[a]);
    }
  }
}

// float32 form of sigma_rows: a thread item is (row r, column quad hq,
// right-hand side j), j fastest so that a thread keeps one j (kBT is a
// multiple of K); S[r, 4hq..4hq+3, j] = sum_g U[r, g, j] Omega[g, 4hq..]
// takes one shared load of U and one float4 (broadcast) load of an Omega row
// per four FMAs.  Two items per thread in flight.  Calls epi(e, r, h, j, S)
// for every h < G of the item.
template <int K, typename Epi>
__device__ __forceinline__ void sigma_rows4(const float* __restrict__ U, int tr, int G, int Gq,
                                            const float* __restrict__ om, Epi epi) {
  const int nhq = Gq >> 2;
  const int n = tr * nhq * K;
  const int j = threadIdx.x % K;
  for (int i0 = threadIdx.x; i0 < n; i0 += 2 * kBT) {
    int rr[2], h0[2];
    float sv[2][4];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const int item = i0 + a * kBT < n ? i0 + a * kBT : i0;
      const int rest = item / K;
      rr[a] = rest / nhq;
      h0[a] = 4 * (rest - rr[a] * nhq);
#pragma unroll
      for (int c = 0; c < 4; ++c) sv[a][c] = 0.f;
    }
    for (int g = 0; g < G; ++g) {
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const float u = U[(rr[a] * G + g) * K + j];
        const float4 o = *reinterpret_cast<const float4*>(om + g * Gq + h0[a]);
        sv[a][0] += u * o.x;
        sv[a][1] += u * o.y;
        sv[a][2] += u * o.z;
        sv[a][3] += u * o.w;
      }
    }
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      if (i0 + a * kBT < n) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int h = h0[a] + c;
          if (h < G) epi((rr[a] * G + h) * K + j, rr[a], h, j, sv[a][c]);
        }
      }
    }
  }
}

// One instance, K right-hand sides, by one CTA.
template <int K, int kTR>
struct Inst {
  const BatchInst& d;
  const Smem& sm;
  const BatchPools& P;

  __device__ int G() const { return d.G; }
  __device__ int64_t GK() const { return (int64_t)d.G * K; }

  // Copy rows t0 .. t0+tr-1 of the instance's Q (np values each, 16-byte
  // aligned rows) into the shared tile Qt, all threads together.
  template <typename TQ>
  __device__ void stage_q(const TQ* Q, int64_t t0, int tr, TQ* Qt) const {
    using V = typename Vec4<TQ>::type;
    const V* src = reinterpret_cast<const V*>(Q + d.q_off + t0 * d.np);
    V* dst = reinterpret_cast<V*>(Qt);
    const int n = tr * d.nq;
    int e = threadIdx.x;
    for (; e + kBT < n; e += 2 * kBT) {
      V a, b;
      Vec4<TQ>::copy(src + e, &a);
      Vec4<TQ>::copy(src + e + kBT, &b);
      dst[e] = a;
      dst[e + kBT] = b;
    }
    for (; e < n; e += kBT) Vec4<TQ>::copy(src + e, dst + e);
  }

  // Accumulate acc(pair) += sum_{rows of tile} Qt[r, 4q+c] * tile[r][blk(q)][j]
  // for the thread's (quad, column) pairs (Qt: the staged rows of Q).
  template <typename TQ, typename TT, typename TA>
  __device__ void accumulate(const TQ* Qt, const TT* tile, int tr, TA (&acc)[kPairsPerThread][4]) const {
    const int npairs = d.nq * K;
#pragma unroll
    for (int a = 0; a < kPairsPerThread; ++a) {
      const int pr = threadIdx.x + a * kBT;
      if (pr < npairs) {
        const int q = pr / K, j = pr % K;
        const int blk = P.quad_blk[d.quad0 + q];
#pragma unroll 4
        for (int r = 0; r < tr; ++r) {
          TQ qv[4];
          Vec4<TQ>::load(Qt + r * d.np + 4 * q, qv);
          const TA sv = (TA)tile[((int64_t)r * d.G + blk) * K + j];
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[a][c] += (TA)qv[c] * sv;
        }
      }
    }
  }

  // (Q e)[row r of the staged float64 tile, i, j] with e in the [col][K] layout
  __device__ double qe_tile_d(const double* Qt, const double* e, int r, int i, int j) const {
    const double* qp = Qt + r * d.np + sm.poff[i];
    const double* ep = e + sm.poff[i] * K + j;
    double s = 0.0;
    for (int c = 0; c < sm.n_i[i]; ++c) s += qp[c] * ep[c * K];
    return s;
  }

  // Write the float32 accumulators transposed, eT[j * np + col], so that one
  // right-hand side's coefficients are contiguous (float4 reads in qe_tile).
  __device__ void store_acc_t(float (&acc)[kPairsPerThread][4], float* eT) const {
    const int npairs = d.nq * K;
#pragma unroll
    for (int a = 0; a < kPairsPerThread; ++a) {
      const int pr = threadIdx.x + a * kBT;
      if (pr < npairs) {
        const int q = pr / K, j = pr % K;
        *reinterpret_cast<float4*>(eT + j * d.np + 4 * q) = make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
      }
    }
  }

  // (Q e)[row r of the staged tile, i, j] = sum over block i's (padded) columns,
  // four at a time (the pad columns of Q are zero)
  __device__ float qe_tile(const float* Qt, const float* eT, int r, int i, int j) const {
    const int c0 = sm.poff[i], nq_i = (sm.poff[i + 1] - c0) >> 2;
    const float4* qp = reinterpret_cast<const float4*>(Qt + r * d.np + c0);
    const float4* ep = reinterpret_cast<const float4*>(eT + j * d.np + c0);
    float s = 0.f;
    for (int q = 0; q < nq_i; ++q) {
      const float4 a = qp[q], b = ep[q];
      s += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
    }
    return s;
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

};

template <int K, int kTR>
__device__ void solve_instance(const BatchInst& dsc, const BatchPools& P, const BatchOpts& o, const Smem& sm) {
  Inst<K, kTR> I{dsc, sm, P};
  double* tile64 = sm.tile64;
  float* tile32 = sm.tile32;
  double* e64 = sm.e64;
  float* e32 = sm.e32;
  double* qt64 = reinterpret_cast<double*>(sm.qtile);
  // 16-byte asynchronous copies need 16-byte aligned row tiles: G K a
  // multiple of 4 and a 16-byte aligned instance offset in the vector pools
  const bool vec_ok = ((dsc.G * K) % 4 == 0) && (dsc.v_off % 4 == 0);
  const int G = dsc.G, Gq = dsc.Gq;
  const int64_t M = dsc.M, GK = (int64_t)G * K;
  const int64_t nv = M * GK;
  const int tid = threadIdx.x;
  const long long clk0 = clock64();
  int cta_steps = 0;
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
      sigma_rows<K>(w64 + t0 * GK, tr, G, Gq, sm.om64, [&](int e, int r, int h, int j, double sv) {
        const double ev = Y[(int64_t)j * m + (int64_t)h * M + t0 + r] - sv;
        tile64[e] = ev;
        E64[t0 * GK + e] = ev;
      });
      I.stage_q(P.q64, t0, tr, qt64);
      __syncthreads();
      I.accumulate(qt64, tile64, tr, acc64);
      __syncthreads();
    }
    I.store_acc(acc64, e64);
    __syncthreads();
    double nrm = 0.0;
    for (int64_t t0 = 0; t0 < M; t0 += kTR) {
      const int tr = (int)((M - t0) < kTR ? (M - t0) : kTR);
      I.stage_q(P.q64, t0, tr, qt64);
      __syncthreads();
      for (int e = tid; e < tr * GK; e += kBT) {
        const int j = e % K, rest = e / K, h = rest % G, r = rest / G;
        const int64_t gi = t0 * GK + e;
        const double rho = E64[gi] - I.qe_tile_d(qt64, e64, r, h, j);
        nrm += rho * rho;
        g32[gi] = (float)(-rho);
      }
      __syncthreads();
    }
    cta_sum_strided<K>(nrm, sm.red, sm.colv);
    // ---- per-column decisions (reference: the single-instance refinement loop)
    if (tid < K) {
      const int j = tid;
      const double cur = sqrt(sm.colv[j]);
      revert[j] = 0;
      if (outer == 0) rho0[j] = P.rho_extra ? sqrt(cur * cur + P.rho_extra[(int64_t)dsc.index * kBatchMaxK + j]) : cur;
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
    // Per-column state of the inner solve.  It is the same for every thread,
    // so it lives in shared memory, written by thread j < K between barriers.
    __shared__ double s_c1[K], s_c[K], s_cbest[K], s_csnap[K], s_cstop[K], s_mu[K], s_lam[K];
    __shared__ float s_mu32[K], s_lam32[K];   // float copies read per element (no conversions there)
    __shared__ int s_ibest[K], s_act[K], s_done[K], s_snap[K], s_conv[K];
    {
      double cs = 0.0;
      __syncthreads();
      for (int64_t e = tid; e < nv; e += kBT) cs += (double)g32[e] * (double)g32[e];
      cta_sum_strided<K>(cs, sm.red, sm.colv + K);
      if (tid < K) {
        const double v = sm.colv[K + tid];
        s_c1[tid] = s_c[tid] = s_cbest[tid] = s_csnap[tid] = s_cstop[tid] = v;
        s_ibest[tid] = 0;
        s_act[tid] = (v > 0.0) && isfinite(v);
        s_done[tid] = 0;
        s_snap[tid] = 0;
        s_conv[tid] = 0;
        s_mu[tid] = 0.0;
        s_lam[tid] = 0.0;
        s_mu32[tid] = 0.f;
        s_lam32[tid] = 0.f;
      }
      __syncthreads();
    }
    for (int it = 1; it <= o.inner_maxit; ++it) {
      int anyact = 0;
#pragma unroll
      for (int j = 0; j < K; ++j) anyact |= s_act[j];
      if (!anyact) break;
      ++cta_steps;
      // pass A: u = g + mu u ; S = U Omega ; d = u.S ; e = Q^T S
      float acc32[kPairsPerThread][4] = {};
      double dd = 0.0;
      const int ntiles = (int)((M + kTR - 1) / kTR);
      const size_t sf = stage_floats(K, kTR, sm.maxG, sm.maxNp);
      // stage layout: u | g | w | Q (tile strides of the largest instance)
      auto stage = [&](int b) { return sm.ibuf + b * sf; };
      const int tstride = kTR * sm.maxG * K;
      auto issue = [&](int t, bool with_w) {
        const int64_t t0 = (int64_t)t * kTR;
        const int tr = (int)((M - t0) < kTR ? (M - t0) : kTR);
        float* st = stage(t & 1);
        copy_async(u32 + t0 * GK, st, tr * (int)GK, vec_ok);
        copy_async(g32 + t0 * GK, st + tstride, tr * (int)GK, vec_ok);
        if (with_w) copy_async(w32 + t0 * GK, st + 2 * tstride, tr * (int)GK, vec_ok);
        copy_async(P.q32 + dsc.q_off + t0 * dsc.np, st + 3 * tstride, tr * dsc.np, true);
        cp_async_commit();
      };
      issue(0, false);
      for (int t = 0; t < ntiles; ++t) {
        const int64_t t0 = (int64_t)t * kTR;
        const int tr = (int)((M - t0) < kTR ? (M - t0) : kTR);
        if (t + 1 < ntiles) {
          issue(t + 1, false);
          cp_async_wait<1>();
        } else {
          cp_async_wait<0>();
        }
        __syncthreads();
        float* ut = stage(t & 1);
        const float* gt = ut + tstride;
        const float* qt = ut + 3 * tstride;
        for (int e = tid; e < tr * GK; e += kBT) {
          const int j = e % K;
          if (s_act[j]) {
            const float un = gt[e] + s_mu32[j] * ut[e];
            ut[e] = un;
            u32[t0 * GK + e] = un;
          }
        }
        __syncthreads();
        // S tile into tile32, d partials
        float* St = tile32;
        float ddt = 0.f;
        sigma_rows4<K>(ut, tr, G, Gq, sm.om32, [&](int e, int, int, int, float sv) {
          St[e] = sv;
          ddt += sv * ut[e];
        });
        dd += (double)ddt;
        __syncthreads();
        I.accumulate(qt, St, tr, acc32);
        __syncthreads();
      }
      I.store_acc_t(acc32, e32);
      cta_sum_strided<K>(dd, sm.red, sm.colv + 2 * K);
      if (tid < K) {
        const double dj = sm.colv[2 * K + tid];
        s_lam[tid] = 0.0;
        if (s_act[tid]) {
          if (!(dj > 0.0) || !isfinite(dj)) s_act[tid] = 0;
          else s_lam[tid] = s_c[tid] / dj;
        }
        s_lam32[tid] = (float)s_lam[tid];
      }
      __syncthreads();
      // pass B: t = S - Q e ; g -= lam t ; w -= lam u ; c' = g.g
      double cn = 0.0;
      issue(0, true);
      for (int t = 0; t < ntiles; ++t) {
        const int64_t t0 = (int64_t)t * kTR;
        const int tr = (int)((M - t0) < kTR ? (M - t0) : kTR);
        if (t + 1 < ntiles) {
          issue(t + 1, true);
          cp_async_wait<1>();
        } else {
          cp_async_wait<0>();
        }
        __syncthreads();
        const float* ut = stage(t & 1);
        const float* gt = ut + tstride;
        const float* wt = ut + 2 * tstride;
        const float* qt = ut + 3 * tstride;
        float cnt = 0.f;
        sigma_rows4<K>(ut, tr, G, Gq, sm.om32, [&](int e, int r, int h, int j, float sv) {
          const int64_t gi = t0 * GK + e;
          const float lj = s_lam32[j];
          const float tval = sv - I.qe_tile(qt, e32, r, h, j);
          const float gn = gt[e] - lj * tval;
          g32[gi] = gn;
          const float wo = wt[e];
          if (s_snap[j]) wb32[gi] = wo;   // the w whose c was a new quarter-low
          w32[gi] = wo - lj * ut[e];
          cnt += gn * gn;
        });
        cn += (double)cnt;
        __syncthreads();
      }
      cta_sum_strided<K>(cn, sm.red, sm.colv + 3 * K);
      if (tid < K) {
        const int j = tid;
        s_snap[j] = 0;
        if (!s_act[j]) {
          s_mu[j] = 0.0;
        } else {
          const double cj = sm.colv[3 * K + j];
          s_done[j] = it;
          s_cstop[j] = cj;
          if (cj < s_cbest[j]) { s_cbest[j] = cj; s_ibest[j] = it; }
          const bool done_conv = isfinite(cj) && cj >= 0.0 && sqrt(cj / s_c1[j]) <= o.inner_tol;
          if (done_conv || !isfinite(cj) || cj < 0.0 || it - s_ibest[j] >= o.inner_window || it >= o.inner_maxit) {
            s_act[j] = 0;
            s_mu[j] = 0.0;
            s_conv[j] = done_conv;
          } else {
            if (cj < 0.25 * s_csnap[j]) { s_csnap[j] = cj; s_snap[j] = 1; }   // saved in the next pass B
            s_mu[j] = cj / s_c[j];
            s_c[j] = cj;
          }
        }
        s_mu32[j] = (float)s_mu[j];
      }
      __syncthreads();
    }
    // columns that stopped without converging take their saved best w
    {
      int any_restore = 0;
#pragma unroll
      for (int j = 0; j < K; ++j) any_restore |= (!s_conv[j] && !(s_cstop[j] <= s_csnap[j]));
      if (any_restore) {
        for (int64_t e = tid; e < nv; e += kBT) {
          const int j = (int)(e % K);
          if (!s_conv[j] && !(s_cstop[j] <= s_csnap[j])) w32[e] = wb32[e];
        }
        __syncthreads();
      }
    }
    if (tid < K) iters_acc[tid] += s_done[tid];
    // ---- d = P (double) w32 ; w64 += d on the live columns
    double accp[kPairsPerThread][4] = {};
    for (int64_t t0 = 0; t0 < M; t0 += kTR) {
      const int tr = (int)((M - t0) < kTR ? (M - t0) : kTR);
      for (int e = tid; e < tr * GK; e += kBT) tile64[e] = (double)w32[t0 * GK + e];
      I.stage_q(P.q64, t0, tr, qt64);
      __syncthreads();
      I.accumulate(qt64, tile64, tr, accp);
      __syncthreads();
    }
    I.store_acc(accp, e64);
    __syncthreads();
    for (int64_t t0 = 0; t0 < M; t0 += kTR) {
      const int tr = (int)((M - t0) < kTR ? (M - t0) : kTR);
      I.stage_q(P.q64, t0, tr, qt64);
      __syncthreads();
      for (int e = tid; e < tr * GK; e += kBT) {
        const int j = e % K, rest = e / K, h = rest % G, r = rest / G;
        const int64_t gi = t0 * GK + e;
        const double dv = live[j] ? (double)w32[gi] - I.qe_tile_d(qt64, e64, r, h, j) : 0.0;
        d64[gi] = dv;
        w64[gi] += dv;
      }
      __syncthreads();
    }
  }
  // ---- b = R^-1 Q^T (y - Sigma w64)
  double accb[kPairsPerThread][4] = {};
  for (int64_t t0 = 0; t0 < M; t0 += kTR) {
    const int tr = (int)((M - t0) < kTR ? (M - t0) : kTR);
    sigma_rows<K>(w64 + t0 * GK, tr, G, Gq, sm.om64, [&](int e, int r, int h, int j, double sv) {
      tile64[e] = Y[(int64_t)j * m + (int64_t)h * M + t0 + r] - sv;
    });
    I.stage_q(P.q64, t0, tr, qt64);
    __syncthreads();
    I.accumulate(qt64, tile64, tr, accb);
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
  if (tid == 0) {
    P.steps[dsc.index] = cta_steps;
    P.cycles[dsc.index] = clock64() - clk0;
  }
  __syncthreads();
}

template <int K, int kTR>
__global__ void __launch_bounds__(kBT, 1)
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
