// Fused float32 PCG-Aug step with the Sigma-apply on the fifth-generation
// tensor cores (Algorithm glmpcg2 with D = I, Sec. 4.3).
//
// One step is three launches:
//   pass A : prologue (c_i, stop tests, mu_{i-1}); u_i = g_i + mu_{i-1} u_{i-1};
//            S = U Omega (Sigma u, Sec. 4.3) on the tensor cores; partial sums
//            of d_i = u_i^T S (step 5) and of C = Q_i^T S_i per block (the
//            projection's X*^T-like apply without R^-1).
//   reduce : C = sum of the partials, lambda_i = c_i / d_i (k_reduce).
//   pass B : S = U Omega again (recomputed: it is never stored);
//            w_{i+1} = w_i - lambda_i u_i (step 6); t = S - Q C (= P Sigma u);
//            g_{i+1} = g_i - lambda_i t (steps 7-8); partial sums of
//            c_{i+1} = g^T g.
// Per step the vectors are read or written eight times (pass A: g, u read,
// u written; pass B: u, g, w read, g, w written) and Q twice: the floor of a
// two-pass step.
//
// Tensor-core Sigma-apply.  A row tile of TV = 128 / KK observations holds
// 128 (row t, right-hand side j) pairs; S[t][h][j] = sum_g U[t][g][j] Om[g][h]
// is the 128 x Gp x Gp product D = A B^T with A[(t, j)][g] = U[t][g][j] and
// B[h][g] = Om[g][h] (Gp = G padded to 32 or 64), issued as tcgen05.mma
// kind::tf32: A in tensor memory, B in shared memory, the accumulator in
// tensor memory.  float32 accuracy comes from splitting both operands into
// tf32 high and low parts (hi = x with the low 13 mantissa bits cleared,
// lo = x - hi exactly) and summing three products, A_hi B_hi + A_hi B_lo +
// A_lo B_hi (the dropped A_lo B_lo term is of relative size 2^-20).  Per
// eight values of K one MMA of N = 2 Gp multiplies A_hi by [B_hi; B_lo]
// (columns 0 .. Gp - 1 and Gp .. 2 Gp - 1 of the accumulator) and one of
// N = Gp adds A_lo B_hi to the first half; S is the sum of the two halves.
// Thread (warp w, lane l) owns MMA row r = 32 (w % 4) + l (its quarter of the
// tensor-memory lanes) and the HB columns h = HB (w / 4) ...: it stores
// exactly the operand entries whose products it reads back, so u and S never
// change hands between threads.  Tensor-memory columns: accumulator at 0
// (2 Gp), A_hi at 128, A_lo at 192; pass B keeps the C values of its (block,
// rhs) pairs at 256 ...
//
// Overlap.  Pass A issues the MMA of tile i, writes the updated u tile back
// by a bulk copy and refills the stage from a warp without projection work,
// and projects tile i - 1 meanwhile; pass B forms (Q C) of tile i while the
// MMA of tile i runs.
//
// Memory: vector row tiles (contiguous in the (M, G, k) layout) and Q row
// sub-tiles of TQ rows are brought into shared memory by 1-D bulk copies
// (cp.async.bulk) completing on mbarriers; every wait is bounded and an
// expired wait sets the error word, drains the copies in flight and releases
// the tensor memory before the CTA leaves.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "pcg.h"
#include "pcg_dev.cuh"
#include "tc.cuh"
#include "tma.cuh"

namespace glmsur {

namespace {

constexpr int kTcThreads = 512;
constexpr int kTcRows = 128;   // MMA rows (t, j) per tile
// tensor-memory columns: accumulator, A operand (tf32 high, low parts), C of pass B
constexpr uint32_t kColAhi = 128, kColAlo = 192, kColC = 256;

__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ void st_smem_f(float* base, uint32_t byte_off, float v) {
  *reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(base) + byte_off) = v;
}

// Omega as the B operand, split into tf32 high and low parts:
// B[h][g] = Om[g][h] for g, h < G, zero in the padding; the low parts are the
// rows Gp .. 2 Gp - 1 of the same K-major operand.
template <int Gp>
__device__ void load_omega_split(const float* __restrict__ Om, int G, int Gq, float* Bhi) {
  float* Blo = Bhi + Gp * Gp;
  for (int e = threadIdx.x; e < Gp * Gp; e += blockDim.x) {
    const int h = e / Gp, gg = e % Gp;
    const float v = (h < G && gg < G) ? Om[(int64_t)gg * Gq + h] : 0.f;
    const float hi = tf32_trunc(v);
    const uint32_t off = kmajor_offset(h, gg, Gp);
    st_smem_f(Bhi, off, hi);
    st_smem_f(Blo, off, v - hi);
  }
}

// Row r of the A operand (tensor memory), columns h0 .. h0 + HB - 1, from HB
// float32 values: tf32 high parts at column 128 + h0, low parts at 192 + h0.
template <int HB>
__device__ __forceinline__ void store_a_split_tmem(uint32_t tmem_row, int h0, const float (&v)[HB]) {
  float t[HB];
#pragma unroll
  for (int c = 0; c < HB; ++c) t[c] = tf32_trunc(v[c]);
  tmem_st<HB>(tmem_row + kColAhi + (uint32_t)h0, t);
#pragma unroll
  for (int c = 0; c < HB; ++c) t[c] = v[c] - tf32_trunc(v[c]);
  tmem_st<HB>(tmem_row + kColAlo + (uint32_t)h0, t);
}

// S of the thread's row and columns h0 .. h0 + HB - 1: the sum of the two
// accumulator halves.
template <int HB, int Gp>
__device__ __forceinline__ void load_s(uint32_t tmem_row, int h0, float (&s)[HB]) {
  float s1[HB];
  tmem_ld<HB>(tmem_row + (uint32_t)h0, s);
  tmem_ld<HB>(tmem_row + (uint32_t)(Gp + h0), s1);
  tmem_ld_wait();
#pragma unroll
  for (int c = 0; c < HB; ++c) s[c] += s1[c];
}

// The tf32 products of one tile (16 MMAs for Gp = 64), one thread.
template <int Gp>
__device__ __forceinline__ void issue_sigma_mma(uint32_t tmem, const float* Bhi, uint64_t* bar) {
  const uint32_t id2 = tf32_idesc(kTcRows, 2 * Gp), id1 = tf32_idesc(kTcRows, Gp);
  const uint32_t bh = smem_u32(Bhi);
#pragma unroll
  for (int ks = 0; ks < Gp / 8; ++ks) {
    const uint64_t bd = kmajor_desc(bh + ks * 256, Gp);   // eight tf32 values of K: two core matrices
    mma_tf32_ts(tmem, tmem + kColAhi + 8 * ks, bd, id2, ks > 0);   // A_hi [B_hi; B_lo]
    mma_tf32_ts(tmem, tmem + kColAlo + 8 * ks, bd, id1, 1);        // + A_lo B_hi
  }
  mma_commit(bar);
}

// Copies that a CTA leaving early still has in flight: wait for them (bounded).
__device__ void drain_bar(uint64_t* bar, int issued, int consumed, int nslots) {
  for (int t = consumed; t < issued; ++t) mbar_wait_bounded(&bar[t % nslots], (t / nslots) & 1, kWaitLimitNs);
}

// Bounded wait by thread 0 for phase `parity` of `bar`; the CTA learns the
// outcome at the next barrier through `abort_flag`.
__device__ __forceinline__ void lead_wait(uint64_t* bar, uint32_t parity, int* abort_flag, int* err) {
  if (threadIdx.x == 0 && !mbar_wait_bounded(bar, parity, kWaitLimitNs)) {
    *abort_flag = 1;
    atomicExch(err, 1);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// pass A
// smem: [bars 128 B][Om_hi Om_lo: 2 Gp^2][g u: 2 TV G KK][S tile: TV G KK][Q ring NSQ x TQ np]
// bars: 0 vector tile, 1 MMA, 2 .. 2 + NSQ Q sub-tiles
// Iteration i: u of tile i and its operand (E), MMA of tile i, projection of
// tile i - 1 (P), then S of tile i into shared memory and d (R).
// ---------------------------------------------------------------------------
template <int KK, int HB>
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_pass_a(int64_t M, int G, int Gq, int np, int nq, int TQ, int NSQ, const float* __restrict__ Om,
            const float* __restrict__ Q, const float* __restrict__ g, float* __restrict__ u,
            const float* __restrict__ w, float* __restrict__ wbest, const int* __restrict__ quad_blk, PcgState st,
            const double* __restrict__ cpart, int ncpart, double* __restrict__ dpart, float* __restrict__ Cpart) {
  constexpr int Gp = 4 * HB, TV = kTcRows / KK;
  extern __shared__ __align__(1024) unsigned char smraw[];
  const TcSmem L = tc_smem_layout(0, G, Gp, KK, np, TQ, NSQ, 0);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smraw);
  float* Bhi = reinterpret_cast<float*>(smraw + L.om);
  const int GKP = tc_row_stride(0, G, KK);   // shared-memory row stride of the staged tiles
  float* gs = reinterpret_cast<float*>(smraw + L.vec);
  float* us = gs + TV * GKP;
  float* Ss = reinterpret_cast<float*>(smraw + L.tile);   // S of the tile being projected
  float* qring = reinterpret_cast<float*>(smraw + L.q);
  __shared__ double red[16 * 16];
  __shared__ float mu_s[KK];
  __shared__ int act_s[KK], snap_s[KK], anyp_s, abort_s;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  griddep_launch_dependents();
  griddep_wait();        // the previous step's pass B, the reduce or the init kernels
  if (*st.err) return;   // an earlier bounded wait gave up: the run is being abandoned
  if (tid == 0) anyp_s = 0;
  const double csum = sum_partials<KK>(cpart, ncpart, KK, 0, red);
  if (tid < KK) {
    const StepScalars sc = step_prologue(st, tid, KK, csum, blockIdx.x == 0);
    mu_s[tid] = (float)sc.mu;
    act_s[tid] = sc.act;
    snap_s[tid] = sc.snap;
    if (sc.act_prev) atomicOr(&anyp_s, 1);
  }
  __syncthreads();
  if (!anyp_s) return;   // every column already stopped: nothing changes
  load_omega_split<Gp>(Om, G, Gq, Bhi);
  const int64_t r0 = M * blockIdx.x / gridDim.x, r1 = M * (blockIdx.x + 1) / gridDim.x;
  const int ntiles = (int)((r1 - r0 + TV - 1) / TV);
  const int nsub = (int)((r1 - r0 + TQ - 1) / TQ);
  const int GK = G * KK;
  // warps with column quads run the projection; the last warp, when it has
  // none, issues the MMAs and the vector copies meanwhile
  const int pwarps = (nq + 31) >> 5;
  const int issuer = pwarps < kTcThreads / 32 ? kTcThreads - 32 : 0;
  const int iwarp = issuer >> 5;   // its warp issues the row copies, lane by lane
  if (tid == 0) {
    for (int q = 0; q < 2 + NSQ; ++q) mbar_init(&bars[q], 1);
    fence_mbar_init();
    abort_s = 0;
  }
  if (warp == 0) {
    tmem_alloc(&tslot, 256);
    tmem_relinquish();
  }
  fence_proxy_async_smem();   // the Omega operand is read by the tensor cores
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);   // this warp's lane quarter
  int vec_issued = 0, q_issued = 0, q_used = 0;   // (bookkeeping of the issuing threads)
  bool mma_pending = false;
  int mma_count = 0;
  // (all lanes of the issuing warp) the g and u rows of a tile, one row per lane
  auto issue_vec = [&](int tile) {
    const int64_t row0 = r0 + (int64_t)tile * TV;
    const int tr = (int)((r1 - row0) < TV ? (r1 - row0) : TV);
    const uint32_t rb = (uint32_t)(GK * sizeof(float));
    if (lane == 0) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&bars[0], 2u * (uint32_t)tr * rb);
    }
    __syncwarp();
    if (lane < tr) {
      fence_proxy_async_smem();
      tma_load_1d(gs + lane * GKP, g + (row0 + lane) * GK, rb, &bars[0]);
      tma_load_1d(us + lane * GKP, u + (row0 + lane) * GK, rb, &bars[0]);
    }
  };
  auto issue_q = [&](int s) {
    const int slot = s % NSQ;
    const int64_t row0 = r0 + (int64_t)s * TQ;
    const int tq = (int)((r1 - row0) < TQ ? (r1 - row0) : TQ);
    const uint32_t bytes = (uint32_t)(tq * np * sizeof(float));
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bars[2 + slot], bytes);
    tma_load_1d(qring + (int64_t)slot * TQ * np, Q + row0 * np, bytes, &bars[2 + slot]);
  };
  if (warp == iwarp && ntiles > 0) issue_vec(vec_issued++);
  if (tid == 0)
    for (; q_issued < NSQ && q_issued < nsub; ++q_issued) issue_q(q_issued);
  const int r = 32 * (warp & 3) + lane;   // MMA row of this thread: (t_r, j_r)
  const int t_r = r / KK, j_r = r % KK;
  const int hb = HB * (warp >> 2);
  const bool has_q = tid < nq;
  const int blk = has_q ? quad_blk[tid] : 0;
  const float mu_j = mu_s[j_r];
  const int act_j = act_s[j_r], snap_j = snap_s[j_r];
  float acc[4][KK];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int jj = 0; jj < KK; ++jj) acc[c][jj] = 0.f;
  double dsum = 0.0;
  for (int it = 0; it <= ntiles; ++it) {
    const int64_t row0 = r0 + (int64_t)it * TV;
    const int tr = it < ntiles ? (int)((r1 - row0) < TV ? (r1 - row0) : TV) : 0;
    if (it < ntiles) {
      // E: u = g + mu u on the live columns, over the staged u; row r of the A
      // operand.  Eight columns at a time: the loads of a chunk are issued
      // before its stores, which write the same tile.
      lead_wait(&bars[0], it & 1, &abort_s, st.err);
      __syncthreads();
      if (abort_s) break;
      const bool rowok = t_r < tr;
#pragma unroll
      for (int c0 = 0; c0 < HB; c0 += 8) {
        float uo[8], gv[8], v[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int h = hb + c0 + c;
          const bool ok = rowok && h < G;
          const int es = t_r * GKP + h * KK + j_r;
          uo[c] = ok ? us[es] : 0.f;
          gv[c] = ok ? gs[es] : 0.f;
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = act_j ? gv[c] + mu_j * uo[c] : uo[c];
        if (act_j && rowok) {
#pragma unroll
          for (int c = 0; c < 8; ++c)
            if (hb + c0 + c < G) us[t_r * GKP + (hb + c0 + c) * KK + j_r] = v[c];
        }
        if (snap_j && rowok) {   // the w whose c is a new quarter-low
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const int h = hb + c0 + c;
            if (h < G) {
              const int64_t e = row0 * GK + (t_r * G + h) * KK + j_r;
              wbest[e] = w[e];
            }
          }
        }
        store_a_split_tmem<8>(trow, hb + c0, v);
      }
      tmem_st_wait();
      fence_proxy_async_smem();   // the staged u is written back by a bulk copy
      tc_fence_before();
      __syncthreads();
      if (warp == iwarp) {
        if (lane == 0) {
          tc_fence_after();
          issue_sigma_mma<Gp>(tmem, Bhi, &bars[1]);
        }
        mma_pending = true;
        ++mma_count;
        if (lane < tr) {   // one row of u per lane
          tma_store_1d(u + (row0 + lane) * GK, us + lane * GKP, (uint32_t)(GK * sizeof(float)));
          bulk_commit();
          bulk_wait_read_all();   // the stage may be refilled once the store has read it
        }
        __syncwarp();
        if (vec_issued < ntiles) issue_vec(vec_issued++);
      }
    }
    if (it > 0 && warp < pwarps) {
      // P: projection partials of tile it - 1 (thread q owns column quad q),
      // by the warps that own column quads (named barrier 1)
      const int64_t prow0 = r0 + (int64_t)(it - 1) * TV;
      const int s0 = (it - 1) * (TV / TQ);
      const int s1 = min(nsub, s0 + TV / TQ);
      for (int s = s0; s < s1; ++s) {
        const int slot = s % NSQ;
        lead_wait(&bars[2 + slot], (s / NSQ) & 1, &abort_s, st.err);
        if (tid == 0) q_used = s + 1;
        named_bar_sync(1, 32 * pwarps);
        if (abort_s) break;
        const int64_t qrow0 = r0 + (int64_t)s * TQ;
        const int tq = (int)((r1 - qrow0) < TQ ? (r1 - qrow0) : TQ);
        const int tl0 = (int)(qrow0 - prow0);
        if (has_q) {
          const float* qs = qring + (int64_t)slot * TQ * np + 4 * tid;
          for (int rr = 0; rr < tq; ++rr) {
            const float4 qv = *reinterpret_cast<const float4*>(qs + (int64_t)rr * np);
            const float4* sp = reinterpret_cast<const float4*>(Ss + (tl0 + rr) * GKP + blk * KK);
            const float qc[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
            for (int a = 0; a < KK / 4; ++a) {
              const float4 sv = sp[a];
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                acc[c][4 * a] += qc[c] * sv.x;
                acc[c][4 * a + 1] += qc[c] * sv.y;
                acc[c][4 * a + 2] += qc[c] * sv.z;
                acc[c][4 * a + 3] += qc[c] * sv.w;
              }
            }
          }
        }
        named_bar_sync(1, 32 * pwarps);
        if (tid == 0 && q_issued < nsub) issue_q(q_issued++);
      }
    }
    __syncthreads();
    if (abort_s) break;
    if (it < ntiles) {
      // R: S of tile it from tensor memory; d = u^T S; S into shared memory
      if (tid == 0) {
        if (!mbar_wait_bounded(&bars[1], it & 1, kWaitLimitNs)) {
          abort_s = 1;
          atomicExch(st.err, 1);
        }
      }
      __syncthreads();
      if (abort_s) break;
      if (tid == issuer) mma_pending = false;
      tc_fence_after();
      // S = the two accumulator halves; u = A_hi + A_lo read back from tensor
      // memory (the split is exact), so u needs no registers across the step
      float dl = 0.f;
#pragma unroll
      for (int c0 = 0; c0 < HB; c0 += 8) {
        float sv[8], s1[8], ah[8], al[8];
        tmem_ld<8>(trow + (uint32_t)(hb + c0), sv);
        tmem_ld<8>(trow + (uint32_t)(Gp + hb + c0), s1);
        tmem_ld<8>(trow + kColAhi + (uint32_t)(hb + c0), ah);
        tmem_ld<8>(trow + kColAlo + (uint32_t)(hb + c0), al);
        tmem_ld_wait();
        if (t_r < tr) {
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const int h = hb + c0 + c;
            if (h < G) {
              const float sc = sv[c] + s1[c];
              dl += (ah[c] + al[c]) * sc;
              Ss[t_r * GKP + h * KK + j_r] = sc;
            }
          }
        }
      }
      if (t_r < tr) dsum += (double)dl;   // d = u^T S: per-tile float partials added in float64
      tc_fence_before();
      __syncthreads();
    }
  }
  if (abort_s) {
    if (tid == issuer) {
      if (mma_pending) mbar_wait_bounded(&bars[1], (mma_count - 1) & 1, kWaitLimitNs);
      drain_bar(bars, vec_issued, vec_issued - 1, 1);
    }
    if (tid == 0) drain_bar(bars + 2, q_issued, q_used, NSQ);
  } else {
    const double d = reduce_cols_strided<KK>(dsum, red);   // thread's column: tid % KK == j_r
    if (tid < KK) dpart[(int64_t)blockIdx.x * KK + tid] = d;
    if (has_q) {
      float* dst = Cpart + ((int64_t)blockIdx.x * np + 4 * tid) * KK;
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int a = 0; a < KK / 4; ++a)
          reinterpret_cast<float4*>(dst + c * KK)[a] =
              make_float4(acc[c][4 * a], acc[c][4 * a + 1], acc[c][4 * a + 2], acc[c][4 * a + 3]);
    }
  }
  if (warp == iwarp) bulk_wait_all();   // the stores of u (one per lane) have completed
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 256);
  }
}

// ---------------------------------------------------------------------------
// pass B
// smem: [bars][Om_hi Om_lo][u: TV G KK][g: NSG x TV G KK][(Q C) tile][Q ring]
// bars: 0 u tile, 1 MMA, 2 .. 2 + NSG g tiles, 2 + NSG .. Q sub-tiles
// Iteration i: operand from u and w -= lambda u (E), MMA of tile i, (Q C) of
// tile i while it runs (QC), then g -= lambda (S - Q C) and c' (U).
// ---------------------------------------------------------------------------
template <int KK, int HB>
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_pass_b(int64_t M, int G, int Gq, int np, int TQ, int NSQ, int NSG, const float* __restrict__ Om,
            const float* __restrict__ Q, float* __restrict__ g, const float* __restrict__ u, float* __restrict__ w,
            const float* __restrict__ C, const int* __restrict__ poff, PcgState st, double* __restrict__ cpart) {
  constexpr int Gp = 4 * HB, TV = kTcRows / KK;
  constexpr int NP = (Gp * KK + kTcThreads - 1) / kTcThreads;   // (block, rhs) pairs per thread (<= 2)
  extern __shared__ __align__(1024) unsigned char smraw[];
  const TcSmem L = tc_smem_layout(1, G, Gp, KK, np, TQ, NSQ, NSG);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smraw);
  uint64_t* gbar = bars + 2;
  uint64_t* qbar = bars + 2 + NSG;
  float* Bhi = reinterpret_cast<float*>(smraw + L.om);
  float* us = reinterpret_cast<float*>(smraw + L.vec);
  float* gstage = us + TV * G * KK;
  float* QCs = reinterpret_cast<float*>(smraw + L.tile);
  float* qring = reinterpret_cast<float*>(smraw + L.q);
  __shared__ double red[16 * 16];
  __shared__ float lam_s[KK];
  __shared__ int abort_s;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  griddep_launch_dependents();
  griddep_wait();        // the reduce of this step (after pass A)
  if (*st.err) return;
  {
    const int slot = (*st.it - 1) & 1;   // reduce has already advanced the counter
    int any = 0;
    for (int jj = 0; jj < KK; ++jj) any |= st.active[slot][jj];
    if (!any) {
      if (tid < KK) cpart[(int64_t)blockIdx.x * KK + tid] = 0.0;
      return;
    }
  }
  if (tid < KK) lam_s[tid] = (float)st.lam[tid];
  load_omega_split<Gp>(Om, G, Gq, Bhi);
  const int64_t r0 = M * blockIdx.x / gridDim.x, r1 = M * (blockIdx.x + 1) / gridDim.x;
  const int ntiles = (int)((r1 - r0 + TV - 1) / TV);
  const int nsub = (int)((r1 - r0 + TQ - 1) / TQ);
  const int GK = G * KK;
  if (tid == 0) {
    for (int q = 0; q < 2 + NSG + NSQ; ++q) mbar_init(&bars[q], 1);
    fence_mbar_init();
    abort_s = 0;
  }
  if (warp == 0) {
    tmem_alloc(&tslot, 512);
    tmem_relinquish();
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  // (block i, right-hand side j) pairs of this thread; their C = Q_i^T S_i
  // values wait in this thread's lane of tensor memory, columns
  // 256 + 64 (warp / 4) + 32 a ...
  const int npairs = G * KK;
  int pc0[NP], nqi[NP], pi[NP], pj[NP];
  const uint32_t ccol = kColC + 64u * (uint32_t)(warp >> 2);
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    const int p = tid + a * kTcThreads;
    const bool has = p < npairs;
    pi[a] = has ? p / KK : 0;
    pj[a] = p % KK;
    pc0[a] = has ? poff[pi[a]] : 0;
    nqi[a] = has ? (poff[pi[a] + 1] - poff[pi[a]]) >> 2 : 0;
    float cv[16];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int cc = 16 * half + e;   // column pc0 + cc of block pi
        cv[e] = (cc < 4 * nqi[a]) ? C[(int64_t)(pc0[a] + cc) * KK + pj[a]] : 0.f;
      }
      tmem_st16(trow + ccol + 32u * a + 16u * half, cv);
    }
  }
  tmem_st_wait();
  int u_issued = 0, g_issued = 0, g_used = 0, q_issued = 0, q_used = 0;
  bool mma_pending = false;
  int mma_count = 0;
  auto tile_rows = [&](int tile) {
    const int64_t row0 = r0 + (int64_t)tile * TV;
    return (int)((r1 - row0) < TV ? (r1 - row0) : TV);
  };
  auto issue_u = [&](int tile) {
    const uint32_t bytes = (uint32_t)(tile_rows(tile) * GK * sizeof(float));
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bars[0], bytes);
    tma_load_1d(us, u + (r0 + (int64_t)tile * TV) * GK, bytes, &bars[0]);
  };
  auto issue_g = [&](int tile) {
    const int slot = tile % NSG;
    const uint32_t bytes = (uint32_t)(tile_rows(tile) * GK * sizeof(float));
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&gbar[slot], bytes);
    tma_load_1d(gstage + (int64_t)slot * TV * GK, g + (r0 + (int64_t)tile * TV) * GK, bytes, &gbar[slot]);
  };
  auto issue_q = [&](int s) {
    const int slot = s % NSQ;
    const int64_t row0 = r0 + (int64_t)s * TQ;
    const int tq = (int)((r1 - row0) < TQ ? (r1 - row0) : TQ);
    const uint32_t bytes = (uint32_t)(tq * np * sizeof(float));
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&qbar[slot], bytes);
    tma_load_1d(qring + (int64_t)slot * TQ * np, Q + row0 * np, bytes, &qbar[slot]);
  };
  if (tid == 0) {
    if (ntiles > 0) issue_u(u_issued++);
    for (; g_issued < NSG && g_issued < ntiles; ++g_issued) issue_g(g_issued);
    for (; q_issued < NSQ && q_issued < nsub; ++q_issued) issue_q(q_issued);
  }
  const int r = 32 * (warp & 3) + lane;
  const int t_r = r / KK, j_r = r % KK;
  const int hb = HB * (warp >> 2);
  __syncthreads();
  const float lam_j = lam_s[j_r];
  // w of the thread's elements of the next tile, loaded one tile ahead
  float wv[HB];
  auto load_w = [&](int tile) {
    const int64_t row0 = r0 + (int64_t)tile * TV;
    const bool rowok = t_r < tile_rows(tile) && lam_j != 0.f;
#pragma unroll
    for (int c = 0; c < HB; ++c) {
      const int h = hb + c;
      wv[c] = (rowok && h < G) ? w[row0 * GK + (t_r * G + h) * KK + j_r] : 0.f;
    }
  };
  if (ntiles > 0) load_w(0);
  double csd = 0.0;
  for (int tile = 0; tile < ntiles; ++tile) {
    const int64_t row0 = r0 + (int64_t)tile * TV;
    const int tr = tile_rows(tile);
    lead_wait(&bars[0], tile & 1, &abort_s, st.err);
    __syncthreads();
    if (abort_s) break;
    // E: the A operand from u; w -= lambda u
    {
      float uv[HB];
      const bool rowok = t_r < tr;
#pragma unroll
      for (int c = 0; c < HB; ++c) {
        const int h = hb + c;
        uv[c] = (rowok && h < G) ? us[(t_r * G + h) * KK + j_r] : 0.f;
      }
      store_a_split_tmem<HB>(trow, hb, uv);
      if (rowok && lam_j != 0.f) {
#pragma unroll
        for (int c = 0; c < HB; ++c) {
          const int h = hb + c;
          if (h < G) w[row0 * GK + (t_r * G + h) * KK + j_r] = wv[c] - lam_j * uv[c];
        }
      }
    }
    tmem_st_wait();
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      if (u_issued < ntiles) issue_u(u_issued++);
      issue_sigma_mma<Gp>(tmem, Bhi, &bars[1]);
      mma_pending = true;
      ++mma_count;
    }
    if (tile + 1 < ntiles) load_w(tile + 1);
    // QC: (Q C)[t][i][j] = sum over block i's columns of Q[t][c] C[c][j] (pair threads)
    const int s0 = tile * (TV / TQ);
    const int s1 = min(nsub, s0 + TV / TQ);
    for (int s = s0; s < s1; ++s) {
      const int slot = s % NSQ;
      lead_wait(&qbar[slot], (s / NSQ) & 1, &abort_s, st.err);
      if (tid == 0) q_used = s + 1;
      __syncthreads();
      if (abort_s) break;
      const int64_t qrow0 = r0 + (int64_t)s * TQ;
      const int tq = (int)((r1 - qrow0) < TQ ? (r1 - qrow0) : TQ);
      const int tl0 = (int)(qrow0 - row0);
      const float* qs = qring + (int64_t)slot * TQ * np;
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        float cv[32];
        {
          float c0[16], c1[16];
          tmem_ld16(trow + ccol + 32u * a, c0);
          tmem_ld16(trow + ccol + 32u * a + 16u, c1);
          tmem_ld_wait();
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            cv[e] = c0[e];
            cv[16 + e] = c1[e];
          }
        }
        if (tid + a * kTcThreads < npairs) {
          for (int rr = 0; rr < tq; ++rr) {
            const float* qrow = qs + (int64_t)rr * np + pc0[a];
            float sum = 0.f;
#pragma unroll
            for (int qq = 0; qq < 8; ++qq) {
              if (qq < nqi[a]) {
                const float4 qv = *reinterpret_cast<const float4*>(qrow + 4 * qq);
                sum += qv.x * cv[4 * qq] + qv.y * cv[4 * qq + 1] + qv.z * cv[4 * qq + 2] + qv.w * cv[4 * qq + 3];
              }
            }
            QCs[((tl0 + rr) * G + pi[a]) * KK + pj[a]] = sum;
          }
        }
      }
      __syncthreads();
      if (tid == 0 && q_issued < nsub) issue_q(q_issued++);
    }
    if (abort_s) break;
    // U: t = S - Q C ; g -= lambda t ; c' = g^T g
    const int gslot = tile % NSG;
    lead_wait(&gbar[gslot], (tile / NSG) & 1, &abort_s, st.err);
    if (tid == 0) {
      g_used = tile + 1;
      if (!mbar_wait_bounded(&bars[1], tile & 1, kWaitLimitNs)) {
        abort_s = 1;
        atomicExch(st.err, 1);
      } else {
        mma_pending = false;
      }
    }
    __syncthreads();
    if (abort_s) break;
    tc_fence_after();
    {
      const float* gs = gstage + (int64_t)gslot * TV * GK;
      float sv[HB];
      load_s<HB, Gp>(trow, hb, sv);
      if (t_r < tr) {
        float cs = 0.f;
#pragma unroll
        for (int c = 0; c < HB; ++c) {
          const int h = hb + c;
          if (h < G) {
            const int e = (t_r * G + h) * KK + j_r;
            float gn = gs[e];
            if (lam_j != 0.f) {
              gn -= lam_j * (sv[c] - QCs[e]);
              g[row0 * GK + e] = gn;
            }
            cs += gn * gn;
          }
        }
        csd += (double)cs;   // per-tile float partials added in float64
      }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && g_issued < ntiles) issue_g(g_issued++);
  }
  if (abort_s) {
    if (tid == 0) {
      if (mma_pending) mbar_wait_bounded(&bars[1], (mma_count - 1) & 1, kWaitLimitNs);
      drain_bar(bars, u_issued, u_issued - 1, 1);
      drain_bar(gbar, g_issued, g_used, NSG);
      drain_bar(qbar, q_issued, q_used, NSQ);
    }
  } else {
    const double tot = reduce_cols_strided<KK>(csd, red);
    if (tid < KK) cpart[(int64_t)blockIdx.x * KK + tid] = tot;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
bool tc_step_eligible(int G, int k, int np, int nmax_cols) {
  return (k == 8 || k == 16) && G >= 1 && G <= 64 && np / 4 <= kTcThreads && nmax_cols <= 32;
}

template <int KK, int HB>
static cudaError_t tc_set_attrs(size_t a_bytes, size_t b_bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_tc_pass_a<KK, HB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)a_bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_pass_b<KK, HB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b_bytes);
  return e;
}

cudaError_t tc_prepare(int k, int Gp, size_t a_bytes, size_t b_bytes) {
  if (k == 16) return Gp == 64 ? tc_set_attrs<16, 16>(a_bytes, b_bytes) : tc_set_attrs<16, 8>(a_bytes, b_bytes);
  return Gp == 64 ? tc_set_attrs<8, 16>(a_bytes, b_bytes) : tc_set_attrs<8, 8>(a_bytes, b_bytes);
}

#define TC_DISPATCH(k, Gp, CALL)          \
  do {                                    \
    if ((k) == 16) {                      \
      if ((Gp) == 64) CALL(16, 16);       \
      else CALL(16, 8);                   \
    } else {                              \
      if ((Gp) == 64) CALL(8, 16);        \
      else CALL(8, 8);                    \
    }                                     \
  } while (0)

void launch_tc_pass_a(const IterPlan& p, const Geom& gm, int k, const float* Om, const float* Q, const float* g,
                      float* u, const float* w, float* wbest, const PcgState& st, const double* cpart, int ncpart,
                      double* dpart, float* Cpart, cudaStream_t s) {
#define A_(KK, HB)                                                                                          \
  launch_pdl(k_tc_pass_a<KK, HB>, dim3(p.n_sigma), dim3(kTcThreads), p.tc_a_smem, s, gm.M, gm.G, gm.Gq, gm.np, \
             gm.nq, p.tc_tq_a, p.tc_nsq_a, Om, Q, g, u, w, wbest, gm.d_quad_blk, st, cpart, ncpart, dpart, Cpart)
  TC_DISPATCH(k, p.tc_gp, A_);
#undef A_
}

void launch_tc_pass_b(const IterPlan& p, const Geom& gm, int k, const float* Om, const float* Q, float* g,
                      const float* u, float* w, const float* C, const PcgState& st, double* cpart, cudaStream_t s) {
#define B_(KK, HB)                                                                                          \
  launch_pdl(k_tc_pass_b<KK, HB>, dim3(p.n_update), dim3(kTcThreads), p.tc_b_smem, s, gm.M, gm.G, gm.Gq, gm.np, \
             p.tc_tq_b, p.tc_nsq_b, p.tc_nsg, Om, Q, g, u, w, C, gm.d_poff, st, cpart)
  TC_DISPATCH(k, p.tc_gp, B_);
#undef B_
}

}  // namespace glmsur
