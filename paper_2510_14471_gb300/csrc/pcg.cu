// PCG-Aug iteration kernels for the SUR model (Algorithm glmpcg2 with D = I,
// Sec. 4.3).  With D = I the preconditioner block Pi = (+)_i (I - Q_i Q_i^T)
// =: P is an orthogonal projector, so the iteration keeps g = P r
// (c = r^T Pi r = g^T g) and, because P X v = 0, updates it by
// g <- g - lambda P (Sigma u): the X v term of step 7 never has to be formed.
//
// One step i of the iteration is four launches (all stream-ordered):
//   sigma_step     : c_i from the partial sums of the previous step, the stop
//                    tests and mu_{i-1} = c_i / c_{i-1} (every CTA computes the
//                    same values); the lagged w_i = w_{i-1} - lambda_{i-1} u_{i-1};
//                    u_i = g_i + mu_{i-1} u_{i-1}; S = U Omega (Sigma u, Sec. 4.3);
//                    partial sums of d_i = u_i^T S (step 5).
//   proj_partial   : partial sums over row ranges of C_i = Q_i^T S_i (X*^T-like
//                    apply of Sec. 4.3 without the R^-1).
//   reduce         : C = sum of partials (fixed order); lambda_i = c_i / d_i
//                    (step 6) and the breakdown test d_i <= 0.
//   proj_update    : t = S - Q C (= P Sigma u), g_{i+1} = g_i - lambda_i t
//                    (steps 7-8), partial sums of c_{i+1} = g^T g.
// Vectors are (M, G, k) row-major so that one row tile holds every block and
// every right-hand side of a set of observations.
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"
#include "pcg.h"
#include "pcg_dev.cuh"
#include "tma.cuh"

namespace glmsur {

// ---------------------------------------------------------------------------
// sigma_step: prologue, lagged w update, u update, S = U Omega, d partials.
// grid (nrowcta, 1, k / JJ); dynamic smem: Omega (G x Gq) + U tile (TR x G x JJ)
// ---------------------------------------------------------------------------
template <typename T, int JJ>
__global__ void __launch_bounds__(256)
k_sigma_step(int64_t M, int64_t Ms, int G, int Gq, int k, int TR, const T* __restrict__ Om, const T* __restrict__ g,
             T* __restrict__ u, T* __restrict__ w, T* __restrict__ S, T* __restrict__ wbest,
             PcgState st, const double* __restrict__ cpart, int ncpart, double* __restrict__ dpart) {
  extern __shared__ __align__(128) unsigned char smraw[];
  T* Om_s = reinterpret_cast<T*>(smraw);
  T* U_s = Om_s + (int64_t)G * Gq;
  __shared__ double red[8 * 16];
  __shared__ double mu_s[JJ], lamp_s[JJ];
  __shared__ int act_s[JJ], snap_s[JJ], anyp_s;
  const int jg = blockIdx.z;
  if (threadIdx.x == 0) anyp_s = 0;
  const double csum = sum_partials<JJ>(cpart, ncpart, k, jg * JJ, red);
  if (threadIdx.x < JJ) {
    const int j = jg * JJ + threadIdx.x;
    const StepScalars sc = step_prologue(st, j, k, csum, blockIdx.x == 0);
    mu_s[threadIdx.x] = sc.mu;
    lamp_s[threadIdx.x] = sc.lam_prev;
    act_s[threadIdx.x] = sc.act;
    snap_s[threadIdx.x] = sc.snap;
    if (sc.act_prev) atomicOr(&anyp_s, 1);
  }
  __syncthreads();
  if (!anyp_s) return;   // every column of this group already stopped: nothing changes
  for (int64_t e = threadIdx.x; e < (int64_t)G * Gq; e += blockDim.x) Om_s[e] = Om[e];
  const int64_t r0 = M * blockIdx.x / gridDim.x, r1 = M * (blockIdx.x + 1) / gridDim.x;
  const int nhq = Gq >> 2;
  const int jj_t = threadIdx.x % JJ;
  double dsum = 0.0;
  __syncthreads();
  for (int64_t t0 = r0; t0 < r1; t0 += TR) {
    const int tr = (int)((r1 - t0) < (int64_t)TR ? (r1 - t0) : (int64_t)TR);
    // elementwise: w -= lam_prev u_old ; u = g + mu u_old (live columns).
    // Arithmetic in T: the float32 bulk path issues no float64 instruction
    // per element (float64 throughput is 1/58 of float32 on this part).
    // Units of V consecutive right-hand sides, EB units per thread in flight.
    constexpr int V = (JJ >= 4) ? 4 : JJ;
    constexpr int EB = 4;
    const int nu = tr * G * (JJ / V);
    for (int e0 = threadIdx.x; e0 < nu; e0 += EB * blockDim.x) {
      T uo[EB][V], gv[EB][V], wv[EB][V];
      int64_t gi[EB];
      int ee[EB];
      bool live[EB];
#pragma unroll
      for (int b = 0; b < EB; ++b) {
        const int e = e0 + b * blockDim.x;
        ee[b] = e;
        live[b] = false;
        if (e < nu) {
          const int jv = e % (JJ / V), rest = e / (JJ / V);
          const int i = rest % G, t = rest / G;
          gi[b] = ((t0 + t) * G + i) * k + jg * JJ + jv * V;
          live[b] = t0 + t < Ms;
#pragma unroll
          for (int c = 0; c < V; ++c) {
            uo[b][c] = u[gi[b] + c];
            gv[b][c] = g[gi[b] + c];
            wv[b][c] = w[gi[b] + c];
          }
        }
      }
#pragma unroll
      for (int b = 0; b < EB; ++b) {
        if (ee[b] < nu) {
          const int jv = ee[b] % (JJ / V);
#pragma unroll
          for (int c = 0; c < V; ++c) {
            const int jj = jv * V + c;
            const T lp = (T)lamp_s[jj];
            T un = uo[b][c];
            const T wn = wv[b][c] - lp * un;
            if (lp != (T)0) w[gi[b] + c] = wn;
            if (snap_s[jj]) wbest[gi[b] + c] = wn;
            if (act_s[jj]) {
              un = gv[b][c] + (T)mu_s[jj] * un;
              u[gi[b] + c] = un;
            }
            // rows t >= Ms have Sigma = 0 (restriction rows): S = U Omega sees zeros there
            U_s[(int64_t)ee[b] * V + c] = live[b] ? un : (T)0;
          }
        }
      }
    }
    __syncthreads();
    // S = U Omega on the tile; thread item (t, hq, jj) with jj = tid % JJ
    const int nitems = tr * nhq * JJ;
    T dloc = 0;
    for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
      const int rest = it / JJ;
      const int hq = rest % nhq, t = rest / nhq;
      T acc[4] = {0, 0, 0, 0};
      const T* urow = U_s + (int64_t)t * G * JJ + jj_t;
      for (int gg = 0; gg < G; ++gg) {
        T om[4];
        Vec4<T>::load(Om_s + (int64_t)gg * Gq + 4 * hq, om);
        const T uv = urow[gg * JJ];
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] += uv * om[c];
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int h = 4 * hq + c;
        if (h < G) {
          S[((t0 + t) * G + h) * k + jg * JJ + jj_t] = acc[c];
          dloc += acc[c] * urow[h * JJ];
        }
      }
    }
    dsum += (double)dloc;
    __syncthreads();
  }
  const double d = reduce_cols_strided<JJ>(dsum, red);
  if (threadIdx.x < JJ) dpart[(int64_t)blockIdx.x * k + jg * JJ + threadIdx.x] = d;
}

// ---------------------------------------------------------------------------
// sigma_resid: E = Y - W Omega on rows t < Ms, E = Y on the rows t >= Ms
// (Sigma = 0 there), Y = 0 when null; no state; used for b = X*^T (y - Sigma w)
// ---------------------------------------------------------------------------
template <typename T, int JJ>
__global__ void __launch_bounds__(256)
k_sigma_resid(int64_t M, int64_t Ms, int G, int Gq, int k, int TR, const T* __restrict__ Om, const T* __restrict__ Y,
              const T* __restrict__ Wv, T* E) {
  extern __shared__ __align__(128) unsigned char smraw[];
  T* Om_s = reinterpret_cast<T*>(smraw);
  T* U_s = Om_s + (int64_t)G * Gq;
  const int jg = blockIdx.z;
  for (int64_t e = threadIdx.x; e < (int64_t)G * Gq; e += blockDim.x) Om_s[e] = Om[e];
  const int64_t r0 = M * blockIdx.x / gridDim.x, r1 = M * (blockIdx.x + 1) / gridDim.x;
  const int nhq = Gq >> 2;
  const int jj_t = threadIdx.x % JJ;
  __syncthreads();
  for (int64_t t0 = r0; t0 < r1; t0 += TR) {
    const int tr = (int)((r1 - t0) < (int64_t)TR ? (r1 - t0) : (int64_t)TR);
    const int ne = tr * G * JJ;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
      const int jj = e % JJ, rest = e / JJ;
      const int i = rest % G, t = rest / G;
      U_s[e] = t0 + t < Ms ? Wv[((t0 + t) * G + i) * k + jg * JJ + jj] : (T)0;
    }
    __syncthreads();
    const int nitems = tr * nhq * JJ;
    for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
      const int rest = it / JJ;
      const int hq = rest % nhq, t = rest / nhq;
      T acc[4] = {0, 0, 0, 0};
      const T* urow = U_s + (int64_t)t * G * JJ + jj_t;
      for (int gg = 0; gg < G; ++gg) {
        T om[4];
        Vec4<T>::load(Om_s + (int64_t)gg * Gq + 4 * hq, om);
        const T uv = urow[gg * JJ];
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] += uv * om[c];
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int h = 4 * hq + c;
        if (h < G) {
          const int64_t gi = ((t0 + t) * G + h) * k + jg * JJ + jj_t;
          E[gi] = (Y ? Y[gi] : (T)0) - acc[c];
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// proj_partial: Cpart[rb] = sum_{t in rows(rb)} Q[t, col] * S[t, blk(col), j]
// grid (nrb, nqgroups, k / JJ); thread = one column quad of the group.
// ---------------------------------------------------------------------------
template <typename T, int JJ>
__global__ void __launch_bounds__(256)
k_proj_partial(int64_t M, int G, int np, int nq, int k, const T* __restrict__ Q, const T* __restrict__ S,
               const int* __restrict__ quad_blk, T* __restrict__ Cpart, PcgState st, int use_state) {
  const int jg = blockIdx.z;
  if (use_state) {
    const int slot = (*st.it) & 1;
    int any = 0;
    for (int jj = 0; jj < JJ; ++jj) any |= st.active[slot][jg * JJ + jj];
    if (!any) return;
  }
  const int qpg = (int)ceil_div(nq, gridDim.y);
  const int q = blockIdx.y * qpg + threadIdx.x;
  if (threadIdx.x >= qpg || q >= nq) return;
  const int64_t r0 = M * blockIdx.x / gridDim.x, r1 = M * (blockIdx.x + 1) / gridDim.x;
  const int blk = quad_blk[q];
  T acc[4][JJ];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int jj = 0; jj < JJ; ++jj) acc[c][jj] = 0;
  const T* qp = Q + r0 * np + 4 * q;
  const T* sp = S + (r0 * G + blk) * k + jg * JJ;
  const int64_t sstride = (int64_t)G * k;
#pragma unroll 2
  for (int64_t t = r0; t < r1; ++t) {
    T qv[4];
    Vec4<T>::load(qp, qv);
    T sv[JJ];
    if constexpr (JJ >= 4) {
#pragma unroll
      for (int a = 0; a < JJ / 4; ++a) {
        T tmp[4];
        Vec4<T>::load(sp + 4 * a, tmp);
#pragma unroll
        for (int b = 0; b < 4; ++b) sv[4 * a + b] = tmp[b];
      }
    } else {
#pragma unroll
      for (int jj = 0; jj < JJ; ++jj) sv[jj] = sp[jj];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int jj = 0; jj < JJ; ++jj) acc[c][jj] += qv[c] * sv[jj];
    qp += np;
    sp += sstride;
  }
  T* dst = Cpart + ((int64_t)blockIdx.x * np + 4 * q) * k + jg * JJ;
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int jj = 0; jj < JJ; ++jj) dst[(int64_t)c * k + jj] = acc[c][jj];
}

// ---------------------------------------------------------------------------
// reduce: C[idx] = sum_rb Cpart[rb][idx] (fixed order), and in the last CTA
// the scalar step lambda_i = c_i / d_i with the breakdown test.
// grid (ceil(np*k / 32) + (scalar ? 1 : 0)); block 256 = 8 slices x 32 lanes
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_reduce(int64_t nidx, int nrb, const T* __restrict__ Cpart, T* __restrict__ C, PcgState st, int scalar,
         const double* __restrict__ dpart, int ndpart) {
  __shared__ double part[8][33];
  __shared__ int nact_s;
  griddep_launch_dependents();
  griddep_wait();
  const int k = st.k;
  if (scalar && blockIdx.x == gridDim.x - 1) {
    // scalar step for all k columns
    const int it = *st.it;
    const int slot = it & 1;
    __shared__ double red_s[256], dsum_s[kMaxRhs];
    if (threadIdx.x == 0) nact_s = 0;
    sum_partials_cols(dpart, ndpart, k, red_s, dsum_s);
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
      const double d = dsum_s[j];
      int act = st.active[slot][j];
      double lam = 0.0;
      if (act) {
        if (!(d > 0.0) || !isfinite(d)) {
          act = 0;
          st.active[slot][j] = 0;
          st.status[j] = GLM_SUR_BREAKDOWN;
          st.iters[j] = it;
        } else {
          lam = st.c[slot][j] / d;
        }
      }
      st.lam[j] = lam;
      if (act) atomicAdd(&nact_s, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (nact_s == 0) *st.done = 1;
      *st.it = it + 1;
    }
    return;
  }
  // (the reduction CTAs never read the step counter: the scalar CTA of this
  // same launch advances it)
  const int lane = threadIdx.x & 31, sl = threadIdx.x >> 5;
  const int64_t idx = (int64_t)blockIdx.x * 32 + lane;
  // each slice sums its partials in the working precision (four independent
  // chains, fixed order), the eight slices are added in float64
  T s4[4] = {(T)0, (T)0, (T)0, (T)0};
  if (idx < nidx) {
    int r = sl;
    for (; r + 24 < nrb; r += 32) {
#pragma unroll
      for (int a = 0; a < 4; ++a) s4[a] += Cpart[(int64_t)(r + 8 * a) * nidx + idx];
    }
    for (int a = 0; r < nrb; r += 8, a = (a + 1) & 3) s4[a] += Cpart[(int64_t)r * nidx + idx];
  }
  part[sl][lane] = ((double)s4[0] + (double)s4[1]) + ((double)s4[2] + (double)s4[3]);
  __syncthreads();
  if (sl == 0 && idx < nidx) {
    double tot = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) tot += part[q][lane];
    C[idx] = (T)tot;
  }
}

// ---------------------------------------------------------------------------
// proj_update: t = S - Q C;  g = alpha g - lam_j t;  partials of g^T g.
// lam_j = lam[j] when lam != nullptr, else lam_const.
// grid (n_update row ranges, n_ugroups block groups, k / JJ).  A block group
// is a run of whole blocks; thread q of the CTA owns one column quad of the
// group and keeps its 4 x JJ entries of C in registers.  Per row tile:
//   phase 1  part[r][q][jj] = sum_{c < 4} Q[t, 4q + c] C[4q + c, jj]
//   phase 2  t[r, i, jj] = S[t, i, jj] - sum_{q in block i} part[r][q][jj]
// so Q streams once with coalesced 16-byte loads and every C value is read
// from L2 once per CTA.
// ---------------------------------------------------------------------------
template <typename T, int JJ>
__global__ void __launch_bounds__(512)
k_proj_update(int64_t M, int G, int np, int k, int TRB, const T* __restrict__ Q, const T* __restrict__ S,
              T* __restrict__ g, const T* __restrict__ C, const int* __restrict__ poff,
              const int* __restrict__ ug_blk0, int alpha, const double* __restrict__ lam, double lam_const,
              double* __restrict__ cpart, PcgState st, int use_state) {
  extern __shared__ __align__(128) unsigned char smraw[];
  T* part = reinterpret_cast<T*>(smraw);
  __shared__ double red[16 * 16];
  __shared__ T lam_s[JJ];
  const int jg = blockIdx.z, grp = blockIdx.y;
  const int64_t cp_idx = ((int64_t)blockIdx.x * gridDim.y + grp) * k + jg * JJ;
  if (use_state) {
    const int slot = (*st.it - 1) & 1;   // reduce has already advanced the counter
    int any = 0;
    for (int jj = 0; jj < JJ; ++jj) any |= st.active[slot][jg * JJ + jj];
    if (!any) {
      if (threadIdx.x < JJ) cpart[cp_idx + threadIdx.x] = 0.0;
      return;
    }
  }
  if (threadIdx.x < JJ) lam_s[threadIdx.x] = (T)(lam ? lam[jg * JJ + threadIdx.x] : lam_const);
  const int b0 = ug_blk0[grp], b1 = ug_blk0[grp + 1];
  const int q0 = poff[b0] >> 2, nqg = (poff[b1] >> 2) - q0, nbg = b1 - b0;
  const int nqp = nqg + ((33 - (nqg & 31)) & 31);   // padded so that nqp % 32 == 1
  const int tid = threadIdx.x;
  T creg[4][JJ];
  if (tid < nqg) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const T* cr = C + (int64_t)(4 * (q0 + tid) + c) * k + jg * JJ;
#pragma unroll
      for (int jj = 0; jj < JJ; ++jj) creg[c][jj] = cr[jj];
    }
  }
  const int64_t r0 = M * blockIdx.x / gridDim.x, r1 = M * (blockIdx.x + 1) / gridDim.x;
  // g^T g: per-tile partial sums in the working precision, added in float64
  double csd = 0.0;
  __syncthreads();
  for (int64_t t0 = r0; t0 < r1; t0 += TRB) {
    const int tr = (int)((r1 - t0) < (int64_t)TRB ? (r1 - t0) : (int64_t)TRB);
    T cs = 0;
    if (tid < nqg) {
      const T* qp = Q + t0 * np + 4 * (q0 + tid);
      for (int r = 0; r < tr; r += 2) {
        T qv[2][4];
        Vec4<T>::load(qp + (int64_t)r * np, qv[0]);
        if (r + 1 < tr) Vec4<T>::load(qp + (int64_t)(r + 1) * np, qv[1]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (r + h < tr) {
            T* dst = part + (int64_t)(r + h) * JJ * nqp + tid;
#pragma unroll
            for (int jj = 0; jj < JJ; ++jj) {
              T acc = qv[h][0] * creg[0][jj];
#pragma unroll
              for (int c = 1; c < 4; ++c) acc += qv[h][c] * creg[c][jj];
              dst[(int64_t)jj * nqp] = acc;
            }
          }
        }
      }
    }
    __syncthreads();
    const int nout = tr * nbg * JJ;
    constexpr int EB = 4;
    for (int o0 = tid; o0 < nout; o0 += EB * blockDim.x) {
      T sv[EB], gv[EB];
      int64_t gi[EB];
#pragma unroll
      for (int b = 0; b < EB; ++b) {
        const int o = o0 + b * blockDim.x;
        gi[b] = -1;
        if (o < nout) {
          const int rest = o / JJ, ib = rest % nbg, r = rest / nbg;
          gi[b] = ((t0 + r) * G + b0 + ib) * k + jg * JJ + (o % JJ);
          sv[b] = S[gi[b]];
          gv[b] = alpha ? g[gi[b]] : (T)0;
        }
      }
#pragma unroll
      for (int b = 0; b < EB; ++b) {
        const int o = o0 + b * blockDim.x;
        if (o < nout) {
          const int jj = o % JJ, rest = o / JJ, ib = rest % nbg, r = rest / nbg;
          const int qa = (poff[b0 + ib] >> 2) - q0, qb = (poff[b0 + ib + 1] >> 2) - q0;
          T sum = 0;
          const T* pr = part + (int64_t)(r * JJ + jj) * nqp;
          for (int qq = qa; qq < qb; ++qq) sum += pr[qq];
          const T gn = gv[b] - lam_s[jj] * (sv[b] - sum);
          g[gi[b]] = gn;
          cs += gn * gn;
        }
      }
    }
    csd += (double)cs;
    __syncthreads();
  }
  const double tot = reduce_cols_strided<JJ>(csd, red);
  if (tid < JJ) cpart[cp_idx + tid] = tot;
}

// ---------------------------------------------------------------------------
// TMA-streamed variants (all k right-hand sides in one CTA: JJ == k, row
// length G*k*sizeof(T) a multiple of 16 bytes).  One CTA per SM processes a
// contiguous row range in tiles; each tile's rows (contiguous in HBM) are
// brought into shared memory by 1-D bulk copies (cp.async.bulk) completing on
// an mbarrier, NST tiles in flight, so the CTA streams at HBM rate with few
// warps.  Waits are bounded: on timeout the CTA records an error and stops.
// ---------------------------------------------------------------------------

// Thread 0: wait for the tiles still in flight (bounded) before leaving.
__device__ void tma_drain(uint64_t* full, int NST, int next_tile, int issued) {
  for (int t = next_tile; t < issued; ++t) mbar_wait_bounded(&full[t % NST], (t / NST) & 1, kWaitLimitNs);
}

// proj_partial, TMA-streamed: one CTA per SM over a contiguous row range;
// thread q owns column quad q (all JJ == k right-hand sides): per row one
// vector of Q and JJ/4 vectors of S (the rows of its block, shared by the
// warp) give 4 JJ FMAs.  Output layout as k_proj_partial (one partial per CTA).
template <typename T, int JJ>
__global__ void __launch_bounds__(512, 1)
k_proj_partial_tma(int64_t M, int G, int np, int nq, int TR, int NST, const T* __restrict__ Q,
                   const T* __restrict__ S, const int* __restrict__ quad_blk, T* __restrict__ Cpart, PcgState st,
                   int use_state) {
  extern __shared__ __align__(128) unsigned char smraw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smraw);
  T* stage0 = reinterpret_cast<T*>(smraw + 128);
  const int64_t GK = (int64_t)G * JJ;
  const int64_t stage_elems = (int64_t)TR * (np + GK);
  __shared__ int abort_s;
  const int tid = threadIdx.x;
  if (*st.err) return;   // an earlier bounded wait gave up: the run is being abandoned
  if (use_state) {
    const int slot = (*st.it) & 1;
    int any = 0;
    for (int jj = 0; jj < JJ; ++jj) any |= st.active[slot][jj];
    if (!any) return;
  }
  const int64_t r0 = M * blockIdx.x / gridDim.x, r1 = M * (blockIdx.x + 1) / gridDim.x;
  const int ntiles = (int)((r1 - r0 + TR - 1) / TR);
  if (tid == 0) {
    for (int q = 0; q < NST; ++q) mbar_init(&full[q], 1);
    fence_mbar_init();
    abort_s = 0;
  }
  __syncthreads();
  int issued = 0;
  auto issue = [&](int tile) {
    const int sidx = tile % NST;
    const int64_t row0 = r0 + (int64_t)tile * TR;
    const int tr = (int)((r1 - row0) < TR ? (r1 - row0) : TR);
    T* Qs = stage0 + sidx * stage_elems;
    T* Ss = Qs + (int64_t)TR * np;
    const uint32_t bq = (uint32_t)(tr * np * sizeof(T)), bs = (uint32_t)(tr * GK * sizeof(T));
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&full[sidx], bq + bs);
    tma_load_1d(Qs, Q + row0 * np, bq, &full[sidx]);
    tma_load_1d(Ss, S + row0 * GK, bs, &full[sidx]);
  };
  if (tid == 0)
    for (; issued < NST && issued < ntiles; ++issued) issue(issued);
  const bool has = tid < nq;
  const int blk = has ? quad_blk[tid] : 0;
  T acc[4][JJ];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int jj = 0; jj < JJ; ++jj) acc[c][jj] = 0;
  for (int tile = 0; tile < ntiles; ++tile) {
    const int sidx = tile % NST;
    if (tid == 0 && !mbar_wait_bounded(&full[sidx], (tile / NST) & 1, kWaitLimitNs)) {
      abort_s = 1;
      atomicExch(st.err, 1);
    }
    __syncthreads();
    if (abort_s) {
      if (tid == 0) tma_drain(full, NST, tile + 1, issued);
      return;
    }
    const int64_t row0 = r0 + (int64_t)tile * TR;
    const int tr = (int)((r1 - row0) < TR ? (r1 - row0) : TR);
    const T* Qs = stage0 + sidx * stage_elems;
    const T* Ss = Qs + (int64_t)TR * np;
    if (has) {
#pragma unroll 2
      for (int r = 0; r < tr; ++r) {
        T qv[4];
        Vec4<T>::load(Qs + (int64_t)r * np + 4 * tid, qv);
        const T* sp = Ss + (int64_t)r * GK + blk * JJ;
        T sv[JJ];
        if constexpr (JJ >= 4) {
#pragma unroll
          for (int a = 0; a < JJ / 4; ++a) {
            T tmp[4];
            Vec4<T>::load(sp + 4 * a, tmp);
#pragma unroll
            for (int b = 0; b < 4; ++b) sv[4 * a + b] = tmp[b];
          }
        } else {
#pragma unroll
          for (int jj = 0; jj < JJ; ++jj) sv[jj] = sp[jj];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int jj = 0; jj < JJ; ++jj) acc[c][jj] += qv[c] * sv[jj];
      }
    }
    __syncthreads();
    if (tid == 0 && issued < ntiles) issue(issued++);
  }
  if (has) {
    T* dst = Cpart + ((int64_t)blockIdx.x * np + 4 * tid) * JJ;
    if constexpr (sizeof(T) == 4 && JJ % 4 == 0) {
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int a = 0; a < JJ / 4; ++a)
          reinterpret_cast<float4*>(dst + c * JJ)[a] =
              make_float4(acc[c][4 * a], acc[c][4 * a + 1], acc[c][4 * a + 2], acc[c][4 * a + 3]);
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int jj = 0; jj < JJ; ++jj) dst[(int64_t)c * JJ + jj] = acc[c][jj];
    }
  }
}

template <typename T, int JJ>
__global__ void __launch_bounds__(512, 1)
k_proj_update_tma(int64_t M, int G, int np, int nq, int TRB, int NST, const T* __restrict__ Q,
                  const T* __restrict__ S, T* __restrict__ g, const T* __restrict__ C, const int* __restrict__ poff,
                  int alpha, const double* __restrict__ lam, double lam_const, double* __restrict__ cpart,
                  PcgState st, int use_state) {
  extern __shared__ __align__(128) unsigned char smraw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smraw);
  T* stage0 = reinterpret_cast<T*>(smraw + 128);
  const int64_t GK = (int64_t)G * JJ;
  const int64_t stage_elems = (int64_t)TRB * (np + (alpha ? 2 : 1) * GK);
  T* part = stage0 + NST * stage_elems;
  const int nqp = nq + ((33 - (nq & 31)) & 31);   // padded so that nqp % 32 == 1
  __shared__ double red[16 * 16];
  __shared__ T lam_s[JJ];
  __shared__ int abort_s;
  const int tid = threadIdx.x;
  if (*st.err) return;   // an earlier bounded wait gave up: the run is being abandoned
  if (use_state) {
    const int slot = (*st.it - 1) & 1;   // reduce has already advanced the counter
    int any = 0;
    for (int jj = 0; jj < JJ; ++jj) any |= st.active[slot][jj];
    if (!any) {
      if (tid < JJ) cpart[(int64_t)blockIdx.x * JJ + tid] = 0.0;
      return;
    }
  }
  if (tid < JJ) lam_s[tid] = (T)(lam ? lam[tid] : lam_const);
  T creg[4][JJ];
  if (tid < nq) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const T* cr = C + (int64_t)(4 * tid + c) * JJ;
#pragma unroll
      for (int jj = 0; jj < JJ; ++jj) creg[c][jj] = cr[jj];
    }
  }
  const int64_t r0 = M * blockIdx.x / gridDim.x, r1 = M * (blockIdx.x + 1) / gridDim.x;
  const int ntiles = (int)((r1 - r0 + TRB - 1) / TRB);
  if (tid == 0) {
    for (int q = 0; q < NST; ++q) mbar_init(&full[q], 1);
    fence_mbar_init();
    abort_s = 0;
  }
  __syncthreads();
  int issued = 0;
  auto issue = [&](int tile) {
    const int sidx = tile % NST;
    const int64_t row0 = r0 + (int64_t)tile * TRB;
    const int tr = (int)((r1 - row0) < TRB ? (r1 - row0) : TRB);
    T* Qs = stage0 + sidx * stage_elems;
    T* Ss = Qs + (int64_t)TRB * np;
    T* gs = Ss + (int64_t)TRB * GK;
    const uint32_t bq = (uint32_t)(tr * np * sizeof(T)), bs = (uint32_t)(tr * GK * sizeof(T));
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&full[sidx], bq + bs + (alpha ? bs : 0u));
    tma_load_1d(Qs, Q + row0 * np, bq, &full[sidx]);
    tma_load_1d(Ss, S + row0 * GK, bs, &full[sidx]);
    if (alpha) tma_load_1d(gs, g + row0 * GK, bs, &full[sidx]);
  };
  if (tid == 0)
    for (; issued < NST && issued < ntiles; ++issued) issue(issued);
  double csd = 0.0;   // g^T g: per-tile partial sums in T, added in float64
  for (int tile = 0; tile < ntiles; ++tile) {
    const int sidx = tile % NST;
    if (tid == 0 && !mbar_wait_bounded(&full[sidx], (tile / NST) & 1, kWaitLimitNs)) {
      abort_s = 1;
      atomicExch(st.err, 1);
    }
    __syncthreads();
    if (abort_s) {
      if (tid == 0) tma_drain(full, NST, tile + 1, issued);
      return;
    }
    const int64_t row0 = r0 + (int64_t)tile * TRB;
    const int tr = (int)((r1 - row0) < TRB ? (r1 - row0) : TRB);
    const T* Qs = stage0 + sidx * stage_elems;
    const T* Ss = Qs + (int64_t)TRB * np;
    const T* gs = Ss + (int64_t)TRB * GK;
    T cs = 0;
    // part[(r*JJ + jj)*nqp + q]: consecutive threads write consecutive words,
    // and the readers below (consecutive jj) hit distinct banks (nqp % 32 == 1)
    if (tid < nq) {
      for (int r = 0; r < tr; ++r) {
        T qv[4];
        Vec4<T>::load(Qs + (int64_t)r * np + 4 * tid, qv);
        T* dst = part + (int64_t)r * JJ * nqp + tid;
#pragma unroll
        for (int jj = 0; jj < JJ; ++jj) {
          T acc = qv[0] * creg[0][jj];
#pragma unroll
          for (int c = 1; c < 4; ++c) acc += qv[c] * creg[c][jj];
          dst[(int64_t)jj * nqp] = acc;
        }
      }
    }
    __syncthreads();
    const int nout = tr * G * JJ;
    for (int o = tid; o < nout; o += blockDim.x) {
      const int jj = o % JJ, rest = o / JJ, i = rest % G, r = rest / G;
      const int qa = __ldg(poff + i) >> 2, qb = __ldg(poff + i + 1) >> 2;
      T sum = 0;
      const T* pr = part + (int64_t)(r * JJ + jj) * nqp;
      for (int qq = qa; qq < qb; ++qq) sum += pr[qq];
      const T gold = alpha ? gs[o] : (T)0;
      const T gn = gold - lam_s[jj] * (Ss[o] - sum);
      g[row0 * GK + o] = gn;
      cs += gn * gn;
    }
    csd += (double)cs;
    __syncthreads();
    if (tid == 0 && issued < ntiles) issue(issued++);
  }
  const double tot = reduce_cols_strided<JJ>(csd, red);
  if (tid < JJ) cpart[(int64_t)blockIdx.x * JJ + tid] = tot;
}

// Projection update, "block x column" form (TMA-streamed, JJ == k, n_i <= 32):
// thread = (block i, right-hand side jj) [x row group], holding C[c, jj] of
// its block's columns in registers; per row it forms
//   t = S[t, i, jj] - sum_{c in block i} Q[t, c] C[c, jj]
// directly (no partial buffer, one barrier pair per tile), reading Q from the
// staged tile with 16-byte loads that all threads of a block share.
template <typename T, int JJ, int NP>
__global__ void __launch_bounds__(512, 1)
k_proj_update_bj(int64_t M, int G, int np, int TRB, int NST, const T* __restrict__ Q, const T* __restrict__ S,
                 T* __restrict__ g, const T* __restrict__ C, const int* __restrict__ poff, int alpha,
                 const double* __restrict__ lam, double lam_const, double* __restrict__ cpart, PcgState st,
                 int use_state) {
  extern __shared__ __align__(128) unsigned char smraw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smraw);
  T* stage0 = reinterpret_cast<T*>(smraw + 128);
  const int64_t GK = (int64_t)G * JJ;
  const int64_t stage_elems = (int64_t)TRB * (np + (alpha ? 2 : 1) * GK);
  __shared__ double red[16 * 16];
  __shared__ T lam_s[JJ];
  __shared__ int abort_s;
  const int tid = threadIdx.x;
  if (*st.err) return;
  if (use_state) {
    const int slot = (*st.it - 1) & 1;
    int any = 0;
    for (int jj = 0; jj < JJ; ++jj) any |= st.active[slot][jj];
    if (!any) {
      if (tid < JJ) cpart[(int64_t)blockIdx.x * JJ + tid] = 0.0;
      return;
    }
  }
  if (tid < JJ) lam_s[tid] = (T)(lam ? lam[tid] : lam_const);
  const int npairs = G * JJ;
  const int nrg = npairs >= (int)blockDim.x ? 1 : (int)blockDim.x / npairs;
  const int rg = tid / (npairs < (int)blockDim.x ? npairs : (int)blockDim.x);
  const bool busy = rg < nrg;
  // the pairs of this thread, their quad ranges and C values
  int pc0[NP], nqi[NP], jjp[NP], ip[NP];
  bool has[NP];
  T creg[NP][8][4];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    const int pr = (npairs < (int)blockDim.x ? tid % npairs : tid) + a * blockDim.x;
    has[a] = busy && pr < npairs;
    const int i = has[a] ? pr / JJ : 0, jj = pr % JJ;
    ip[a] = i;
    jjp[a] = jj;
    pc0[a] = has[a] ? poff[i] : 0;
    nqi[a] = has[a] ? (poff[i + 1] - poff[i]) >> 2 : 0;
#pragma unroll
    for (int qq = 0; qq < 8; ++qq)
#pragma unroll
      for (int c = 0; c < 4; ++c)
        creg[a][qq][c] = (qq < nqi[a]) ? C[(int64_t)(pc0[a] + 4 * qq + c) * JJ + jj] : (T)0;
  }
  const int64_t r0 = M * blockIdx.x / gridDim.x, r1 = M * (blockIdx.x + 1) / gridDim.x;
  const int ntiles = (int)((r1 - r0 + TRB - 1) / TRB);
  if (tid == 0) {
    for (int q = 0; q < NST; ++q) mbar_init(&full[q], 1);
    fence_mbar_init();
    abort_s = 0;
  }
  __syncthreads();
  int issued = 0;
  auto issue = [&](int tile) {
    const int sidx = tile % NST;
    const int64_t row0 = r0 + (int64_t)tile * TRB;
    const int tr = (int)((r1 - row0) < TRB ? (r1 - row0) : TRB);
    T* Qs = stage0 + sidx * stage_elems;
    T* Ss = Qs + (int64_t)TRB * np;
    T* gs = Ss + (int64_t)TRB * GK;
    const uint32_t bq = (uint32_t)(tr * np * sizeof(T)), bs = (uint32_t)(tr * GK * sizeof(T));
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&full[sidx], bq + bs + (alpha ? bs : 0u));
    tma_load_1d(Qs, Q + row0 * np, bq, &full[sidx]);
    tma_load_1d(Ss, S + row0 * GK, bs, &full[sidx]);
    if (alpha) tma_load_1d(gs, g + row0 * GK, bs, &full[sidx]);
  };
  if (tid == 0)
    for (; issued < NST && issued < ntiles; ++issued) issue(issued);
  double csd = 0.0;   // g^T g: per-tile partial sums in T, added in float64
  for (int tile = 0; tile < ntiles; ++tile) {
    const int sidx = tile % NST;
    if (tid == 0 && !mbar_wait_bounded(&full[sidx], (tile / NST) & 1, kWaitLimitNs)) {
      abort_s = 1;
      atomicExch(st.err, 1);
    }
    __syncthreads();
    if (abort_s) {
      if (tid == 0) tma_drain(full, NST, tile + 1, issued);
      return;
    }
    const int64_t row0 = r0 + (int64_t)tile * TRB;
    const int tr = (int)((r1 - row0) < TRB ? (r1 - row0) : TRB);
    const T* Qs = stage0 + sidx * stage_elems;
    const T* Ss = Qs + (int64_t)TRB * np;
    const T* gs = Ss + (int64_t)TRB * GK;
    T cs = 0;
    for (int r = rg; r < tr; r += nrg) {
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        if (has[a]) {
          const T* qrow = Qs + (int64_t)r * np + pc0[a];
          T sum = 0;
#pragma unroll
          for (int qq = 0; qq < 8; ++qq) {
            if (qq < nqi[a]) {
              T qv[4];
              Vec4<T>::load(qrow + 4 * qq, qv);
#pragma unroll
              for (int c = 0; c < 4; ++c) sum += qv[c] * creg[a][qq][c];
            }
          }
          const int64_t o = (int64_t)r * GK + (int64_t)ip[a] * JJ + jjp[a];
          const T gold = alpha ? gs[o] : (T)0;
          const T gn = gold - lam_s[jjp[a]] * (Ss[o] - sum);
          g[row0 * GK + o] = gn;
          cs += gn * gn;
        }
      }
    }
    csd += (double)cs;
    __syncthreads();
    if (tid == 0 && issued < ntiles) issue(issued++);
  }
  // per-column sums: thread's columns are jjp[a]; with npairs a multiple of JJ
  // and blockDim a multiple of JJ every thread's jj is tid % JJ
  const double tot = reduce_cols_strided<JJ>(csd, red);
  if (tid < JJ) cpart[(int64_t)blockIdx.x * JJ + tid] = tot;
}

// S = U Omega on a staged row tile of float32 U (row stride GK = G JJ), items
// (RR rows, h quad, jj quad); dq[c] accumulates d = u.S of the thread's
// right-hand sides 4 (tid % (JJ/4)) + c in float64 per tile.
template <int RR, int JJ>
__device__ __forceinline__ void sigma_quads(const float* __restrict__ us, const float* __restrict__ Om_s,
                                            float* __restrict__ S, int64_t row0, int tr, int G, int Gq, int64_t GK,
                                            double (&dsq)[4]) {
  constexpr int JQ = JJ / 4;
  const int nhq = Gq >> 2;
  const int ngrp = (tr + RR - 1) / RR;
  const int nitems = ngrp * nhq * JQ;
  const int jq = threadIdx.x % JQ;   // fixed per thread: blockDim is a multiple of JQ
  float dq[4] = {0.f, 0.f, 0.f, 0.f};
  for (int itm = threadIdx.x; itm < nitems; itm += blockDim.x) {
    const int rest = itm / JQ;
    const int hq = rest % nhq, tg = rest / nhq;
    const float* ur[RR];
#pragma unroll
    for (int a = 0; a < RR; ++a) {
      const int t = RR * tg + a;
      ur[a] = us + (int64_t)(t < tr ? t : RR * tg) * GK + 4 * jq;
    }
    float4 acc[RR][4];
#pragma unroll
    for (int a = 0; a < RR; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][c] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int gg = 0; gg < G; ++gg) {
      const float4 om = *reinterpret_cast<const float4*>(Om_s + (int64_t)gg * Gq + 4 * hq);
      const float oc[4] = {om.x, om.y, om.z, om.w};
#pragma unroll
      for (int a = 0; a < RR; ++a) {
        const float4 v = *reinterpret_cast<const float4*>(ur[a] + gg * JJ);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          acc[a][c].x += v.x * oc[c];
          acc[a][c].y += v.y * oc[c];
          acc[a][c].z += v.z * oc[c];
          acc[a][c].w += v.w * oc[c];
        }
      }
    }
#pragma unroll
    for (int a = 0; a < RR; ++a) {
      const int t = RR * tg + a;
      if (t < tr) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int h = 4 * hq + c;
          if (h < G) {
            *reinterpret_cast<float4*>(S + (row0 + t) * GK + h * JJ + 4 * jq) = acc[a][c];
            const float4 uh = *reinterpret_cast<const float4*>(ur[a] + h * JJ);
            dq[0] += acc[a][c].x * uh.x;
            dq[1] += acc[a][c].y * uh.y;
            dq[2] += acc[a][c].z * uh.z;
            dq[3] += acc[a][c].w * uh.w;
          }
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) dsq[c] += (double)dq[c];
}

// S = U Omega for one right-hand side (row stride G, G a multiple of 4):
// items (RR rows, h quad); per four g one float4 of U per row and four float4
// Omega rows give 16 RR FMAs.  Returns the thread's part of d = u.S.
template <int RR>
__device__ __forceinline__ float sigma_k1(const float* __restrict__ us, const float* __restrict__ Om_s,
                                          float* __restrict__ S, int64_t row0, int tr, int G, int Gq) {
  const int nhq = Gq >> 2;
  const int ngrp = (tr + RR - 1) / RR;
  const int nitems = ngrp * nhq;
  float dl = 0.f;
  for (int itm = threadIdx.x; itm < nitems; itm += blockDim.x) {
    const int hq = itm % nhq, tg = itm / nhq;
    const float* ur[RR];
#pragma unroll
    for (int a = 0; a < RR; ++a) {
      const int t = RR * tg + a;
      ur[a] = us + (int64_t)(t < tr ? t : RR * tg) * G;
    }
    float acc[RR][4];
#pragma unroll
    for (int a = 0; a < RR; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;
    for (int g0 = 0; g0 < G; g0 += 4) {
      float4 uv[RR];
#pragma unroll
      for (int a = 0; a < RR; ++a) uv[a] = *reinterpret_cast<const float4*>(ur[a] + g0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 om = *reinterpret_cast<const float4*>(Om_s + (int64_t)(g0 + q) * Gq + 4 * hq);
#pragma unroll
        for (int a = 0; a < RR; ++a) {
          const float x = q == 0 ? uv[a].x : q == 1 ? uv[a].y : q == 2 ? uv[a].z : uv[a].w;
          acc[a][0] += x * om.x;
          acc[a][1] += x * om.y;
          acc[a][2] += x * om.z;
          acc[a][3] += x * om.w;
        }
      }
    }
#pragma unroll
    for (int a = 0; a < RR; ++a) {
      const int t = RR * tg + a;
      if (t < tr) {
        // the h quad lies inside the row: G is a multiple of 4
        *reinterpret_cast<float4*>(S + (row0 + t) * G + 4 * hq) = make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
        const float4 uh = *reinterpret_cast<const float4*>(ur[a] + 4 * hq);
        dl += acc[a][0] * uh.x + acc[a][1] * uh.y + acc[a][2] * uh.z + acc[a][3] * uh.w;
      }
    }
  }
  return dl;
}

// float32 with whole quads of right-hand sides: the TMA sigma step works on
// float4 (four right-hand sides) per thread
template <typename T, int JJ>
constexpr bool kQuadSigma = sizeof(T) == 4 && JJ % 4 == 0 && JJ >= 4;

template <typename T, int JJ, int RI>
__global__ void __launch_bounds__(512, 1)
k_sigma_step_tma(int64_t M, int64_t Ms, int G, int Gq, int TR, int NST, const T* __restrict__ Om, const T* __restrict__ g,
                 T* __restrict__ u, T* __restrict__ w, T* __restrict__ S, T* __restrict__ wbest, PcgState st,
                 const double* __restrict__ cpart, int ncpart, double* __restrict__ dpart) {
  extern __shared__ __align__(128) unsigned char smraw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smraw);
  T* Om_s = reinterpret_cast<T*>(smraw + 128);
  T* stage0 = Om_s + (int64_t)G * Gq;
  const int64_t GK = (int64_t)G * JJ;
  const int64_t stage_elems = (int64_t)TR * 3 * GK;
  __shared__ double red[16 * 16];
  __shared__ T mu_s[JJ], lamp_s[JJ];   // in the working precision: no conversion per element
  __shared__ int act_s[JJ], snap_s[JJ], anyp_s, abort_s;
  const int tid = threadIdx.x;
  if (*st.err) return;   // an earlier bounded wait gave up: the run is being abandoned
  if (tid == 0) anyp_s = 0;
  const double csum = sum_partials<JJ>(cpart, ncpart, JJ, 0, red);
  if (tid < JJ) {
    const StepScalars sc = step_prologue(st, tid, JJ, csum, blockIdx.x == 0);
    mu_s[tid] = (T)sc.mu;
    lamp_s[tid] = (T)sc.lam_prev;
    act_s[tid] = sc.act;
    snap_s[tid] = sc.snap;
    if (sc.act_prev) atomicOr(&anyp_s, 1);
  }
  __syncthreads();
  if (!anyp_s) return;   // every column already stopped: nothing changes
  for (int64_t e = tid; e < (int64_t)G * Gq; e += blockDim.x) Om_s[e] = Om[e];
  const int64_t r0 = M * blockIdx.x / gridDim.x, r1 = M * (blockIdx.x + 1) / gridDim.x;
  const int ntiles = (int)((r1 - r0 + TR - 1) / TR);
  if (tid == 0) {
    for (int q = 0; q < NST; ++q) mbar_init(&full[q], 1);
    fence_mbar_init();
    abort_s = 0;
  }
  __syncthreads();
  int issued = 0;
  auto issue = [&](int tile) {
    const int sidx = tile % NST;
    const int64_t row0 = r0 + (int64_t)tile * TR;
    const int tr = (int)((r1 - row0) < TR ? (r1 - row0) : TR);
    T* gs = stage0 + sidx * stage_elems;
    const uint32_t bs = (uint32_t)(tr * GK * sizeof(T));
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&full[sidx], 3 * bs);
    tma_load_1d(gs, g + row0 * GK, bs, &full[sidx]);
    tma_load_1d(gs + (int64_t)TR * GK, u + row0 * GK, bs, &full[sidx]);
    tma_load_1d(gs + (int64_t)2 * TR * GK, w + row0 * GK, bs, &full[sidx]);
  };
  if (tid == 0)
    for (; issued < NST && issued < ntiles; ++issued) issue(issued);
  const int nhq = Gq >> 2;
  const int jj_t = tid % JJ;
  double dsum = 0.0;
  double dsq[4] = {0.0, 0.0, 0.0, 0.0};   // quad path: columns 4 (tid % (JJ/4)) + c
  for (int tile = 0; tile < ntiles; ++tile) {
    const int sidx = tile % NST;
    if (tid == 0 && !mbar_wait_bounded(&full[sidx], (tile / NST) & 1, kWaitLimitNs)) {
      abort_s = 1;
      atomicExch(st.err, 1);
    }
    __syncthreads();
    if (abort_s) {
      if (tid == 0) tma_drain(full, NST, tile + 1, issued);
      return;
    }
    const int64_t row0 = r0 + (int64_t)tile * TR;
    const int tr = (int)((r1 - row0) < TR ? (r1 - row0) : TR);
    const T* gs = stage0 + sidx * stage_elems;
    T* us = const_cast<T*>(gs) + (int64_t)TR * GK;
    const T* ws = gs + (int64_t)2 * TR * GK;
    // elementwise (contiguous tile): w -= lam_prev u_old ; u = g + mu u_old
    const int ne = tr * (int)GK;
    if constexpr (kQuadSigma<T, JJ>) {
      // four consecutive right-hand sides per thread (float4 in shared and global memory)
      for (int e4 = tid; e4 < (ne >> 2); e4 += blockDim.x) {
        const int jj0 = (4 * e4) % JJ;
        float4 uo = reinterpret_cast<const float4*>(us)[e4];
        const float4 wo = reinterpret_cast<const float4*>(ws)[e4];
        const float4 go = reinterpret_cast<const float4*>(gs)[e4];
        const float4 lp = make_float4(lamp_s[jj0], lamp_s[jj0 + 1], lamp_s[jj0 + 2], lamp_s[jj0 + 3]);
        const float4 wn = make_float4(wo.x - lp.x * uo.x, wo.y - lp.y * uo.y, wo.z - lp.z * uo.z, wo.w - lp.w * uo.w);
        float4* wg = reinterpret_cast<float4*>(w + row0 * GK) + e4;
        if (lp.x != 0.f || lp.y != 0.f || lp.z != 0.f || lp.w != 0.f) *wg = wn;   // unchanged lanes rewrite w
        const int sn = snap_s[jj0] + snap_s[jj0 + 1] + snap_s[jj0 + 2] + snap_s[jj0 + 3];
        if (sn == 4) {
          reinterpret_cast<float4*>(wbest + row0 * GK)[e4] = wn;
        } else if (sn) {
          float* wb = wbest + row0 * GK + 4 * e4;
          if (snap_s[jj0]) wb[0] = wn.x;
          if (snap_s[jj0 + 1]) wb[1] = wn.y;
          if (snap_s[jj0 + 2]) wb[2] = wn.z;
          if (snap_s[jj0 + 3]) wb[3] = wn.w;
        }
        const int na = act_s[jj0] + act_s[jj0 + 1] + act_s[jj0 + 2] + act_s[jj0 + 3];
        if (na) {
          if (act_s[jj0]) uo.x = go.x + mu_s[jj0] * uo.x;
          if (act_s[jj0 + 1]) uo.y = go.y + mu_s[jj0 + 1] * uo.y;
          if (act_s[jj0 + 2]) uo.z = go.z + mu_s[jj0 + 2] * uo.z;
          if (act_s[jj0 + 3]) uo.w = go.w + mu_s[jj0 + 3] * uo.w;
          reinterpret_cast<float4*>(u + row0 * GK)[e4] = uo;   // inactive lanes rewrite their u
          reinterpret_cast<float4*>(us)[e4] = uo;
        }
        // rows t >= Ms have Sigma = 0 (restriction rows): the tile of U that
        // S = U Omega reads is zero there (a float4 never straddles two rows)
        if (row0 + (4 * e4) / GK >= Ms) reinterpret_cast<float4*>(us)[e4] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    } else {
      for (int e = tid; e < ne; e += blockDim.x) {
        const int jj = e % JJ;
        const T uo = us[e];
        const T lp = lamp_s[jj];
        const T wn = ws[e] - lp * uo;
        if (lp != (T)0) w[row0 * GK + e] = wn;
        if (snap_s[jj]) wbest[row0 * GK + e] = wn;
        if (act_s[jj]) {
          const T un = gs[e] + mu_s[jj] * uo;
          u[row0 * GK + e] = un;
          us[e] = un;
        }
        if (row0 + e / GK >= Ms) us[e] = (T)0;   // Sigma = 0 on rows t >= Ms
      }
    }
    __syncthreads();
    if constexpr (kQuadSigma<T, JJ>) {
      // S = U Omega: item = (RR rows, h quad, jj quad); per g one float4 of U
      // per row and one float4 of Omega give 16 RR FMAs.  Two rows per item
      // when the tile has enough items for every thread, else one.
      constexpr int JQ = JJ / 4;
      if (((tr + 1) / 2) * nhq * JQ >= (int)blockDim.x)
        sigma_quads<2, JJ>(reinterpret_cast<const float*>(us), reinterpret_cast<const float*>(Om_s),
                           reinterpret_cast<float*>(S), row0, tr, G, Gq, GK, dsq);
      else
        sigma_quads<1, JJ>(reinterpret_cast<const float*>(us), reinterpret_cast<const float*>(Om_s),
                           reinterpret_cast<float*>(S), row0, tr, G, Gq, GK, dsq);
    } else if (sizeof(T) == 4 && JJ == 1 && (G & 3) == 0) {
      // one right-hand side, G a multiple of 4: items (RR rows, h quad)
      const int nhq1 = Gq >> 2;
      float dl = 0.f;
      if (((tr + 1) / 2) * nhq1 >= (int)blockDim.x)
        dl = sigma_k1<2>(reinterpret_cast<const float*>(us), reinterpret_cast<const float*>(Om_s),
                         reinterpret_cast<float*>(S), row0, tr, G, Gq);
      else
        dl = sigma_k1<1>(reinterpret_cast<const float*>(us), reinterpret_cast<const float*>(Om_s),
                         reinterpret_cast<float*>(S), row0, tr, G, Gq);
      dsum += (double)dl;
    } else {
    // S = U Omega: item = (RI-row group, h quad, jj), RI x 4 outputs per item
    const int ngrp = (tr + RI - 1) / RI;
    const int nitems = ngrp * nhq * JJ;
    T dloc = 0;
    for (int itm = tid; itm < nitems; itm += blockDim.x) {
      const int rest = itm / JJ;
      const int hq = rest % nhq, tg = rest / nhq;
      const T* ur[RI];
#pragma unroll
      for (int a = 0; a < RI; ++a) {
        const int t = RI * tg + a;
        ur[a] = us + (int64_t)(t < tr ? t : RI * tg) * GK + jj_t;
      }
      T acc[RI][4];
#pragma unroll
      for (int a = 0; a < RI; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = 0;
      for (int gg = 0; gg < G; ++gg) {
        T om[4];
        Vec4<T>::load(Om_s + (int64_t)gg * Gq + 4 * hq, om);
#pragma unroll
        for (int a = 0; a < RI; ++a) {
          const T v = ur[a][gg * JJ];
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[a][c] += v * om[c];
        }
      }
#pragma unroll
      for (int a = 0; a < RI; ++a) {
        const int t = RI * tg + a;
        if (t < tr) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int h = 4 * hq + c;
            if (h < G) {
              S[(row0 + t) * GK + h * JJ + jj_t] = acc[a][c];
              dloc += acc[a][c] * ur[a][h * JJ];
            }
          }
        }
      }
    }
    dsum += (double)dloc;
    }
    __syncthreads();
    if (tid == 0 && issued < ntiles) issue(issued++);
  }
  double d;
  if constexpr (kQuadSigma<T, JJ>) d = reduce_cols_quads<JJ>(dsq, red);
  else d = reduce_cols_strided<JJ>(dsum, red);
  if (tid < JJ) dpart[(int64_t)blockIdx.x * JJ + tid] = d;
}

// ---------------------------------------------------------------------------
// layout conversions and small helpers
// ---------------------------------------------------------------------------

// out[(t*G + i)*k + j] = scale * s_i * Y[j*ldy + i*M + t]   (32 x 32 tiles over
// (t, c = i*k + j)); s_i = blk_scale[i], or 1 when blk_scale is null
template <typename Tout>
__global__ void k_colmajor_to_layout(int64_t M, int G, int k, const double* __restrict__ Y, int64_t ldy,
                                     Tout* __restrict__ out, double scale, const double* __restrict__ blk_scale) {
  __shared__ double tile[32][33];
  const int64_t t0 = (int64_t)blockIdx.x * 32;
  const int64_t c0 = (int64_t)blockIdx.y * 32;
  const int64_t ncol = (int64_t)G * k;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 256 threads: 8 rows of 32
  for (int r = ty; r < 32; r += 8) {
    const int64_t c = c0 + r, t = t0 + tx;
    double v = 0.0;
    if (c < ncol && t < M) {
      const int64_t i = c / k, j = c % k;
      v = Y[j * ldy + i * M + t];
    }
    tile[r][tx] = v;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t t = t0 + r, c = c0 + tx;
    if (t < M && c < ncol) {
      const double sc = blk_scale ? scale * blk_scale[c / k] : scale;
      out[t * ncol + c] = (Tout)(sc * tile[tx][r]);
    }
  }
}

// Y[j*ldy + i*M + t] = in[(t*G + i)*k + j]
template <typename Tin>
__global__ void k_layout_to_colmajor(int64_t M, int G, int k, const Tin* __restrict__ in, double* __restrict__ Y,
                                     int64_t ldy, const double* __restrict__ blk_scale) {
  __shared__ double tile[32][33];
  const int64_t t0 = (int64_t)blockIdx.x * 32;
  const int64_t c0 = (int64_t)blockIdx.y * 32;
  const int64_t ncol = (int64_t)G * k;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int64_t t = t0 + r, c = c0 + tx;
    tile[r][tx] = (t < M && c < ncol) ? (double)in[t * ncol + c] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t c = c0 + r, t = t0 + tx;
    if (c < ncol && t < M) {
      const int64_t i = c / k, j = c % k;
      Y[j * ldy + i * M + t] = blk_scale ? blk_scale[i] * tile[tx][r] : tile[tx][r];
    }
  }
}

// b_i = s_i R_i^-1 C_i  (back substitution; one thread per (block, column));
// s_i = blk_scale[i], or 1 when blk_scale is null
__global__ void k_tri_solve(int G, int k, const double* __restrict__ R, const int64_t* __restrict__ r_off,
                            const int* __restrict__ n_i, const int* __restrict__ off,
                            const int* __restrict__ poff, const double* __restrict__ C, double* b, int64_t ldb,
                            const double* __restrict__ blk_scale) {
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
  const double sc = blk_scale ? blk_scale[i] : 1.0;
  for (int r = 0; r < ni; ++r) b[(int64_t)j * ldb + off[i] + r] = sc * x[r];
}

// Preconditioner block D = diag(delta) (x) I_M by row scaling: delta_i =
// omega_ii (kind 2) or max_i omega_ii (kind 1); Om_out = D0^-1/2 Om D0^-1/2,
// sqrtd[i] = sqrt(delta_i), isqrtd[i] = 1 / sqrt(delta_i).  A block whose
// delta is not positive keeps delta_i = 1.  One CTA.
__global__ void k_precond_omega(int G, int Gq, int kind, const double* __restrict__ Om, double* __restrict__ Om_out,
                                double* __restrict__ sqrtd, double* __restrict__ isqrtd) {
  __shared__ double dmax;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int i = 0; i < G; ++i) mx = fmax(mx, Om[(int64_t)i * Gq + i]);
    dmax = mx;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < G; i += blockDim.x) {
    double d = kind == 1 ? dmax : Om[(int64_t)i * Gq + i];
    if (!(d > 0.0) || !isfinite(d)) d = 1.0;
    sqrtd[i] = sqrt(d);
    isqrtd[i] = 1.0 / sqrt(d);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < G * Gq; e += blockDim.x) {
    const int a = e / Gq, c = e % Gq;
    Om_out[e] = c < G ? Om[e] * isqrtd[a] * isqrtd[c] : 0.0;
  }
}

template <typename Tin, typename Tout>
__global__ void k_convert(int64_t n, const Tin* __restrict__ in, Tout* __restrict__ out, double scale) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (Tout)(scale * (double)in[e]);
}

// w64 += d (refinement correction)
template <typename Tin>
__global__ void k_add_to_f64(int64_t n, const Tin* __restrict__ d, double* __restrict__ w) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    w[e] += (double)d[e];
}

// start of a refinement run: g = -(T)rho on live columns (0 elsewhere), u = 0,
// w = 0 unless w is null (a float64 restart keeps its w), partials of g^T g
template <typename T>
__global__ void __launch_bounds__(256)
k_init_inner(int64_t M, int Gk, int k, const double* __restrict__ rho, const int* __restrict__ live, T* g, T* u,
             T* w, double* __restrict__ cpart) {
  __shared__ double red[8 * kMaxRhs];
  __shared__ double sq[256];
  const int64_t r0 = M * blockIdx.x / gridDim.x, r1 = M * (blockIdx.x + 1) / gridDim.x;
  const int64_t e0 = r0 * Gk, e1 = r1 * Gk;
  if (blockDim.x == 256 && 256 % k == 0) {
    // e0 is a multiple of k and so is the stride: thread t always meets
    // column t % k, and sums its squares in the same pass
    const int j = threadIdx.x % k;
    const bool on = live == nullptr || live[j];
    double acc = 0.0;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += 256) {
      const T gv = on ? (T)(-rho[e]) : (T)0;
      g[e] = gv;
      u[e] = (T)0;
      if (w) w[e] = (T)0;
      acc += (double)gv * (double)gv;
    }
    sq[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < k) {
      double t = 0.0;
      for (int q = threadIdx.x; q < 256; q += k) t += sq[q];   // fixed order
      cpart[(int64_t)blockIdx.x * k + threadIdx.x] = t;
    }
    return;
  }
  for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    g[e] = (live == nullptr || live[e % k]) ? (T)(-rho[e]) : (T)0;
    u[e] = (T)0;
    if (w) w[e] = (T)0;
  }
  __syncthreads();
  // second pass for the per-column sums (k <= 64): warp w sums column j = w, w+8, ...
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = warp; j < k; j += 8) {
    double s = 0.0;
    for (int64_t e = e0 + j + (int64_t)lane * k; e < e1; e += (int64_t)32 * k) {
      const double v = (double)g[e];
      s += v * v;
    }
    s = warp_sum(s);
    if (lane == 0) red[j] = s;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < k; j += blockDim.x) cpart[(int64_t)blockIdx.x * k + j] = red[j];
}

// per-column sums of squares of a (M, G, k) vector over row ranges (partials)
template <typename T>
__global__ void __launch_bounds__(256)
k_colsumsq(int64_t M, int Gk, int k, const T* __restrict__ v, double* __restrict__ part) {
  const int64_t r0 = M * blockIdx.x / gridDim.x, r1 = M * (blockIdx.x + 1) / gridDim.x;
  const int64_t e0 = r0 * Gk, e1 = r1 * Gk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = warp; j < k; j += 8) {
    double s = 0.0;
    for (int64_t e = e0 + j + (int64_t)lane * k; e < e1; e += (int64_t)32 * k) {
      const double x = (double)v[e];
      s += x * x;
    }
    s = warp_sum(s);
    if (lane == 0) part[(int64_t)blockIdx.x * k + j] = s;
  }
}

// w[e] += sign * d[e] for the columns j = e % k with mask[j] != 0
__global__ void k_masked_axpy(int64_t n, int k, const int* __restrict__ mask, double sign,
                              const double* __restrict__ d, double* __restrict__ w) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    if (mask[e % k]) w[e] += sign * d[e];
}

// Om32[i][i] += rel * max_i Om64[i][i]   (one thread: G <= 1024)
__global__ void k_shift_diag(int G, int Gq, const double* __restrict__ Om64, float* __restrict__ Om32, double rel) {
  if (threadIdx.x != 0 || blockIdx.x != 0 || rel == 0.0) return;
  double mx = 0.0;
  for (int i = 0; i < G; ++i) mx = fmax(mx, Om64[(int64_t)i * Gq + i]);
  const double sh = rel * mx;
  for (int i = 0; i < G; ++i) Om32[(int64_t)i * Gq + i] = (float)(Om64[(int64_t)i * Gq + i] + sh);
}

__global__ void k_add_int(int n, const int* __restrict__ a, int* __restrict__ acc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) acc[j] += a[j];
}

// After a run: columns that stopped without converging and whose saved w has
// a smaller c than the final one take the saved w (best iterate).
template <typename T>
__global__ void k_restore_best(int64_t n, int k, PcgState st, const T* __restrict__ wbest, T* __restrict__ w) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % k);
    const int slot = (*st.it) & 1;
    const double cs = st.csnap[slot][j] < st.csnap[slot ^ 1][j] ? st.csnap[slot][j] : st.csnap[slot ^ 1][j];
    if (st.status[j] != GLM_SUR_OK && st.status[j] != kStatusRunning && !(st.cstop[j] <= cs)) w[e] = wbest[e];
  }
}
__global__ void k_restore_relres(int k, PcgState st) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  const int slot = (*st.it) & 1;
  const double cs = st.csnap[slot][j] < st.csnap[slot ^ 1][j] ? st.csnap[slot][j] : st.csnap[slot ^ 1][j];
  if (st.status[j] != GLM_SUR_OK && st.status[j] != kStatusRunning && !(st.cstop[j] <= cs) && st.c1[j] > 0)
    st.relres[j] = sqrt(cs / st.c1[j]);
}

// finalize sums of partials: out[j] = sqrt(sum_p part[p*k+j])
__global__ void k_sum_partials_sqrt(int np_, int k, const double* __restrict__ part, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  double s = 0.0;
  for (int p = 0; p < np_; ++p) s += part[(int64_t)p * k + j];
  out[j] = sqrt(s);
}

// Q_cm[c*ldq + t] = Q[t*np + poff(blk(c)) + c - off(blk(c))]   (padded row-major -> column-major)
__global__ void k_unpad_q(int64_t M, int G, int np, const int* __restrict__ off, const int* __restrict__ poff,
                          const double* __restrict__ Q, double* __restrict__ out, int64_t ldq) {
  const int i = blockIdx.y;
  const int ni = off[i + 1] - off[i];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < M * ni; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = e % M;
    const int c = (int)(e / M);
    out[(int64_t)(off[i] + c) * ldq + t] = Q[t * np + poff[i] + c];
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <typename T, int JJ>
static void launch_sigma_step_jj(const IterPlan& p, const Geom& gm, int k, const T* Om, T* g, T* u, T* w, T* S,
                                 T* wbest, const PcgState& st, const double* cpart, double* dpart, cudaStream_t s) {
  if (p.tma_sigma) {
#define SIG_(R)                                                                                                  \
  k_sigma_step_tma<T, JJ, R><<<p.n_sigma, 512, p.sigma_tma_smem, s>>>(gm.M, gm.Ms, gm.G, gm.Gq, p.tr_tma, p.nst_sigma, Om, \
                                                                       g, u, w, S, wbest, st, cpart,          \
                                                                       p.n_cpart + p.extra_cpart, dpart)
    if (p.ri == 4) SIG_(4);
    else if (p.ri == 2) SIG_(2);
    else SIG_(1);
#undef SIG_
    return;
  }
  dim3 grid(p.n_sigma, 1, k / JJ);
  const size_t smem = sizeof(T) * ((size_t)gm.G * gm.Gq + (size_t)p.TR * gm.G * JJ);
  k_sigma_step<T, JJ><<<grid, 256, smem, s>>>(gm.M, gm.Ms, gm.G, gm.Gq, k, p.TR, Om, g, u, w, S, wbest, st, cpart,
                                              p.n_cpart + p.extra_cpart, dpart);
}

template <typename T, int JJ>
static void launch_sigma_resid_jj(const IterPlan& p, const Geom& gm, int k, const T* Om, const T* Y, const T* W,
                                  T* E, cudaStream_t s) {
  dim3 grid(p.n_sigma, 1, k / JJ);
  const size_t smem = sizeof(T) * ((size_t)gm.G * gm.Gq + (size_t)p.TR * gm.G * JJ);
  k_sigma_resid<T, JJ><<<grid, 256, smem, s>>>(gm.M, gm.Ms, gm.G, gm.Gq, k, p.TR, Om, Y, W, E);
}

template <typename T, int JJ>
static void launch_proj_partial_jj(const IterPlan& p, const Geom& gm, int k, const T* Q, const T* S, T* Cpart,
                                   const PcgState& st, int use_state, cudaStream_t s) {
  if (p.tma_partial) {
    k_proj_partial_tma<T, JJ><<<p.n_partial_rows, p.partial_threads, p.partial_tma_smem, s>>>(
        gm.M, gm.G, gm.np, gm.nq, p.tr_partial, p.nst_partial, Q, S, gm.d_quad_blk, Cpart, st, use_state);
    return;
  }
  dim3 grid(p.n_partial_rows, p.n_qgroups, k / JJ);
  const int qpg = (int)ceil_div(gm.nq, p.n_qgroups);
  const int threads = (int)std::min<int64_t>(256, ceil_div(qpg, 32) * 32);
  k_proj_partial<T, JJ><<<grid, threads, 0, s>>>(gm.M, gm.G, gm.np, gm.nq, k, Q, S, gm.d_quad_blk, Cpart, st,
                                                 use_state);
}

template <typename T, int JJ>
static void launch_proj_update_jj(const IterPlan& p, const Geom& gm, int k, const T* Q, const T* S, T* g,
                                  const T* C, int alpha, const double* lam, double lam_const, double* cpart,
                                  const PcgState& st, int use_state, cudaStream_t s) {
  if (p.bj_update) {
    if (p.bj_np == 2)
      k_proj_update_bj<T, JJ, 2><<<p.n_update, 512, p.bj_smem, s>>>(gm.M, gm.G, gm.np, p.trb_bj, p.nst_bj, Q, S, g,
                                                                     C, gm.d_poff, alpha, lam, lam_const, cpart, st,
                                                                     use_state);
    else
      k_proj_update_bj<T, JJ, 1><<<p.n_update, 512, p.bj_smem, s>>>(gm.M, gm.G, gm.np, p.trb_bj, p.nst_bj, Q, S, g,
                                                                     C, gm.d_poff, alpha, lam, lam_const, cpart, st,
                                                                     use_state);
    return;
  }
  if (p.tma_update) {
    k_proj_update_tma<T, JJ><<<p.n_update, p.update_threads, p.update_tma_smem, s>>>(
        gm.M, gm.G, gm.np, gm.nq, p.trb_tma, p.nst_update, Q, S, g, C, gm.d_poff, alpha, lam, lam_const, cpart, st,
        use_state);
    return;
  }
  dim3 grid(p.n_update, p.n_ugroups, k / JJ);
  const size_t smem = p.update_smem;
  k_proj_update<T, JJ><<<grid, p.ug_threads, smem, s>>>(gm.M, gm.G, gm.np, k, p.TRB, Q, S, g, C, gm.d_poff,
                                                         gm.d_ug_blk0, alpha, lam, lam_const, cpart, st, use_state);
}

#define GS_DISPATCH_JJ(JJv, CALL) \
  switch (JJv) {                  \
    case 16: CALL(16); break;     \
    case 8: CALL(8); break;       \
    case 4: CALL(4); break;       \
    case 2: CALL(2); break;       \
    default: CALL(1); break;      \
  }

template <typename T>
void launch_sigma_step(const IterPlan& p, const Geom& gm, int k, const T* Om, T* g, T* u, T* w, T* S, T* wbest,
                       const PcgState& st, const double* cpart, double* dpart, cudaStream_t s) {
#define C_(J) launch_sigma_step_jj<T, J>(p, gm, k, Om, g, u, w, S, wbest, st, cpart, dpart, s)
  GS_DISPATCH_JJ(p.JJ, C_)
#undef C_
}
template <typename T>
void launch_sigma_resid(const IterPlan& p, const Geom& gm, int k, const T* Om, const T* Y, const T* W, T* E,
                        cudaStream_t s) {
#define C_(J) launch_sigma_resid_jj<T, J>(p, gm, k, Om, Y, W, E, s)
  GS_DISPATCH_JJ(p.JJ, C_)
#undef C_
}
template <typename T>
void launch_proj_partial(const IterPlan& p, const Geom& gm, int k, const T* Q, const T* S, T* Cpart,
                         const PcgState& st, int use_state, cudaStream_t s) {
#define C_(J) launch_proj_partial_jj<T, J>(p, gm, k, Q, S, Cpart, st, use_state, s)
  GS_DISPATCH_JJ(p.JJ, C_)
#undef C_
}
template <typename T>
void launch_reduce(const IterPlan& p, const Geom& gm, int k, const T* Cpart, T* C, const PcgState& st, int scalar,
                   const double* dpart, cudaStream_t s, bool pdl) {
  const int64_t nidx = (int64_t)gm.np * k;
  const int nblk = (int)ceil_div(nidx, 32) + (scalar ? 1 : 0);
  if (pdl)
    launch_pdl(k_reduce<T>, dim3(nblk), dim3(256), 0, s, nidx, p.n_partial_rows, Cpart, C, st, scalar, dpart,
               p.n_sigma);
  else
    k_reduce<T><<<nblk, 256, 0, s>>>(nidx, p.n_partial_rows, Cpart, C, st, scalar, dpart, p.n_sigma);
}
template <typename T>
void launch_proj_update(const IterPlan& p, const Geom& gm, int k, const T* Q, const T* S, T* g, const T* C,
                        int alpha, const double* lam, double lam_const, double* cpart, const PcgState& st,
                        int use_state, cudaStream_t s) {
#define C_(J) launch_proj_update_jj<T, J>(p, gm, k, Q, S, g, C, alpha, lam, lam_const, cpart, st, use_state, s)
  GS_DISPATCH_JJ(p.JJ, C_)
#undef C_
}

template <typename Tout>
void launch_colmajor_to_layout(const Geom& gm, int k, const double* Y, int64_t ldy, Tout* out, double scale,
                               cudaStream_t s, const double* blk_scale) {
  dim3 grid((unsigned)ceil_div(gm.M, 32), (unsigned)ceil_div((int64_t)gm.G * k, 32));
  k_colmajor_to_layout<Tout><<<grid, 256, 0, s>>>(gm.M, gm.G, k, Y, ldy, out, scale, blk_scale);
}
template <typename Tin>
void launch_layout_to_colmajor(const Geom& gm, int k, const Tin* in, double* Y, int64_t ldy, cudaStream_t s,
                               const double* blk_scale) {
  dim3 grid((unsigned)ceil_div(gm.M, 32), (unsigned)ceil_div((int64_t)gm.G * k, 32));
  k_layout_to_colmajor<Tin><<<grid, 256, 0, s>>>(gm.M, gm.G, k, in, Y, ldy, blk_scale);
}

void launch_tri_solve(const Geom& gm, int k, const double* R, const double* C, double* b, int64_t ldb,
                      cudaStream_t s, const double* blk_scale) {
  const int n = gm.G * k;
  k_tri_solve<<<(unsigned)ceil_div(n, 128), 128, 0, s>>>(gm.G, k, R, gm.d_r_off, gm.d_n_i, gm.d_off, gm.d_poff, C,
                                                        b, ldb, blk_scale);
}
void launch_precond_omega(int G, int Gq, int kind, const double* Om, double* Om_out, double* sqrtd, double* isqrtd,
                          cudaStream_t s) {
  k_precond_omega<<<1, 256, 0, s>>>(G, Gq, kind, Om, Om_out, sqrtd, isqrtd);
}
template <typename Tin, typename Tout>
void launch_convert(int64_t n, const Tin* in, Tout* out, double scale, cudaStream_t s) {
  k_convert<Tin, Tout><<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 16), 256, 0, s>>>(n, in, out, scale);
}
template <typename Tin>
void launch_add_to_f64(int64_t n, const Tin* d, double* w, cudaStream_t s) {
  k_add_to_f64<Tin><<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 16), 256, 0, s>>>(n, d, w);
}
template void launch_add_to_f64<float>(int64_t, const float*, double*, cudaStream_t);
template void launch_add_to_f64<double>(int64_t, const double*, double*, cudaStream_t);
template <typename T>
void launch_init_inner(const IterPlan& p, const Geom& gm, int k, const double* rho, const int* live, T* g, T* u,
                       T* w, double* cpart, cudaStream_t s) {
  k_init_inner<T><<<p.n_cpart, 256, 0, s>>>(gm.M, gm.G * k, k, rho, live, g, u, w, cpart);
}
template void launch_init_inner<float>(const IterPlan&, const Geom&, int, const double*, const int*, float*, float*,
                                       float*, double*, cudaStream_t);
template void launch_init_inner<double>(const IterPlan&, const Geom&, int, const double*, const int*, double*,
                                        double*, double*, double*, cudaStream_t);
template <typename T>
void launch_colsumsq(const IterPlan& p, const Geom& gm, int k, const T* v, double* part, cudaStream_t s) {
  k_colsumsq<T><<<p.n_cpart, 256, 0, s>>>(gm.M, gm.G * k, k, v, part);
}
void launch_unpad_q(const Geom& gm, const double* Q, double* out, int64_t ldq, cudaStream_t s) {
  dim3 grid((unsigned)std::min<int64_t>(ceil_div(gm.M * 8, 256), 4096), gm.G);
  k_unpad_q<<<grid, 256, 0, s>>>(gm.M, gm.G, gm.np, gm.d_off, gm.d_poff, Q, out, ldq);
}
void launch_masked_axpy(int64_t n, int k, const int* mask, double sign, const double* d, double* w,
                        cudaStream_t s) {
  k_masked_axpy<<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 16), 256, 0, s>>>(n, k, mask, sign, d, w);
}
void launch_shift_diag(int G, int Gq, const double* Om64, float* Om32, double rel, cudaStream_t s) {
  k_shift_diag<<<1, 32, 0, s>>>(G, Gq, Om64, Om32, rel);
}
template <typename T>
void launch_restore_best(int64_t n, int k, const PcgState& st, const T* wbest, T* w, cudaStream_t s) {
  k_restore_best<T><<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 16), 256, 0, s>>>(n, k, st, wbest, w);
  k_restore_relres<<<1, 64, 0, s>>>(k, st);
}
template void launch_restore_best<float>(int64_t, int, const PcgState&, const float*, float*, cudaStream_t);
template void launch_restore_best<double>(int64_t, int, const PcgState&, const double*, double*, cudaStream_t);
void launch_add_int(int n, const int* a, int* acc, cudaStream_t s) {
  k_add_int<<<(unsigned)ceil_div(n, 64), 64, 0, s>>>(n, a, acc);
}
void launch_sum_partials_sqrt(int np_, int k, const double* part, double* out, cudaStream_t s) {
  k_sum_partials_sqrt<<<1, 64, 0, s>>>(np_, k, part, out);
}

template <typename T>
cudaError_t set_smem_attrs(int JJ, size_t bytes, size_t upd_bytes) {
  cudaError_t e = cudaSuccess;
#define C_(J)                                                                                                    \
  e = cudaFuncSetAttribute(k_sigma_step<T, J>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);        \
  if (e == cudaSuccess)                                                                                          \
    e = cudaFuncSetAttribute(k_sigma_resid<T, J>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);     \
  if (e == cudaSuccess)                                                                                          \
    e = cudaFuncSetAttribute(k_proj_update<T, J>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)upd_bytes);
  GS_DISPATCH_JJ(JJ, C_)
#undef C_
  return e;
}

// explicit instantiations
template void launch_sigma_step<double>(const IterPlan&, const Geom&, int, const double*, double*, double*, double*,
                                        double*, double*, const PcgState&, const double*, double*, cudaStream_t);
template void launch_sigma_step<float>(const IterPlan&, const Geom&, int, const float*, float*, float*, float*,
                                       float*, float*, const PcgState&, const double*, double*, cudaStream_t);
template void launch_sigma_resid<double>(const IterPlan&, const Geom&, int, const double*, const double*,
                                         const double*, double*, cudaStream_t);
template void launch_proj_partial<double>(const IterPlan&, const Geom&, int, const double*, const double*, double*,
                                          const PcgState&, int, cudaStream_t);
template void launch_proj_partial<float>(const IterPlan&, const Geom&, int, const float*, const float*, float*,
                                         const PcgState&, int, cudaStream_t);
template void launch_reduce<double>(const IterPlan&, const Geom&, int, const double*, double*, const PcgState&, int,
                                    const double*, cudaStream_t, bool);
template void launch_reduce<float>(const IterPlan&, const Geom&, int, const float*, float*, const PcgState&, int,
                                   const double*, cudaStream_t, bool);
template void launch_proj_update<double>(const IterPlan&, const Geom&, int, const double*, const double*, double*,
                                         const double*, int, const double*, double, double*, const PcgState&, int,
                                         cudaStream_t);
template void launch_proj_update<float>(const IterPlan&, const Geom&, int, const float*, const float*, float*,
                                        const float*, int, const double*, double, double*, const PcgState&, int,
                                        cudaStream_t);
template void launch_colmajor_to_layout<double>(const Geom&, int, const double*, int64_t, double*, double,
                                                cudaStream_t, const double*);
template void launch_layout_to_colmajor<double>(const Geom&, int, const double*, double*, int64_t, cudaStream_t,
                                                const double*);
template void launch_convert<double, float>(int64_t, const double*, float*, double, cudaStream_t);
template void launch_convert<float, double>(int64_t, const float*, double*, double, cudaStream_t);
template void launch_colsumsq<double>(const IterPlan&, const Geom&, int, const double*, double*, cudaStream_t);
template <typename T>
cudaError_t set_tma_smem_attrs(int JJ, size_t sigma_bytes, size_t update_bytes, size_t bj_bytes,
                               size_t partial_bytes) {
  cudaError_t e = cudaSuccess;
#define C_(J)                                                                                                      \
  e = cudaFuncSetAttribute(k_sigma_step_tma<T, J, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sigma_bytes); \
  if (e == cudaSuccess)                                                                                            \
    e = cudaFuncSetAttribute(k_sigma_step_tma<T, J, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,              \
                             (int)sigma_bytes);                                                                    \
  if (e == cudaSuccess)                                                                                            \
    e = cudaFuncSetAttribute(k_sigma_step_tma<T, J, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,              \
                             (int)sigma_bytes);                                                                    \
  if (e == cudaSuccess)                                                                                            \
    e = cudaFuncSetAttribute(k_proj_update_tma<T, J>, cudaFuncAttributeMaxDynamicSharedMemorySize,                 \
                             (int)update_bytes);                                                                   \
  if (e == cudaSuccess)                                                                                            \
    e = cudaFuncSetAttribute(k_proj_update_bj<T, J, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bj_bytes); \
  if (e == cudaSuccess)                                                                                            \
    e = cudaFuncSetAttribute(k_proj_update_bj<T, J, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bj_bytes); \
  if (e == cudaSuccess)                                                                                            \
    e = cudaFuncSetAttribute(k_proj_partial_tma<T, J>, cudaFuncAttributeMaxDynamicSharedMemorySize,               \
                             (int)partial_bytes);
  GS_DISPATCH_JJ(JJ, C_)
#undef C_
  return e;
}
template cudaError_t set_tma_smem_attrs<double>(int, size_t, size_t, size_t, size_t);
template cudaError_t set_tma_smem_attrs<float>(int, size_t, size_t, size_t, size_t);
template cudaError_t set_smem_attrs<double>(int, size_t, size_t);
template cudaError_t set_smem_attrs<float>(int, size_t, size_t);

}  // namespace glmsur
