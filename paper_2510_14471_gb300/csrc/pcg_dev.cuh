// Device helpers shared by the PCG step kernels: the per-column scalar logic
// of the step prologue (stop tests, mu) and deterministic CTA reductions of
// per-thread partial sums.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "internal.h"

namespace glmsur {

// ---------------------------------------------------------------------------
// per-column scalar logic of the step prologue (identical in every CTA)
// ---------------------------------------------------------------------------
struct StepScalars {
  double mu;
  double lam_prev;
  int act;
  int act_prev;
  int snap;   // save w of this step as the best iterate so far
};

__device__ __forceinline__ StepScalars step_prologue(const PcgState& st, int j, int k, double csum, bool writer) {
  StepScalars out{};
  const int it = *st.it;
  out.lam_prev = st.lam[j];
  if (it == 0) {
    const double c1v = csum + (st.c1_extra ? st.c1_extra[j] : 0.0);
    const bool fin = isfinite(csum);
    const bool conv0 = fin && st.c1_extra != nullptr && csum <= st.tol * st.tol * c1v;   // converged at the start
    const bool act = (csum > 0.0) && fin && !conv0;
    out.act = act;
    out.act_prev = 1;
    out.mu = 0.0;
    if (writer) {
      st.c1[j] = c1v;
      st.c[0][j] = csum;
      st.active[0][j] = act;
      st.cbest[0][j] = csum;
      st.itbest[0][j] = 0;
      st.csnap[0][j] = csum;
      st.cstop[j] = csum;
      st.relres[j] = (fin && csum > 0.0) ? sqrt(csum / c1v) : 0.0;
      st.status[j] = act ? kStatusRunning : (fin ? GLM_SUR_OK : GLM_SUR_NONFINITE);
      st.iters[j] = 0;
    }
    return out;
  }
  const int sp = (it - 1) & 1, sc = it & 1;
  const int ap = st.active[sp][j];
  const double cp = st.c[sp][j];
  out.act_prev = ap;
  double cb = st.cbest[sp][j];
  int ib = st.itbest[sp][j];
  const double cs_prev = st.csnap[sp][j];
  if (!ap) {
    out.act = 0;
    out.mu = 0.0;
    if (writer) {
      st.c[sc][j] = cp; st.active[sc][j] = 0; st.cbest[sc][j] = cb; st.itbest[sc][j] = ib;
      st.csnap[sc][j] = cs_prev;
    }
    return out;
  }
  // the w formed in this step (lagged update) is saved when c dropped below
  // a quarter of the c of the previous save
  out.snap = isfinite(csum) && csum < 0.25 * cs_prev;
  const double c1 = st.c1[j];
  const double rr = sqrt(fmax(csum, 0.0) / c1);
  int act = 1, status = kStatusRunning;
  if (csum < cb) { cb = csum; ib = it; }
  // stop tests: breakdown, convergence, stagnation (no new minimum of c for
  // W steps: c need not decrease monotonically), iteration cap
  if (!isfinite(csum) || csum < 0.0) { act = 0; status = GLM_SUR_BREAKDOWN; }
  else if (rr <= st.tol) { act = 0; status = GLM_SUR_OK; }
  else if (st.W > 0 && it - ib >= st.W) { act = 0; status = GLM_SUR_STAGNATED; }
  else if (it >= st.maxit) { act = 0; status = GLM_SUR_NOT_CONVERGED; }
  out.act = act;
  out.mu = act ? csum / cp : 0.0;
  if (writer) {
    st.c[sc][j] = act ? csum : cp;
    st.active[sc][j] = act;
    st.cbest[sc][j] = cb;
    st.itbest[sc][j] = ib;
    st.csnap[sc][j] = out.snap ? csum : cs_prev;
    st.cstop[j] = csum;
    st.relres[j] = rr;
    st.iters[j] = it;
    if (!act) st.status[j] = status;
  }
  return out;
}

// Deterministic CTA reduction of per-thread partial sums, one per column
// jj < JJ, where thread t holds column (t % JJ).  Result valid in threads
// tid < JJ.  `red` needs (blockDim/32) * JJ doubles.
template <int JJ>
__device__ __forceinline__ double reduce_cols_strided(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int off = 16; off >= JJ; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __syncthreads();
  if (lane < JJ) red[warp * JJ + lane] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < JJ)
    for (int w = 0; w < nw; ++w) s += red[w * JJ + threadIdx.x];
  return s;
}

// Same reduction when every thread holds four columns, 4 (tid % (JJ/4)) + c
// (c = 0..3).  Valid in threads tid < JJ.
template <int JJ>
__device__ __forceinline__ double reduce_cols_quads(const double (&v)[4], double* red) {
  constexpr int JQ = JJ / 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double x[4] = {v[0], v[1], v[2], v[3]};
#pragma unroll
  for (int off = 16; off >= JQ; off >>= 1)
#pragma unroll
    for (int c = 0; c < 4; ++c) x[c] += __shfl_xor_sync(0xffffffffu, x[c], off);
  __syncthreads();
  if (lane < JQ)
#pragma unroll
    for (int c = 0; c < 4; ++c) red[warp * JJ + 4 * lane + c] = x[c];
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < JJ)
    for (int w = 0; w < nw; ++w) s += red[w * JJ + threadIdx.x];
  return s;
}

// out[jj] = sum_{p < np} part[p*k + j0 + jj] for jj < JJ, using the whole CTA
// (fixed order: deterministic).  Valid in threads tid < JJ.
template <int JJ>
__device__ __forceinline__ double sum_partials(const double* __restrict__ part, int np, int k, int j0, double* red) {
  const int jj = threadIdx.x % JJ, P = blockDim.x / JJ, q = threadIdx.x / JJ;
  double v = 0.0;
#pragma unroll 4
  for (int p = q; p < np; p += P) v += part[(int64_t)p * k + j0 + jj];
  return reduce_cols_strided<JJ>(v, red);
}

// Same for a runtime number of columns k <= blockDim: out[j] = sum_p part[p*k + j],
// written to out_s[j] (shared).  Tree over a power-of-two number of slices.
__device__ __forceinline__ void sum_partials_cols(const double* __restrict__ part, int np, int k, double* red, double* out_s) {
  int P = 1;
  while (P * 2 * k <= (int)blockDim.x) P *= 2;
  const int j = threadIdx.x % k, q = threadIdx.x / k;
  double v = 0.0;
  if (q < P)
    for (int p = q; p < np; p += P) v += part[(int64_t)p * k + j];
  __syncthreads();
  if (q < P) red[q * k + j] = v;
  __syncthreads();
  for (int h = P / 2; h >= 1; h >>= 1) {
    if (q < h) red[q * k + j] += red[(q + h) * k + j];
    __syncthreads();
  }
  if (threadIdx.x < k) out_s[threadIdx.x] = red[threadIdx.x];
  __syncthreads();
}

// Every thread holds JJ partial sums (one per column); result in tid < JJ.
template <int JJ>
__device__ __forceinline__ double reduce_cols_all(const double (&v)[JJ], double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
#pragma unroll
  for (int jj = 0; jj < JJ; ++jj) {
    const double s = warp_sum(v[jj]);
    if (lane == 0) red[warp * JJ + jj] = s;
  }
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < JJ)
    for (int w = 0; w < nw; ++w) s += red[w * JJ + threadIdx.x];
  return s;
}

}  // namespace glmsur
