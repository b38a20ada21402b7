// PCG-NE kernels: the n-space half of one CG step on the normal equations
// (the m-space half, X p = Q (R p), -Sigma^-1 v and Q^T s, runs on the
// projection and Sigma kernels of the PCG-Aug step).
#include <cuda_runtime.h>

#include "common.cuh"
#include "ne.h"

namespace glmsur {

namespace {

constexpr int kNeThreads = 256;

// deterministic CTA sum: warp sums, then the warps' sums in order by thread 0
__device__ double cta_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kNeThreads / 32; ++w) t += red[w];
    red[32] = t;
  }
  __syncthreads();
  return red[32];
}

__global__ void k_ne_rmul(int n, int k, const double* __restrict__ R, const int64_t* __restrict__ r_off,
                          const int* __restrict__ n_i, const int* __restrict__ off, const int* __restrict__ poff,
                          const int* __restrict__ col_blk, const double* __restrict__ p, double* __restrict__ cvec) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= (int64_t)n * k) return;
  const int col = (int)(id / k), j = (int)(id % k);
  const int i = col_blk[col], ni = n_i[i], r = col - off[i];
  const double* Ri = R + r_off[i];
  double s = 0.0;
  for (int c = r; c < ni; ++c) s += Ri[r * ni + c] * p[(int64_t)(off[i] + c) * k + j];
  cvec[(int64_t)(poff[i] + r) * k + j] = s;
}

// one CTA per right-hand side j
__global__ void __launch_bounds__(kNeThreads)
k_ne_step(int n, int k, const double* __restrict__ R, const int64_t* __restrict__ r_off,
          const int* __restrict__ n_i, const int* __restrict__ off, const int* __restrict__ poff,
          const int* __restrict__ col_blk, const double* __restrict__ C, NeState st, int init) {
  __shared__ double red[33];
  const int j = blockIdx.x;
  if (!init && !st.active[j]) return;
  // q = -[R_i^T C_i]: q[off_i + c] = -sum_{r <= c} R_i[r][c] C[poff_i + r]
  double dp = 0.0;
  for (int col = threadIdx.x; col < n; col += kNeThreads) {
    const int i = col_blk[col], ni = n_i[i], c = col - off[i];
    const double* Ri = R + r_off[i];
    double q = 0.0;
    for (int r = 0; r <= c; ++r) q += Ri[r * ni + c] * C[(int64_t)(poff[i] + r) * k + j];
    q = -q;
    const int64_t e = (int64_t)col * k + j;
    if (init) {
      // beta_1 = 0: f_1 = -h, p_1 = f_1
      st.beta[e] = 0.0;
      st.f[e] = -q;
      st.p[e] = -q;
      dp += q * q;
    } else {
      st.q[e] = q;
      dp += st.p[e] * q;
    }
  }
  const double d = cta_sum(dp, red);
  if (init) {
    if (threadIdx.x == 0) {
      st.c[j] = d;
      st.c1[j] = d;
      st.iters[j] = 0;
      const bool fin = isfinite(d);
      st.active[j] = fin && d > 0.0;
      st.status[j] = !fin ? (int)GLM_SUR_NONFINITE : (d > 0.0 ? kStatusRunning : (int)GLM_SUR_OK);
      st.relres[j] = d > 0.0 ? 1.0 : 0.0;
    }
    return;
  }
  const double c = st.c[j];
  if (!(d > 0.0) || !isfinite(d)) {
    // p^T A p not positive: breakdown (A is positive definite in exact arithmetic)
    if (threadIdx.x == 0) {
      st.active[j] = 0;
      st.status[j] = GLM_SUR_BREAKDOWN;
    }
    return;
  }
  const double lam = c / d;
  double ff = 0.0;
  for (int col = threadIdx.x; col < n; col += kNeThreads) {
    const int64_t e = (int64_t)col * k + j;
    st.beta[e] -= lam * st.p[e];
    const double fn = st.f[e] - lam * st.q[e];
    st.f[e] = fn;
    ff += fn * fn;
  }
  const double cn = cta_sum(ff, red);
  const int it = st.iters[j] + 1;
  const double rr = sqrt(cn / st.c1[j]);
  bool stop = true;
  int status = kStatusRunning;
  if (!isfinite(cn)) status = GLM_SUR_NONFINITE;
  else if (rr <= st.tol) status = GLM_SUR_OK;
  else if (it >= st.maxit) status = GLM_SUR_NOT_CONVERGED;
  else stop = false;
  if (!stop) {
    const double mu = cn / c;
    for (int col = threadIdx.x; col < n; col += kNeThreads) {
      const int64_t e = (int64_t)col * k + j;
      st.p[e] = st.f[e] + mu * st.p[e];
    }
  }
  if (threadIdx.x == 0) {
    st.iters[j] = it;
    st.relres[j] = rr;
    st.c[j] = cn;
    st.status[j] = status;
    if (stop) st.active[j] = 0;
  }
}

__global__ void k_ne_store(int n, int k, const double* __restrict__ beta, double* __restrict__ b, int64_t ldb) {
  const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= (int64_t)n * k) return;
  const int col = (int)(id / k), j = (int)(id % k);
  b[(int64_t)j * ldb + col] = beta[id];
}

}  // namespace

void launch_ne_rmul(const Geom& gm, int k, const double* R, const double* p, double* cvec, cudaStream_t s) {
  const int64_t tot = (int64_t)gm.n * k;
  k_ne_rmul<<<(unsigned)ceil_div(tot, 256), 256, 0, s>>>(gm.n, k, R, gm.d_r_off, gm.d_n_i, gm.d_off, gm.d_poff,
                                                         gm.d_col_blk, p, cvec);
}

void launch_ne_step(const Geom& gm, int k, const double* R, const double* C, const NeState& st, int init,
                    cudaStream_t s) {
  k_ne_step<<<k, kNeThreads, 0, s>>>(gm.n, k, R, gm.d_r_off, gm.d_n_i, gm.d_off, gm.d_poff, gm.d_col_blk, C, st,
                                     init);
}

void launch_ne_store(const Geom& gm, int k, const double* beta, double* b, int64_t ldb, cudaStream_t s) {
  const int64_t tot = (int64_t)gm.n * k;
  k_ne_store<<<(unsigned)ceil_div(tot, 256), 256, 0, s>>>(gm.n, k, beta, b, ldb);
}

}  // namespace glmsur
