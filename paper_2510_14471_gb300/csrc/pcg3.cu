// Vector and scalar kernels of Algorithm glmpcg3 (float64); the projections
// and the Sigma-apply run on the kernels of the PCG-Aug step.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "pcg3.h"

namespace glmsur {

namespace {

constexpr int kP3Threads = 256;

// thread (g, j) of a CTA sums column j over the elements e = j + k (g + G_n t)
// of the CTA's rows, in a fixed order; then the groups in order
__global__ void __launch_bounds__(kP3Threads)
k_pcg3_dot(int64_t M, int GK, int k, const double* __restrict__ u, const double* __restrict__ Sm, Pcg3State st) {
  __shared__ double part[kP3Threads];
  const int groups = kP3Threads / k;
  const int t = threadIdx.x, g = t / k, j = t % k;
  const int64_t r0 = M * blockIdx.x / gridDim.x, r1 = M * (blockIdx.x + 1) / gridDim.x;
  const int64_t e0 = r0 * GK, e1 = r1 * GK;   // e % k == column (GK is a multiple of k)
  double acc = 0.0;
  if (g < groups)
    for (int64_t e = e0 + j + (int64_t)k * g; e < e1; e += (int64_t)k * groups) acc -= u[e] * Sm[e];
  part[t] = acc;
  __syncthreads();
  if (t < k) {
    double tot = 0.0;
    for (int q = 0; q < groups; ++q) tot += part[q * k + t];
    st.dpart[(int64_t)blockIdx.x * k + t] = tot;
  }
}

__global__ void k_pcg3_lambda(Pcg3State st) {
  const int j = threadIdx.x;
  if (j >= st.k) return;
  double d = 0.0;
  for (int b = 0; b < st.nblk; ++b) d += st.dpart[(int64_t)b * st.k + j];
  double lam = 0.0;
  if (st.active[j]) {
    if (!(d > 0.0) || !isfinite(d)) {
      st.active[j] = 0;
      st.status[j] = GLM_SUR_BREAKDOWN;
    } else {
      lam = st.c[j] / d;
    }
  }
  st.lam[j] = lam;
}

__global__ void k_pcg3_wr(int64_t n_elem, int k, Pcg3State st, const double* __restrict__ u,
                          const double* __restrict__ Sm, const double* __restrict__ sv, double* __restrict__ w,
                          double* __restrict__ r) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_elem; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % k);
    if (!st.active[j]) continue;
    const double lam = st.lam[j], ue = u[e];
    w[e] -= lam * ue;
    r[e] -= lam * ((sv[e] - ue) - Sm[e]);   // Sigma u = -Sm
  }
}

__global__ void k_pcg3_after(Pcg3State st, const double* __restrict__ cpart, int ncpart, int init) {
  const int j = threadIdx.x;
  if (j >= st.k) return;
  double cn = 0.0;
  for (int p = 0; p < ncpart; ++p) cn += cpart[(int64_t)p * st.k + j];
  if (init) {
    const double c1v = cn + (st.c1_extra ? st.c1_extra[j] : 0.0);
    st.c[j] = cn;
    st.c1[j] = c1v;
    st.iters[j] = 0;
    const bool fin = isfinite(cn);
    const bool conv0 = fin && st.c1_extra != nullptr && cn <= st.tol * st.tol * c1v;
    st.active[j] = fin && cn > 0.0 && !conv0;
    st.status[j] = !fin ? (int)GLM_SUR_NONFINITE : ((cn > 0.0 && !conv0) ? kStatusRunning : (int)GLM_SUR_OK);
    st.relres[j] = (fin && cn > 0.0) ? sqrt(cn / c1v) : 0.0;
    st.mu[j] = 0.0;
    return;
  }
  if (!st.active[j]) return;
  const int it = st.iters[j] + 1;
  st.iters[j] = it;
  const double rr = sqrt(cn / st.c1[j]);
  st.relres[j] = rr;
  int status = kStatusRunning;
  if (!isfinite(cn) || cn < 0.0) status = GLM_SUR_BREAKDOWN;
  else if (rr <= st.tol) status = GLM_SUR_OK;
  else if (it >= st.maxit) status = GLM_SUR_NOT_CONVERGED;
  if (status != kStatusRunning) {
    st.active[j] = 0;
    st.status[j] = status;
    st.mu[j] = 0.0;
    return;
  }
  st.mu[j] = cn / st.c[j];
  st.c[j] = cn;
}

__global__ void k_pcg3_s(int64_t n_elem, int k, Pcg3State st, const double* __restrict__ r, double* __restrict__ sv,
                         int init) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_elem; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % k);
    if (init) sv[e] = r[e];
    else if (st.active[j]) sv[e] = r[e] + st.mu[j] * sv[e];
  }
}

__global__ void k_pcg3_neg(int64_t n_elem, const double* __restrict__ y, double* __restrict__ r) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_elem; e += (int64_t)gridDim.x * blockDim.x)
    r[e] = -y[e];
}

unsigned elem_grid(int64_t n_elem) { return (unsigned)std::min<int64_t>(ceil_div(n_elem, 256), 152 * 16); }

}  // namespace

void launch_pcg3_dot(int64_t M, int G, int k, const double* u, const double* Sm, const Pcg3State& st, cudaStream_t s) {
  k_pcg3_dot<<<st.nblk, kP3Threads, 0, s>>>(M, G * k, k, u, Sm, st);
}
void launch_pcg3_neg(int64_t n_elem, const double* y, double* r, cudaStream_t s) {
  k_pcg3_neg<<<elem_grid(n_elem), 256, 0, s>>>(n_elem, y, r);
}
void launch_pcg3_lambda(const Pcg3State& st, cudaStream_t s) { k_pcg3_lambda<<<1, 64, 0, s>>>(st); }
void launch_pcg3_wr(int64_t n_elem, int k, const Pcg3State& st, const double* u, const double* Sm, const double* sv,
                    double* w, double* r, cudaStream_t s) {
  k_pcg3_wr<<<elem_grid(n_elem), 256, 0, s>>>(n_elem, k, st, u, Sm, sv, w, r);
}
void launch_pcg3_after(const Pcg3State& st, const double* cpart, int ncpart, int init, cudaStream_t s) {
  k_pcg3_after<<<1, 64, 0, s>>>(st, cpart, ncpart, init);
}
void launch_pcg3_s(int64_t n_elem, int k, const Pcg3State& st, const double* r, double* sv, int init, cudaStream_t s) {
  k_pcg3_s<<<elem_grid(n_elem), 256, 0, s>>>(n_elem, k, st, r, sv, init);
}

}  // namespace glmsur
