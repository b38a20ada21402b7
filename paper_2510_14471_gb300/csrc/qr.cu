// Batched tall-skinny Householder QR of the regressor blocks X_i (setup, once
// per handle).  Sec. 4.3: X_i = Q_i R_i with Q_i (M x n_i) orthonormal columns
// and R_i upper triangular; Sec. 3.2: the factorisations of the auxiliary OLS
// problem are computed once and only applied in the iterations.
//
// Design: a TSQR reduction tree per block.  Leaves are row chunks of X_i
// (<= 256 rows, even split); inner nodes stack the R factors of up to
// floor(TL / n_i) children.  Every node is factored by Householder
// reflections in shared memory (one CTA per node, all blocks of all levels at
// the same depth in one launch).  The explicit thin Q_i is then formed top
// down: node Q = H_0 ... H_{n-1} [E; 0], E = identity at the root and the
// parent's rows for this child elsewhere.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace glmsur {

namespace {

constexpr int kQrThreads = 256;

// Sum of a value over the CTA, returned to every thread (deterministic order).
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();                       // previous users of red[] are done
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// Householder QR of A (rows x nc, column-major, ld = rows) in shared memory.
// On exit the upper triangle holds R, the strict lower part the reflector
// vectors v_j (v_j[j] = 1 implicit) and tau[j] the reflector scalars, so that
// H_j = I - tau_j v_j v_j^T and H_{n-1} ... H_0 A = [R; 0].
__device__ void householder_qr_smem(double* A, int rows, int nc, double* tau, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < nc; ++j) {
    double* a = A + (int64_t)j * rows;
    double part = 0.0;
    for (int r = j + 1 + threadIdx.x; r < rows; r += blockDim.x) part += a[r] * a[r];
    const double sigma = block_sum(part, red);
    const double alpha = a[j];
    double beta = alpha, t = 0.0, scal = 0.0;
    if (sigma > 0.0) {
      beta = -copysign(sqrt(alpha * alpha + sigma), alpha);
      t = (beta - alpha) / beta;
      scal = 1.0 / (alpha - beta);
    }
    for (int r = j + 1 + threadIdx.x; r < rows; r += blockDim.x) a[r] *= scal;
    __syncthreads();
    if (threadIdx.x == 0) { a[j] = beta; tau[j] = t; }
    // apply H_j to the trailing columns: one warp per column
    for (int c = j + 1 + warp; c < nc; c += nw) {
      double* b = A + (int64_t)c * rows;
      double dot = 0.0;
      for (int r = j + 1 + lane; r < rows; r += 32) dot += a[r] * b[r];
      dot = warp_sum(dot) + b[j];
      const double coef = t * dot;
      if (lane == 0) b[j] -= coef;
      for (int r = j + 1 + lane; r < rows; r += 32) b[r] -= coef * a[r];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kQrThreads)
qr_factor_level(const QrNode* __restrict__ nodes, int first, int count, const double* __restrict__ X,
                double* stack, double* V, double* tau_ws, double* Rout, const int64_t* __restrict__ r_off,
                int* setup_flags) {
  extern __shared__ double sm[];
  __shared__ double red[32];
  __shared__ double tau_s[kMaxBlockCols];
  const int id = blockIdx.x;
  if (id >= count) return;
  const QrNode nd = nodes[first + id];
  const int rows = nd.rows, nc = nd.nc;
  double* A = sm;
  // load the node's input
  if (nd.level == 0) {
    const double* src = X + nd.x_base + nd.in_off;
    for (int64_t e = threadIdx.x; e < (int64_t)rows * nc; e += blockDim.x) {
      const int c = (int)(e / rows), r = (int)(e % rows);
      A[e] = src[(int64_t)c * nd.x_ld + r];
    }
  } else {
    const double* src = stack + nd.in_off;
    for (int64_t e = threadIdx.x; e < (int64_t)rows * nc; e += blockDim.x) A[e] = src[e];
  }
  __syncthreads();
  householder_qr_smem(A, rows, nc, tau_s, red);
  // reflectors + R of this node
  double* vdst = V + nd.v_off;
  for (int64_t e = threadIdx.x; e < (int64_t)rows * nc; e += blockDim.x) vdst[e] = A[e];
  for (int c = threadIdx.x; c < nc; c += blockDim.x) tau_ws[nd.tau_off + c] = tau_s[c];
  if (nd.parent < 0) {
    // final R_i, row-major n_i x n_i, and the rank test |R_jj| <= n eps max|R|
    double* R = Rout + r_off[nd.blk];
    double amax = 0.0;
    for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) {
      const int r = e / nc, c = e % nc;
      const double v = (r <= c) ? A[(int64_t)c * rows + r] : 0.0;
      R[e] = v;
      amax = fmax(amax, fabs(v));
    }
    // max via sum of a per-warp max is not needed: recompute max serially
    __syncthreads();
    if (threadIdx.x == 0) {
      double mx = 0.0, mn = 1e300;
      for (int c = 0; c < nc; ++c) {
        for (int r = 0; r <= c; ++r) mx = fmax(mx, fabs(A[(int64_t)c * rows + r]));
        mn = fmin(mn, fabs(A[(int64_t)c * rows + c]));
      }
      const bool finite = isfinite(mx) && isfinite(mn);
      if (!finite) atomicOr(setup_flags, 2);
      else if (!(mn > (double)nc * 2.220446049250313e-16 * mx)) atomicOr(setup_flags, 1);
    }
    (void)amax;
  } else {
    // R into the parent's stacked input (column-major, ld = parent rows)
    double* dst = stack + nd.out_off;
    for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) {
      const int c = e / nc, r = e % nc;
      dst[(int64_t)c * nd.parent_rows + r] = (r <= c) ? A[(int64_t)c * rows + r] : 0.0;
    }
  }
}

// Explicit Q of one node: B = H_0 ... H_{nc-1} [E; 0].
__global__ void __launch_bounds__(kQrThreads)
qr_form_q_level(const QrNode* __restrict__ nodes, int first, int count, double* stack,
                const double* __restrict__ V, const double* __restrict__ tau_ws, double* Q) {
  extern __shared__ double sm[];
  const int id = blockIdx.x;
  if (id >= count) return;
  const QrNode nd = nodes[first + id];
  const int rows = nd.rows, nc = nd.nc;
  double* Vs = sm;
  double* B = sm + (int64_t)rows * nc;
  __shared__ double tau_s[kMaxBlockCols];
  const double* vsrc = V + nd.v_off;
  for (int64_t e = threadIdx.x; e < (int64_t)rows * nc; e += blockDim.x) {
    Vs[e] = vsrc[e];
    const int c = (int)(e / rows), r = (int)(e % rows);
    double b = 0.0;
    if (r < nc) {
      if (nd.parent < 0) b = (r == c) ? 1.0 : 0.0;
      else b = stack[nd.parent_in_off + (int64_t)c * nd.parent_rows + nd.child_row + r];
    }
    B[e] = b;
  }
  for (int c = threadIdx.x; c < nc; c += blockDim.x) tau_s[c] = tau_ws[nd.tau_off + c];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = nc - 1; j >= 0; --j) {
    const double* v = Vs + (int64_t)j * rows;
    const double t = tau_s[j];
    for (int c = warp; c < nc; c += nw) {
      double* b = B + (int64_t)c * rows;
      double dot = 0.0;
      for (int r = j + 1 + lane; r < rows; r += 32) dot += v[r] * b[r];
      dot = warp_sum(dot) + b[j];
      const double coef = t * dot;
      __syncwarp();
      if (lane == 0) b[j] -= coef;
      for (int r = j + 1 + lane; r < rows; r += 32) b[r] -= coef * v[r];
    }
    __syncthreads();
  }
  if (nd.level == 0) {
    // leaf: rows of Q_i into the padded row-major Q
    double* dst = Q + nd.q_base + nd.in_off * nd.q_ld;
    for (int64_t e = threadIdx.x; e < (int64_t)rows * nc; e += blockDim.x) {
      const int r = (int)(e / nc), c = (int)(e % nc);
      dst[(int64_t)r * nd.q_ld + c] = B[(int64_t)c * rows + r];
    }
  } else {
    double* dst = stack + nd.in_off;
    for (int64_t e = threadIdx.x; e < (int64_t)rows * nc; e += blockDim.x) dst[e] = B[e];
  }
}

}  // namespace

// Build the TSQR forest of a list of blocks (host).  Block b is R factor b
// (r_off[b]) of the caller.
void build_qr_plan(const std::vector<QrBlock>& blocks, QrPlan& plan) {
  plan.nodes.clear();
  plan.level_first.clear();
  plan.level_count.clear();
  std::vector<std::vector<QrNode>> by_level;
  int64_t stack_sz = 0, v_sz = 0, tau_sz = 0;
  const int G = (int)blocks.size();
  for (int b = 0; b < G; ++b) {
    const int nc = blocks[b].nc;
    const int64_t M = blocks[b].rows;
    const int TL = (nc <= 32) ? 256 : 128;
    // level 0: even row chunks
    const int64_t nch = std::max<int64_t>(1, ceil_div(M, TL));
    std::vector<QrNode> cur;
    for (int64_t c = 0; c < nch; ++c) {
      QrNode nd{};
      nd.blk = b; nd.nc = nc; nd.level = 0;
      nd.x_base = blocks[b].x_base; nd.x_ld = blocks[b].x_ld;
      nd.q_base = blocks[b].q_base; nd.q_ld = blocks[b].q_ld;
      const int64_t s = (M * c) / nch, e = (M * (c + 1)) / nch;
      nd.rows = (int)(e - s);
      nd.in_off = s;
      cur.push_back(nd);
    }
    int level = 0;
    std::vector<std::vector<QrNode>> levels;
    levels.push_back(cur);
    while (levels.back().size() > 1) {
      auto& ch = levels.back();
      const int F = std::max(2, TL / nc);
      const int64_t N = (int64_t)ch.size();
      const int64_t np = ceil_div(N, F);
      std::vector<QrNode> par;
      for (int64_t p = 0; p < np; ++p) {
        const int64_t s = (N * p) / np, e = (N * (p + 1)) / np;
        QrNode nd{};
        nd.blk = b; nd.nc = nc; nd.level = level + 1;
        nd.rows = (int)((e - s) * nc);
        nd.in_off = stack_sz;                 // its stacked input lives in the stack workspace
        stack_sz += (int64_t)nd.rows * nc;
        nd.parent = -1;
        for (int64_t c = s; c < e; ++c) {
          ch[c].parent = 1;                   // marker; resolved to index below
          ch[c].child_row = (int)((c - s) * nc);
          ch[c].parent_rows = nd.rows;
          ch[c].parent_in_off = nd.in_off;
          ch[c].out_off = nd.in_off + ch[c].child_row;
        }
        par.push_back(nd);
      }
      levels.push_back(par);
      ++level;
    }
    levels.back()[0].parent = -1;
    for (size_t l = 0; l < levels.size(); ++l) {
      if (by_level.size() <= l) by_level.resize(l + 1);
      for (auto& nd : levels[l]) {
        nd.v_off = v_sz;
        v_sz += (int64_t)nd.rows * nd.nc;
        nd.tau_off = tau_sz;
        tau_sz += nd.nc;
        by_level[l].push_back(nd);
      }
    }
  }
  for (auto& lv : by_level) {
    plan.level_first.push_back((int)plan.nodes.size());
    plan.level_count.push_back((int)lv.size());
    for (auto& nd : lv) plan.nodes.push_back(nd);
  }
  plan.stack_elems = std::max<int64_t>(stack_sz, 1);
  plan.v_elems = std::max<int64_t>(v_sz, 1);
  plan.tau_elems = std::max<int64_t>(tau_sz, 1);
  plan.max_smem_factor = 0;
  plan.max_smem_form = 0;
  for (auto& nd : plan.nodes) {
    const size_t a = (size_t)nd.rows * nd.nc * sizeof(double);
    plan.max_smem_factor = std::max(plan.max_smem_factor, a);
    plan.max_smem_form = std::max(plan.max_smem_form, 2 * a);
  }
}

glm_sur_status run_qr(const QrPlan& plan, const double* X, const int64_t* d_r_off, double* Q, double* R,
                      int* d_setup_flags, cudaStream_t st) {
  QrNode* d_nodes = nullptr;
  double *stack = nullptr, *V = nullptr, *tau = nullptr;
  const size_t nb = plan.nodes.size() * sizeof(QrNode);
  glm_sur_status rc = GLM_SUR_OK;
  auto fail = [&](cudaError_t e, const char* what) {
    set_last_error(e, what, __FILE__, __LINE__);
    rc = (e == cudaErrorMemoryAllocation) ? GLM_SUR_OOM : GLM_SUR_CUDA_ERROR;
  };
  cudaError_t e;
  if ((e = cudaMallocAsync(&d_nodes, nb, st)) != cudaSuccess) { fail(e, "malloc nodes"); return rc; }
  if ((e = cudaMallocAsync(&stack, plan.stack_elems * sizeof(double), st)) != cudaSuccess) fail(e, "malloc stack");
  if (rc == GLM_SUR_OK && (e = cudaMallocAsync(&V, plan.v_elems * sizeof(double), st)) != cudaSuccess) fail(e, "malloc V");
  if (rc == GLM_SUR_OK && (e = cudaMallocAsync(&tau, plan.tau_elems * sizeof(double), st)) != cudaSuccess) fail(e, "malloc tau");
  if (rc == GLM_SUR_OK && (e = cudaMemcpyAsync(d_nodes, plan.nodes.data(), nb, cudaMemcpyHostToDevice, st)) != cudaSuccess) fail(e, "copy nodes");
  if (rc == GLM_SUR_OK) {
    if ((e = cudaFuncSetAttribute(qr_factor_level, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)plan.max_smem_factor)) != cudaSuccess) fail(e, "smem attr factor");
    if ((e = cudaFuncSetAttribute(qr_form_q_level, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)plan.max_smem_form)) != cudaSuccess) fail(e, "smem attr form");
  }
  const int L = (int)plan.level_first.size();
  for (int l = 0; rc == GLM_SUR_OK && l < L; ++l) {
    qr_factor_level<<<plan.level_count[l], kQrThreads, plan.max_smem_factor, st>>>(
        d_nodes, plan.level_first[l], plan.level_count[l], X, stack, V, tau, R, d_r_off, d_setup_flags);
    if ((e = cudaGetLastError()) != cudaSuccess) fail(e, "qr_factor_level");
  }
  for (int l = L - 1; rc == GLM_SUR_OK && l >= 0; --l) {
    qr_form_q_level<<<plan.level_count[l], kQrThreads, plan.max_smem_form, st>>>(
        d_nodes, plan.level_first[l], plan.level_count[l], stack, V, tau, Q);
    if ((e = cudaGetLastError()) != cudaSuccess) fail(e, "qr_form_q_level");
  }
  if (tau) cudaFreeAsync(tau, st);
  if (V) cudaFreeAsync(V, st);
  if (stack) cudaFreeAsync(stack, st);
  cudaFreeAsync(d_nodes, st);
  return rc;
}

}  // namespace glmsur
