// C ABI of the batched solver: setup of many SUR instances (TSQR of all their
// blocks in shared level launches), and one-launch solves with a small
// autotuner for the tile height.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "batch.h"
#include "common.cuh"
#include "glm_sur.h"
#include "internal.h"
#include "pcg.h"
#include "reduce.h"
#include "rglm.h"

using namespace glmsur;

struct glm_sur_batch_ctx {
  int count = 0, sms = 148, maxG = 0, maxNp = 0, maxNq = 0;
  glm_sur_opts opts;
  std::vector<int> G, M, n, np, nq, blk0, quad0;
  std::vector<int64_t> q_off, om_off, x_off, m_sum;   // per instance
  int nblk = 0, nquad = 0;
  int64_t q_elems = 0, om_elems = 0, r_elems = 0, v_rows = 0;  // v_rows = sum M*G
  double *q64 = nullptr, *R = nullptr, *om64 = nullptr;
  float *q32 = nullptr, *om32 = nullptr;
  int *d_n_i = nullptr, *d_poff = nullptr, *d_quad_blk = nullptr, *setup_flags = nullptr;
  int64_t* d_r_off = nullptr;
  // solve workspace
  int kcap = 0;
  double *w64 = nullptr, *E64 = nullptr, *d64 = nullptr;
  float *g32 = nullptr, *u32 = nullptr, *w32 = nullptr, *wb32 = nullptr;
  int *status = nullptr, *iters_d = nullptr, *counter = nullptr, *steps_d = nullptr;
  double* relres_d = nullptr;
  long long* cycles_d = nullptr;
  BatchInst* d_insts = nullptr;
  int insts_k = 0;
  int last_k = 0;
  int tile = 0;          // autotuned tile height (0 = not tuned yet)
  float tune_ms[3] = {0, 0, 0};
  int grid = 0;
  cudaGraphExec_t graph = nullptr;
  const void* graph_key[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int graph_k = 0;
  int64_t launches = 0;
  // row reduction (Remark rem:reduction, opts.reduce_rows): the solves run on
  // `inner`, the batch of the reduced instances (n_j rows per equation);
  // reduced instance j keeps Q_W (M_j x n_j column-major) at qw_off[j]
  glm_sur_batch_ctx* inner = nullptr;
  std::vector<int> red;                 // 1: instance reduced
  std::vector<int64_t> qw_off, y_off, yr_off;
  int64_t y_rows = 0, yr_rows = 0;      // sum G M, sum G M'
  double* qw = nullptr;
  double* yred = nullptr;
  int yred_k = 0;
  DgemmProblem* d_rot = nullptr;        // rotation problems of the last (Y, k)
  const double* rot_y = nullptr;
  int rot_k = 0, rot_count = 0, rot_tiles = 0;
  // energy of every instance's responses outside range(W_j) (count x K), the
  // reference term of the reduced instances' relres and tol; on `inner` the
  // outer handle's buffer
  struct RedRows { int64_t y_off, yr_off, m, mr; int red; };
  RedRows* d_redrows = nullptr;
  double* d_extra = nullptr;
  const double* rho_extra = nullptr;
};

namespace {

template <typename T>
cudaError_t balloc(T** p, size_t n) {
  *p = nullptr;
  return cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T));
}

// out[j K + c] = max(0, ||y_jc||^2 - ||Q_W^T y_jc||^2) for a reduced instance
// j (0 for the others): one CTA per (instance, right-hand side)
__global__ void __launch_bounds__(256)
k_batch_complement(int k, const glm_sur_batch_ctx::RedRows* __restrict__ rr, const double* __restrict__ Y,
                   const double* __restrict__ Yr, double* __restrict__ out) {
  __shared__ double red[256];
  const int j = blockIdx.x, c = blockIdx.y;
  const glm_sur_batch_ctx::RedRows d = rr[j];
  double a = 0.0;
  if (d.red) {
    const double* y = Y + d.y_off * k + (int64_t)c * d.m;
    const double* yr = Yr + d.yr_off * k + (int64_t)c * d.mr;
    for (int64_t t = threadIdx.x; t < d.m; t += 256) a += y[t] * y[t];
    for (int64_t t = threadIdx.x; t < d.mr; t += 256) a -= yr[t] * yr[t];
  }
  red[threadIdx.x] = a;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[(int64_t)j * kBatchMaxK + c] = red[0] > 0.0 ? red[0] : 0.0;
}
template <typename T>
void bfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_solve(glm_sur_batch_ctx* h) {
  bfree(h->w64); bfree(h->E64); bfree(h->d64); bfree(h->g32); bfree(h->u32); bfree(h->w32); bfree(h->wb32);
  bfree(h->status); bfree(h->iters_d); bfree(h->relres_d); bfree(h->d_insts); bfree(h->steps_d);
  bfree(h->cycles_d);
  h->kcap = 0;
  h->insts_k = 0;
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
}

// Omega of every instance into the padded G x Gq pools (float64 and float32).
__global__ void k_pad_omegas(int count, const int* __restrict__ G, const int64_t* __restrict__ src_off,
                             const int64_t* __restrict__ dst_off, const double* __restrict__ Om, double* om64,
                             float* om32) {
  const int j = blockIdx.x;
  if (j >= count) return;
  const int g = G[j], gq = (g + 3) & ~3;
  for (int e = threadIdx.x; e < g * gq; e += blockDim.x) {
    const int r = e / gq, c = e % gq;
    const double v = c < g ? Om[src_off[j] + (int64_t)c * g + r] : 0.0;
    om64[dst_off[j] + e] = v;
    om32[dst_off[j] + e] = (float)v;
  }
}

}  // namespace

// Descriptors of every instance in work order: decreasing `cost` (longest
// processing time first, so that the persistent CTAs finish together).
static cudaError_t write_work_order(glm_sur_batch_ctx* h, int k, const std::vector<double>& cost) {
  std::vector<int> order(h->count);
  for (int j = 0; j < h->count; ++j) order[j] = j;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
  std::vector<int64_t> voff(h->count), yoff(h->count), boff(h->count);
  int64_t v = 0, y = 0, bo = 0;
  for (int j = 0; j < h->count; ++j) {
    voff[j] = v; yoff[j] = y; boff[j] = bo;
    v += (int64_t)h->M[j] * h->G[j] * k;
    y += (int64_t)h->M[j] * h->G[j] * k;
    bo += (int64_t)h->n[j] * k;
  }
  std::vector<BatchInst> insts(h->count);
  for (int r = 0; r < h->count; ++r) {
    const int j = order[r];
    BatchInst& d = insts[r];
    d.index = j;
    d.G = h->G[j]; d.Gq = round_up4(h->G[j]); d.M = h->M[j]; d.n = h->n[j]; d.np = h->np[j]; d.nq = h->nq[j];
    d.blk0 = h->blk0[j]; d.quad0 = h->quad0[j];
    d.q_off = h->q_off[j]; d.om_off = h->om_off[j]; d.v_off = voff[j]; d.y_off = yoff[j]; d.b_off = boff[j];
  }
  return cudaMemcpy(h->d_insts, insts.data(), sizeof(BatchInst) * h->count, cudaMemcpyHostToDevice);
}

// Remark rem:reduction for every instance with M_j >= 2 n_j: Q_W (M_j x n_j
// orthonormal, range(Q_W) = range(W_j), W_j = [X_1 ... X_G]) by Cholesky QR
// twice and R_W = L2^T L1^T; the reduced instance has the regressor blocks
// R_W[:, block i] (n_j rows) and the responses Q_W^T y_i.  The products of
// all instances run as one batched launch per stage; the Cholesky
// factorisations and triangular inverses are one-CTA launches per instance.
// Returns GLM_SUR_RANK_DEFICIENT when some W_j has no full column rank (the
// caller then keeps the batch whole).
static glm_sur_status batch_setup_reduced(glm_sur_batch_t* out, int count, const int* G, const int* M,
                                          const int* n_i, const double* X, const double* Omega,
                                          const glm_sur_opts& o, cudaStream_t s) {
  glm_sur_batch_ctx* h = new glm_sur_batch_ctx();
  h->count = count;
  h->opts = o;
  std::vector<int> n(count), Mr(count);
  std::vector<int64_t> x_off(count), xr_off(count), nn_off(count);
  int64_t xo = 0, xro = 0, qwo = 0, nb = 0, nno = 0;
  for (int j = 0; j < count; ++j) {
    int nj = 0;
    for (int i = 0; i < G[j]; ++i) nj += n_i[nb + i];
    nb += G[j];
    n[j] = nj;
    const bool r = M[j] >= 2 * nj && nj <= kMaxReducedCols;
    h->red.push_back(r ? 1 : 0);
    Mr[j] = r ? nj : M[j];
    x_off[j] = xo;
    xr_off[j] = xro;
    nn_off[j] = nno;
    h->qw_off.push_back(r ? qwo : -1);
    h->y_off.push_back(h->y_rows);
    h->yr_off.push_back(h->yr_rows);
    xo += (int64_t)M[j] * nj;
    xro += (int64_t)Mr[j] * nj;
    if (r) {
      qwo += (int64_t)M[j] * nj;
      nno += (int64_t)nj * nj;
    }
    h->y_rows += (int64_t)G[j] * M[j];
    h->yr_rows += (int64_t)G[j] * Mr[j];
  }
  double *xr = nullptr, *G1 = nullptr, *Li1 = nullptr, *G2 = nullptr, *Li2 = nullptr, *Q1 = nullptr;
  int* flags = nullptr;
  DgemmProblem* dprob = nullptr;
  auto release = [&]() {
    bfree(xr); bfree(G1); bfree(Li1); bfree(G2); bfree(Li2); bfree(Q1); bfree(flags); bfree(dprob);
  };
  auto fail = [&](cudaError_t e, const char* what) {
    set_last_error(e, what, __FILE__, __LINE__);
    release();
    bfree(h->qw);
    bfree(h->d_rot);
    delete h;
    return e == cudaErrorMemoryAllocation ? GLM_SUR_OOM : GLM_SUR_CUDA_ERROR;
  };
  cudaError_t e;
#define RTRY(x) if ((e = (x)) != cudaSuccess) return fail(e, #x)
  RTRY(balloc(&xr, (size_t)xro));
  RTRY(balloc(&h->qw, (size_t)qwo));
  RTRY(balloc(&G1, (size_t)nno)); RTRY(balloc(&Li1, (size_t)nno));
  RTRY(balloc(&G2, (size_t)nno)); RTRY(balloc(&Li2, (size_t)nno));
  RTRY(balloc(&Q1, (size_t)qwo));
  RTRY(balloc(&flags, (size_t)count));
  RTRY(balloc(&dprob, (size_t)count));
  RTRY(balloc(&h->d_rot, (size_t)count));
  RTRY(cudaMemsetAsync(flags, 0, sizeof(int) * count, s));
  std::vector<DgemmProblem> pr;
  // one stage of products, one problem per reduced instance
  auto stage = [&](auto make) -> cudaError_t {
    pr.clear();
    int tiles = 0;
    for (int j = 0; j < count; ++j)
      if (h->red[j]) {
        pr.push_back(make(j));
        tiles = std::max(tiles, dgemm_tiles(pr.back().m, pr.back().n));
      }
    if (pr.empty()) return cudaSuccess;
    cudaError_t ce = cudaMemcpyAsync(dprob, pr.data(), sizeof(DgemmProblem) * pr.size(), cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) return ce;
    launch_dgemm_batched(dprob, (int)pr.size(), tiles, s);
    ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);   // `pr` is reused by the next stage
    h->launches += 1;
    return ce;
  };
  // per-instance Cholesky and inverse of a stage's n x n Gram matrices
  auto factor = [&](double* Gm, double* Li) -> cudaError_t {
    for (int j = 0; j < count; ++j) {
      if (!h->red[j]) continue;
      const int nj = n[j];
      const double piv_tol = 64.0 * nj * 2.220446049250313e-16;   // below: W treated as rank deficient
      cudaError_t ce = cholesky_lower(nj, Gm + nn_off[j], flags + j, piv_tol, s);
      if (ce != cudaSuccess) return ce;
      launch_zero_upper(nj, Gm + nn_off[j], s);
      ce = launch_tri_inverse(nj, Gm + nn_off[j], Li + nn_off[j], s);
      if (ce != cudaSuccess) return ce;
      h->launches += 3;
    }
    return cudaGetLastError();
  };
  for (int j = 0; j < count; ++j)
    if (!h->red[j])
      RTRY(cudaMemcpyAsync(xr + xr_off[j], X + x_off[j], sizeof(double) * (size_t)M[j] * n[j],
                           cudaMemcpyDeviceToDevice, s));
  // W^T W = L1 L1^T ;  Q1 = W L1^-T ;  Q1^T Q1 = L2 L2^T ;  Q = Q1 L2^-T ;  R_W = L2^T L1^T
  RTRY(stage([&](int j) {
    const int64_t Mj = M[j];
    const double* W = X + x_off[j];
    return DgemmProblem{n[j], n[j], Mj, W, Mj, 1, W, 1, Mj, G1 + nn_off[j], n[j], 1};
  }));
  RTRY(factor(G1, Li1));
  RTRY(stage([&](int j) {
    const int64_t Mj = M[j];
    return DgemmProblem{(int)Mj, n[j], n[j], X + x_off[j], 1, Mj, Li1 + nn_off[j], 1, n[j],
                        Q1 + h->qw_off[j], 1, Mj};
  }));
  RTRY(stage([&](int j) {
    const int64_t Mj = M[j];
    const double* A = Q1 + h->qw_off[j];
    return DgemmProblem{n[j], n[j], Mj, A, Mj, 1, A, 1, Mj, G2 + nn_off[j], n[j], 1};
  }));
  RTRY(factor(G2, Li2));
  RTRY(stage([&](int j) {
    const int64_t Mj = M[j];
    return DgemmProblem{(int)Mj, n[j], n[j], Q1 + h->qw_off[j], 1, Mj, Li2 + nn_off[j], 1, n[j],
                        h->qw + h->qw_off[j], 1, Mj};
  }));
  RTRY(stage([&](int j) {
    return DgemmProblem{n[j], n[j], n[j], G2 + nn_off[j], 1, n[j], G1 + nn_off[j], 1, n[j], xr + xr_off[j], 1, n[j]};
  }));
  std::vector<int> hflags(count, 0);
  RTRY(cudaMemcpyAsync(hflags.data(), flags, sizeof(int) * count, cudaMemcpyDeviceToHost, s));
  RTRY(cudaStreamSynchronize(s));
  for (int j = 0; j < count; ++j)
    if (hflags[j]) {
      release();
      bfree(h->qw);
      bfree(h->d_rot);
      delete h;
      return GLM_SUR_RANK_DEFICIENT;
    }
  glm_sur_opts so = o;
  so.reduce_rows = 0;
  glm_sur_batch_t inner = nullptr;
  glm_sur_status rc = glm_sur_batch_setup(&inner, count, G, Mr.data(), n_i, xr, Omega, &so,
                                          reinterpret_cast<glm_sur_stream_t>(s));
  cudaStreamSynchronize(s);
  release();
  if (rc != GLM_SUR_OK) {
    bfree(h->qw);
    bfree(h->d_rot);
    delete h;
    return rc;
  }
#undef RTRY
  h->inner = inner;
  h->G.assign(G, G + count);
  h->M.assign(M, M + count);
  h->n = n;
  {
    std::vector<glm_sur_batch_ctx::RedRows> rows(count);
    for (int j = 0; j < count; ++j)
      rows[j] = {h->y_off[j], h->yr_off[j], (int64_t)G[j] * M[j], (int64_t)G[j] * Mr[j], h->red[j]};
    cudaError_t e = balloc(&h->d_redrows, (size_t)count);
    if (e == cudaSuccess) e = balloc(&h->d_extra, (size_t)count * kBatchMaxK);
    if (e == cudaSuccess)
      e = cudaMemcpy(h->d_redrows, rows.data(), sizeof(glm_sur_batch_ctx::RedRows) * count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      set_last_error(e, "cudaMalloc (batch row reduction)", __FILE__, __LINE__);
      glm_sur_batch_destroy(h);
      return GLM_SUR_CUDA_ERROR;
    }
  }
  *out = h;
  return GLM_SUR_OK;
}

extern "C" {

glm_sur_status glm_sur_batch_setup(glm_sur_batch_t* out, int count, const int* G, const int* M, const int* n_i,
                                   const double* X, const double* Omega, const glm_sur_opts* opts,
                                   glm_sur_stream_t stream) {
  if (!out || count < 1 || !G || !M || !n_i || !X || !Omega) return GLM_SUR_INVALID_ARG;
  *out = nullptr;
  glm_sur_opts o;
  glm_sur_default_opts(&o);
  if (opts) o = *opts;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (o.reduce_rows) {
    // validate the instances first: the reduced setup assumes their sizes
    int64_t nb = 0;
    for (int j = 0; j < count; ++j) {
      if (G[j] < 1 || G[j] > kBatchMaxG || M[j] < 1) return GLM_SUR_INVALID_ARG;
      for (int i = 0; i < G[j]; ++i)
        if (n_i[nb + i] < 1 || n_i[nb + i] > kBatchMaxCols || n_i[nb + i] > M[j]) return GLM_SUR_INVALID_ARG;
      nb += G[j];
    }
    glm_sur_status rr = batch_setup_reduced(out, count, G, M, n_i, X, Omega, o, s);
    if (rr != GLM_SUR_RANK_DEFICIENT) return rr;
    // some W_j without full column rank: the batch is kept whole
    o.reduce_rows = 0;
  }
  glm_sur_batch_ctx* h = new glm_sur_batch_ctx();
  h->count = count;
  h->opts = o;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
  std::vector<int> blk_n, blk_poff, quad_blk;
  std::vector<int64_t> blk_roff;
  std::vector<QrBlock> qb;
  int64_t xo = 0, mo = 0;
  for (int j = 0; j < count; ++j) {
    const int g = G[j], mm = M[j];
    if (g < 1 || g > kBatchMaxG || mm < 1) { delete h; return GLM_SUR_INVALID_ARG; }
    int n = 0, np = 0;
    h->blk0.push_back(h->nblk);
    h->quad0.push_back(h->nquad);
    h->q_off.push_back(h->q_elems);
    h->om_off.push_back(h->om_elems);
    h->x_off.push_back(xo);
    h->m_sum.push_back(mo);
    for (int i = 0; i < g; ++i) {
      const int ni = n_i[h->nblk + i];
      if (ni < 1 || ni > kBatchMaxCols || ni > mm) { delete h; return GLM_SUR_INVALID_ARG; }
      blk_n.push_back(ni);
      blk_poff.push_back(np);
      blk_roff.push_back(h->r_elems);
      qb.push_back(QrBlock{ni, mm, xo + (int64_t)n * mm, mm, h->q_elems + np, 0});
      for (int q = 0; q < round_up4(ni) / 4; ++q) quad_blk.push_back(i);
      n += ni;
      np += round_up4(ni);
      h->r_elems += (int64_t)ni * ni;
    }
    if (np > kBatchMaxNp || (np / 4) * kBatchMaxK > kBatchMaxPairs) { delete h; return GLM_SUR_INVALID_ARG; }
    for (int i = 0; i < g; ++i) qb[h->nblk + i].q_ld = np;
    h->G.push_back(g); h->M.push_back(mm); h->n.push_back(n); h->np.push_back(np); h->nq.push_back(np / 4);
    h->nblk += g;
    h->nquad += np / 4;
    h->q_elems += (int64_t)mm * np;
    h->om_elems += (int64_t)g * round_up4(g);
    h->v_rows += (int64_t)mm * g;
    h->maxG = std::max(h->maxG, g);
    h->maxNp = std::max(h->maxNp, np);
    h->maxNq = std::max(h->maxNq, np / 4);
    xo += (int64_t)mm * n;
    mo += (int64_t)g * g;
  }
  auto fail = [&](cudaError_t e, const char* what) {
    set_last_error(e, what, __FILE__, __LINE__);
    glm_sur_batch_destroy(h);
    return e == cudaErrorMemoryAllocation ? GLM_SUR_OOM : GLM_SUR_CUDA_ERROR;
  };
  cudaError_t e;
#define BTRY(x) if ((e = (x)) != cudaSuccess) return fail(e, #x)
  BTRY(balloc(&h->q64, h->q_elems));
  BTRY(balloc(&h->q32, h->q_elems));
  BTRY(balloc(&h->R, h->r_elems));
  BTRY(balloc(&h->om64, h->om_elems));
  BTRY(balloc(&h->om32, h->om_elems));
  BTRY(balloc(&h->d_n_i, h->nblk));
  BTRY(balloc(&h->d_poff, h->nblk));
  BTRY(balloc(&h->d_r_off, h->nblk));
  BTRY(balloc(&h->d_quad_blk, h->nquad));
  BTRY(balloc(&h->setup_flags, 1));
  BTRY(balloc(&h->counter, 1));
  BTRY(cudaMemcpy(h->d_n_i, blk_n.data(), sizeof(int) * h->nblk, cudaMemcpyHostToDevice));
  BTRY(cudaMemcpy(h->d_poff, blk_poff.data(), sizeof(int) * h->nblk, cudaMemcpyHostToDevice));
  BTRY(cudaMemcpy(h->d_r_off, blk_roff.data(), sizeof(int64_t) * h->nblk, cudaMemcpyHostToDevice));
  BTRY(cudaMemcpy(h->d_quad_blk, quad_blk.data(), sizeof(int) * h->nquad, cudaMemcpyHostToDevice));
  BTRY(cudaMemsetAsync(h->q64, 0, sizeof(double) * h->q_elems, s));
  BTRY(cudaMemsetAsync(h->setup_flags, 0, sizeof(int), s));
  // Omega pools
  {
    int* dG = nullptr;
    int64_t *dsrc = nullptr, *ddst = nullptr;
    BTRY(balloc(&dG, count));
    BTRY(balloc(&dsrc, count));
    BTRY(balloc(&ddst, count));
    BTRY(cudaMemcpy(dG, h->G.data(), sizeof(int) * count, cudaMemcpyHostToDevice));
    BTRY(cudaMemcpy(dsrc, h->m_sum.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice));
    BTRY(cudaMemcpy(ddst, h->om_off.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice));
    k_pad_omegas<<<count, 128, 0, s>>>(count, dG, dsrc, ddst, Omega, h->om64, h->om32);
    BTRY(cudaGetLastError());
    BTRY(cudaStreamSynchronize(s));
    cudaFree(dG); cudaFree(dsrc); cudaFree(ddst);
  }
  // TSQR of every block of every instance
  QrPlan plan;
  build_qr_plan(qb, plan);
  glm_sur_status rc = run_qr(plan, X, h->d_r_off, h->q64, h->R, h->setup_flags, s);
  if (rc != GLM_SUR_OK) { glm_sur_batch_destroy(h); return rc; }
  launch_convert<double, float>(h->q_elems, h->q64, h->q32, 1.0, s);
  BTRY(cudaGetLastError());
  h->launches += 2 * (int64_t)plan.level_first.size() + 2;
#undef BTRY
  *out = h;
  return GLM_SUR_OK;
}

glm_sur_status glm_sur_batch_get_setup_status(glm_sur_batch_t h) {
  if (h && h->inner) return glm_sur_batch_get_setup_status(h->inner);
  if (!h) return GLM_SUR_INVALID_ARG;
  int flags = 0;
  GS_CUDA_TRY(cudaMemcpy(&flags, h->setup_flags, sizeof(int), cudaMemcpyDeviceToHost));
  if (flags & 2) return GLM_SUR_NONFINITE;
  if (flags & 1) return GLM_SUR_RANK_DEFICIENT;
  return GLM_SUR_OK;
}

glm_sur_status glm_sur_batch_solve(glm_sur_batch_t h, const double* Y, int k, double* b, int* iters,
                                   double* relres, glm_sur_stream_t stream) {
  if (!h || !Y || !b) return GLM_SUR_INVALID_ARG;
  if (k != 1 && k != 2 && k != 4 && k != 8) return GLM_SUR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (h->inner) {
    // Remark rem:reduction: y' = Q_W^T y per reduced instance (one float64
    // product of its G_j k columns), the other instances copied; then the
    // batch of the reduced instances
    if (k > h->yred_k) {
      GS_CUDA_TRY(cudaStreamSynchronize(s));   // an earlier solve may still read the old buffer
      bfree(h->yred);
      h->yred_k = 0;
      GS_CUDA_TRY(balloc(&h->yred, (size_t)h->yr_rows * k));
      h->yred_k = k;
      h->rot_y = nullptr;                      // the rotation problems point at the old buffer
    }
    if (Y != h->rot_y || k != h->rot_k) {
      // the rotation problems of this (Y, k): one batched float64 launch per solve
      std::vector<DgemmProblem> pr;
      int tiles = 0;
      for (int j = 0; j < h->count; ++j) {
        if (!h->red[j]) continue;
        const int64_t Mj = h->M[j];
        pr.push_back(DgemmProblem{h->n[j], h->G[j] * k, Mj, h->qw + h->qw_off[j], Mj, 1, Y + h->y_off[j] * k, 1, Mj,
                                  h->yred + h->yr_off[j] * k, 1, h->n[j]});
        tiles = std::max(tiles, dgemm_tiles(pr.back().m, pr.back().n));
      }
      if (!pr.empty())
        GS_CUDA_TRY(cudaMemcpy(h->d_rot, pr.data(), sizeof(DgemmProblem) * pr.size(), cudaMemcpyHostToDevice));
      h->rot_y = Y;
      h->rot_k = k;
      h->rot_count = (int)pr.size();
      h->rot_tiles = tiles;
    }
    launch_dgemm_batched(h->d_rot, h->rot_count, h->rot_tiles, s);
    h->launches += 1;
    for (int j = 0; j < h->count; ++j)
      if (!h->red[j])
        GS_CUDA_TRY(cudaMemcpyAsync(h->yred + h->yr_off[j] * k, Y + h->y_off[j] * k,
                                    sizeof(double) * (size_t)h->G[j] * h->M[j] * k, cudaMemcpyDeviceToDevice, s));
    // tol and relres of every reduced instance refer to its M-row model's
    // ||P y||: the reduced ||P' y'||^2 plus the energy of y outside range(W)
    k_batch_complement<<<dim3((unsigned)h->count, (unsigned)k), 256, 0, s>>>(k, h->d_redrows, Y, h->yred,
                                                                             h->d_extra);
    h->launches += 1;
    GS_CUDA_TRY(cudaGetLastError());
    h->last_k = k;
    h->inner->rho_extra = h->d_extra;
    return glm_sur_batch_solve(h->inner, h->yred, k, b, iters, relres, stream);
  }
  if (h->maxNq * k > kBatchMaxPairs) return GLM_SUR_INVALID_ARG;
  if (k > h->kcap) {
    free_solve(h);
    const size_t nv = (size_t)h->v_rows * k;
    GS_CUDA_TRY(balloc(&h->w64, nv)); GS_CUDA_TRY(balloc(&h->E64, nv)); GS_CUDA_TRY(balloc(&h->d64, nv));
    GS_CUDA_TRY(balloc(&h->g32, nv)); GS_CUDA_TRY(balloc(&h->u32, nv)); GS_CUDA_TRY(balloc(&h->w32, nv));
    GS_CUDA_TRY(balloc(&h->wb32, nv));
    GS_CUDA_TRY(balloc(&h->status, (size_t)h->count * k));
    GS_CUDA_TRY(balloc(&h->iters_d, (size_t)h->count * k));
    GS_CUDA_TRY(balloc(&h->relres_d, (size_t)h->count * k));
    GS_CUDA_TRY(balloc(&h->steps_d, (size_t)h->count));
    GS_CUDA_TRY(balloc(&h->cycles_d, (size_t)h->count));
    GS_CUDA_TRY(balloc(&h->d_insts, (size_t)h->count));
    h->kcap = k;
  }
  if (h->insts_k != k) {
    // the descriptors are rewritten below: an earlier solve on this stream must be done
    GS_CUDA_TRY(cudaStreamSynchronize(s));
    // first work order: most expensive steps first (cost ~ M (G^2 + 2 n'));
    // replaced by the measured times once the autotuner has run the batch
    std::vector<double> cost(h->count);
    for (int j = 0; j < h->count; ++j) cost[j] = (double)h->M[j] * (h->G[j] * h->G[j] + 2.0 * h->np[j]);
    GS_CUDA_TRY(write_work_order(h, k, cost));
    h->insts_k = k;
    h->tile = 0;
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  BatchPools P{h->q64, h->q32, h->R, h->om64, h->om32, h->d_n_i, h->d_poff, h->d_r_off, h->d_quad_blk,
               h->w64, h->E64, h->d64, h->g32, h->u32, h->w32, h->wb32, Y, b, h->status, h->iters_d,
               h->relres_d, h->steps_d, h->cycles_d, h->rho_extra};
  BatchOpts bo{h->opts.tol, h->opts.inner_tol, h->opts.max_refine, 4000, 25};
  if (h->tile == 0) {
    // autotune: time one batch solve per tile height, tallest first, keep the
    // fastest; stop once a candidate is 10% slower than the best so far
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    std::vector<long long> best_cycles(h->count, 0);   // per-instance times of the fastest tile height
    for (int t = 2; t >= 0; --t) {
      const int TR = kBatchTiles[t];
      int ctas = 0;
      if (batch_prepare(k, TR, h->maxG, h->maxNp, &ctas) != cudaSuccess) {
        cudaGetLastError();   // tile height whose shared memory does not fit
        ctas = 0;
      }
      if (ctas < 1) { h->tune_ms[t] = -1; continue; }
      const int grid = h->sms * ctas;
      cudaEventRecord(e0, s);
      GS_CUDA_TRY(batch_solve_launch(k, TR, h->d_insts, h->count, P, bo, h->counter, grid, h->maxG, h->maxNp, s));
      cudaEventRecord(e1, s);
      GS_CUDA_TRY(cudaEventSynchronize(e1));
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      h->tune_ms[t] = ms;
      h->launches += 2;
      if (ms < best) {
        best = ms; h->tile = TR; h->grid = grid;
        GS_CUDA_TRY(cudaMemcpy(best_cycles.data(), h->cycles_d, sizeof(long long) * h->count,
                               cudaMemcpyDeviceToHost));
      } else if (ms > 1.1f * best) {
        break;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (h->tile == 0) return GLM_SUR_INVALID_ARG;
    // re-order by the measured time of every instance at the chosen tile height
    std::vector<double> cost(best_cycles.begin(), best_cycles.end());
    GS_CUDA_TRY(write_work_order(h, k, cost));
  }
  // one persistent launch, replayed from a captured graph while the buffers stay the same
  const void* key[5] = {Y, b, iters, relres, h->rho_extra};
  if (!h->graph || h->graph_k != k || std::memcmp(key, h->graph_key, sizeof key) != 0) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    cudaStream_t cs;
    GS_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    GS_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    batch_solve_launch(k, h->tile, h->d_insts, h->count, P, bo, h->counter, h->grid, h->maxG, h->maxNp, cs);
    if (iters) cudaMemcpyAsync(iters, h->iters_d, sizeof(int) * h->count * k, cudaMemcpyDeviceToDevice, cs);
    if (relres) cudaMemcpyAsync(relres, h->relres_d, sizeof(double) * h->count * k, cudaMemcpyDeviceToDevice, cs);
    GS_CUDA_TRY(cudaStreamEndCapture(cs, &g));
    cudaError_t e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      set_last_error(e, "cudaGraphInstantiate(batch)", __FILE__, __LINE__);
      h->graph = nullptr;
      return GLM_SUR_CUDA_ERROR;
    }
    std::memcpy(h->graph_key, key, sizeof key);
    h->graph_k = k;
  }
  GS_CUDA_TRY(cudaGraphLaunch(h->graph, s));
  h->launches += 2;
  h->last_k = k;
  return GLM_SUR_OK;
}

glm_sur_status glm_sur_batch_get_status(glm_sur_batch_t h, int* status) {
  if (h && h->inner) return glm_sur_batch_get_status(h->inner, status);
  if (!h || !status || h->last_k < 1) return GLM_SUR_INVALID_ARG;
  GS_CUDA_TRY(cudaDeviceSynchronize());
  GS_CUDA_TRY(cudaMemcpy(status, h->status, sizeof(int) * h->count * h->last_k, cudaMemcpyDeviceToHost));
  glm_sur_status worst = GLM_SUR_OK;
  for (int j = 0; j < h->count * h->last_k; ++j) {
    if (status[j] == kStatusRunning) status[j] = GLM_SUR_NOT_CONVERGED;
    if (status[j] != GLM_SUR_OK && status[j] != GLM_SUR_STAGNATED && worst == GLM_SUR_OK)
      worst = (glm_sur_status)status[j];
  }
  return worst;
}

glm_sur_status glm_sur_batch_get_work(glm_sur_batch_t h, int* steps, long long* cycles) {
  if (h && h->inner) return glm_sur_batch_get_work(h->inner, steps, cycles);
  if (!h || (!steps && !cycles)) return GLM_SUR_INVALID_ARG;
  if (!h->steps_d) return GLM_SUR_INVALID_ARG;   // no solve yet
  GS_CUDA_TRY(cudaDeviceSynchronize());
  if (steps) GS_CUDA_TRY(cudaMemcpy(steps, h->steps_d, sizeof(int) * h->count, cudaMemcpyDeviceToHost));
  if (cycles) GS_CUDA_TRY(cudaMemcpy(cycles, h->cycles_d, sizeof(long long) * h->count, cudaMemcpyDeviceToHost));
  return GLM_SUR_OK;
}

int glm_sur_batch_tile(glm_sur_batch_t h, float* tune_ms) {
  if (h && h->inner) return glm_sur_batch_tile(h->inner, tune_ms);
  if (!h) return -1;
  if (tune_ms)
    for (int t = 0; t < 3; ++t) tune_ms[t] = h->tune_ms[t];
  return h->tile;
}

int glm_sur_batch_grid(glm_sur_batch_t h) {
  if (h && h->inner) return glm_sur_batch_grid(h->inner);
  if (!h) return -1;
  return h->tile ? h->grid : 0;
}

int64_t glm_sur_batch_launch_count(glm_sur_batch_t h) {
  if (!h) return -1;
  return h->launches + (h->inner ? glm_sur_batch_launch_count(h->inner) : 0);
}

void glm_sur_batch_destroy(glm_sur_batch_t h) {
  if (!h) return;
  if (h->inner) {
    glm_sur_batch_destroy(h->inner);
    bfree(h->qw);
    bfree(h->yred);
    bfree(h->d_rot);
    bfree(h->d_redrows);
    bfree(h->d_extra);
    delete h;
    return;
  }
  cudaDeviceSynchronize();
  free_solve(h);
  bfree(h->q64); bfree(h->q32); bfree(h->R); bfree(h->om64); bfree(h->om32);
  bfree(h->d_n_i); bfree(h->d_poff); bfree(h->d_r_off); bfree(h->d_quad_blk); bfree(h->setup_flags);
  bfree(h->counter);
  delete h;
}

}  // extern "C"
