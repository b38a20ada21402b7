// C ABI of the SUR PCG-Aug library: handle, workspace, setup (TSQR), solve
// (float64 PCG, or float32 bulk inside float64 iterative refinement) and the
// b recovery of Algorithm glmpcg2 step 10.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "adjoint.h"
#include "glm_sur.h"
#include "internal.h"
#include "mvrglm.h"
#include "ne.h"
#include "noalloc.h"
#include "pcg.h"
#include "pcg3.h"
#include "reduce.h"
#include "rglm.h"

namespace glmsur {

static thread_local std::string g_last_error;
void set_last_error(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  g_last_error = buf;
}

template <typename T>
static cudaError_t dalloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  return cudaMalloc((void**)p, n * sizeof(T));
}
template <typename T>
static void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

// One cached CUDA graph holding `chunk` PCG steps of one configuration.
struct StepGraph {
  cudaGraphExec_t exec = nullptr;
  int key_prec = -1, key_k = -1, key_chunk = -1;
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    key_prec = key_k = key_chunk = -1;
  }
};

}  // namespace glmsur

using namespace glmsur;

struct glm_sur_ctx {
  int dev = 0, sms = 148;
  Geom gm;
  std::vector<int> n_i, off, poff;
  glm_sur_opts opts;
  // factors
  double* Q64 = nullptr;
  float* Q32 = nullptr;
  double* R = nullptr;
  double* Om64 = nullptr;      // Omega of the iteration (scaled: D0^-1/2 Omega D0^-1/2 when precond != identity)
  float* Om32 = nullptr;
  double* Omraw = nullptr;     // Omega as given
  double* d_sqrtd = nullptr;   // sqrt(delta_i) and 1 / sqrt(delta_i) of the preconditioner block (G each)
  double* d_isqrtd = nullptr;
  int* setup_flags = nullptr;
  // solve workspace (capacity kcap right-hand sides)
  int kcap = 0;
  double *y64 = nullptr, *w64 = nullptr, *g64 = nullptr, *u64 = nullptr, *S64 = nullptr, *E64 = nullptr;
  float *g32 = nullptr, *u32 = nullptr, *w32 = nullptr, *S32 = nullptr;
  double* wb64 = nullptr;       // best-iterate snapshots of w
  float* wb32 = nullptr;
  double* d64 = nullptr;        // last projected refinement correction
  int* d_mask = nullptr;        // 2 x k column masks (live columns, columns to revert)
  void* Cpart = nullptr;
  void* Cfin = nullptr;
  double* C64 = nullptr;
  double *dpart = nullptr, *cpart = nullptr, *norms = nullptr;
  // PCG state arrays
  double* st_buf = nullptr;
  int* st_ibuf = nullptr;
  PcgState st;
  int* h_done = nullptr;           // pinned
  double* h_norms = nullptr;       // pinned
  int last_k = 0;
  int* h_status = nullptr;         // host copy of the last per-column status (k)
  int* d_status_final = nullptr;   // device per-column final status
  int* d_iters_acc = nullptr;      // accumulated iterations (refinement)
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  StepGraph graph;
  IterPlan plan;
  int plan_k = -1, plan_prec = -1;
  bool has_w = false;
  int64_t launches = 0;        // kernel launches issued (graph nodes included)
  // linear restrictions C b = d (Sec. 4.1)
  int kc = 0;
  double* Cmat = nullptr;      // kc x n column-major (ld = kc)
  double* Nmat = nullptr;      // n x n: X_aug^T X_aug, then its Cholesky factor
  double* Minv = nullptr;      // n x n: (X_aug^T X_aug)^-1
  double* cbuf = nullptr;      // n x k coefficients c = N^-1 a
  double* fbuf = nullptr;      // n' x k f_i = R_i c_i
  double* gC = nullptr;        // kc x k restriction rows of g
  int rcap = 0;                // k capacity of cbuf / fbuf / gC
  bool w_restricted = false;   // w64 came from a restricted solve
  // row reduction (Remark rem:reduction): the solves run on `sub`, the model
  // with the n rows Q^T y_i of every equation
  glm_sur_ctx* sub = nullptr;
  double* Qw = nullptr;        // M x n column-major orthonormal basis of range(W)
  double* yred = nullptr;      // reduced responses / gradients, (G n) x k column-major
  int64_t yred_cap = 0;
  double* rot_ws = nullptr;    // depth-split partial products of the rotation
  int64_t rot_ws_cap = 0;
  // (on the reduced model) energy of the responses outside range(W), k
  // values, added to the reference of relres and tol while c1x_on
  double* c1x = nullptr;
  double* c1x_part = nullptr;  // G x kMaxRhs workspace
  bool c1x_on = false;
  // adjoint (glm_sur_backward)
  double* wfwd = nullptr;      // the forward w while the adjoint solve runs
  double* lam1 = nullptr;      // particular solution lam_1 = Q R^-T dL/db
  double* opart = nullptr;     // chunk partials of the Omega gradient
  int acap = 0;                // k capacity of wfwd / lam1
  int64_t ocap = 0;            // doubles in opart
  // PCG-NE comparator (glm_sur_solve_ne)
  double* ne_buf = nullptr;    // beta, f, p, q (n x k each), cvec (n' x k), c, c1, relres (k each)
  int* ne_ibuf = nullptr;      // active, iters, status (k each)
  double* ne_om = nullptr;     // Omega^-1 (G x Gq), then the Cholesky factor and its inverse (G x G each)
  int* ne_hact = nullptr;      // pinned copy of the active flags
  int necap = 0;
  // Algorithm glmpcg3 (opts.algorithm): per-column state and d partials
  double* p3_buf = nullptr;
  int* p3_ibuf = nullptr;
  int* p3_hact = nullptr;      // pinned copy of the active flags
  int p3cap = 0;
  // restricted multivariate GLM (glm_sur_mvrglm_setup): the solves run on
  // `sub`, the G equations [R0; C_i] (N + kmax rows each) with Sigma = 0 on
  // the restriction rows
  int mv_N = 0, mv_kmax = 0, mv_ktot = 0;
  int* mv_koff = nullptr;      // device, G + 1: first restriction row of each equation
  double* mv_Q0 = nullptr;     // M x N row-major, Z0 = Q0 R0
  double* mv_y = nullptr;      // assembled responses, (G (N + kmax)) x k column-major
  int64_t mv_ycap = 0;
};

namespace {

constexpr int kStateDoubles = 10;
constexpr int kStateInts = 6;
// stagnation window of the float32 inner solves (at least; a longer outer
// window W applies to them too)
constexpr int kInnerStagnation = 25;

// float64 PCG steps rather than float32 inner runs inside refinement
bool fp64_steps(const glm_sur_opts& o) { return o.precision != GLM_SUR_PREC_FP32_REFINE; }

glm_sur_status validate_opts(const glm_sur_opts* o) {
  if (o->precision != GLM_SUR_PREC_FP64 && o->precision != GLM_SUR_PREC_FP32_REFINE) return GLM_SUR_INVALID_ARG;
  if (!(o->tol >= 0.0) || !(o->inner_tol > 0.0)) return GLM_SUR_INVALID_ARG;
  if (o->chunk < 2 || (o->chunk & 1)) return GLM_SUR_INVALID_ARG;
  if (!(o->inner_shift >= 0.0) || o->inner_shift > 1e-2) return GLM_SUR_INVALID_ARG;
  if (o->step_kernels != GLM_SUR_STEP_AUTO && o->step_kernels != GLM_SUR_STEP_SIMT) return GLM_SUR_INVALID_ARG;
  if (o->precond < GLM_SUR_PRECOND_IDENTITY || o->precond > GLM_SUR_PRECOND_DIAG) return GLM_SUR_INVALID_ARG;
  if (o->algorithm != GLM_SUR_ALG_GLMPCG2 && o->algorithm != GLM_SUR_ALG_GLMPCG3) return GLM_SUR_INVALID_ARG;
  return GLM_SUR_OK;
}

int pick_jj(int k, bool is_double) {
  const int cap = is_double ? 8 : 16;
  for (int jj = cap; jj > 1; jj >>= 1)
    if (k % jj == 0) return jj;
  return 1;
}

glm_sur_status make_plan(glm_sur_ctx* h, int k, bool is_double, IterPlan& p) {
  const Geom& gm = h->gm;
  const size_t sz = is_double ? 8 : 4;
  p.JJ = pick_jj(k, is_double);
  const int njg = k / p.JJ;
  const size_t om_bytes = sz * (size_t)gm.G * gm.Gq;
  const size_t row_bytes = sz * (size_t)gm.G * p.JJ;
  const size_t budget = 200 * 1024;
  if (gm.G > kMaxSolveG || om_bytes + row_bytes > budget) return GLM_SUR_INVALID_ARG;   // Omega must fit shared memory
  p.TR = (int)std::max<size_t>(1, std::min<size_t>(16, (budget / 2 - std::min(om_bytes, budget / 2)) / row_bytes));
  if (p.TR < 1) p.TR = 1;
  p.sigma_smem = om_bytes + (size_t)p.TR * row_bytes;
  const int target = 2 * h->sms;
  p.n_sigma = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(gm.M, p.TR), ceil_div(target, njg)));
  p.n_qgroups = (int)std::max<int64_t>(1, ceil_div(gm.nq, 256));
  p.n_partial_rows = (int)std::max<int64_t>(1, std::min<int64_t>(gm.M, ceil_div(target, (int64_t)p.n_qgroups * njg)));
  p.n_ugroups = gm.n_ugroups;
  p.ug_max_quads = gm.ug_max_quads;
  p.ug_threads = (int)std::min<int64_t>(512, ceil_div(gm.ug_max_quads, 32) * 32);
  p.n_update = (int)std::max<int64_t>(1, std::min<int64_t>(gm.M, ceil_div(target, (int64_t)njg * p.n_ugroups)));
  p.n_cpart = p.n_update * p.n_ugroups;
  p.extra_cpart = h->kc > 0 ? 1 : 0;
  const size_t upd_row = sz * (size_t)(gm.ug_max_quads + 32) * p.JJ;   // padded quad stride
  p.TRB = (int)std::max<size_t>(2, std::min<size_t>(32, (48 * 1024) / upd_row));
  p.update_smem = (size_t)p.TRB * upd_row;
  // TMA-streamed step kernels: one CTA per SM, whole rows (all k) per tile
  const size_t GK_bytes = sz * (size_t)gm.G * k;
  const size_t budget_tma = 200 * 1024;
  int nmax = 0;
  for (int v : h->n_i) nmax = std::max(nmax, v);
  if (p.JJ == k && GK_bytes % 16 == 0) {
    // Sigma step: items are (RI-row group, column quad of Omega, rhs); pick RI
    // and the tile height TR so that a tile holds >= 512 items when shared
    // memory allows (3 stages, else 2)
    const size_t om = sz * (size_t)gm.G * gm.Gq;
    const size_t sig_budget = 210 * 1024;
    const int per_row_items = (gm.Gq / 4) * p.JJ;
    p.ri = per_row_items >= 256 ? 4 : (per_row_items >= 64 ? 2 : 1);
    int tr_want = p.ri * (int)ceil_div(512, per_row_items);
    if (!is_double && p.JJ == 1 && gm.G % 4 == 0) {
      // float4 runs of one right-hand side: two rows per item when the tile is tall enough
      p.ri = 2;
      tr_want = 2 * (int)ceil_div(512, gm.Gq / 4);
    }
    tr_want = std::max(p.ri, std::min(64, tr_want));
    for (int tr = tr_want; tr >= 1 && !p.tma_sigma; tr = (tr > p.ri ? tr - p.ri : tr - 1)) {
      for (int nst = 3; nst >= 2; --nst) {
        if (128 + om + (size_t)nst * tr * 3 * GK_bytes <= sig_budget) {
          p.tr_tma = tr; p.nst_sigma = nst; p.tma_sigma = true;
          break;
        }
      }
    }
    if (p.tma_sigma) p.sigma_tma_smem = 128 + om + (size_t)p.nst_sigma * p.tr_tma * 3 * GK_bytes;
    if (gm.n_ugroups == 1) {
      p.nst_update = 3;
      const size_t row_stage = sz * (size_t)gm.np + 2 * GK_bytes, row_part = sz * (size_t)(gm.nq + 32) * p.JJ;
      const size_t per_row = p.nst_update * row_stage + row_part;
      if (per_row + 128 <= budget_tma) {
        p.trb_tma = (int)std::min<size_t>(16, (budget_tma - 128) / per_row);
        p.tma_update = true;
        p.update_tma_smem = 128 + (size_t)p.trb_tma * per_row;
        p.update_threads = (int)std::max<int64_t>(256, std::min<int64_t>(512, ceil_div(gm.nq, 32) * 32));
      }
    }
    // block x column update: every block at most 32 columns, G*k pairs on <= 2 per thread
    const int npairs = gm.G * k;
    if (nmax <= 32 && npairs <= 1024 && (!is_double || npairs <= 512)) {
      p.bj_np = npairs > 512 ? 2 : 1;
      p.nst_bj = 3;
      const size_t row_stage = sz * (size_t)gm.np + 2 * GK_bytes;
      const size_t trb = (budget_tma - 128) / (p.nst_bj * row_stage);
      if (trb >= 1) {
        p.trb_bj = (int)std::min<size_t>(16, trb);
        p.bj_smem = 128 + (size_t)p.nst_bj * p.trb_bj * row_stage;
        p.bj_update = true;
        p.tma_update = true;   // same grid and partial layout
      }
    }
    // projection partials: a thread per column quad, rows of Q and S streamed
    if (gm.nq <= 512) {
      const size_t row_stage = sz * (size_t)gm.np + GK_bytes;
      p.nst_partial = 3;
      const size_t trp = (budget_tma - 128) / (p.nst_partial * row_stage);
      if (trp >= 1) {
        p.tr_partial = (int)std::min<size_t>(16, trp);
        p.partial_tma_smem = 128 + (size_t)p.nst_partial * p.tr_partial * row_stage;
        p.partial_threads = (int)std::max<int64_t>(64, ceil_div(gm.nq, 32) * 32);
        p.tma_partial = true;
        p.n_partial_rows = h->sms;
        p.n_qgroups = 1;
      }
    }
    if (p.tma_sigma) p.n_sigma = h->sms;
    if (p.tma_update) {
      p.n_update = h->sms;
      p.n_cpart = h->sms;
    }
    p.extra_cpart = h->kc > 0 ? 1 : 0;
    // fused float32 step with the tensor-core Sigma-apply (pcg_tc.cu)
    if (!is_double && h->kc == 0 && gm.Ms == gm.M && h->opts.step_kernels != GLM_SUR_STEP_SIMT &&
        tc_step_eligible(gm.G, k, gm.np, nmax)) {
      p.tc_gp = gm.G <= 32 ? 32 : 64;
      const int TV = 128 / k;
      const size_t tc_budget = 224 * 1024;
      // Q ring of each pass: the largest number of rows in flight (tq x nsq,
      // nsq >= 2) that fits next to the fixed buffers; pass B keeps two g tiles
      // in flight when it can
      auto pick_q = [&](int pass, int nsg, int& tq_out, int& nsq_out) {
        int best = 0;
        for (int tq = TV; tq >= 1; tq >>= 1)
          for (int nsq = 2; nsq <= 4; ++nsq) {
            const TcSmem L = tc_smem_layout(pass, gm.G, p.tc_gp, k, gm.np, tq, nsq, nsg);
            if (L.total <= tc_budget && tq * nsq > best) {
              best = tq * nsq;
              tq_out = tq;
              nsq_out = nsq;
            }
          }
        return best > 0;
      };
      bool ok = pick_q(0, 0, p.tc_tq_a, p.tc_nsq_a);
      // pass B: two g tiles in flight when the Q ring still holds a full
      // vector tile of rows, else one
      int tq2 = 0, nsq2 = 0, tq1 = 0, nsq1 = 0;
      const bool ok2 = pick_q(1, 2, tq2, nsq2), ok1 = pick_q(1, 1, tq1, nsq1);
      const bool okb = ok2 || ok1;
      if (tc_smem_layout(1, gm.G, p.tc_gp, k, gm.np, TV, 2, 1).total <= tc_budget) {
        // one Q sub-tile per vector tile, two in flight, one staged g tile:
        // the fastest ring measured at G = 64, k = 16 (pass B 0.143 ms against
        // 0.152 with two g tiles and half-height Q sub-tiles)
        p.tc_nsg = 1; p.tc_tq_b = TV; p.tc_nsq_b = 2;
      } else if (ok2 && (tq2 * nsq2 >= TV || !ok1)) {
        p.tc_nsg = 2; p.tc_tq_b = tq2; p.tc_nsq_b = nsq2;
      } else if (ok1) {
        p.tc_nsg = 1; p.tc_tq_b = tq1; p.tc_nsq_b = nsq1;
      }
      if (const char* env = getenv("GLMSUR_TC_RING")) {   // tuning override: "tqa,nsqa,tqb,nsqb,nsg"
        int a0, a1, b0, b1, b2;
        if (sscanf(env, "%d,%d,%d,%d,%d", &a0, &a1, &b0, &b1, &b2) == 5 && a0 >= 1 && TV % a0 == 0 &&
            b0 >= 1 && TV % b0 == 0 && a1 >= 1 && b1 >= 1 && b2 >= 1 && a1 + 2 <= 16 && b1 + b2 + 2 <= 16 &&
            tc_smem_layout(0, gm.G, p.tc_gp, k, gm.np, a0, a1, 0).total <= tc_budget &&
            tc_smem_layout(1, gm.G, p.tc_gp, k, gm.np, b0, b1, b2).total <= tc_budget) {
          p.tc_tq_a = a0; p.tc_nsq_a = a1; p.tc_tq_b = b0; p.tc_nsq_b = b1; p.tc_nsg = b2;
        }
      }
      if (ok && okb) {
        p.tc_a_smem = tc_smem_layout(0, gm.G, p.tc_gp, k, gm.np, p.tc_tq_a, p.tc_nsq_a, 0).total;
        p.tc_b_smem = tc_smem_layout(1, gm.G, p.tc_gp, k, gm.np, p.tc_tq_b, p.tc_nsq_b, p.tc_nsg).total;
        p.tc_step = true;
        p.launches_per_step = 3;
        p.n_sigma = p.n_partial_rows = p.n_update = p.n_cpart = h->sms;
        p.n_qgroups = 1;
      }
    }
  }
  cudaError_t e = is_double ? set_smem_attrs<double>(p.JJ, p.sigma_smem, p.update_smem)
                            : set_smem_attrs<float>(p.JJ, p.sigma_smem, p.update_smem);
  if (e == cudaSuccess && (p.tma_sigma || p.tma_update || p.tma_partial))
    e = is_double ? set_tma_smem_attrs<double>(p.JJ, std::max<size_t>(p.sigma_tma_smem, 1024),
                                               std::max<size_t>(p.update_tma_smem, 1024),
                                               std::max<size_t>(p.bj_smem, 1024),
                                               std::max<size_t>(p.partial_tma_smem, 1024))
                  : set_tma_smem_attrs<float>(p.JJ, std::max<size_t>(p.sigma_tma_smem, 1024),
                                              std::max<size_t>(p.update_tma_smem, 1024),
                                              std::max<size_t>(p.bj_smem, 1024),
                                              std::max<size_t>(p.partial_tma_smem, 1024));
  if (e == cudaSuccess && p.tc_step) e = tc_prepare(k, p.tc_gp, p.tc_a_smem, p.tc_b_smem);
  if (e != cudaSuccess) {
    set_last_error(e, "cudaFuncSetAttribute", __FILE__, __LINE__);
    return GLM_SUR_CUDA_ERROR;
  }
  return GLM_SUR_OK;
}

void free_workspace(glm_sur_ctx* h) {
  dfree(h->y64); dfree(h->w64); dfree(h->g64); dfree(h->u64); dfree(h->S64); dfree(h->E64);
  dfree(h->g32); dfree(h->u32); dfree(h->w32); dfree(h->S32); dfree(h->wb64); dfree(h->wb32);
  if (h->Cpart) cudaFree(h->Cpart);
  if (h->Cfin) cudaFree(h->Cfin);
  h->Cpart = h->Cfin = nullptr;
  dfree(h->C64); dfree(h->dpart); dfree(h->cpart); dfree(h->norms);
  dfree(h->st_buf); dfree(h->st_ibuf); dfree(h->d_status_final); dfree(h->d_iters_acc);
  dfree(h->d64); dfree(h->d_mask);
  if (h->h_status) { delete[] h->h_status; h->h_status = nullptr; }
  h->kcap = 0;
  h->graph.reset();
  h->has_w = false;   // the forward w went with the workspace (no adjoint without a new solve)
}

// Allocate every buffer a solve with k right-hand sides needs (both precisions).
glm_sur_status ensure_workspace(glm_sur_ctx* h, int k) {
  if (k <= h->kcap) return GLM_SUR_OK;
  free_workspace(h);
  const Geom& gm = h->gm;
  const size_t mk = (size_t)gm.M * gm.G * k;
  const int maxrows = 2 * h->sms + gm.n_ugroups + 8;   // upper bound of every partial count in make_plan
  const size_t cpart_n = (size_t)maxrows * gm.np * k;
  GS_CUDA_TRY(dalloc(&h->y64, mk));
  GS_CUDA_TRY(dalloc(&h->w64, mk));
  GS_CUDA_TRY(dalloc(&h->g64, mk));
  GS_CUDA_TRY(dalloc(&h->E64, mk));
  if (fp64_steps(h->opts)) {
    GS_CUDA_TRY(dalloc(&h->u64, mk));
    GS_CUDA_TRY(dalloc(&h->S64, mk));
    GS_CUDA_TRY(dalloc(&h->wb64, mk));
  } else {
    GS_CUDA_TRY(dalloc(&h->g32, mk));
    GS_CUDA_TRY(dalloc(&h->u32, mk));
    GS_CUDA_TRY(dalloc(&h->w32, mk));
    GS_CUDA_TRY(dalloc(&h->S32, mk));
    GS_CUDA_TRY(dalloc(&h->wb32, mk));
  }
  GS_CUDA_TRY(cudaMalloc(&h->Cpart, cpart_n * sizeof(double)));
  GS_CUDA_TRY(cudaMalloc(&h->Cfin, (size_t)gm.np * k * sizeof(double)));
  GS_CUDA_TRY(dalloc(&h->C64, (size_t)gm.np * k));
  GS_CUDA_TRY(dalloc(&h->dpart, (size_t)maxrows * k));
  GS_CUDA_TRY(dalloc(&h->cpart, (size_t)maxrows * k));
  GS_CUDA_TRY(dalloc(&h->norms, (size_t)2 * k));
  if (h->opts.precision != GLM_SUR_PREC_FP64) GS_CUDA_TRY(dalloc(&h->d64, mk));
  // doubles: c[2], c1, lam, relres, cbest[2];  ints: active[2], iters, status, itbest[2], it, done
  GS_CUDA_TRY(dalloc(&h->st_buf, (size_t)kStateDoubles * k));
  GS_CUDA_TRY(dalloc(&h->st_ibuf, (size_t)kStateInts * k + 3));
  GS_CUDA_TRY(dalloc(&h->d_status_final, (size_t)k));
  GS_CUDA_TRY(dalloc(&h->d_iters_acc, (size_t)k));
  GS_CUDA_TRY(dalloc(&h->d_mask, (size_t)2 * k));
  h->h_status = new int[k];
  PcgState& st = h->st;
  st.k = k;
  st.c[0] = h->st_buf;
  st.c[1] = h->st_buf + k;
  st.c1 = h->st_buf + 2 * k;
  st.lam = h->st_buf + 3 * k;
  st.relres = h->st_buf + 4 * k;
  st.cbest[0] = h->st_buf + 5 * k;
  st.cbest[1] = h->st_buf + 6 * k;
  st.csnap[0] = h->st_buf + 7 * k;
  st.csnap[1] = h->st_buf + 8 * k;
  st.cstop = h->st_buf + 9 * k;
  st.active[0] = h->st_ibuf;
  st.active[1] = h->st_ibuf + k;
  st.iters = h->st_ibuf + 2 * k;
  st.status = h->st_ibuf + 3 * k;
  st.itbest[0] = h->st_ibuf + 4 * k;
  st.itbest[1] = h->st_ibuf + 5 * k;
  st.it = h->st_ibuf + 6 * k;
  st.done = h->st_ibuf + 6 * k + 1;
  st.err = h->st_ibuf + 6 * k + 2;
  h->kcap = k;
  return GLM_SUR_OK;
}

// Reset the per-column PCG state before a run (stream-ordered).
glm_sur_status reset_state(glm_sur_ctx* h, int k, double tol, int maxit, int W, cudaStream_t s) {
  PcgState& st = h->st;
  st.k = k;
  st.tol = tol;
  st.maxit = maxit;
  st.W = W;
  st.c1_extra = nullptr;
  GS_CUDA_TRY(cudaMemsetAsync(h->st_buf, 0, sizeof(double) * (size_t)kStateDoubles * h->kcap, s));
  GS_CUDA_TRY(cudaMemsetAsync(h->st_ibuf, 0, sizeof(int) * ((size_t)kStateInts * h->kcap + 2), s));
  // (the error word after them is cleared per solve, not per inner run)
  return GLM_SUR_OK;
}

template <typename T>
struct Bufs;
template <>
struct Bufs<double> {
  static double* g(glm_sur_ctx* h) { return h->g64; }
  static double* u(glm_sur_ctx* h) { return h->u64; }
  static double* w(glm_sur_ctx* h) { return h->w64; }
  static double* S(glm_sur_ctx* h) { return h->S64; }
  static double* Q(glm_sur_ctx* h) { return h->Q64; }
  static double* Om(glm_sur_ctx* h) { return h->Om64; }
  static double* wb(glm_sur_ctx* h) { return h->wb64; }
};
template <>
struct Bufs<float> {
  static float* g(glm_sur_ctx* h) { return h->g32; }
  static float* u(glm_sur_ctx* h) { return h->u32; }
  static float* w(glm_sur_ctx* h) { return h->w32; }
  static float* S(glm_sur_ctx* h) { return h->S32; }
  static float* Q(glm_sur_ctx* h) { return h->Q32; }
  static float* Om(glm_sur_ctx* h) { return h->Om32; }
  static float* wb(glm_sur_ctx* h) { return h->wb32; }
};

// Enqueue n PCG steps (four launches each).
template <typename T>
void enqueue_steps(glm_sur_ctx* h, int k, int n, cudaStream_t s) {
  const IterPlan& p = h->plan;
  T* Cpart = reinterpret_cast<T*>(h->Cpart);
  T* C = reinterpret_cast<T*>(h->Cfin);
  for (int i = 0; i < n; ++i) {
    if constexpr (sizeof(T) == sizeof(float)) {
      if (p.tc_step) {
        // pass A (u, S = U Omega on the tensor cores, d and C partials), reduce, pass B
        launch_tc_pass_a(p, h->gm, k, h->Om32, h->Q32, h->g32, h->u32, h->w32, h->wb32, h->st, h->cpart,
                         p.n_cpart + p.extra_cpart, h->dpart, Cpart, s);
        launch_reduce<float>(p, h->gm, k, Cpart, C, h->st, 1, h->dpart, s, true);
        launch_tc_pass_b(p, h->gm, k, h->Om32, h->Q32, h->g32, h->u32, h->w32, C, h->st, h->cpart, s);
        continue;
      }
    }
    launch_sigma_step<T>(p, h->gm, k, Bufs<T>::Om(h), Bufs<T>::g(h), Bufs<T>::u(h), Bufs<T>::w(h), Bufs<T>::S(h),
                         Bufs<T>::wb(h), h->st, h->cpart, h->dpart, s);
    launch_proj_partial<T>(p, h->gm, k, Bufs<T>::Q(h), Bufs<T>::S(h), Cpart, h->st, 1, s);
    launch_reduce<T>(p, h->gm, k, Cpart, C, h->st, 1, h->dpart, s);
    const T* Cupd = C;
    if (h->kc > 0 && sizeof(T) == sizeof(double)) {
      // restricted GLM (Sec. 4.1): c = N^-1 [R_i^T e_i], f_i = R_i c_i, g_C += lambda C c
      rglm_coef(h->gm, k, reinterpret_cast<const double*>(C), h->R, h->Minv, h->Cmat, h->kc, h->kc, nullptr, 0, 0.0,
                h->cbuf, h->fbuf, nullptr, 0, s);
      rglm_gc(h->gm, k, h->kc, h->Cmat, h->kc, h->cbuf, nullptr, 0, h->st.lam, 0, h->gC, h->cpart, p.n_cpart, s);
      Cupd = reinterpret_cast<const T*>(h->fbuf);
    }
    launch_proj_update<T>(p, h->gm, k, Bufs<T>::Q(h), Bufs<T>::S(h), Bufs<T>::g(h), Cupd, 1, h->st.lam, 0.0,
                          h->cpart, h->st, 1, s);
  }
}

// Run PCG steps until every column stopped: a captured graph of `chunk`
// steps is replayed, and the host reads the done flag one replay behind.
template <typename T>
glm_sur_status run_steps(glm_sur_ctx* h, int k, int maxit, cudaStream_t s) {
  const int prec = sizeof(T) == 8 ? 0 : 1;
  const int chunk = h->opts.chunk;
  StepGraph& gr = h->graph;
  if (!gr.exec || gr.key_prec != prec || gr.key_k != k || gr.key_chunk != chunk) {
    gr.reset();
    cudaGraph_t graph = nullptr;
    GS_CUDA_TRY(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    enqueue_steps<T>(h, k, chunk, h->cap_stream);
    GS_CUDA_TRY(cudaStreamEndCapture(h->cap_stream, &graph));
    cudaError_t e = cudaGraphInstantiate(&gr.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      set_last_error(e, "cudaGraphInstantiate", __FILE__, __LINE__);
      gr.exec = nullptr;
      return GLM_SUR_CUDA_ERROR;
    }
    gr.key_prec = prec; gr.key_k = k; gr.key_chunk = chunk;
  }
  const int64_t max_launch = (int64_t)maxit / chunk + 3;
  for (int64_t c = 0; c < max_launch; ++c) {
    GS_CUDA_TRY(cudaGraphLaunch(gr.exec, s));
    h->launches += (h->kc > 0 ? 6 : h->plan.launches_per_step) * (int64_t)chunk;
    // done flag and error word side by side: h_done[2*slot], h_done[2*slot + 1]
    GS_CUDA_TRY(cudaMemcpyAsync(&h->h_done[2 * (c & 1)], h->st.done, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    GS_CUDA_TRY(cudaEventRecord(h->ev[c & 1], s));
    if (c >= 1) {
      GS_CUDA_TRY(cudaEventSynchronize(h->ev[(c - 1) & 1]));
      if (h->h_done[2 * ((c - 1) & 1)] || h->h_done[2 * ((c - 1) & 1) + 1]) break;
    }
  }
  // columns that stopped without converging keep their best saved w
  launch_restore_best<T>(h->gm.M * h->gm.G * k, k, h->st, Bufs<T>::wb(h), Bufs<T>::w(h), s);
  h->launches += 2;
  GS_CUDA_TRY(cudaGetLastError());
  return GLM_SUR_OK;
}

// g = -P y  (first residual of the PCG started at w = 0), u = w = 0, partials of g^T g.
// Restricted (d != null or kc > 0): g = -Pi y_aug, y_aug = [y; d] (Sec. 4.1).
template <typename T>
glm_sur_status pcg_init(glm_sur_ctx* h, int k, const T* y_layout, cudaStream_t s, const double* d = nullptr,
                        int64_t ldd = 0) {
  const IterPlan& p = h->plan;
  T* Cpart = reinterpret_cast<T*>(h->Cpart);
  T* C = reinterpret_cast<T*>(h->Cfin);
  const size_t mk = (size_t)h->gm.M * h->gm.G * k;
  launch_proj_partial<T>(p, h->gm, k, Bufs<T>::Q(h), y_layout, Cpart, h->st, 0, s);
  launch_reduce<T>(p, h->gm, k, Cpart, C, h->st, 0, nullptr, s);
  const T* Cupd = C;
  if (h->kc > 0 && sizeof(T) == sizeof(double)) {
    GS_CUDA_TRY(rglm_coef(h->gm, k, reinterpret_cast<const double*>(C), h->R, h->Minv, h->Cmat, h->kc, h->kc, d, ldd,
                          1.0, h->cbuf, h->fbuf, nullptr, 0, s));
    Cupd = reinterpret_cast<const T*>(h->fbuf);
  }
  launch_proj_update<T>(p, h->gm, k, Bufs<T>::Q(h), y_layout, Bufs<T>::g(h), Cupd, 0, nullptr, 1.0, h->cpart, h->st,
                        0, s);
  if (h->kc > 0 && sizeof(T) == sizeof(double)) {
    if (d == nullptr) GS_CUDA_TRY(cudaMemsetAsync(h->gC, 0, sizeof(double) * (size_t)h->kc * k, s));
    // g_C = C c - d (d = 0 when not given)
    GS_CUDA_TRY(rglm_gc(h->gm, k, h->kc, h->Cmat, h->kc, h->cbuf, d, ldd, nullptr, d ? 1 : 2, h->gC, h->cpart,
                        p.n_cpart, s));
    h->launches += 2;
  }
  h->launches += 3;
  GS_CUDA_TRY(cudaMemsetAsync(Bufs<T>::u(h), 0, mk * sizeof(T), s));
  GS_CUDA_TRY(cudaMemsetAsync(Bufs<T>::w(h), 0, mk * sizeof(T), s));
  GS_CUDA_TRY(cudaMemsetAsync(Bufs<T>::wb(h), 0, mk * sizeof(T), s));
  return GLM_SUR_OK;
}

// rho = P (y - Sigma w64) in float64 (into g64), partials of rho^T rho in cpart.
glm_sur_status true_residual(glm_sur_ctx* h, int k, const IterPlan& p64, cudaStream_t s) {
  double* Cpart = reinterpret_cast<double*>(h->Cpart);
  launch_sigma_resid<double>(p64, h->gm, k, h->Om64, h->y64, h->w64, h->E64, s);
  launch_proj_partial<double>(p64, h->gm, k, h->Q64, h->E64, Cpart, h->st, 0, s);
  launch_reduce<double>(p64, h->gm, k, Cpart, h->C64, h->st, 0, nullptr, s);
  launch_proj_update<double>(p64, h->gm, k, h->Q64, h->E64, h->g64, h->C64, 0, nullptr, -1.0, h->cpart, h->st, 0, s);
  h->launches += 4;
  return GLM_SUR_OK;
}

// d64 = P (double) w32;  w64 += d64 on the live columns (mask d_mask[0..k))
glm_sur_status project_correction(glm_sur_ctx* h, int k, const IterPlan& p64, cudaStream_t s) {
  double* Cpart = reinterpret_cast<double*>(h->Cpart);
  const int64_t mk = h->gm.M * h->gm.G * k;
  launch_convert<float, double>(mk, h->w32, h->E64, 1.0, s);
  launch_proj_partial<double>(p64, h->gm, k, h->Q64, h->E64, Cpart, h->st, 0, s);
  launch_reduce<double>(p64, h->gm, k, Cpart, h->C64, h->st, 0, nullptr, s);
  launch_proj_update<double>(p64, h->gm, k, h->Q64, h->E64, h->d64, h->C64, 0, nullptr, -1.0, h->cpart, h->st, 0, s);
  launch_masked_axpy(mk, k, h->d_mask, 1.0, h->d64, h->w64, s);
  h->launches += 5;
  GS_CUDA_TRY(cudaGetLastError());
  return GLM_SUR_OK;
}

// b = R^-1 Q^T (y - Sigma w64)   (Algorithm glmpcg2 step 10, Sec. 4.3);
// restricted: b = N^-1 ([R_i^T Q_i^T (y - Sigma w)_i] + C^T d)  (eq. rglm1m)
// c_fresh: C64 already holds Q^T (y - Sigma w64) for the current w64 (the
// last float64 residual of the refinement, with no correction taken back
// since), so only the triangular solve remains.
glm_sur_status recover_b(glm_sur_ctx* h, int k, const IterPlan& p64, double* b, int64_t ldb, cudaStream_t s,
                         const double* d = nullptr, int64_t ldd = 0, bool c_fresh = false) {
  double* Cpart = reinterpret_cast<double*>(h->Cpart);
  if (!c_fresh || h->kc > 0) {
    launch_sigma_resid<double>(p64, h->gm, k, h->Om64, h->y64, h->w64, h->E64, s);
    launch_proj_partial<double>(p64, h->gm, k, h->Q64, h->E64, Cpart, h->st, 0, s);
    launch_reduce<double>(p64, h->gm, k, Cpart, h->C64, h->st, 0, nullptr, s);
    h->launches += 3;
  }
  if (h->kc > 0) {
    GS_CUDA_TRY(rglm_coef(h->gm, k, h->C64, h->R, h->Minv, h->Cmat, h->kc, h->kc, d, ldd, 1.0, h->cbuf, h->fbuf, b,
                          ldb, s));
    h->launches += 1;
    return GLM_SUR_OK;
  }
  // (a row-scaled model has R_i / sqrt(delta_i): b_i = sqrt(delta_i) R_i^-1 Q_i^T (y' - Sigma' w')_i)
  launch_tri_solve(h->gm, k, h->R, h->C64, b, ldb, s, h->opts.precond ? h->d_sqrtd : nullptr);
  h->launches += 1;
  GS_CUDA_TRY(cudaGetLastError());
  return GLM_SUR_OK;
}

// Remark rem:reduction.  Q (M x n) orthonormal with range(Q) = range(W), by
// Cholesky QR twice; R_W = L2^T L1^T (n x n, upper), so X_i = Q R_W[:, block i]
// and the reduced model has X_i' = R_W[:, block i] and y_i' = Q^T y_i (M' = n).
// GLM_SUR_RANK_DEFICIENT (nothing kept) when W^T W is not positive definite.
glm_sur_status setup_reduced(glm_sur_t* out, int G, int64_t M, const int* n_i, int n, const double* X, int64_t ldx,
                             const double* Omega, glm_sur_opts o, cudaStream_t s) {
  double *G1 = nullptr, *Li1 = nullptr, *G2 = nullptr, *Li2 = nullptr, *Q1 = nullptr, *Q = nullptr, *Rw = nullptr;
  int* flag = nullptr;
  auto release = [&]() {
    dfree(G1); dfree(Li1); dfree(G2); dfree(Li2); dfree(Q1); dfree(Rw); dfree(flag);
  };
  const size_t nn = (size_t)n * n, Mn = (size_t)M * n;
  cudaError_t e = cudaSuccess;
  if ((e = dalloc(&G1, nn)) != cudaSuccess || (e = dalloc(&Li1, nn)) != cudaSuccess ||
      (e = dalloc(&G2, nn)) != cudaSuccess || (e = dalloc(&Li2, nn)) != cudaSuccess ||
      (e = dalloc(&Q1, Mn)) != cudaSuccess || (e = dalloc(&Q, Mn)) != cudaSuccess ||
      (e = dalloc(&Rw, nn)) != cudaSuccess || (e = dalloc(&flag, 1)) != cudaSuccess) {
    release();
    dfree(Q);
    set_last_error(e, "cudaMalloc (row reduction)", __FILE__, __LINE__);
    return e == cudaErrorMemoryAllocation ? GLM_SUR_OOM : GLM_SUR_CUDA_ERROR;
  }
  cudaMemsetAsync(flag, 0, sizeof(int), s);
  // W^T W = L1 L1^T ;  Q1 = W L1^-T
  // a pivot below 64 n eps of the largest diagonal entry: W is treated as rank deficient
  const double piv_tol = 64.0 * n * 2.220446049250313e-16;
  launch_dgemm(n, n, M, X, ldx, 1, X, 1, ldx, G1, n, 1, s);
  cholesky_lower(n, G1, flag, piv_tol, s);
  launch_zero_upper(n, G1, s);
  launch_tri_inverse(n, G1, Li1, s);
  launch_dgemm((int)M, n, n, X, 1, ldx, Li1, 1, n, Q1, 1, M, s);
  // Q1^T Q1 = L2 L2^T ;  Q = Q1 L2^-T
  launch_dgemm(n, n, M, Q1, M, 1, Q1, 1, M, G2, n, 1, s);
  cholesky_lower(n, G2, flag, piv_tol, s);
  launch_zero_upper(n, G2, s);
  launch_tri_inverse(n, G2, Li2, s);
  launch_dgemm((int)M, n, n, Q1, 1, M, Li2, 1, n, Q, 1, M, s);
  // R_W = L2^T L1^T (column-major n x n: the reduced regressors)
  launch_dgemm(n, n, n, G2, 1, n, G1, 1, n, Rw, 1, n, s);
  int hflag = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess || hflag) {
    release();
    dfree(Q);
    if (e != cudaSuccess) {
      set_last_error(e, "row reduction", __FILE__, __LINE__);
      return GLM_SUR_CUDA_ERROR;
    }
    return GLM_SUR_RANK_DEFICIENT;
  }
  glm_sur_opts so = o;
  so.reduce_rows = 0;
  glm_sur_t sub = nullptr;
  glm_sur_status rc = glm_sur_setup(&sub, G, n, n_i, Rw, n, Omega, &so, reinterpret_cast<glm_sur_stream_t>(s));
  cudaStreamSynchronize(s);
  release();
  if (rc != GLM_SUR_OK) {
    dfree(Q);
    return rc;
  }
  glm_sur_ctx* h = new glm_sur_ctx();
  h->opts = o;
  h->sub = sub;
  h->Qw = Q;
  h->gm.G = G;
  h->gm.Gq = round_up4(G);
  h->gm.M = M;
  h->gm.Ms = M;
  h->gm.n = n;
  h->n_i.assign(n_i, n_i + G);
  h->dev = sub->dev;
  h->sms = sub->sms;
  h->launches = 11;
  *out = h;
  return GLM_SUR_OK;
}

// Reduced responses of every right-hand side: yred[(j G + i) n + r] = (Q^T y_ij)[r]
glm_sur_status rotate_in(glm_sur_ctx* h, const double* Y, int64_t ldy, int k, cudaStream_t s) {
  const int64_t M = h->gm.M, n = h->gm.n, G = h->gm.G;
  const int64_t need = G * n * k;
  if (need > h->yred_cap) {
    dfree(h->yred);
    h->yred_cap = 0;
    GS_CUDA_TRY(dalloc(&h->yred, (size_t)need));
    h->yred_cap = need;
  }
  // depth-split products when the n x G k output has too few tiles for the SMs
  const bool one = ldy == M * G;
  const int ncols = (int)(one ? G * k : G);
  const int nz = dgemm_split((int)n, ncols, M, h->sms);
  if (nz > 1 && (int64_t)nz * n * ncols > h->rot_ws_cap) {
    dfree(h->rot_ws);
    h->rot_ws_cap = 0;
    GS_CUDA_TRY(dalloc(&h->rot_ws, (size_t)nz * n * ncols));
    h->rot_ws_cap = (int64_t)nz * n * ncols;
  }
  double* ws = nz > 1 ? h->rot_ws : nullptr;
  const int per = nz > 1 ? 2 : 1;
  if (one) {
    launch_dgemm((int)n, ncols, M, h->Qw, M, 1, Y, 1, M, h->yred, 1, n, s, ws, nz);
    h->launches += per;
  } else {
    for (int j = 0; j < k; ++j)
      launch_dgemm((int)n, ncols, M, h->Qw, M, 1, Y + (int64_t)j * ldy, 1, M, h->yred + j * G * n, 1, n, s, ws, nz);
    h->launches += per * k;
  }
  GS_CUDA_TRY(cudaGetLastError());
  return GLM_SUR_OK;
}

// Omega of the iteration from the given one: for the preconditioner block
// D = D0 (x) I_M (D0 = alpha I or diag(Omega), eq. invprec with the choices of
// the VAR experiments), PCG-Aug on (y, X, Sigma) with D runs the iterates of
// PCG-Aug with D = I on the row-scaled model (S y, S X, S Sigma S), S =
// D0^-1/2 (x) I_M: the augmented matrices are congruent by diag(S, I), so KG
// is similar and w' = S^-1 w, while the GLS estimator is unchanged.  Here
// Omega' = D0^-1/2 Omega D0^-1/2; the solve scales y and b.
glm_sur_status derive_omega(glm_sur_ctx* h, cudaStream_t s) {
  const Geom& gm = h->gm;
  if (h->opts.precond == GLM_SUR_PRECOND_IDENTITY) {
    GS_CUDA_TRY(cudaMemcpyAsync(h->Om64, h->Omraw, sizeof(double) * (size_t)gm.G * gm.Gq, cudaMemcpyDeviceToDevice,
                                s));
  } else {
    launch_precond_omega(gm.G, gm.Gq, h->opts.precond, h->Omraw, h->Om64, h->d_sqrtd, h->d_isqrtd, s);
  }
  launch_convert<double, float>((int64_t)gm.G * gm.Gq, h->Om64, h->Om32, 1.0, s);
  // float32 copy used only by the inner solves of FP32_REFINE: Omega + s I
  launch_shift_diag(gm.G, gm.Gq, h->Om64, h->Om32, h->opts.inner_shift, s);
  GS_CUDA_TRY(cudaGetLastError());
  return GLM_SUR_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void glm_sur_default_opts(glm_sur_opts* o) {
  if (!o) return;
  o->precision = GLM_SUR_PREC_FP64;
  o->tol = 1e-13;
  o->maxit = 0;
  o->stagnation_window = 25;
  o->inner_tol = 1e-5;
  o->max_refine = 8;
  o->chunk = 16;
  o->inner_shift = 0.0;
  o->reduce_rows = 0;
  o->step_kernels = GLM_SUR_STEP_AUTO;
  o->precond = GLM_SUR_PRECOND_IDENTITY;
  o->algorithm = GLM_SUR_ALG_GLMPCG2;
}

const char* glm_sur_status_string(glm_sur_status s) {
  switch (s) {
    case GLM_SUR_OK: return "ok";
    case GLM_SUR_INVALID_ARG: return "invalid argument";
    case GLM_SUR_RANK_DEFICIENT: return "rank deficient regressor block";
    case GLM_SUR_BREAKDOWN: return "PCG breakdown (d <= 0 or not finite)";
    case GLM_SUR_STAGNATED: return "PCG stagnated";
    case GLM_SUR_NOT_CONVERGED: return "maximum iterations reached";
    case GLM_SUR_TIMEOUT: return "device wait timed out";
    case GLM_SUR_NONFINITE: return "non-finite input";
    case GLM_SUR_OOM: return "out of device memory";
    case GLM_SUR_CUDA_ERROR: return g_last_error.empty() ? "CUDA error" : g_last_error.c_str();
  }
  return "unknown status";
}

const char* glm_sur_version(void) { return "glm_sur 0.1 (sm_103a, PCG-Aug SUR)"; }

glm_sur_status glm_sur_setup(glm_sur_t* out, int G, int64_t M, const int* n_i, const double* X, int64_t ldx,
                             const double* Omega, const glm_sur_opts* opts, glm_sur_stream_t stream) {
  if (!out || !n_i || !X || !Omega) return GLM_SUR_INVALID_ARG;
  *out = nullptr;
  if (G < 1 || G > kMaxG || M < 1 || ldx < M) return GLM_SUR_INVALID_ARG;
  int nmax = 0;
  for (int i = 0; i < G; ++i) {
    if (n_i[i] < 1 || n_i[i] > kMaxBlockCols) return GLM_SUR_INVALID_ARG;
    nmax = std::max(nmax, n_i[i]);
  }
  if (M < nmax) return GLM_SUR_INVALID_ARG;
  glm_sur_opts o;
  glm_sur_default_opts(&o);
  if (opts) o = *opts;
  if (validate_opts(&o) != GLM_SUR_OK) return GLM_SUR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (o.reduce_rows) {
    int64_t n = 0;
    for (int i = 0; i < G; ++i) n += n_i[i];
    // the basis costs a one-CTA Cholesky of n x n (n^3 / 3 flops): kept to n <= 2048
    if (M >= 2 * n && n <= kMaxReducedCols) {
      glm_sur_status rr = setup_reduced(out, G, M, n_i, (int)n, X, ldx, Omega, o, s);
      if (rr != GLM_SUR_RANK_DEFICIENT) return rr;
      // W without full column rank: the unreduced model below
    }
    o.reduce_rows = 0;
  }

  glm_sur_ctx* h = new glm_sur_ctx();
  h->opts = o;
  cudaGetDevice(&h->dev);
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->dev);
  Geom& gm = h->gm;
  gm.G = G;
  gm.Gq = round_up4(G);
  gm.M = M;
  gm.Ms = M;
  h->n_i.assign(n_i, n_i + G);
  h->off.assign(G + 1, 0);
  h->poff.assign(G + 1, 0);
  std::vector<int> quad_blk;
  std::vector<int64_t> r_off(G + 1, 0);
  for (int i = 0; i < G; ++i) {
    h->off[i + 1] = h->off[i] + n_i[i];
    h->poff[i + 1] = h->poff[i] + round_up4(n_i[i]);
    for (int q = 0; q < round_up4(n_i[i]) / 4; ++q) quad_blk.push_back(i);
    r_off[i + 1] = r_off[i] + (int64_t)n_i[i] * n_i[i];
  }
  gm.n = h->off[G];
  gm.np = h->poff[G];
  gm.nq = gm.np / 4;
  // block groups of the projection update (runs of whole blocks, <= kMaxGroupQuads quads)
  std::vector<int> ug_blk0(1, 0);
  {
    int cur = 0;
    for (int i = 0; i < G; ++i) {
      const int qi = round_up4(n_i[i]) / 4;
      if (cur > 0 && cur + qi > kMaxGroupQuads) {
        ug_blk0.push_back(i);
        gm.ug_max_quads = std::max(gm.ug_max_quads, cur);
        cur = 0;
      }
      cur += qi;
    }
    gm.ug_max_quads = std::max(gm.ug_max_quads, cur);
    ug_blk0.push_back(G);
    gm.n_ugroups = (int)ug_blk0.size() - 1;
  }
  glm_sur_status rc = GLM_SUR_OK;
  auto bail = [&](glm_sur_status r) {
    glm_sur_destroy(h);
    return r;
  };
#define SETUP_TRY(expr)                                            \
  do {                                                             \
    cudaError_t e_ = (expr);                                       \
    if (e_ != cudaSuccess) {                                       \
      set_last_error(e_, #expr, __FILE__, __LINE__);               \
      return bail(e_ == cudaErrorMemoryAllocation ? GLM_SUR_OOM : GLM_SUR_CUDA_ERROR); \
    }                                                              \
  } while (0)
  SETUP_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  SETUP_TRY(cudaEventCreateWithFlags(&h->ev[0], cudaEventDisableTiming));
  SETUP_TRY(cudaEventCreateWithFlags(&h->ev[1], cudaEventDisableTiming));
  SETUP_TRY(cudaMallocHost(&h->h_done, 4 * sizeof(int)));
  SETUP_TRY(cudaMallocHost(&h->h_norms, 2 * kMaxRhs * sizeof(double)));
  SETUP_TRY(dalloc(&gm.d_n_i, G));
  SETUP_TRY(dalloc(&gm.d_off, G + 1));
  SETUP_TRY(dalloc(&gm.d_poff, G + 1));
  SETUP_TRY(dalloc(&gm.d_quad_blk, gm.nq));
  SETUP_TRY(dalloc(&gm.d_r_off, G + 1));
  SETUP_TRY(dalloc(&gm.d_ug_blk0, gm.n_ugroups + 1));
  {
    std::vector<int> col_blk(gm.n);
    for (int i = 0; i < G; ++i)
      for (int c = h->off[i]; c < h->off[i + 1]; ++c) col_blk[c] = i;
    SETUP_TRY(dalloc(&gm.d_col_blk, gm.n));
    SETUP_TRY(cudaMemcpy(gm.d_col_blk, col_blk.data(), gm.n * sizeof(int), cudaMemcpyHostToDevice));
  }
  SETUP_TRY(cudaMemcpyAsync(gm.d_ug_blk0, ug_blk0.data(), (gm.n_ugroups + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  SETUP_TRY(cudaMemcpyAsync(gm.d_n_i, n_i, G * sizeof(int), cudaMemcpyHostToDevice, s));
  SETUP_TRY(cudaMemcpyAsync(gm.d_off, h->off.data(), (G + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  SETUP_TRY(cudaMemcpyAsync(gm.d_poff, h->poff.data(), (G + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  SETUP_TRY(cudaMemcpyAsync(gm.d_quad_blk, quad_blk.data(), gm.nq * sizeof(int), cudaMemcpyHostToDevice, s));
  SETUP_TRY(cudaMemcpyAsync(gm.d_r_off, r_off.data(), (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  SETUP_TRY(dalloc(&h->Q64, (size_t)M * gm.np));
  SETUP_TRY(dalloc(&h->R, (size_t)r_off[G]));
  SETUP_TRY(dalloc(&h->Om64, (size_t)G * gm.Gq));
  SETUP_TRY(dalloc(&h->Om32, (size_t)G * gm.Gq));
  SETUP_TRY(dalloc(&h->Omraw, (size_t)G * gm.Gq));
  SETUP_TRY(dalloc(&h->d_sqrtd, (size_t)G));
  SETUP_TRY(dalloc(&h->d_isqrtd, (size_t)G));
  SETUP_TRY(dalloc(&h->setup_flags, 1));
  SETUP_TRY(cudaMemsetAsync(h->Q64, 0, sizeof(double) * (size_t)M * gm.np, s));
  SETUP_TRY(cudaMemsetAsync(h->setup_flags, 0, sizeof(int), s));
  // TSQR of every block
  QrPlan plan;
  std::vector<QrBlock> qb(G);
  for (int i = 0; i < G; ++i)
    qb[i] = QrBlock{n_i[i], M, (int64_t)h->off[i] * ldx, ldx, (int64_t)h->poff[i], (int64_t)gm.np};
  build_qr_plan(qb, plan);
  rc = run_qr(plan, X, gm.d_r_off, h->Q64, h->R, h->setup_flags, s);
  if (rc != GLM_SUR_OK) return bail(rc);
  if (o.precision == GLM_SUR_PREC_FP32_REFINE) {
    SETUP_TRY(dalloc(&h->Q32, (size_t)M * gm.np));
    launch_convert<double, float>((int64_t)M * gm.np, h->Q64, h->Q32, 1.0, s);
    SETUP_TRY(cudaGetLastError());
  }
  *out = h;
  rc = glm_sur_set_omega(h, Omega, stream);
  if (rc != GLM_SUR_OK) {
    *out = nullptr;
    return bail(rc);
  }
#undef SETUP_TRY
  return GLM_SUR_OK;
}

glm_sur_status glm_sur_mvrglm_setup(glm_sur_t* out, int G, int64_t M, int N, const double* Z0, int64_t ldz,
                                    const double* Omega0, const int* k_i, const double* C, int64_t ldc,
                                    const glm_sur_opts* opts, glm_sur_stream_t stream) {
  if (!out || !Z0 || !Omega0 || !k_i) return GLM_SUR_INVALID_ARG;
  *out = nullptr;
  if (G < 1 || G > kMaxG || N < 1 || N > kMaxBlockCols || M < N || ldz < M) return GLM_SUR_INVALID_ARG;
  int kmax = 0, ktot = 0;
  std::vector<int> koff(G + 1, 0);
  for (int i = 0; i < G; ++i) {
    if (k_i[i] < 0 || k_i[i] > N) return GLM_SUR_INVALID_ARG;   // at most N independent restrictions
    kmax = std::max(kmax, k_i[i]);
    ktot += k_i[i];
    koff[i + 1] = ktot;
  }
  if (ktot > 0 && (!C || ldc < ktot)) return GLM_SUR_INVALID_ARG;
  glm_sur_opts o;
  glm_sur_default_opts(&o);
  if (opts) o = *opts;
  if (validate_opts(&o) != GLM_SUR_OK) return GLM_SUR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int Mp = N + kmax;
  double *Q0 = nullptr, *R0 = nullptr, *Xt = nullptr;
  int64_t* roff = nullptr;
  int *flags = nullptr, *dkoff = nullptr;
  auto release = [&]() {
    dfree(R0); dfree(Xt); dfree(roff); dfree(flags);
  };
  auto fail = [&](cudaError_t e, const char* what) {
    set_last_error(e, what, __FILE__, __LINE__);
    release();
    dfree(Q0);
    dfree(dkoff);
    return e == cudaErrorMemoryAllocation ? GLM_SUR_OOM : GLM_SUR_CUDA_ERROR;
  };
#define MV_TRY(expr)                       \
  do {                                     \
    cudaError_t e_ = (expr);               \
    if (e_ != cudaSuccess) return fail(e_, #expr); \
  } while (0)
  MV_TRY(dalloc(&Q0, (size_t)M * N));
  MV_TRY(dalloc(&R0, (size_t)N * N));
  MV_TRY(dalloc(&Xt, (size_t)Mp * G * N));
  MV_TRY(dalloc(&roff, 2));
  MV_TRY(dalloc(&flags, 1));
  MV_TRY(dalloc(&dkoff, G + 1));
  const int64_t roff_h[2] = {0, (int64_t)N * N};
  MV_TRY(cudaMemcpyAsync(roff, roff_h, sizeof(roff_h), cudaMemcpyHostToDevice, s));
  MV_TRY(cudaMemcpyAsync(dkoff, koff.data(), (G + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  MV_TRY(cudaMemsetAsync(flags, 0, sizeof(int), s));
  MV_TRY(cudaMemsetAsync(Q0, 0, sizeof(double) * (size_t)M * N, s));
  // model reduction: Householder TSQR of Z0 (Q0 row-major M x N, R0 row-major)
  {
    QrPlan plan;
    std::vector<QrBlock> qb(1, QrBlock{N, M, 0, ldz, 0, (int64_t)N});
    build_qr_plan(qb, plan);
    glm_sur_status rc = run_qr(plan, Z0, roff, Q0, R0, flags, s);
    if (rc != GLM_SUR_OK) {
      release();
      dfree(Q0);
      dfree(dkoff);
      return rc;
    }
  }
  int hflag = 0;
  MV_TRY(cudaMemcpyAsync(&hflag, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  MV_TRY(cudaStreamSynchronize(s));
  if (hflag) {
    release();
    dfree(Q0);
    dfree(dkoff);
    return (hflag & 2) ? GLM_SUR_NONFINITE : GLM_SUR_RANK_DEFICIENT;   // Z0 not finite / not of full column rank
  }
  // the G blocks [R0; C_i; 0] and their setup (the updating QRDs)
  launch_mv_build_x(G, N, Mp, R0, C, ldc, dkoff, Xt, s);
  MV_TRY(cudaGetLastError());
  std::vector<int> n_i(G, N);
  glm_sur_opts so = o;
  so.reduce_rows = 0;
  glm_sur_t sub = nullptr;
  glm_sur_status rc = glm_sur_setup(&sub, G, Mp, n_i.data(), Xt, Mp, Omega0, &so, stream);
  MV_TRY(cudaStreamSynchronize(s));
  release();
  if (rc != GLM_SUR_OK) {
    dfree(Q0);
    dfree(dkoff);
    return rc;
  }
  sub->gm.Ms = N;                    // Sigma = 0 on the restriction rows
  glm_sur_ctx* h = new glm_sur_ctx();
  h->opts = o;
  h->sub = sub;
  h->mv_N = N;
  h->mv_kmax = kmax;
  h->mv_ktot = ktot;
  h->mv_koff = dkoff;
  h->mv_Q0 = Q0;
  h->gm.G = G;
  h->gm.Gq = round_up4(G);
  h->gm.M = M;
  h->gm.Ms = M;
  h->gm.n = G * N;
  h->n_i.assign(G, N);
  h->launches = 3;
  *out = h;
#undef MV_TRY
  return GLM_SUR_OK;
}

glm_sur_status glm_sur_get_setup_status(glm_sur_t h) {
  if (h && h->sub) return glm_sur_get_setup_status(h->sub);
  if (!h) return GLM_SUR_INVALID_ARG;
  int flags = 0;
  GS_CUDA_TRY(cudaMemcpy(&flags, h->setup_flags, sizeof(int), cudaMemcpyDeviceToHost));
  if (flags & 2) return GLM_SUR_NONFINITE;
  if (flags & 1) return GLM_SUR_RANK_DEFICIENT;
  return GLM_SUR_OK;
}

glm_sur_status glm_sur_set_omega(glm_sur_t h, const double* Omega, glm_sur_stream_t stream) {
  if (h && h->sub) return glm_sur_set_omega(h->sub, Omega, stream);
  if (!h || !Omega) return GLM_SUR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const Geom& gm = h->gm;
  GS_CUDA_TRY(cudaMemsetAsync(h->Omraw, 0, sizeof(double) * (size_t)gm.G * gm.Gq, s));
  GS_CUDA_TRY(cudaMemcpy2DAsync(h->Omraw, gm.Gq * sizeof(double), Omega, gm.G * sizeof(double),
                                gm.G * sizeof(double), gm.G, cudaMemcpyDeviceToDevice, s));
  glm_sur_status rc = derive_omega(h, s);
  if (rc != GLM_SUR_OK) return rc;
  h->has_w = false;
  return GLM_SUR_OK;
}

glm_sur_status glm_sur_set_opts(glm_sur_t h, const glm_sur_opts* opts) {
  if (h && h->sub && opts) {
    glm_sur_opts so = *opts;
    so.reduce_rows = 0;
    glm_sur_status rc = glm_sur_set_opts(h->sub, &so);
    if (rc == GLM_SUR_OK) h->opts = *opts;
    return rc;
  }
  if (!h || !opts) return GLM_SUR_INVALID_ARG;
  if (validate_opts(opts) != GLM_SUR_OK) return GLM_SUR_INVALID_ARG;
  const bool need_q32 = opts->precision == GLM_SUR_PREC_FP32_REFINE && !h->Q32;
  const bool prec_change = opts->precision != h->opts.precision || opts->stagnation_window != h->opts.stagnation_window;
  h->opts = *opts;
  if (need_q32) {
    GS_CUDA_TRY(dalloc(&h->Q32, (size_t)h->gm.M * h->gm.np));
    launch_convert<double, float>((int64_t)h->gm.M * h->gm.np, h->Q64, h->Q32, 1.0, nullptr);
    GS_CUDA_TRY(cudaDeviceSynchronize());
  }
  if (prec_change) free_workspace(h);
  glm_sur_status rc = derive_omega(h, nullptr);
  if (rc != GLM_SUR_OK) return rc;
  GS_CUDA_TRY(cudaDeviceSynchronize());
  h->plan_k = -1;
  return GLM_SUR_OK;
}

}  // extern "C"

namespace {

glm_sur_status ensure_restriction_workspace(glm_sur_ctx* h, int k) {
  if (h->kc == 0 || k <= h->rcap) return GLM_SUR_OK;
  dfree(h->cbuf); dfree(h->fbuf); dfree(h->gC);
  h->rcap = 0;
  GS_CUDA_TRY(dalloc(&h->cbuf, (size_t)h->gm.n * k));
  GS_CUDA_TRY(dalloc(&h->fbuf, (size_t)h->gm.np * k));
  GS_CUDA_TRY(dalloc(&h->gC, (size_t)h->kc * k));
  h->rcap = k;
  return GLM_SUR_OK;
}

// Workspace and iteration plans for k right-hand sides; p64 receives the
// float64 plan of the residual and recovery passes.
glm_sur_status prepare_solve(glm_sur_t h, int k, IterPlan& p64) {
  glm_sur_status rc = ensure_workspace(h, k);
  if (rc != GLM_SUR_OK) return rc;
  rc = ensure_restriction_workspace(h, k);
  if (rc != GLM_SUR_OK) return rc;
  rc = make_plan(h, k, true, p64);
  if (rc != GLM_SUR_OK) return rc;
  if (h->plan_k != k || h->plan_prec != h->opts.precision) {
    IterPlan pit;
    rc = make_plan(h, k, fp64_steps(h->opts), pit);
    if (rc != GLM_SUR_OK) return rc;
    h->plan = pit;
    h->plan_k = k;
    h->plan_prec = h->opts.precision;
    h->graph.reset();
  }
  return GLM_SUR_OK;
}

// PCG-Aug (float64, or float32 inside float64 refinement) on the right-hand
// sides already in y64; b = R^-1 Q^T (y - Sigma w) unless b is null.
glm_sur_status solve_core(glm_sur_t h, const IterPlan& p64, const double* d, int64_t ldd, int k, double* b,
                          int64_t ldb, int* iters, double* relres, cudaStream_t s) {
  glm_sur_status rc = GLM_SUR_OK;
  const Geom& gm = h->gm;
  const int64_t m = gm.M * gm.G;
  const bool fp64 = fp64_steps(h->opts);
  const int64_t mk = m * k;
  const int maxit = h->opts.maxit > 0 ? h->opts.maxit : (int)std::min<int64_t>(m - gm.n + 1, 1 << 30);
  GS_CUDA_TRY(cudaMemsetAsync(h->st.err, 0, sizeof(int), s));
  h->last_k = k;
  bool c_fresh = false;
  if (fp64) {
    rc = reset_state(h, k, h->opts.tol, maxit, h->opts.stagnation_window, s);
    if (rc != GLM_SUR_OK) return rc;
    h->st.c1_extra = h->c1x_on ? h->c1x : nullptr;
    rc = pcg_init<double>(h, k, h->y64, s, d, ldd);
    if (rc != GLM_SUR_OK) return rc;
    GS_CUDA_TRY(cudaGetLastError());
    rc = run_steps<double>(h, k, maxit, s);
    if (rc != GLM_SUR_OK) return rc;
    GS_CUDA_TRY(cudaMemcpyAsync(h->d_status_final, h->st.status, k * sizeof(int), cudaMemcpyDeviceToDevice, s));
    GS_CUDA_TRY(cudaMemcpyAsync(h->d_iters_acc, h->st.iters, k * sizeof(int), cudaMemcpyDeviceToDevice, s));
    if (relres) GS_CUDA_TRY(cudaMemcpyAsync(relres, h->st.relres, k * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    // float64 iterative refinement on P Sigma w = P y (w in null(X^T)) with
    // float32 inner PCG.  A correction that increases a column's float64
    // residual is taken back and the column stops (its best w is kept); one
    // that does not at least halve it is kept and the column stops too: the
    // residual has reached its float64 rounding floor.
    GS_CUDA_TRY(cudaMemsetAsync(h->w64, 0, mk * sizeof(double), s));
    GS_CUDA_TRY(cudaMemsetAsync(h->d_iters_acc, 0, k * sizeof(int), s));
    std::vector<double> rho0(k, 0.0), prev(k, 0.0), cur(k, 0.0), rr_out(k, 0.0), extra(k, 0.0);
    std::vector<int> fin(k, kStatusRunning), mask(2 * k, 0);
    if (h->c1x_on)   // (read after the first synchronisation below)
      GS_CUDA_TRY(cudaMemcpyAsync(extra.data(), h->c1x, k * sizeof(double), cudaMemcpyDeviceToHost, s));
    for (int outer = 0;; ++outer) {
      c_fresh = false;
      rc = true_residual(h, k, p64, s);
      if (rc != GLM_SUR_OK) return rc;
      launch_sum_partials_sqrt(p64.n_cpart, k, h->cpart, h->norms, s);
      h->launches += 1;
      GS_CUDA_TRY(cudaMemcpyAsync(h->h_norms, h->norms, k * sizeof(double), cudaMemcpyDeviceToHost, s));
      GS_CUDA_TRY(cudaStreamSynchronize(s));
      bool all_done = true, any_revert = false;
      for (int j = 0; j < k; ++j) {
        cur[j] = h->h_norms[j];
        if (outer == 0) rho0[j] = std::sqrt(cur[j] * cur[j] + extra[j]);
        mask[k + j] = 0;
        if (fin[j] == kStatusRunning) {
          const double rr = rho0[j] > 0 ? cur[j] / rho0[j] : 0.0;
          if (!std::isfinite(cur[j])) {
            fin[j] = GLM_SUR_NONFINITE;
          } else if (outer > 0 && cur[j] >= prev[j]) {
            mask[k + j] = 1;            // take the last correction back
            any_revert = true;
            fin[j] = (rr_out[j] <= h->opts.tol) ? GLM_SUR_OK : GLM_SUR_STAGNATED;
          } else {
            rr_out[j] = rr;
            const bool floor = outer > 0 && cur[j] > kRefineMinGain * prev[j];
            prev[j] = cur[j];
            if (rr <= h->opts.tol) fin[j] = GLM_SUR_OK;
            else if (floor) fin[j] = GLM_SUR_STAGNATED;
            else if (outer >= h->opts.max_refine) fin[j] = GLM_SUR_NOT_CONVERGED;
          }
        }
        mask[j] = fin[j] == kStatusRunning;
        if (mask[j]) all_done = false;
      }
      GS_CUDA_TRY(cudaMemcpyAsync(h->d_mask, mask.data(), 2 * k * sizeof(int), cudaMemcpyHostToDevice, s));
      if (any_revert) {
        launch_masked_axpy(mk, k, h->d_mask + k, -1.0, h->d64, h->w64, s);
        h->launches += 1;
      }
      // (the host vector `mask` must outlive the copy above)
      GS_CUDA_TRY(cudaStreamSynchronize(s));
      if (all_done) {
        c_fresh = !any_revert && d == nullptr;   // C64 = Q^T (y - Sigma w64) of the final w64
        break;
      }
      // inner float32 PCG on P Sigma_e d = rho (live columns)
      rc = reset_state(h, k, h->opts.inner_tol, maxit, std::max(kInnerStagnation, h->opts.stagnation_window), s);
      if (rc != GLM_SUR_OK) return rc;
      launch_init_inner<float>(h->plan, gm, k, h->g64, h->d_mask, h->g32, h->u32, h->w32, h->cpart, s);
      GS_CUDA_TRY(cudaMemsetAsync(h->wb32, 0, mk * sizeof(float), s));
      h->launches += 1;
      GS_CUDA_TRY(cudaGetLastError());
      rc = run_steps<float>(h, k, maxit, s);
      if (rc != GLM_SUR_OK) return rc;
      // d = P (double) w32; w64 += d on the live columns.  The float32
      // iterates leave null(X^T) by rounding while the solution w of
      // eq. (aug1) lies in it (X^T w = 0), so the correction is projected
      // in float64 before it is added.
      rc = project_correction(h, k, p64, s);
      if (rc != GLM_SUR_OK) return rc;
      launch_add_int(k, h->st.iters, h->d_iters_acc, s);
      h->launches += 1;
      GS_CUDA_TRY(cudaGetLastError());
    }
    for (int j = 0; j < k; ++j) {
      h->h_status[j] = fin[j];
      h->h_norms[kMaxRhs + j] = rr_out[j];
    }
    GS_CUDA_TRY(cudaMemcpyAsync(h->d_status_final, h->h_status, k * sizeof(int), cudaMemcpyHostToDevice, s));
    if (relres)
      GS_CUDA_TRY(cudaMemcpyAsync(relres, h->h_norms + kMaxRhs, k * sizeof(double), cudaMemcpyHostToDevice, s));
    GS_CUDA_TRY(cudaStreamSynchronize(s));
  }
  if (iters) GS_CUDA_TRY(cudaMemcpyAsync(iters, h->d_iters_acc, k * sizeof(int), cudaMemcpyDeviceToDevice, s));
  if (b) {
    rc = recover_b(h, k, p64, b, ldb, s, d, ldd, c_fresh);
    if (rc != GLM_SUR_OK) return rc;
  }
  return GLM_SUR_OK;
}

glm_sur_status solve_impl(glm_sur_t h, const double* Y, int64_t ldy, const double* d, int64_t ldd, int k, double* b,
                          int64_t ldb, int* iters, double* relres, cudaStream_t s);

// Algorithm glmpcg3 in float64 on the right-hand sides in y64 (D = I on the
// model of the handle: a preconditioner block acts through the row scaling).
// Per step: u = P s (two passes over Q), S = Sigma u with d = u^T S, w and r,
// g = P r with c' = g^T g (two passes over Q), s = r + mu s.
glm_sur_status pcg3_core(glm_sur_t h, const IterPlan& p64, int k, double* b, int64_t ldb, int* iters, double* relres,
                         cudaStream_t s) {
  const Geom& gm = h->gm;
  const int64_t m = gm.M * gm.G, mk = m * k;
  const int nblk = 2 * h->sms;
  if (k > h->p3cap) {
    dfree(h->p3_buf);
    dfree(h->p3_ibuf);
    if (h->p3_hact) cudaFreeHost(h->p3_hact);
    h->p3_hact = nullptr;
    h->p3cap = 0;
    GS_CUDA_TRY(dalloc(&h->p3_buf, (size_t)k * (5 + nblk)));
    GS_CUDA_TRY(dalloc(&h->p3_ibuf, (size_t)3 * k));
    GS_CUDA_TRY(cudaMallocHost(&h->p3_hact, kMaxRhs * sizeof(int)));
    h->p3cap = k;
  }
  Pcg3State st;
  st.k = k;
  st.tol = h->opts.tol;
  st.maxit = h->opts.maxit > 0 ? h->opts.maxit : (int)std::min<int64_t>(m - gm.n + 1, 1 << 30);
  st.c = h->p3_buf;
  st.c1 = st.c + k;
  st.lam = st.c1 + k;
  st.mu = st.lam + k;
  st.relres = st.mu + k;
  st.dpart = st.relres + k;
  st.nblk = nblk;
  st.c1_extra = h->c1x_on ? h->c1x : nullptr;
  st.active = h->p3_ibuf;
  st.iters = st.active + k;
  st.status = st.iters + k;
  double *sv = h->wb64, *r = h->E64, *u = h->u64, *Sm = h->S64, *gP = h->g64, *w = h->w64;
  double* Cpart = reinterpret_cast<double*>(h->Cpart);
  const int ncp = p64.n_cpart;
  GS_CUDA_TRY(cudaMemsetAsync(h->st.err, 0, sizeof(int), s));
  GS_CUDA_TRY(cudaMemsetAsync(w, 0, mk * sizeof(double), s));
  launch_pcg3_neg(mk, h->y64, r, s);                                   // r_1 = -y
  auto project = [&](const double* x, double* px) {                    // px = P x; cpart: partials of px^T px
    launch_proj_partial<double>(p64, gm, k, h->Q64, x, Cpart, h->st, 0, s);
    launch_reduce<double>(p64, gm, k, Cpart, h->C64, h->st, 0, nullptr, s);
    launch_proj_update<double>(p64, gm, k, h->Q64, x, px, h->C64, 0, nullptr, -1.0, h->cpart, h->st, 0, s);
  };
  project(r, gP);
  launch_pcg3_after(st, h->cpart, ncp, 1, s);                          // c_1 = r^T Pi r
  launch_pcg3_s(mk, k, st, r, sv, 1, s);                               // s_1 = r_1
  h->launches += 6;
  GS_CUDA_TRY(cudaGetLastError());
  const int chunk = std::max(1, h->opts.chunk);
  for (int it = 0; it < st.maxit;) {
    const int steps = std::min(chunk, st.maxit - it);
    for (int c = 0; c < steps; ++c) {
      project(sv, u);                                                  // u = Pi s
      launch_sigma_resid<double>(p64, gm, k, h->Om64, nullptr, u, Sm, s);   // Sm = -Sigma u
      launch_pcg3_dot(gm.M, gm.G, k, u, Sm, st, s);
      launch_pcg3_lambda(st, s);                                       // lambda = c / (u^T Sigma u)
      launch_pcg3_wr(mk, k, st, u, Sm, sv, w, r, s);                   // w, r
      project(r, gP);
      launch_pcg3_after(st, h->cpart, ncp, 0, s);                      // c' = r^T Pi r, stop tests, mu
      launch_pcg3_s(mk, k, st, r, sv, 0, s);                           // s = r + mu s
    }
    h->launches += 12 * steps;
    GS_CUDA_TRY(cudaGetLastError());
    it += steps;
    GS_CUDA_TRY(cudaMemcpyAsync(h->p3_hact, st.active, k * sizeof(int), cudaMemcpyDeviceToHost, s));
    GS_CUDA_TRY(cudaStreamSynchronize(s));
    bool any = false;
    for (int j = 0; j < k; ++j) any |= h->p3_hact[j] != 0;
    if (!any) break;
  }
  GS_CUDA_TRY(cudaMemcpyAsync(h->d_status_final, st.status, k * sizeof(int), cudaMemcpyDeviceToDevice, s));
  GS_CUDA_TRY(cudaMemcpyAsync(h->d_iters_acc, st.iters, k * sizeof(int), cudaMemcpyDeviceToDevice, s));
  if (iters) GS_CUDA_TRY(cudaMemcpyAsync(iters, st.iters, k * sizeof(int), cudaMemcpyDeviceToDevice, s));
  if (relres) GS_CUDA_TRY(cudaMemcpyAsync(relres, st.relres, k * sizeof(double), cudaMemcpyDeviceToDevice, s));
  h->last_k = k;
  return recover_b(h, k, p64, b, ldb, s);
}

// MVRGLM solve: Y0 = Q0^T Y (model reduction), y' = [Y0_i; gamma_i; 0] per
// equation, then the SUR iteration of the masked model; b = vec(B).
glm_sur_status mv_solve(glm_sur_t h, const double* Y, int64_t ldy, const double* gamma, int64_t ldd, int k,
                        double* b, int64_t ldb, int* iters, double* relres, cudaStream_t s) {
  const int G = h->gm.G, N = h->mv_N, Mp = N + h->mv_kmax;
  const int64_t M = h->gm.M;
  if (k < 1 || k > kMaxRhs || ldy < M * G || ldb < (int64_t)G * N) return GLM_SUR_INVALID_ARG;
  if (gamma && ldd < h->mv_ktot) return GLM_SUR_INVALID_ARG;
  const int64_t need0 = (int64_t)N * G * k, need1 = (int64_t)G * Mp * k;
  if (need0 > h->yred_cap) {
    dfree(h->yred);
    h->yred_cap = 0;
    GS_CUDA_TRY(dalloc(&h->yred, (size_t)need0));
    h->yred_cap = need0;
  }
  if (need1 > h->mv_ycap) {
    dfree(h->mv_y);
    h->mv_ycap = 0;
    GS_CUDA_TRY(dalloc(&h->mv_y, (size_t)need1));
    h->mv_ycap = need1;
  }
  // Y0(:, j G + i) = Q0^T y_ij  (Q0 row-major M x N)
  if (ldy == M * G) {
    launch_dgemm(N, G * k, M, h->mv_Q0, 1, N, Y, 1, M, h->yred, 1, N, s);
    h->launches += 1;
  } else {
    for (int j = 0; j < k; ++j)
      launch_dgemm(N, G, M, h->mv_Q0, 1, N, Y + (int64_t)j * ldy, 1, M, h->yred + (int64_t)j * G * N, 1, N, s);
    h->launches += k;
  }
  launch_mv_assemble(G, N, Mp, k, h->yred, gamma, ldd, h->mv_koff, h->mv_y, s);
  h->launches += 1;
  GS_CUDA_TRY(cudaGetLastError());
  return solve_impl(h->sub, h->mv_y, (int64_t)G * Mp, nullptr, 0, k, b, ldb, iters, relres, s);
}

glm_sur_status solve_impl(glm_sur_t h, const double* Y, int64_t ldy, const double* d, int64_t ldd, int k, double* b,
                          int64_t ldb, int* iters, double* relres, cudaStream_t s) {
  if (!h || !Y || !b) return GLM_SUR_INVALID_ARG;
  if (h->mv_N) return mv_solve(h, Y, ldy, d, ldd, k, b, ldb, iters, relres, s);
  if (h->sub) {
    // Remark rem:reduction: the same estimate from the n rotated rows
    if (k < 1 || k > kMaxRhs || ldy < h->gm.M * h->gm.G) return GLM_SUR_INVALID_ARG;
    glm_sur_status rc = rotate_in(h, Y, ldy, k, s);
    if (rc != GLM_SUR_OK) return rc;
    // tol and relres refer to the M-row model's ||P y||: its square is the
    // reduced model's plus the energy of y outside range(W), where the
    // model has no regressor and no restriction (scaled by D0^-1 under a
    // preconditioner block, as the iteration sees it)
    glm_sur_ctx* sb = h->sub;
    if (!sb->c1x) {
      GS_CUDA_TRY(dalloc(&sb->c1x, (size_t)kMaxRhs));
      GS_CUDA_TRY(dalloc(&sb->c1x_part, (size_t)h->gm.G * kMaxRhs));
    }
    launch_complement_energy(h->gm.G, h->gm.M, h->gm.n, k, Y, ldy, h->yred,
                             sb->opts.precond != GLM_SUR_PRECOND_IDENTITY ? sb->d_isqrtd : nullptr, sb->c1x_part,
                             sb->c1x, s);
    h->launches += 2;
    GS_CUDA_TRY(cudaGetLastError());
    sb->c1x_on = true;
    rc = solve_impl(sb, h->yred, (int64_t)h->gm.G * h->gm.n, d, ldd, k, b, ldb, iters, relres, s);
    sb->c1x_on = false;
    return rc;
  }
  const Geom& gm = h->gm;
  const int64_t m = gm.M * gm.G;
  if (k < 1 || k > kMaxRhs || ldy < m || ldb < gm.n) return GLM_SUR_INVALID_ARG;
  if (h->kc > 0 && (h->opts.precision != GLM_SUR_PREC_FP64 || (d && ldd < h->kc))) return GLM_SUR_INVALID_ARG;
  if (h->kc > 0 && h->opts.precond != GLM_SUR_PRECOND_IDENTITY) return GLM_SUR_INVALID_ARG;
  const bool pcg3 = h->opts.algorithm == GLM_SUR_ALG_GLMPCG3;
  if (pcg3 && (h->kc > 0 || h->opts.precision != GLM_SUR_PREC_FP64)) return GLM_SUR_INVALID_ARG;
  IterPlan p64;
  glm_sur_status rc = prepare_solve(h, k, p64);
  if (rc != GLM_SUR_OK) return rc;
  h->has_w = false;
  // preconditioner block D = D0 (x) I_M: the iteration runs on the row-scaled
  // model (y_i / sqrt(delta_i), X_i / sqrt(delta_i), D0^-1/2 Omega D0^-1/2)
  launch_colmajor_to_layout<double>(gm, k, Y, ldy, h->y64, 1.0, s, h->opts.precond ? h->d_isqrtd : nullptr);
  h->launches += 1;
  GS_CUDA_TRY(cudaGetLastError());
  rc = pcg3 ? pcg3_core(h, p64, k, b, ldb, iters, relres, s) : solve_core(h, p64, d, ldd, k, b, ldb, iters, relres, s);
  if (rc != GLM_SUR_OK) return rc;
  h->has_w = true;
  h->w_restricted = h->kc > 0;
  return GLM_SUR_OK;
}

// Buffers of the adjoint: the saved forward w, lam_1 and the Omega-gradient partials.
glm_sur_status ensure_adjoint_workspace(glm_sur_ctx* h, int k, int nch) {
  const size_t mk = (size_t)h->gm.M * h->gm.G * k;
  if (k > h->acap) {
    dfree(h->wfwd); dfree(h->lam1);
    h->acap = 0;
    GS_CUDA_TRY(dalloc(&h->wfwd, mk));
    GS_CUDA_TRY(dalloc(&h->lam1, mk));
    h->acap = k;
  }
  const int64_t need = (int64_t)nch * h->gm.G * h->gm.G;
  if (need > h->ocap) {
    dfree(h->opart);
    h->ocap = 0;
    GS_CUDA_TRY(dalloc(&h->opart, (size_t)need));
    h->ocap = need;
  }
  return GLM_SUR_OK;
}

glm_sur_status ensure_ne_workspace(glm_sur_ctx* h, int k) {
  const Geom& gm = h->gm;
  if (!h->ne_om) {
    GS_CUDA_TRY(dalloc(&h->ne_om, (size_t)gm.G * gm.Gq + 2 * (size_t)gm.G * gm.G));
    GS_CUDA_TRY(cudaMallocHost(&h->ne_hact, kMaxRhs * sizeof(int)));
  }
  if (k > h->necap) {
    dfree(h->ne_buf);
    dfree(h->ne_ibuf);
    h->necap = 0;
    GS_CUDA_TRY(dalloc(&h->ne_buf, (size_t)k * (4 * (size_t)gm.n + gm.np + 3)));
    GS_CUDA_TRY(dalloc(&h->ne_ibuf, (size_t)3 * k));
    h->necap = k;
  }
  return GLM_SUR_OK;
}

// PCG-NE (the comparator of Sec. "Statistical properties of the PCG-Aug
// estimator" and Sec. "Experimental Tests"): Algorithm pcg with K = I on
// (X^T Sigma^-1 X) beta = X^T Sigma^-1 y, beta_1 = 0, float64.  A beta =
// R^T Q^T Sigma^-1 Q R beta with Sigma^-1 = Omega^-1 (x) I_M; Omega^-1 =
// L^-T L^-1 from the Cholesky factor of the given Omega (the preconditioner
// block of the PCG-Aug solves plays no part).  Stops per column when
// ||f|| <= tol ||f_1|| or after maxit steps (opts.maxit, 0: 4 n).
glm_sur_status ne_solve(glm_sur_t h, const double* Y, int64_t ldy, int k, double* b, int64_t ldb, int* iters,
                        double* relres, cudaStream_t s) {
  if (!h || !Y || !b || h->mv_N) return GLM_SUR_INVALID_ARG;
  if (h->sub) {
    if (k < 1 || k > kMaxRhs || ldy < h->gm.M * h->gm.G) return GLM_SUR_INVALID_ARG;
    glm_sur_status rc = rotate_in(h, Y, ldy, k, s);
    if (rc != GLM_SUR_OK) return rc;
    return ne_solve(h->sub, h->yred, (int64_t)h->gm.G * h->gm.n, k, b, ldb, iters, relres, s);
  }
  const Geom& gm = h->gm;
  const int64_t m = gm.M * gm.G, mk = m * k;
  if (k < 1 || k > kMaxRhs || ldy < m || ldb < gm.n || h->kc > 0) return GLM_SUR_INVALID_ARG;
  IterPlan p64;
  glm_sur_status rc = prepare_solve(h, k, p64);
  if (rc != GLM_SUR_OK) return rc;
  rc = ensure_ne_workspace(h, k);
  if (rc != GLM_SUR_OK) return rc;
  h->has_w = false;
  h->last_k = k;
  const int G = gm.G;
  double* Oinv = h->ne_om;
  double* Lw = Oinv + (size_t)G * gm.Gq;
  double* Linv = Lw + (size_t)G * G;
  // Omega^-1 (positive definite Omega only: the normal equations need Sigma^-1)
  GS_CUDA_TRY(cudaMemcpy2DAsync(Lw, G * sizeof(double), h->Omraw, gm.Gq * sizeof(double), G * sizeof(double), G,
                                cudaMemcpyDeviceToDevice, s));
  GS_CUDA_TRY(cudaMemsetAsync(h->setup_flags, 0, sizeof(int), s));
  GS_CUDA_TRY(cholesky_lower(G, Lw, h->setup_flags, 1e-13, s));
  int flag = 0;
  GS_CUDA_TRY(cudaMemcpyAsync(&flag, h->setup_flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  GS_CUDA_TRY(cudaStreamSynchronize(s));
  if (flag) return GLM_SUR_INVALID_ARG;
  GS_CUDA_TRY(launch_tri_inverse(G, Lw, Linv, s));
  GS_CUDA_TRY(cudaMemsetAsync(Oinv, 0, sizeof(double) * (size_t)G * gm.Gq, s));
  launch_dgemm(G, G, G, Linv, 1, G, Linv, G, 1, Oinv, gm.Gq, 1, s);
  // state
  NeState st;
  st.k = k;
  st.tol = h->opts.tol;
  st.maxit = h->opts.maxit > 0 ? h->opts.maxit : 4 * gm.n;
  const size_t nk = (size_t)gm.n * k;
  st.beta = h->ne_buf;
  st.f = st.beta + nk;
  st.p = st.f + nk;
  st.q = st.p + nk;
  double* cvec = st.q + nk;
  st.c = cvec + (size_t)gm.np * k;
  st.c1 = st.c + k;
  st.relres = st.c1 + k;
  st.active = h->ne_ibuf;
  st.iters = st.active + k;
  st.status = st.iters + k;
  GS_CUDA_TRY(cudaMemsetAsync(cvec, 0, sizeof(double) * (size_t)gm.np * k, s));
  GS_CUDA_TRY(cudaMemsetAsync(h->st.err, 0, sizeof(int), s));
  double* Cpart = reinterpret_cast<double*>(h->Cpart);
  double* zero = h->u64;        // m x k zeros: S of the update and Y of the residual kernel
  GS_CUDA_TRY(cudaMemsetAsync(zero, 0, mk * sizeof(double), s));
  launch_colmajor_to_layout<double>(gm, k, Y, ldy, h->y64, 1.0, s);
  // h = X^T Sigma^-1 y:  E = 0 - y Omega^-1,  C = Q^T E,  h = -[R_i^T C_i]
  launch_sigma_resid<double>(p64, gm, k, Oinv, zero, h->y64, h->E64, s);
  launch_proj_partial<double>(p64, gm, k, h->Q64, h->E64, Cpart, h->st, 0, s);
  launch_reduce<double>(p64, gm, k, Cpart, h->C64, h->st, 0, nullptr, s);
  launch_ne_step(gm, k, h->R, h->C64, st, 1, s);
  h->launches += 7;
  GS_CUDA_TRY(cudaGetLastError());
  const int chunk = std::max(1, h->opts.chunk);
  for (int it = 0; it < st.maxit;) {
    const int steps = std::min(chunk, st.maxit - it);
    for (int c = 0; c < steps; ++c) {
      // v = Q (R p)  (update kernel: g = 0 g - 1 (0 - Q c))
      launch_ne_rmul(gm, k, h->R, st.p, cvec, s);
      launch_proj_update<double>(p64, gm, k, h->Q64, zero, h->g64, cvec, 0, nullptr, 1.0, h->cpart, h->st, 0, s);
      // E = -Sigma^-1 v;  C = Q^T E;  q = -[R_i^T C_i] = A p, then the CG step
      launch_sigma_resid<double>(p64, gm, k, Oinv, zero, h->g64, h->E64, s);
      launch_proj_partial<double>(p64, gm, k, h->Q64, h->E64, Cpart, h->st, 0, s);
      launch_reduce<double>(p64, gm, k, Cpart, h->C64, h->st, 0, nullptr, s);
      launch_ne_step(gm, k, h->R, h->C64, st, 0, s);
    }
    h->launches += 6 * steps;
    GS_CUDA_TRY(cudaGetLastError());
    it += steps;
    GS_CUDA_TRY(cudaMemcpyAsync(h->ne_hact, st.active, k * sizeof(int), cudaMemcpyDeviceToHost, s));
    GS_CUDA_TRY(cudaStreamSynchronize(s));
    bool any = false;
    for (int j = 0; j < k; ++j) any |= h->ne_hact[j] != 0;
    if (!any) break;
  }
  launch_ne_store(gm, k, st.beta, b, ldb, s);
  h->launches += 1;
  GS_CUDA_TRY(cudaMemcpyAsync(h->d_status_final, st.status, k * sizeof(int), cudaMemcpyDeviceToDevice, s));
  if (iters) GS_CUDA_TRY(cudaMemcpyAsync(iters, st.iters, k * sizeof(int), cudaMemcpyDeviceToDevice, s));
  if (relres) GS_CUDA_TRY(cudaMemcpyAsync(relres, st.relres, k * sizeof(double), cudaMemcpyDeviceToDevice, s));
  GS_CUDA_TRY(cudaGetLastError());
  return GLM_SUR_OK;
}

}  // namespace

extern "C" {

glm_sur_status glm_sur_solve_ne(glm_sur_t h, const double* Y, int64_t ldy, int k, double* b, int64_t ldb,
                                int* iters, double* relres, glm_sur_stream_t stream) {
  return ne_solve(h, Y, ldy, k, b, ldb, iters, relres, reinterpret_cast<cudaStream_t>(stream));
}

glm_sur_status glm_sur_solve(glm_sur_t h, const double* Y, int64_t ldy, int k, double* b, int64_t ldb, int* iters,
                             double* relres, glm_sur_stream_t stream) {
  return solve_impl(h, Y, ldy, nullptr, 0, k, b, ldb, iters, relres, reinterpret_cast<cudaStream_t>(stream));
}

glm_sur_status glm_sur_solve_restricted(glm_sur_t h, const double* Y, int64_t ldy, const double* d, int64_t ldd,
                                        int k, double* b, int64_t ldb, int* iters, double* relres,
                                        glm_sur_stream_t stream) {
  if (!h) return GLM_SUR_INVALID_ARG;
  if (h->mv_N == 0 && (h->sub ? h->sub->kc : h->kc) == 0) return GLM_SUR_INVALID_ARG;   // no restrictions
  return solve_impl(h, Y, ldy, d, ldd, k, b, ldb, iters, relres, reinterpret_cast<cudaStream_t>(stream));
}

glm_sur_status glm_sur_backward(glm_sur_t h, const double* dL_db, int64_t ldg, int k, double* dL_dY, int64_t ldy,
                                double* dL_dOmega, int64_t ldo, int* iters, double* relres, glm_sur_stream_t stream) {
  if (!h || !dL_db || (!dL_dY && !dL_dOmega) || h->mv_N) return GLM_SUR_INVALID_ARG;
  if (h->sub) {
    // the adjoint of the reduced model; dL/dy = Q dL/dy' (the rows outside
    // range(W) have lam = 0) and dL/dOmega is the reduced model's
    const int64_t M = h->gm.M, n = h->gm.n, G = h->gm.G;
    if (k < 1 || k > kMaxRhs || (dL_dY && ldy < M * G) || G * n * k > h->yred_cap) return GLM_SUR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    glm_sur_status rc = glm_sur_backward(h->sub, dL_db, ldg, k, dL_dY ? h->yred : nullptr, G * n, dL_dOmega, ldo,
                                         iters, relres, stream);
    if (rc != GLM_SUR_OK || !dL_dY) return rc;
    for (int j = 0; j < k; ++j)
      launch_dgemm((int)M, (int)G, n, h->Qw, 1, M, h->yred + j * G * n, 1, n, dL_dY + (int64_t)j * ldy, 1, M, s);
    h->launches += k;
    GS_CUDA_TRY(cudaGetLastError());
    return GLM_SUR_OK;
  }
  const Geom& gm = h->gm;
  const int64_t m = gm.M * gm.G;
  if (k < 1 || k != h->last_k || !h->has_w || h->w_restricted || h->kc > 0 || ldg < gm.n || (dL_dY && ldy < m) || (dL_dOmega && ldo < gm.G))
    return GLM_SUR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  IterPlan p64;
  glm_sur_status rc = prepare_solve(h, k, p64);
  if (rc != GLM_SUR_OK) return rc;
  const int nch = adj_omega_chunks(gm, k, h->sms);
  rc = ensure_adjoint_workspace(h, k, nch);
  if (rc != GLM_SUR_OK) return rc;
  const int64_t mk = m * k;
  GS_CUDA_TRY(cudaMemcpyAsync(h->wfwd, h->w64, mk * sizeof(double), cudaMemcpyDeviceToDevice, s));
  // lam_1 = Q R^-T dL/db: block by block X_i^T lam_1 = R_i^T Q_i^T Q_i R_i^-T g_i = g_i.
  // With a preconditioner block the iteration's model is the row-scaled one
  // (X_i / sqrt(delta_i), Omega~ = D0^-1/2 Omega D0^-1/2, y~ = S y, S =
  // D0^-1/2 (x) I_M), whose R_i^-T is sqrt(delta_i) R_i^-T.  b does not depend
  // on D0, so dL/dy = S dL/dy~ and dL/dOmega = D0^-1/2 dL/dOmega~ D0^-1/2.
  const double* sq = h->opts.precond != GLM_SUR_PRECOND_IDENTITY ? h->d_sqrtd : nullptr;
  const double* isq = h->opts.precond != GLM_SUR_PRECOND_IDENTITY ? h->d_isqrtd : nullptr;
  launch_adj_seed(gm, k, h->R, dL_db, ldg, h->C64, s, sq);
  GS_CUDA_TRY(cudaMemsetAsync(h->E64, 0, mk * sizeof(double), s));
  launch_proj_update<double>(p64, gm, k, h->Q64, h->E64, h->lam1, h->C64, 0, nullptr, 1.0, h->cpart, h->st, 0, s);
  // y' = 0 - Sigma lam_1; the remaining lam_2 solves eq. (aug1) for y'
  launch_sigma_resid<double>(p64, gm, k, h->Om64, h->E64, h->lam1, h->y64, s);
  h->launches += 3;
  GS_CUDA_TRY(cudaGetLastError());
  h->has_w = false;
  rc = solve_core(h, p64, nullptr, 0, k, nullptr, 0, iters, relres, s);
  if (rc != GLM_SUR_OK) return rc;
  // lam = lam_1 + lam_2 (into w64), outputs, then the forward w back in place
  launch_add_to_f64<double>(mk, h->lam1, h->w64, s);
  h->launches += 1;
  if (dL_dY) {
    launch_layout_to_colmajor<double>(gm, k, h->w64, dL_dY, ldy, s, isq);
    h->launches += 1;
  }
  if (dL_dOmega) {
    launch_adj_omega(gm, k, h->w64, h->wfwd, h->opart, nch, dL_dOmega, ldo, s, isq);
    h->launches += 2;
  }
  GS_CUDA_TRY(cudaMemcpyAsync(h->w64, h->wfwd, mk * sizeof(double), cudaMemcpyDeviceToDevice, s));
  GS_CUDA_TRY(cudaGetLastError());
  h->has_w = true;
  return GLM_SUR_OK;
}

glm_sur_status glm_sur_set_restrictions(glm_sur_t h, const double* C, int64_t ldc, int kc, glm_sur_stream_t stream) {
  if (h && h->mv_N) return GLM_SUR_INVALID_ARG;   // the restrictions are the model's own
  if (h && h->sub) return glm_sur_set_restrictions(h->sub, C, ldc, kc, stream);
  if (!h || kc < 0 || (kc > 0 && (!C || ldc < kc))) return GLM_SUR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const Geom& gm = h->gm;
  if (kc > 0 && (size_t)gm.n * sizeof(double) > 200 * 1024) return GLM_SUR_INVALID_ARG;   // n <= 25600
  dfree(h->Cmat); dfree(h->Nmat); dfree(h->Minv); dfree(h->cbuf); dfree(h->fbuf); dfree(h->gC);
  dfree(h->wfwd); dfree(h->lam1); dfree(h->opart);
  h->rcap = 0;
  h->kc = 0;
  h->plan_k = -1;
  h->graph.reset();
  h->has_w = false;
  if (kc == 0) return GLM_SUR_OK;
  GS_CUDA_TRY(dalloc(&h->Cmat, (size_t)kc * gm.n));
  GS_CUDA_TRY(dalloc(&h->Nmat, (size_t)gm.n * gm.n));
  GS_CUDA_TRY(dalloc(&h->Minv, (size_t)gm.n * gm.n));
  GS_CUDA_TRY(cudaMemcpy2DAsync(h->Cmat, kc * sizeof(double), C, ldc * sizeof(double), kc * sizeof(double), gm.n,
                                cudaMemcpyDeviceToDevice, s));
  GS_CUDA_TRY(rglm_factor(gm, h->R, h->Cmat, kc, kc, gm.d_col_blk, h->Nmat, h->Minv, h->setup_flags, s));
  h->launches += 3;
  h->kc = kc;
  return GLM_SUR_OK;
}

glm_sur_status glm_sur_get_status(glm_sur_t h, int* status, int k) {
  if (h && h->sub) return glm_sur_get_status(h->sub, status, k);
  if (!h || !status || k < 1 || k > h->last_k) return GLM_SUR_INVALID_ARG;
  GS_CUDA_TRY(cudaDeviceSynchronize());
  GS_CUDA_TRY(cudaMemcpy(status, h->d_status_final, k * sizeof(int), cudaMemcpyDeviceToHost));
  int err = 0;
  GS_CUDA_TRY(cudaMemcpy(&err, h->st.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    for (int j = 0; j < k; ++j) status[j] = GLM_SUR_TIMEOUT;
    return GLM_SUR_TIMEOUT;
  }
  glm_sur_status worst = GLM_SUR_OK;
  for (int j = 0; j < k; ++j) {
    if (status[j] == kStatusRunning) status[j] = GLM_SUR_NOT_CONVERGED;
    if (status[j] != GLM_SUR_OK && worst == GLM_SUR_OK) worst = (glm_sur_status)status[j];
  }
  return worst;
}

glm_sur_status glm_sur_get_w(glm_sur_t h, double* w, int64_t ldw, glm_sur_stream_t stream) {
  if (h && h->sub) return GLM_SUR_INVALID_ARG;   // w of the unreduced rows is not formed
  if (!h || !w || !h->has_w || ldw < h->gm.M * h->gm.G) return GLM_SUR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // the row-scaled model's w~ solves it for S^-1 w: w = S w~, S = D0^-1/2 (x) I_M
  launch_layout_to_colmajor<double>(h->gm, h->last_k, h->w64, w, ldw, s,
                                    h->opts.precond != GLM_SUR_PRECOND_IDENTITY ? h->d_isqrtd : nullptr);
  GS_CUDA_TRY(cudaGetLastError());
  return GLM_SUR_OK;
}

glm_sur_status glm_sur_get_factors(glm_sur_t h, double* Q, int64_t ldq, double* R, glm_sur_stream_t stream) {
  if (h && h->sub) return GLM_SUR_INVALID_ARG;   // the factors belong to the reduced model
  if (!h || (Q && ldq < h->gm.M)) return GLM_SUR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const Geom& gm = h->gm;
  if (Q) {
    // padded row-major M x np  ->  column-major M x n
    launch_unpad_q(gm, h->Q64, Q, ldq, s);
    GS_CUDA_TRY(cudaGetLastError());
  }
  if (R) {
    int64_t relems = 0;
    for (int i = 0; i < gm.G; ++i) relems += (int64_t)h->n_i[i] * h->n_i[i];
    GS_CUDA_TRY(cudaMemcpyAsync(R, h->R, relems * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  return GLM_SUR_OK;
}

int glm_sur_step_path(glm_sur_t h) {
  if (h && h->sub) return glm_sur_step_path(h->sub);
  if (!h || h->plan_k < 1) return -1;
  return h->plan.tc_step ? 1 : 0;
}

int64_t glm_sur_launch_count(glm_sur_t h) {
  if (!h) return -1;
  return h->launches + (h->sub ? glm_sur_launch_count(h->sub) : 0);
}

glm_sur_status glm_sur_profile_steps(glm_sur_t h, int reps, double* ms, glm_sur_stream_t stream) {
  if (h && h->sub) return glm_sur_profile_steps(h->sub, reps, ms, stream);
  if (!h || !ms || reps < 1 || h->last_k < 1 || h->plan_k != h->last_k) return GLM_SUR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int k = h->last_k;
  const bool fp64 = fp64_steps(h->opts);
  glm_sur_status rc = reset_state(h, k, 0.0, 1 << 30, 0, s);   // no stop tests
  if (rc != GLM_SUR_OK) return rc;
  if (fp64) rc = pcg_init<double>(h, k, h->y64, s);
  else launch_init_inner<float>(h->plan, h->gm, k, h->y64, nullptr, h->g32, h->u32, h->w32, h->cpart, s);
  cudaEvent_t ev[5];
  for (auto& e : ev) cudaEventCreate(&e);
  double acc[5] = {0, 0, 0, 0, 0};
  const IterPlan& p = h->plan;
  auto one = [&](bool timed) {
    if (timed) cudaEventRecord(ev[0], s);
    if (fp64) {
      double* Cp = reinterpret_cast<double*>(h->Cpart);
      double* C = reinterpret_cast<double*>(h->Cfin);
      launch_sigma_step<double>(p, h->gm, k, h->Om64, h->g64, h->u64, h->w64, h->S64, h->wb64, h->st, h->cpart,
                                h->dpart, s);
      if (timed) cudaEventRecord(ev[1], s);
      launch_proj_partial<double>(p, h->gm, k, h->Q64, h->S64, Cp, h->st, 1, s);
      if (timed) cudaEventRecord(ev[2], s);
      launch_reduce<double>(p, h->gm, k, Cp, C, h->st, 1, h->dpart, s);
      if (timed) cudaEventRecord(ev[3], s);
      launch_proj_update<double>(p, h->gm, k, h->Q64, h->S64, h->g64, C, 1, h->st.lam, 0.0, h->cpart, h->st, 1, s);
    } else {
      float* Cp = reinterpret_cast<float*>(h->Cpart);
      float* C = reinterpret_cast<float*>(h->Cfin);
      if (p.tc_step) {
        // ms[0] pass A, ms[1] 0 (its projection partials are inside pass A), ms[2] reduce, ms[3] pass B
        launch_tc_pass_a(p, h->gm, k, h->Om32, h->Q32, h->g32, h->u32, h->w32, h->wb32, h->st, h->cpart,
                         p.n_cpart + p.extra_cpart, h->dpart, Cp, s);
        if (timed) cudaEventRecord(ev[1], s);
        if (timed) cudaEventRecord(ev[2], s);
        launch_reduce<float>(p, h->gm, k, Cp, C, h->st, 1, h->dpart, s);
        if (timed) cudaEventRecord(ev[3], s);
        launch_tc_pass_b(p, h->gm, k, h->Om32, h->Q32, h->g32, h->u32, h->w32, C, h->st, h->cpart, s);
      } else {
        launch_sigma_step<float>(p, h->gm, k, h->Om32, h->g32, h->u32, h->w32, h->S32, h->wb32, h->st, h->cpart,
                                 h->dpart, s);
        if (timed) cudaEventRecord(ev[1], s);
        launch_proj_partial<float>(p, h->gm, k, h->Q32, h->S32, Cp, h->st, 1, s);
        if (timed) cudaEventRecord(ev[2], s);
        launch_reduce<float>(p, h->gm, k, Cp, C, h->st, 1, h->dpart, s);
        if (timed) cudaEventRecord(ev[3], s);
        launch_proj_update<float>(p, h->gm, k, h->Q32, h->S32, h->g32, C, 1, h->st.lam, 0.0, h->cpart, h->st, 1,
                                  s);
      }
    }
    if (timed) cudaEventRecord(ev[4], s);
    h->launches += p.launches_per_step;
  };
  for (int r = 0; r < 3; ++r) one(false);
  for (int r = 0; r < reps; ++r) {
    one(true);
    cudaError_t e = cudaEventSynchronize(ev[4]);
    if (e != cudaSuccess) {
      set_last_error(e, "profile step", __FILE__, __LINE__);
      rc = GLM_SUR_CUDA_ERROR;
      break;
    }
    float t;
    for (int q = 0; q < 4; ++q) {
      cudaEventElapsedTime(&t, ev[q], ev[q + 1]);
      acc[q] += t;
    }
    cudaEventElapsedTime(&t, ev[0], ev[4]);
    acc[4] += t;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  for (int q = 0; q < 5; ++q) ms[q] = acc[q] / reps;
  h->has_w = false;
  h->graph.reset();   // the captured graph baked the previous tolerance
  return rc;
}

glm_sur_status glm_sur_ols_static(glm_sur_t h, const double* Y, int64_t ldy, int k, double* b, int64_t ldb,
                                  glm_sur_stream_t stream) {
  if (h && h->sub) return GLM_SUR_INVALID_ARG;   // a rotation needs device workspace
  if (!h || !Y || !b || k < 1 || k > kMaxRhs) return GLM_SUR_INVALID_ARG;
  const Geom& gm = h->gm;
  if (ldy < gm.M * gm.G || ldb < gm.n) return GLM_SUR_INVALID_ARG;
  if ((long long)gm.np * k * 2 > kOlsScratchDoubles) return GLM_SUR_INVALID_ARG;
  // the scratch address is looked up on the current device: it must be the handle's
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != h->dev) return GLM_SUR_INVALID_ARG;
  return ols_static(gm, h->Q64, h->R, Y, ldy, k, b, ldb, h->sms, reinterpret_cast<cudaStream_t>(stream));
}

void glm_sur_destroy(glm_sur_t h) {
  if (!h) return;
  if (h->sub) {
    glm_sur_destroy(h->sub);
    cudaDeviceSynchronize();
    dfree(h->Qw);
    dfree(h->yred);
    dfree(h->rot_ws);
    dfree(h->mv_koff);
    dfree(h->mv_Q0);
    dfree(h->mv_y);
    delete h;
    return;
  }
  cudaDeviceSynchronize();
  free_workspace(h);
  dfree(h->Q64); dfree(h->Q32); dfree(h->R); dfree(h->Om64); dfree(h->Om32); dfree(h->setup_flags);
  dfree(h->Omraw); dfree(h->d_sqrtd); dfree(h->d_isqrtd);
  dfree(h->gm.d_n_i); dfree(h->gm.d_off); dfree(h->gm.d_poff); dfree(h->gm.d_quad_blk); dfree(h->gm.d_r_off);
  dfree(h->gm.d_ug_blk0); dfree(h->gm.d_col_blk);
  dfree(h->Cmat); dfree(h->Nmat); dfree(h->Minv); dfree(h->cbuf); dfree(h->fbuf); dfree(h->gC);
  dfree(h->wfwd); dfree(h->lam1); dfree(h->opart);
  dfree(h->ne_buf); dfree(h->ne_ibuf); dfree(h->ne_om);
  dfree(h->p3_buf); dfree(h->p3_ibuf);
  dfree(h->c1x); dfree(h->c1x_part);
  if (h->p3_hact) cudaFreeHost(h->p3_hact);
  if (h->ne_hact) cudaFreeHost(h->ne_hact);
  if (h->h_done) cudaFreeHost(h->h_done);
  if (h->h_norms) cudaFreeHost(h->h_norms);
  if (h->ev[0]) cudaEventDestroy(h->ev[0]);
  if (h->ev[1]) cudaEventDestroy(h->ev[1]);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

}  // extern "C"
