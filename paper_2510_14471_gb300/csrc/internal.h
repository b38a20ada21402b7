// Internal declarations shared by the translation units of the library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "glm_sur.h"

namespace glmsur {

constexpr int kMaxBlockCols = 64;   // max n_i (TSQR leaves hold <= 256 x 32 or 128 x 64)
constexpr int kMaxRhs = 64;         // max k
constexpr int kMaxG = 1024;         // max number of equations of a handle
constexpr int kMaxReducedCols = 2048;   // largest n of a row-reduced model (its setup Cholesky is n^3 / 3)
constexpr int kMaxSolveG = 156;     // max equations of a solve: float64 Omega and one row tile of
                                    // eight right-hand sides within 200 KB of shared memory

// One node of the TSQR forest (setup).
struct QrNode {
  int blk;             // block (equation) index
  int nc;              // n_i
  int rows;            // rows of the node's input matrix
  int level;           // 0 = leaf (rows of X_i)
  int parent;          // -1 at the root
  int child_row;       // first row of this node's R inside the parent's stack
  int parent_rows;     // rows of the parent's stack (its leading dimension)
  int pad_;
  int64_t in_off;      // leaf: first row in X_i; inner: offset of its stack in the workspace
  int64_t parent_in_off;
  int64_t out_off;     // where this node's R goes inside the parent's stack
  int64_t v_off;       // reflectors (rows x nc, col-major)
  int64_t tau_off;
  int64_t x_base;      // leaf input: element offset of the block's first column in X
  int64_t x_ld;        //   and its leading dimension (column-major)
  int64_t q_base;      // explicit Q: element offset of the block's (row 0, column 0) in Q
  int64_t q_ld;        //   and its row stride (row-major)
};

// One regressor block to factor: rows x nc, read from X and written to Q.
struct QrBlock {
  int nc;
  int64_t rows, x_base, x_ld, q_base, q_ld;
};

struct QrPlan {
  std::vector<QrNode> nodes;          // sorted by level
  std::vector<int> level_first, level_count;
  int64_t stack_elems = 0, v_elems = 0, tau_elems = 0;
  size_t max_smem_factor = 0, max_smem_form = 0;
};

void build_qr_plan(const std::vector<QrBlock>& blocks, QrPlan& plan);
glm_sur_status run_qr(const QrPlan& plan, const double* X, const int64_t* d_r_off, double* Q, double* R,
                      int* d_setup_flags, cudaStream_t st);

// Geometry of one SUR problem on the device.
//   vectors (g, u, w, S, ...) : (M, G, k) row-major, element (t, i, j) at (t*G + i)*k + j
//   Q                          : M x np row-major, block i in columns poff[i] .. poff[i]+n_i-1,
//                                columns padded with zeros to a multiple of 4 per block
//   Omega                      : G x Gq row-major (Gq = G rounded up to 4, zero padded)
//   R                          : block i row-major n_i x n_i at r_off[i]
struct Geom {
  int G = 0, Gq = 0, n = 0, np = 0, nq = 0;   // nq = np / 4 column quads
  int64_t M = 0;
  int64_t Ms = 0;            // rows t < Ms carry Sigma = Omega (x) I; Sigma = 0 on rows t >= Ms
                             // (the restriction rows of the restricted multivariate model)
  int* d_n_i = nullptr;
  int* d_off = nullptr;      // unpadded column offsets (G+1)
  int* d_poff = nullptr;     // padded column offsets (G+1)
  int* d_quad_blk = nullptr; // block of every column quad (nq)
  int* d_col_blk = nullptr;  // block of every (unpadded) column (n)
  int64_t* d_r_off = nullptr;
  // block groups of the projection update: runs of whole blocks with at most
  // kMaxGroupQuads column quads each; group g = blocks [ug_blk0[g], ug_blk0[g+1])
  int n_ugroups = 1, ug_max_quads = 1;
  int* d_ug_blk0 = nullptr;
};

constexpr int kMaxGroupQuads = 512;

// Device state of one batch of k PCG columns (one solve).
struct PcgState {
  int k = 0;
  int W = 10;
  double tol = 1e-12;
  int maxit = 0;
  double* c[2] = {nullptr, nullptr};   // c_i, parity slots
  int* active[2] = {nullptr, nullptr};
  double* c1 = nullptr;
  double* lam = nullptr;
  double* cbest[2] = {nullptr, nullptr};  // running minimum of c (parity slots)
  int* itbest[2] = {nullptr, nullptr};     // step at which it was reached
  double* csnap[2] = {nullptr, nullptr};   // c at the last saved w (best-iterate snapshot)
  double* cstop = nullptr;                 // c when the column stopped
  int* iters = nullptr;
  int* status = nullptr;
  double* relres = nullptr;
  int* it = nullptr;                   // completed steps (written by the reduce kernel)
  int* done = nullptr;
  int* err = nullptr;                  // set when a bounded device wait gave up
  // (nullable, k) energy added to the first c as the reference of relres and
  // the tolerance: a row-reduced model's share of the M-row model's
  // ||P y||^2 that the reduction leaves out
  const double* c1_extra = nullptr;
};

}  // namespace glmsur
