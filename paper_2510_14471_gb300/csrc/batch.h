// Batched solves of independent SUR instances (one persistent launch).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace glmsur {

constexpr int kBatchMaxG = 32;      // equations per instance
constexpr int kBatchMaxCols = 32;   // columns per block
constexpr int kBatchMaxNp = 512;    // padded columns per instance
constexpr int kBatchMaxPairs = 1024;  // column quads x right-hand sides an instance's CTA accumulates
constexpr int kBatchMaxK = 8;       // right-hand sides per instance (1, 2, 4 or 8)

// Device descriptor of one instance (offsets into the batch pools).
struct BatchInst {
  int index;                 // position in the caller's order
  int G, Gq, M, n, np, nq;
  int blk0, quad0;           // first block / quad in the global block / quad arrays
  int64_t q_off;             // Q (M x np, row-major) in the Q pools
  int64_t om_off;            // Omega (G x Gq) in the Omega pools
  int64_t v_off;             // (M, G, K) vectors in the vector pools
  int64_t y_off;             // caller's Y: m x K column-major, ld = m = G*M
  int64_t b_off;             // caller's b: n x K column-major, ld = n
};

struct BatchPools {
  const double* q64;
  const float* q32;
  const double* R;
  const double* om64;
  const float* om32;
  const int* n_i;
  const int* poff;           // padded column offset of every block within its instance
  const int64_t* r_off;
  const int* quad_blk;       // block (within the instance) of every quad
  double *w64, *E64, *d64;
  float *g32, *u32, *w32, *wb32;
  const double* Y;
  double* b;
  int* status;
  int* iters;
  double* relres;
  int* steps;                // per instance: float32 steps the CTA ran (all refinement rounds)
  long long* cycles;         // per instance: SM clock cycles from start to end
  // (nullable, count x kBatchMaxK) energy added to the first float64 residual as the
  // reference of relres and tol: a row-reduced instance's share of the
  // M-row model's ||P y||^2 that the reduction leaves out
  const double* rho_extra;
};

struct BatchOpts {
  double tol, inner_tol;
  int max_refine, inner_maxit, inner_window;
};

// Tile heights the kernel is built for (rows per shared-memory tile); the
// autotuner of glm_sur_batch_solve times them and keeps the fastest.
constexpr int kBatchTiles[3] = {8, 16, 32};

cudaError_t batch_prepare(int K, int TR, int maxG, int maxNp, int* ctas_per_sm);
cudaError_t batch_solve_launch(int K, int TR, const BatchInst* insts, int count, const BatchPools& P,
                               const BatchOpts& o, int* counter, int grid, int maxG, int maxNp, cudaStream_t s);

}  // namespace glmsur
