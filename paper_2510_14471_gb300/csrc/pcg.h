// Launch plans and host launchers of the PCG-Aug iteration kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "internal.h"

namespace glmsur {

// Grid shapes of one PCG configuration (fixed for a handle, k and precision).
struct IterPlan {
  int JJ = 1;              // right-hand sides per thread tile (divides k)
  int TR = 1;              // rows per Sigma-apply tile
  int n_sigma = 1;         // row CTAs of the Sigma-apply kernels (d partials)
  int n_partial_rows = 1;  // row ranges of proj_partial (C partials)
  int n_qgroups = 1;       // column-quad groups of proj_partial
  int n_update = 1;        // row CTAs of proj_update
  int n_ugroups = 1;       // block groups of proj_update
  int n_cpart = 1;         // c partials written per step (n_update * n_ugroups)
  int extra_cpart = 0;     // + 1 partial for the restriction rows (Sec. 4.1)
  int ug_threads = 32;     // threads of a proj_update CTA (>= quads of any group)
  int ug_max_quads = 1;    // quads of the largest block group
  int TRB = 1;             // rows per proj_update tile
  size_t sigma_smem = 0;
  size_t update_smem = 0;
  // TMA-streamed kernels (used when JJ == k and rows are 16-byte multiples)
  bool tma_sigma = false, tma_update = false;
  int tr_tma = 1, nst_sigma = 3, trb_tma = 1, nst_update = 3, update_threads = 256;
  int ri = 4;              // rows per Sigma-apply item of the TMA step
  size_t sigma_tma_smem = 0, update_tma_smem = 0;
  bool bj_update = false;  // block x column projection update (n_i <= 32, G*k <= 1024)
  int bj_np = 1, trb_bj = 1, nst_bj = 3;
  size_t bj_smem = 0;
  bool tma_partial = false;  // TMA-streamed projection partials (n' / 4 <= 512 quads)
  int tr_partial = 1, nst_partial = 3, partial_threads = 64;
  size_t partial_tma_smem = 0;
  // fused float32 step with the Sigma-apply on the tensor cores (pcg_tc.cu):
  // pass A, reduce, pass B; Gp = G padded to 32 or 64; Q sub-tiles of tc_tq_*
  // rows in rings of tc_nsq_* stages; tc_nsg staged g tiles in pass B
  bool tc_step = false;
  int tc_gp = 64, tc_tq_a = 4, tc_nsq_a = 2, tc_tq_b = 2, tc_nsq_b = 2, tc_nsg = 2;
  size_t tc_a_smem = 0, tc_b_smem = 0;
  int launches_per_step = 4;
};

// Shared-memory layout of the tensor-core step kernels (byte offsets); pass 0
// stages g and u tiles and keeps the S tile, pass 1 stages one u tile and NSG
// g tiles and keeps the (Q C) tile.  The U operand of the MMA and the
// accumulator live in tensor memory.  Pass 0 keeps a staged row of G k
// values in (G + 1) k floats: the pad puts the rows that one warp touches at
// once on different banks.
struct TcSmem {
  uint32_t om, vec, tile, q, total;
};
__host__ __device__ inline int tc_row_stride(int pass, int G, int KK) { return (pass == 0 ? G + 1 : G) * KK; }
__host__ __device__ inline TcSmem tc_smem_layout(int pass, int G, int Gp, int KK, int np, int TQ, int NSQ, int NSG) {
  TcSmem L;
  const uint32_t TV = 128u / (uint32_t)KK;
  const uint32_t tile_bytes = TV * (uint32_t)tc_row_stride(pass, G, KK) * 4u;
  uint32_t off = 128;   // mbarriers (at most 16)
  L.om = off;
  off += 2u * Gp * Gp * 4u;
  L.vec = off;
  off += (pass == 0 ? 2u : 1u + (uint32_t)NSG) * tile_bytes;
  L.tile = off;
  off += tile_bytes;
  L.q = off;
  off += (uint32_t)NSQ * TQ * (uint32_t)np * 4u;
  L.total = off;
  return L;
}

bool tc_step_eligible(int G, int k, int np, int nmax_cols);
cudaError_t tc_prepare(int k, int Gp, size_t a_bytes, size_t b_bytes);
void launch_tc_pass_a(const IterPlan& p, const Geom& gm, int k, const float* Om, const float* Q, const float* g,
                      float* u, const float* w, float* wbest, const PcgState& st, const double* cpart, int ncpart,
                      double* dpart, float* Cpart, cudaStream_t s);
void launch_tc_pass_b(const IterPlan& p, const Geom& gm, int k, const float* Om, const float* Q, float* g,
                      const float* u, float* w, const float* C, const PcgState& st, double* cpart, cudaStream_t s);

template <typename T>
void launch_sigma_step(const IterPlan& p, const Geom& gm, int k, const T* Om, T* g, T* u, T* w, T* S, T* wbest,
                       const PcgState& st, const double* cpart, double* dpart, cudaStream_t s);
template <typename T>
void launch_restore_best(int64_t n, int k, const PcgState& st, const T* wbest, T* w, cudaStream_t s);
template <typename T>
void launch_sigma_resid(const IterPlan& p, const Geom& gm, int k, const T* Om, const T* Y, const T* W, T* E,
                        cudaStream_t s);
template <typename T>
void launch_proj_partial(const IterPlan& p, const Geom& gm, int k, const T* Q, const T* S, T* Cpart,
                         const PcgState& st, int use_state, cudaStream_t s);
template <typename T>
void launch_reduce(const IterPlan& p, const Geom& gm, int k, const T* Cpart, T* C, const PcgState& st, int scalar,
                   const double* dpart, cudaStream_t s, bool pdl = false);
template <typename T>
void launch_proj_update(const IterPlan& p, const Geom& gm, int k, const T* Q, const T* S, T* g, const T* C,
                        int alpha, const double* lam, double lam_const, double* cpart, const PcgState& st,
                        int use_state, cudaStream_t s);
template <typename Tout>
void launch_colmajor_to_layout(const Geom& gm, int k, const double* Y, int64_t ldy, Tout* out, double scale,
                               cudaStream_t s, const double* blk_scale = nullptr);
template <typename Tin>
void launch_layout_to_colmajor(const Geom& gm, int k, const Tin* in, double* Y, int64_t ldy, cudaStream_t s,
                               const double* blk_scale = nullptr);
void launch_tri_solve(const Geom& gm, int k, const double* R, const double* C, double* b, int64_t ldb,
                      cudaStream_t s, const double* blk_scale = nullptr);
void launch_precond_omega(int G, int Gq, int kind, const double* Om, double* Om_out, double* sqrtd, double* isqrtd,
                          cudaStream_t s);
template <typename Tin, typename Tout>
void launch_convert(int64_t n, const Tin* in, Tout* out, double scale, cudaStream_t s);
template <typename Tin>
void launch_add_to_f64(int64_t n, const Tin* d, double* w, cudaStream_t s);
template <typename T>
void launch_init_inner(const IterPlan& p, const Geom& gm, int k, const double* rho, const int* live, T* g, T* u,
                       T* w, double* cpart, cudaStream_t s);
void launch_masked_axpy(int64_t n, int k, const int* mask, double sign, const double* d, double* w,
                        cudaStream_t s);
template <typename T>
void launch_colsumsq(const IterPlan& p, const Geom& gm, int k, const T* v, double* part, cudaStream_t s);
void launch_sum_partials_sqrt(int np_, int k, const double* part, double* out, cudaStream_t s);
void launch_add_int(int n, const int* a, int* acc, cudaStream_t s);
void launch_shift_diag(int G, int Gq, const double* Om64, float* Om32, double rel, cudaStream_t s);
void launch_unpad_q(const Geom& gm, const double* Q, double* out, int64_t ldq, cudaStream_t s);
template <typename T>
cudaError_t set_smem_attrs(int JJ, size_t bytes, size_t upd_bytes);
template <typename T>
cudaError_t set_tma_smem_attrs(int JJ, size_t sigma_bytes, size_t update_bytes, size_t bj_bytes,
                               size_t partial_bytes);

}  // namespace glmsur
