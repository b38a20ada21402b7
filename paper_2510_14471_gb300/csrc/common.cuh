// Shared device/host helpers of the SUR PCG-Aug library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>

#include "glm_sur.h"

namespace glmsur {

// ---------------------------------------------------------------------------
// status and error plumbing (host)
// ---------------------------------------------------------------------------
#define GS_CUDA_TRY(expr)                                                      \
  do {                                                                         \
    cudaError_t e_ = (expr);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      glmsur::set_last_error(e_, #expr, __FILE__, __LINE__);                   \
      return e_ == cudaErrorMemoryAllocation ? GLM_SUR_OOM : GLM_SUR_CUDA_ERROR; \
    }                                                                          \
  } while (0)

void set_last_error(cudaError_t e, const char* what, const char* file, int line);

// Per-column run status codes kept on the device while a PCG runs.  Column
// states use the public glm_sur_status values; RUNNING marks a live column.
constexpr int kStatusRunning = -1;
// An iterative-refinement step whose float64 residual is above this fraction
// of the previous one has met the rounding floor of the residual itself.
constexpr double kRefineMinGain = 0.5;

// ---------------------------------------------------------------------------
// programmatic dependent launch (PTX griddepcontrol, sm_90 and later).  A
// kernel launched with the programmatic-serialization attribute may start
// before the kernel ahead of it in the stream has finished; it must call
// griddep_wait() before its first access to anything that kernel writes: the
// wait returns once the prerequisite grid has completed and its memory
// operations are visible.  griddep_launch_dependents() lets the next kernel
// start launching (its blocks are placed as resources free up).  Both are
// no-ops for a kernel launched without the attribute.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch of `kern` with the programmatic-serialization attribute (host).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int round_up4(int x) { return (x + 3) & ~3; }

// Vector load/store of 4 consecutive scalars (16 B for float, 2x16 B for double).
template <typename T> struct Vec4;
template <> struct Vec4<float> {
  using type = float4;
  __device__ __forceinline__ static void copy(const type* src, type* dst) { *dst = *src; }
  __device__ __forceinline__ static void load(const float* p, float (&v)[4]) {
    float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
  __device__ __forceinline__ static void load_stream(const float* p, float (&v)[4]) {
    float4 t = __ldcs(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
};
template <> struct Vec4<double> {
  struct __align__(16) type { double2 a, b; };
  __device__ __forceinline__ static void copy(const type* src, type* dst) {
    dst->a = src->a;
    dst->b = src->b;
  }
  __device__ __forceinline__ static void load(const double* p, double (&v)[4]) {
    double2 a = reinterpret_cast<const double2*>(p)[0];
    double2 b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  __device__ __forceinline__ static void load_stream(const double* p, double (&v)[4]) {
    double2 a = __ldcs(reinterpret_cast<const double2*>(p));
    double2 b = __ldcs(reinterpret_cast<const double2*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
};

}  // namespace glmsur
