// Shared device helpers: the arithmetic traits that let every kernel be
// written once for IEEE FP64 vectors and for double-word FP32-pair vectors,
// and the warp/block reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dw.cuh"

template <typename T>
struct num;

template <>
struct num<double> {
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double to_d(double x) { return x; }
  static __device__ __forceinline__ double from_d(double x) { return x; }
};

template <>
struct num<float> {
  static __device__ __forceinline__ float zero() { return 0.f; }
  static __device__ __forceinline__ double to_d(float x) { return (double)x; }
  static __device__ __forceinline__ float from_d(double x) { return __double2float_rn(x); }
};

template <>
struct num<dw> {
  static __device__ __forceinline__ dw zero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ double to_d(dw x) { return dw_to_double(x); }
  static __device__ __forceinline__ dw from_d(double x) { return dw_from_double(x); }
};

// Accumulator of a linear combination in the vector arithmetic: plain FP64
// for double; the lazy compensated pair (dw.cuh) for double-word.
template <typename T>
struct acc_of;
template <>
struct acc_of<double> {
  using type = double;
};
template <>
struct acc_of<float> {
  using type = float;
};
template <>
struct acc_of<dw> {
  using type = dwacc;
};

__device__ __forceinline__ void acc_set(double &a, double x) { a = x; }
__device__ __forceinline__ void acc_add(double &a, double x) { a += x; }
__device__ __forceinline__ void acc_sub(double &a, double x) { a -= x; }
__device__ __forceinline__ void acc_set_prod(double &a, double c, double x) { a = c * x; }
__device__ __forceinline__ void acc_add_prod(double &a, double c, double x) { a = fma(c, x, a); }
__device__ __forceinline__ double acc_get(const double &a) { return a; }
__device__ __forceinline__ double acc_raw(const double &a) { return a; }
// FP32: plain FP32 arithmetic with FMA (the mixed-precision chain accumulates in FP32)
__device__ __forceinline__ void acc_set(float &a, float x) { a = x; }
__device__ __forceinline__ void acc_add(float &a, float x) { a = __fadd_rn(a, x); }
__device__ __forceinline__ void acc_sub(float &a, float x) { a = __fsub_rn(a, x); }
__device__ __forceinline__ void acc_set_prod(float &a, float c, float x) { a = __fmul_rn(c, x); }
__device__ __forceinline__ void acc_add_prod(float &a, float c, float x) { a = __fmaf_rn(c, x, a); }
__device__ __forceinline__ float acc_get(const float &a) { return a; }
__device__ __forceinline__ float acc_raw(const float &a) { return a; }

// Vectorised 8-byte loads through the read-only path.
template <typename T>
__device__ __forceinline__ T ldg(const T *p) {
  return __ldg(p);
}
template <>
__device__ __forceinline__ dw ldg<dw>(const dw *p) {
  float2 f = __ldg(reinterpret_cast<const float2 *>(p));
  return {f.x, f.y};
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; every thread gets the result.  `red` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double *red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  // fixed order: deterministic
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

// Programmatic dependent launch.  Kernels of the solve are launched with
// pdl_launch, which lets the next grid in the stream be scheduled while the
// previous one drains (its CTAs then wait in pdl_wait).  Every such kernel
// calls pdl_wait() before touching device memory (it returns once the
// preceding grid has completed and its writes are visible) and
// pdl_trigger() to let its own dependents launch; on a grid launched without
// the attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
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
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

#define PP_CUDA_TRY(expr)                                      \
  do {                                                         \
    cudaError_t _e = (expr);                                   \
    if (_e != cudaSuccess) return pp_cuda_fail(_e, #expr);     \
  } while (0)

int pp_cuda_fail(cudaError_t e, const char *what);
