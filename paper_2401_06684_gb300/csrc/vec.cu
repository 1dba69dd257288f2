// Vector kernels of the Krylov process: conversions at the API boundary,
// inner products (per-block partials reduced in a fixed order, so results are
// bitwise reproducible), the Lanczos three-term update, classical
// Gram-Schmidt sweeps against the stored basis (Algorithm 1, lines 5-9, done
// as two CGS passes), and the reconstruction f_m = V_m z (Algorithm 1, last
// line).  Per-element products accumulate in the vector arithmetic (FP64 or
// double-word); per-thread sums are widened to FP64 before any cross-thread
// reduction.
#include "common.cuh"
#include "internal.h"

namespace {

template <typename T>
__device__ __forceinline__ T ldv(const T *p) {
  return *p;
}

template <typename T>
__device__ __forceinline__ double sq_d(T v) {
  double d = num<T>::to_d(v);
  return d * d;
}

template <typename T>
__global__ void k_from_f64(const double *__restrict__ in, T *__restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = num<T>::from_d(in[i]);
}

template <typename T>
__global__ void k_to_f64(const T *__restrict__ in, double *__restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = num<T>::to_d(in[i]);
}

template <typename T>
__global__ void k_scale(const T *__restrict__ in, T *__restrict__ out, int64_t n, double c,
                        const double *__restrict__ c_dev) {
  const double cc = c_dev ? c * (*c_dev) : c;
  const T ct = num<T>::from_d(cc);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i] * ct;
}

template <typename T>
__global__ void k_copy(const T *__restrict__ in, T *__restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}

template <typename T>
__global__ void __launch_bounds__(256) k_dot(const T *__restrict__ x, const T *__restrict__ y, int64_t n,
                                             double *__restrict__ partials) {
  __shared__ double red[32];
  T acc = num<T>::zero();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc = acc + x[i] * y[i];
  const double s = block_sum(num<T>::to_d(acc), red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <typename T>
__global__ void __launch_bounds__(256) k_lanczos_update(T *__restrict__ w, const T *__restrict__ vj,
                                                        const T *__restrict__ vjm1, int64_t n,
                                                        const double *__restrict__ alpha,
                                                        const double *__restrict__ beta_prev,
                                                        double *__restrict__ partials) {
  __shared__ double red[32];
  const T a = num<T>::from_d(-(*alpha));
  const T b = num<T>::from_d(vjm1 ? -(*beta_prev) : 0.0);
  T acc = num<T>::zero();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T r = w[i] + a * vj[i];
    if (vjm1) r = r + b * vjm1[i];
    w[i] = r;
    acc = acc + r * r;
  }
  const double s = block_sum(num<T>::to_d(acc), red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Multi-dot: columns in groups of G; per-thread G accumulators over the
// thread's rows, warp shuffles, then one smem pass over the warps.
constexpr int G = 8;
template <typename T>
__global__ void __launch_bounds__(256) k_multi_dot(const T *__restrict__ V, int64_t ldv, int J,
                                                   const T *__restrict__ w, int64_t n,
                                                   double *__restrict__ partials) {
  __shared__ double red[8][G];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c0 = 0; c0 < J; c0 += G) {
    T acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = num<T>::zero();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
      const T wi = w[i];
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (c0 + g < J) acc[g] = acc[g] + V[(int64_t)(c0 + g) * ldv + i] * wi;
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      double s = warp_sum(num<T>::to_d(acc[g]));
      if (lane == 0) red[wid][g] = s;
    }
    __syncthreads();
    if (threadIdx.x < G && c0 + (int)threadIdx.x < J) {
      double s = 0.0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q][threadIdx.x];
      partials[(int64_t)blockIdx.x * J + c0 + threadIdx.x] = s;
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_multi_update(const T *__restrict__ V, int64_t ldv, int J,
                                                      const double *__restrict__ h, T *__restrict__ w,
                                                      int64_t n, double *__restrict__ partials) {
  extern __shared__ unsigned char smem_raw[];
  T *hs = reinterpret_cast<T *>(smem_raw);
  __shared__ double red[32];
  for (int c = threadIdx.x; c < J; c += blockDim.x) hs[c] = num<T>::from_d(-h[c]);
  __syncthreads();
  T nrm = num<T>::zero();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T r = w[i];
    for (int c = 0; c < J; ++c) r = r + V[(int64_t)c * ldv + i] * hs[c];
    w[i] = r;
    nrm = nrm + r * r;
  }
  if (partials) {
    const double s = block_sum(num<T>::to_d(nrm), red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_reconstruct(const T *__restrict__ V, int64_t ldv, int m,
                                                     const double *__restrict__ z, double *__restrict__ x,
                                                     int64_t n) {
  extern __shared__ unsigned char smem_raw[];
  T *zs = reinterpret_cast<T *>(smem_raw);
  for (int c = threadIdx.x; c < m; c += blockDim.x) zs[c] = num<T>::from_d(z[c]);
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T r = num<T>::zero();
    for (int c = 0; c < m; ++c) r = r + V[(int64_t)c * ldv + i] * zs[c];
    x[i] = num<T>::to_d(r);
  }
}

__global__ void __launch_bounds__(256) k_reduce_cols(const double *__restrict__ partials, int nb, int ncols,
                                                     int mode, double *__restrict__ out_a,
                                                     double *__restrict__ out_b) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partials[(int64_t)b * ncols + c];
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    out_a[c] = s;
    if (mode == 1) out_b[c] = s;
    if (mode == 2) out_b[c] += s;
  }
}

__global__ void __launch_bounds__(256) k_norm_finalize(const double *__restrict__ partials, int nb,
                                                       double *beta_out, double *inv_out,
                                                       const double *__restrict__ ref, int nref,
                                                       double rel, int m_here, DevStatus *st) {
  __shared__ double red[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partials[b];
  s = block_sum(s, red);
  double r2 = 0.0;
  for (int i = threadIdx.x; i < nref; i += blockDim.x) r2 += ref[i] * ref[i];
  r2 = block_sum(r2, red);
  if (threadIdx.x == 0) {
    const double beta = sqrt(s);
    const bool finite = isfinite(beta);
    bool bd = !(beta > 0.0) || (nref > 0 && beta <= rel * sqrt(r2));
    if (!finite) {
      st->bad = 1;
      bd = true;
    }
    if (bd && !st->breakdown) {
      st->breakdown = 1;
      st->m_bd = m_here;
    }
    *beta_out = finite ? (bd ? 0.0 : beta) : 0.0;
    *inv_out = bd ? 0.0 : 1.0 / beta;
  }
}

inline int grid_for(int64_t n, int bs, int max_blocks) {
  int64_t g = (n + bs - 1) / bs;
  if (g > max_blocks) g = max_blocks;
  if (g < 1) g = 1;
  return (int)g;
}

constexpr int kMaxGrid = 152 * 8;

}  // namespace

template <typename T>
int vec_from_f64(const double *in, T *out, int64_t n, cudaStream_t s) {
  k_from_f64<T><<<grid_for(n, 256, kMaxGrid), 256, 0, s>>>(in, out, n);
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template <typename T>
int vec_to_f64(const T *in, double *out, int64_t n, cudaStream_t s) {
  k_to_f64<T><<<grid_for(n, 256, kMaxGrid), 256, 0, s>>>(in, out, n);
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template <typename T>
int vec_scale(const T *in, T *out, int64_t n, double c, const double *c_dev, cudaStream_t s) {
  k_scale<T><<<grid_for(n, 256, kMaxGrid), 256, 0, s>>>(in, out, n, c, c_dev);
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template <typename T>
int vec_copy(const T *in, T *out, int64_t n, cudaStream_t s) {
  k_copy<T><<<grid_for(n, 256, kMaxGrid), 256, 0, s>>>(in, out, n);
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template <typename T>
int vec_dot_partials(const T *x, const T *y, int64_t n, double *partials, int nb, cudaStream_t s) {
  k_dot<T><<<nb, 256, 0, s>>>(x, y, n, partials);
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template <typename T>
int vec_lanczos_update(T *w, const T *vj, const T *vjm1, int64_t n, const double *alpha,
                       const double *beta_prev, double *partials, int nb, cudaStream_t s) {
  k_lanczos_update<T><<<nb, 256, 0, s>>>(w, vj, vjm1, n, alpha, beta_prev, partials);
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template <typename T>
int vec_multi_dot(const T *V, int64_t ldv, int J, const T *w, int64_t n, double *partials, int nb,
                  cudaStream_t s) {
  k_multi_dot<T><<<nb, 256, 0, s>>>(V, ldv, J, w, n, partials);
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template <typename T>
int vec_multi_update(const T *V, int64_t ldv, int J, const double *h, T *w, int64_t n,
                     double *partials, int nb, cudaStream_t s) {
  const size_t sm = (size_t)J * sizeof(T);
  if (sm > 48 * 1024) PP_CUDA_TRY(cudaFuncSetAttribute(k_multi_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_multi_update<T><<<nb, 256, sm, s>>>(V, ldv, J, h, w, n, partials);
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template <typename T>
int vec_reconstruct(const T *V, int64_t ldv, int m, const double *z, double *x, int64_t n,
                    cudaStream_t s) {
  const size_t sm = (size_t)m * sizeof(T);
  if (sm > 48 * 1024) PP_CUDA_TRY(cudaFuncSetAttribute(k_reconstruct<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_reconstruct<T><<<grid_for(n, 256, kMaxGrid), 256, sm, s>>>(V, ldv, m, z, x, n);
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}

int reduce_cols(const double *partials, int nb, int ncols, int mode, double *out_a, double *out_b,
                cudaStream_t s) {
  k_reduce_cols<<<ncols, 256, 0, s>>>(partials, nb, ncols, mode, out_a, out_b);
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}

int norm_finalize(const double *partials, int nb, double *beta_out, double *inv_out,
                  const double *ref, int nref, double rel, int m_here, DevStatus *st,
                  cudaStream_t s) {
  k_norm_finalize<<<1, 256, 0, s>>>(partials, nb, beta_out, inv_out, ref, nref, rel, m_here, st);
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}

#define PP_INST(T)                                                                                  \
  template int vec_from_f64<T>(const double *, T *, int64_t, cudaStream_t);                       \
  template int vec_to_f64<T>(const T *, double *, int64_t, cudaStream_t);                         \
  template int vec_scale<T>(const T *, T *, int64_t, double, const double *, cudaStream_t);       \
  template int vec_copy<T>(const T *, T *, int64_t, cudaStream_t);                                \
  template int vec_dot_partials<T>(const T *, const T *, int64_t, double *, int, cudaStream_t);   \
  template int vec_lanczos_update<T>(T *, const T *, const T *, int64_t, const double *,          \
                                     const double *, double *, int, cudaStream_t);                \
  template int vec_multi_dot<T>(const T *, int64_t, int, const T *, int64_t, double *, int,       \
                                cudaStream_t);                                                    \
  template int vec_multi_update<T>(const T *, int64_t, int, const double *, T *, int64_t, double *, \
                                   int, cudaStream_t);                                            \
  template int vec_reconstruct<T>(const T *, int64_t, int, const double *, double *, int64_t,     \
                                  cudaStream_t);
PP_INST(double)
PP_INST(dw)
