// Vector kernels of the Krylov process: conversions at the API boundary,
// inner products, the Lanczos three-term update, classical Gram-Schmidt
// sweeps against the stored basis (the orthogonalization loop of
// Algorithm 1, done as two CGS passes), and the reconstruction f_m = V_m z
// (the final step of Algorithm 1).
//
// Layout: every block owns a chunk of CHUNK = 2048 consecutive rows; thread t
// owns rows chunk + t + 256 u, u < 8, so each column sweep issues 8
// independent coalesced loads per thread.  Products accumulate in the vector
// arithmetic (FP64, FP32, or the compensated double-word accumulator); warp
// reductions stay in that arithmetic and only the 8 warp sums of a block are
// widened to FP64, so every block writes one FP64 partial per column and a
// fixed-order pass over the partials finishes the sum (results are bitwise
// reproducible run to run).
//
// Segments (Seg): a vector may be the concatenation of several independent
// problems ("segments", each padded to whole chunks, padding kept at zero).
// A block finds its segment from the chunk table, skips inactive segments,
// and reads its per-segment FP64 scalars at base + segment * dstride.  A
// single vector is the case nseg = 1.
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int TPB = 256;
constexpr int U = 8;
constexpr int CHUNK = TPB * U;
constexpr int CG = 8;  // columns per block in the multi-dot
constexpr int kUpdateDotTileMaxJ = 32;  // widest J of the shared-memory fused sweep

__device__ __forceinline__ double warp_reduce_d(double v) { return warp_sum(v); }
__device__ __forceinline__ float warp_reduce_d(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ dw warp_reduce_d(dw v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dw t = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = v + t;
  }
  return v;
}

// Block sum of per-thread values in arithmetic T; result (FP64) valid in thread 0.
template <typename T>
__device__ __forceinline__ double block_reduce_to_d(T v, double *red) {
  v = warp_reduce_d(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = num<T>::to_d(v);
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < TPB / 32; ++i) s += red[i];
  return s;
}

// Segment of the chunk a block owns, and whether it still iterates.
__device__ __forceinline__ int chunk_seg(const Seg &S, int64_t chunk) {
  return S.chunk_seg ? __ldg(S.chunk_seg + chunk) : 0;
}
__device__ __forceinline__ bool seg_active(const Seg &S, int seg) {
  return !S.active || __ldg(S.active + seg) != 0;
}

template <typename T>
__global__ void k_from_f64(const double *__restrict__ in, T *__restrict__ out, int64_t n) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = num<T>::from_d(in[i]);
}

template <typename T>
__global__ void k_to_f64(const T *__restrict__ in, double *__restrict__ out, int64_t n) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = num<T>::to_d(in[i]);
}

// Fixed pseudo-random vector in [-1, 1): splitmix64 of (seed + index).
template <typename T>
__global__ void k_fill_hash(T *__restrict__ out, int64_t n, uint64_t seed) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    out[i] = num<T>::from_d((double)(z >> 11) * 0x1p-52 - 1.0);
  }
}

template <typename TI, typename TO>
__global__ void k_convert(const TI *__restrict__ in, TO *__restrict__ out, int64_t n) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (std::is_same<TI, dw>::value && std::is_same<TO, float>::value) {
      // one FP32 addition rounds hi + lo correctly (no FP64 pipe, no double rounding)
      const dw v = in[i];
      out[i] = __fadd_rn(v.hi, v.lo);
    } else {
      out[i] = num<TO>::from_d(num<TI>::to_d(in[i]));
    }
  }
}

// out = in * (c * c_dev[segment]) (c_dev may be NULL); inactive segments untouched
template <typename T>
__global__ void __launch_bounds__(TPB) k_scale(const T *__restrict__ in, T *__restrict__ out, int64_t n, double c,
                                               const double *__restrict__ c_dev, Seg S) {
  pdl_wait();
  pdl_trigger();
  const int seg = chunk_seg(S, blockIdx.x);
  if (!seg_active(S, seg)) return;
  const double cc = c_dev ? c * c_dev[seg * S.dstride] : c;
  const T ct = num<T>::from_d(cc);
  const int64_t base = (int64_t)blockIdx.x * CHUNK + threadIdx.x;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t r = base + (int64_t)u * TPB;
    if (r < n) out[r] = in[r] * ct;
  }
}

// out = 1 / in (0 for in = 0), one value
__global__ void k_recip(const double *__restrict__ in, double *__restrict__ out) {
  pdl_wait();
  pdl_trigger();
  if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = in[0] != 0.0 ? 1.0 / in[0] : 0.0;
}

template <typename T>
__global__ void k_copy(const T *__restrict__ in, T *__restrict__ out, int64_t n) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}

// partials[chunk] = sum over the chunk of x.y
template <typename T>
__global__ void __launch_bounds__(TPB) k_dot(const T *__restrict__ x, const T *__restrict__ y, int64_t n,
                                             double *__restrict__ partials, Seg S) {
  pdl_wait();
  pdl_trigger();
  using A = typename acc_of<T>::type;
  __shared__ double red[TPB / 32];
  if (!seg_active(S, chunk_seg(S, blockIdx.x))) {
    if (threadIdx.x == 0) partials[blockIdx.x] = 0.0;
    return;
  }
  const int64_t base = (int64_t)blockIdx.x * CHUNK + threadIdx.x;
  A acc;
  acc_set(acc, num<T>::zero());
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t r = base + (int64_t)u * TPB;
    if (r < n) acc_add_prod(acc, ldg(x + r), ldg(y + r));
  }
  const double s = block_reduce_to_d(acc_get(acc), red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// w -= alpha v_j + beta v_{j-1}; partials[chunk] = ||w||^2 over the chunk
template <typename T>
__global__ void __launch_bounds__(TPB) k_lanczos_update(T *__restrict__ w, const T *__restrict__ vj,
                                                        const T *__restrict__ vjm1, int64_t n,
                                                        const double *__restrict__ alpha,
                                                        const double *__restrict__ beta_prev,
                                                        double *__restrict__ partials, Seg S) {
  pdl_wait();
  pdl_trigger();
  using A = typename acc_of<T>::type;
  __shared__ double red[TPB / 32];
  const int seg = chunk_seg(S, blockIdx.x);
  if (!seg_active(S, seg)) {
    if (threadIdx.x == 0) partials[blockIdx.x] = 0.0;
    return;
  }
  const T a = num<T>::from_d(-alpha[seg * S.dstride]);
  const T b = num<T>::from_d(vjm1 ? -beta_prev[seg * S.dstride] : 0.0);
  const int64_t base = (int64_t)blockIdx.x * CHUNK + threadIdx.x;
  A nrm;
  acc_set(nrm, num<T>::zero());
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t r = base + (int64_t)u * TPB;
    if (r < n) {
      A acc;
      acc_set(acc, w[r]);
      acc_add_prod(acc, a, ldg(vj + r));
      if (vjm1) acc_add_prod(acc, b, ldg(vjm1 + r));
      const T wr = acc_get(acc);
      w[r] = wr;
      acc_add_prod(nrm, wr, wr);
    }
  }
  const double s = block_reduce_to_d(acc_get(nrm), red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__device__ __forceinline__ float bfly_shfl(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double bfly_shfl(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ dw bfly_shfl(dw v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

// Warp reduce-scatter of K (8 or 16) values per lane by recursive halving:
// at the offsets 16, 8, ... (log2 K of them) a lane keeps one half of its
// values, sends the other half to its partner and adds what it receives;
// the remaining offsets complete the sum.  K - 1 + 5 - log2 K additions
// instead of 5 K for K separate reductions, with the same pairing of lanes
// as warp_reduce_d (offset 16 first), so each total is bit for bit the
// separate reduction's.  Afterwards lane l holds the warp total of value
// rs_index<K>(l); rs_writer<K>(l) picks one lane per value.
template <int K>
__device__ __forceinline__ int rs_index(int lane) {
  static_assert(K == 8 || K == 16, "reduce-scatter of 8 or 16 values");
  return K == 16 ? (lane >> 1) & 15 : (lane >> 2) & 7;
}
template <int K>
__device__ __forceinline__ bool rs_writer(int lane) {
  return (lane & (32 / K - 1)) == 0;
}
template <int K, typename T>
__device__ __forceinline__ T warp_reduce_scatter(T (&v)[K], int lane) {
  static_assert(K == 8 || K == 16, "reduce-scatter of 8 or 16 values");
#pragma unroll
  for (int h = K / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const T send = up ? v[i] : v[i + h];
      const T keep = up ? v[i + h] : v[i];
      v[i] = keep + bfly_shfl(send, o);
    }
  }
  T r = v[0];
#pragma unroll
  for (int o = K == 16 ? 1 : 2; o >= 1; o >>= 1) r = r + bfly_shfl(r, o);
  return r;
}

// partials[chunk*J + c] = sum over the chunk of V_c . w, for the CG columns
// c = blockIdx.y*CG + g of this block.
template <typename T>
__global__ void __launch_bounds__(TPB, sizeof(T) == 4 ? 4 : 3) k_multi_dot(const T *__restrict__ V, int64_t ldv, int J,
                                                   const T *__restrict__ w, int64_t n,
                                                   double *__restrict__ partials, Seg S) {
  pdl_wait();
  pdl_trigger();
  using A = typename acc_of<T>::type;
  __shared__ double red[CG][TPB / 32];
  const int c0 = blockIdx.y * CG;
  const int ncol = min(CG, J - c0);
  if (!seg_active(S, chunk_seg(S, blockIdx.x))) {
    if (threadIdx.x < ncol) partials[(int64_t)blockIdx.x * J + c0 + threadIdx.x] = 0.0;
    return;
  }
  const int64_t base = (int64_t)blockIdx.x * CHUNK + threadIdx.x;
  T wv[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t r = base + (int64_t)u * TPB;
    wv[u] = (r < n) ? ldg(w + r) : num<T>::zero();
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // CU columns per pass, their loads issued together; the block's CG column
  // sums stay in registers until one reduce-scatter
  constexpr int CU = sizeof(T) == 4 ? 4 : 2;
  A acc[CG];
#pragma unroll
  for (int q = 0; q < CG; ++q) acc_set(acc[q], num<T>::zero());
#pragma unroll
  for (int g0 = 0; g0 < CG; g0 += CU) {
    if (g0 < ncol) {  // uniform over the block
      T vals[CU][U];
#pragma unroll
      for (int q = 0; q < CU; ++q) {
        const T *col = V + (int64_t)(c0 + min(g0 + q, ncol - 1)) * ldv;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t r = base + (int64_t)u * TPB;
          vals[q][u] = (r < n && g0 + q < ncol) ? ldg(col + r) : num<T>::zero();
        }
      }
#pragma unroll
      for (int q = 0; q < CU; ++q)
        if (g0 + q < ncol) {
#pragma unroll
          for (int u = 0; u < U; ++u)
            if (base + (int64_t)u * TPB < n) acc_add_prod(acc[g0 + q], vals[q][u], wv[u]);
        }
    }
  }
  T v[CG];
#pragma unroll
  for (int q = 0; q < CG; ++q) v[q] = acc_get(acc[q]);
  const T tot = warp_reduce_scatter<CG>(v, lane);
  const int idx = rs_index<CG>(lane);
  if (rs_writer<CG>(lane) && idx < ncol) red[idx][wid] = num<T>::to_d(tot);
  __syncthreads();
  if (threadIdx.x < ncol) {
    double s = 0.0;
    for (int q = 0; q < TPB / 32; ++q) s += red[threadIdx.x][q];
    partials[(int64_t)blockIdx.x * J + c0 + threadIdx.x] = s;
  }
}

// w -= V h (h: J FP64 values per segment on the device); optional ||w||^2 partials
template <typename T>
__global__ void __launch_bounds__(TPB) k_multi_update(const T *__restrict__ V, int64_t ldv, int J,
                                                      const double *__restrict__ h, T *__restrict__ w,
                                                      int64_t n, double *__restrict__ partials, Seg S) {
  pdl_wait();
  pdl_trigger();
  using A = typename acc_of<T>::type;
  extern __shared__ unsigned char smem_raw[];
  T *hs = reinterpret_cast<T *>(smem_raw);
  __shared__ double red[TPB / 32];
  const int seg = chunk_seg(S, blockIdx.x);
  if (!seg_active(S, seg)) {
    if (partials && threadIdx.x == 0) partials[blockIdx.x] = 0.0;
    return;
  }
  const double *hseg = h + seg * S.dstride;
  for (int c = threadIdx.x; c < J; c += TPB) hs[c] = num<T>::from_d(-hseg[c]);
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * CHUNK + threadIdx.x;
  A acc[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t r = base + (int64_t)u * TPB;
    acc_set(acc[u], (r < n) ? w[r] : num<T>::zero());
  }
  // CU columns per pass: all their loads are issued before the (in-order)
  // accumulation, for more memory-level parallelism
  constexpr int CU = sizeof(T) == 4 ? 4 : 2;
  int c = 0;
  for (; c + CU <= J; c += CU) {
    T vals[CU][U];
#pragma unroll
    for (int q = 0; q < CU; ++q) {
      const T *col = V + (int64_t)(c + q) * ldv;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t r = base + (int64_t)u * TPB;
        vals[q][u] = (r < n) ? ldg(col + r) : num<T>::zero();
      }
    }
#pragma unroll
    for (int q = 0; q < CU; ++q) {
      const T hc = hs[c + q];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (base + (int64_t)u * TPB < n) acc_add_prod(acc[u], hc, vals[q][u]);
    }
  }
  for (; c < J; ++c) {
    const T *col = V + (int64_t)c * ldv;
    const T hc = hs[c];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t r = base + (int64_t)u * TPB;
      if (r < n) acc_add_prod(acc[u], hc, ldg(col + r));
    }
  }
  A nrm;
  acc_set(nrm, num<T>::zero());
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t r = base + (int64_t)u * TPB;
    if (r < n) {
      const T wr = acc_get(acc[u]);
      w[r] = wr;
      acc_add_prod(nrm, wr, wr);
    }
  }
  if (partials) {
    const double s = block_reduce_to_d(acc_get(nrm), red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
  }
}

// First CGS pass's update fused with the second pass's inner products:
// w <- w - V h, then partials[chunk*J + c] = sum over the chunk of V_c . w.
// Each thread keeps its row's J basis entries in registers between the two,
// so V is read from HBM once; w's update and the per-column accumulation
// follow k_multi_update and k_multi_dot step for step (same results).
template <typename T, int JMAX>
__global__ void __launch_bounds__(TPB) k_update_dot(const T *__restrict__ V, int64_t ldv, int J,
                                                    const double *__restrict__ h, T *__restrict__ w, int64_t n,
                                                    double *__restrict__ partials, Seg S) {
  pdl_wait();
  pdl_trigger();
  using A = typename acc_of<T>::type;
  __shared__ T hs[JMAX];
  __shared__ double red[JMAX][TPB / 32];
  const int seg = chunk_seg(S, blockIdx.x);
  if (!seg_active(S, seg)) {
    if (threadIdx.x < J) partials[(int64_t)blockIdx.x * J + threadIdx.x] = 0.0;
    return;
  }
  const double *hseg = h + seg * S.dstride;
  for (int c = threadIdx.x; c < J; c += TPB) hs[c] = num<T>::from_d(-hseg[c]);
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * CHUNK + threadIdx.x;
  A dacc[JMAX];
#pragma unroll
  for (int c = 0; c < JMAX; ++c) acc_set(dacc[c], num<T>::zero());
#pragma unroll 1
  for (int u = 0; u < U; ++u) {
    const int64_t r = base + (int64_t)u * TPB;
    if (r >= n) break;
    T vv[JMAX];
#pragma unroll
    for (int c = 0; c < JMAX; ++c) vv[c] = c < J ? ldg(V + (int64_t)c * ldv + r) : num<T>::zero();
    A acc;
    acc_set(acc, w[r]);
#pragma unroll
    for (int c = 0; c < JMAX; ++c)
      if (c < J) acc_add_prod(acc, hs[c], vv[c]);
    const T wr = acc_get(acc);
    w[r] = wr;
#pragma unroll
    for (int c = 0; c < JMAX; ++c)
      if (c < J) acc_add_prod(dacc[c], vv[c], wr);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T dv[JMAX];
#pragma unroll
  for (int c = 0; c < JMAX; ++c) dv[c] = acc_get(dacc[c]);
  const T tot = warp_reduce_scatter<JMAX>(dv, lane);
  const int idx = rs_index<JMAX>(lane);
  if (rs_writer<JMAX>(lane) && idx < J) red[idx][wid] = num<T>::to_d(tot);
  __syncthreads();
  if (threadIdx.x < J) {
    double sum = 0.0;
    for (int q = 0; q < TPB / 32; ++q) sum += red[threadIdx.x][q];
    partials[(int64_t)blockIdx.x * J + threadIdx.x] = sum;
  }
}

// The same fused sweep for wider J: the chunk's rows go through shared
// memory in tiles of TPB rows (one row per thread): the tile of V (J
// columns) is loaded once, each thread updates its row of w from it, and
// the block then forms the J inner products of the tile with the updated w
// from shared memory (warp g takes columns g, g + 8, ...; lane l rows
// l + 32 k), accumulated over the chunk's tiles in a fixed order.  V is read
// from HBM once instead of twice.
template <typename T>
__global__ void __launch_bounds__(TPB) k_update_dot_tile(const T *__restrict__ V, int64_t ldv, int J,
                                                         const double *__restrict__ h, T *__restrict__ w,
                                                         int64_t n, double *__restrict__ partials, Seg S) {
  pdl_wait();
  pdl_trigger();
  using A = typename acc_of<T>::type;
  extern __shared__ unsigned char smem_raw[];
  T *hs = reinterpret_cast<T *>(smem_raw);  // -h, J entries
  T *wn = hs + J;                            // the tile's updated w, TPB entries
  T *vt = wn + TPB;                          // V tile, [column][row], J x TPB
  const int seg = chunk_seg(S, blockIdx.x);
  if (!seg_active(S, seg)) {
    for (int c = threadIdx.x; c < J; c += TPB) partials[(int64_t)blockIdx.x * J + c] = 0.0;
    return;
  }
  const double *hseg = h + seg * S.dstride;
  for (int c = threadIdx.x; c < J; c += TPB) hs[c] = num<T>::from_d(-hseg[c]);
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int NW = TPB / 32;
  constexpr int CMAX = kUpdateDotTileMaxJ / NW;  // columns per warp
  A dacc[CMAX];
#pragma unroll
  for (int q = 0; q < CMAX; ++q) acc_set(dacc[q], num<T>::zero());
  const int64_t base = (int64_t)blockIdx.x * CHUNK;
  for (int u = 0; u < U; ++u) {
    const int64_t r = base + (int64_t)u * TPB + threadIdx.x;
    const bool ok = r < n;
    for (int c = 0; c < J; ++c) vt[c * TPB + threadIdx.x] = ok ? ldg(V + (int64_t)c * ldv + r) : num<T>::zero();
    A acc;
    acc_set(acc, ok ? w[r] : num<T>::zero());
    for (int c = 0; c < J; ++c) acc_add_prod(acc, hs[c], vt[c * TPB + threadIdx.x]);
    const T wr = acc_get(acc);
    if (ok) w[r] = wr;
    wn[threadIdx.x] = wr;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < CMAX; ++q) {
      const int c = wid + q * NW;
      if (c < J) {
#pragma unroll
        for (int k = 0; k < TPB / 32; ++k)
          acc_add_prod(dacc[q], vt[c * TPB + lane + 32 * k], wn[lane + 32 * k]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < CMAX; ++q) {
    const int c = wid + q * NW;
    if (c < J) {
      const T sc = warp_reduce_d(acc_get(dacc[q]));
      if (lane == 0) partials[(int64_t)blockIdx.x * J + c] = num<T>::to_d(sc);
    }
  }
}

// x = V z (x += V z with accumulate), FP64 output; m columns, or m_seg[segment]
template <typename T>
__global__ void __launch_bounds__(TPB) k_reconstruct(const T *__restrict__ V, int64_t ldv, int m,
                                                     const int *__restrict__ m_seg,
                                                     const double *__restrict__ z, double *__restrict__ x,
                                                     int64_t n, int accumulate, Seg S) {
  pdl_wait();
  pdl_trigger();
  using A = typename acc_of<T>::type;
  extern __shared__ unsigned char smem_raw[];
  T *zs = reinterpret_cast<T *>(smem_raw);
  const int seg = chunk_seg(S, blockIdx.x);
  const int mm = m_seg ? min(m, m_seg[seg]) : m;
  const double *zseg = z + seg * S.dstride;
  for (int c = threadIdx.x; c < mm; c += TPB) zs[c] = num<T>::from_d(zseg[c]);
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * CHUNK + threadIdx.x;
  A acc[U];
#pragma unroll
  for (int u = 0; u < U; ++u) acc_set(acc[u], num<T>::zero());
  double prev[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t r = base + (int64_t)u * TPB;
    prev[u] = (accumulate && r < n) ? x[r] : 0.0;
  }
  for (int c = 0; c < mm; ++c) {
    const T *col = V + (int64_t)c * ldv;
    const T zc = zs[c];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t r = base + (int64_t)u * TPB;
      if (r < n) acc_add_prod(acc[u], zc, ldg(col + r));
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int64_t r = base + (int64_t)u * TPB;
    if (r < n) x[r] = prev[u] + num<T>::to_d(acc_get(acc[u]));
  }
}

// Per (column, segment) sum of the chunk partials of the segment's chunks.
__global__ void __launch_bounds__(256) k_reduce_cols(const double *__restrict__ partials, int nb, int ncols,
                                                     int mode, double *__restrict__ out_a,
                                                     double *__restrict__ out_b, Seg S) {
  pdl_wait();
  pdl_trigger();
  __shared__ double red[32];
  const int c = blockIdx.x, seg = blockIdx.y;
  if (!seg_active(S, seg)) return;
  const int b0 = S.chunk0 ? S.chunk0[seg] : 0, b1 = S.chunk0 ? S.chunk0[seg + 1] : nb;
  double s = 0.0;
  for (int b = b0 + threadIdx.x; b < b1; b += blockDim.x) s += partials[(int64_t)b * ncols + c];
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    const int64_t o = seg * S.dstride + c;
    out_a[o] = s;
    if (mode == 1) out_b[o] = s;
    if (mode == 2) out_b[o] += s;
  }
}

// Per segment: beta = sqrt(sum of the segment's partials), breakdown test
// against ||ref||, 1/beta for the normalisation.
__global__ void __launch_bounds__(256) k_norm_finalize(const double *__restrict__ partials, int nb,
                                                       double *beta_out, double *inv_out,
                                                       const double *__restrict__ ref, int nref,
                                                       double rel, int m_here, DevStatus *st, Seg S) {
  pdl_wait();
  pdl_trigger();
  __shared__ double red[32];
  const int seg = blockIdx.x;
  if (!seg_active(S, seg)) return;
  const int b0 = S.chunk0 ? S.chunk0[seg] : 0, b1 = S.chunk0 ? S.chunk0[seg + 1] : nb;
  const int64_t so = seg * S.dstride;
  DevStatus *sts = st + seg;
  double s = 0.0;
  for (int b = b0 + threadIdx.x; b < b1; b += blockDim.x) s += partials[b];
  s = block_sum(s, red);
  double r2 = 0.0;
  if (ref)
    for (int i = threadIdx.x; i < nref; i += blockDim.x) r2 += ref[so + i] * ref[so + i];
  r2 = block_sum(r2, red);
  if (threadIdx.x == 0) {
    const double beta = sqrt(s);
    const bool finite = isfinite(beta);
    bool bd = !(beta > 0.0) || (nref > 0 && beta <= rel * sqrt(r2));
    if (!finite) {
      sts->bad = 1;
      bd = true;
    }
    if (bd && !sts->breakdown) {
      sts->breakdown = 1;
      sts->m_bd = m_here;
    }
    beta_out[so] = finite ? (bd ? 0.0 : beta) : 0.0;
    inv_out[so] = bd ? 0.0 : 1.0 / beta;
  }
}

inline int grid_for(int64_t n, int bs, int max_blocks) {
  int64_t g = (n + bs - 1) / bs;
  if (g > max_blocks) g = max_blocks;
  if (g < 1) g = 1;
  return (int)g;
}

constexpr int kMaxGrid = 152 * 8;

inline unsigned nchunks(int64_t n) { return (unsigned)((n + CHUNK - 1) / CHUNK); }

// ---- complex vectors ----
// n reals = n/2 complex entries, (re, im) interleaved.  Same chunks as the
// real kernels (CHUNK reals = CHUNK/2 entries per block, so the chunk
// partials line up); thread t owns entries chunk/2 + t + TPB u, u < UC.
constexpr int UC = U / 2;

// partials[chunk*2J + 2c + {0,1}] = sum over the chunk of conj(V_c) w
// (re: vr wr + vi wi, im: vr wi - vi wr), for the CG columns of this block.
template <typename T>
__global__ void __launch_bounds__(TPB) k_multi_dot_c(const T *__restrict__ V, int64_t ldv, int J,
                                                     const T *__restrict__ w, int64_t n,
                                                     double *__restrict__ partials) {
  pdl_wait();
  pdl_trigger();
  using A = typename acc_of<T>::type;
  __shared__ double red[2 * CG][TPB / 32];
  const int c0 = blockIdx.y * CG;
  const int ncol = min(CG, J - c0);
  const int64_t e0 = (int64_t)blockIdx.x * (CHUNK / 2) + threadIdx.x;
  T wr[UC], wi[UC];
#pragma unroll
  for (int u = 0; u < UC; ++u) {
    const int64_t r = 2 * (e0 + (int64_t)u * TPB);
    wr[u] = (r < n) ? ldg(w + r) : num<T>::zero();
    wi[u] = (r < n) ? ldg(w + r + 1) : num<T>::zero();
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int CU = sizeof(T) == 4 ? 4 : 2;
  for (int g0 = 0; g0 < ncol; g0 += CU) {
    T vr[CU][UC], vi[CU][UC];
#pragma unroll
    for (int q = 0; q < CU; ++q) {
      const T *col = V + (int64_t)(c0 + min(g0 + q, ncol - 1)) * ldv;
#pragma unroll
      for (int u = 0; u < UC; ++u) {
        const int64_t r = 2 * (e0 + (int64_t)u * TPB);
        const bool ok = r < n && g0 + q < ncol;
        vr[q][u] = ok ? ldg(col + r) : num<T>::zero();
        vi[q][u] = ok ? ldg(col + r + 1) : num<T>::zero();
      }
    }
#pragma unroll
    for (int q = 0; q < CU; ++q) {
      if (g0 + q >= ncol) break;
      A ar, ai;
      acc_set(ar, num<T>::zero());
      acc_set(ai, num<T>::zero());
#pragma unroll
      for (int u = 0; u < UC; ++u) {
        acc_add_prod(ar, vr[q][u], wr[u]);
        acc_add_prod(ar, vi[q][u], wi[u]);
        acc_add_prod(ai, vr[q][u], wi[u]);
        acc_add_prod(ai, -vi[q][u], wr[u]);
      }
      const T sr = warp_reduce_d(acc_get(ar));
      const T si = warp_reduce_d(acc_get(ai));
      if (lane == 0) {
        red[2 * (g0 + q)][wid] = num<T>::to_d(sr);
        red[2 * (g0 + q) + 1][wid] = num<T>::to_d(si);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * ncol) {
    double sum = 0.0;
    for (int q = 0; q < TPB / 32; ++q) sum += red[threadIdx.x][q];
    partials[(int64_t)blockIdx.x * 2 * J + 2 * c0 + threadIdx.x] = sum;
  }
}

// w -= V h (h: J complex FP64 values); optional ||w||^2 partials
template <typename T>
__global__ void __launch_bounds__(TPB) k_multi_update_c(const T *__restrict__ V, int64_t ldv, int J,
                                                        const double *__restrict__ h, T *__restrict__ w,
                                                        int64_t n, double *__restrict__ partials) {
  pdl_wait();
  pdl_trigger();
  using A = typename acc_of<T>::type;
  extern __shared__ unsigned char smem_raw[];
  T *hr = reinterpret_cast<T *>(smem_raw);  // -Re h, -Im h, +Im h
  T *hi = hr + J;
  T *hni = hi + J;
  __shared__ double red[TPB / 32];
  for (int c = threadIdx.x; c < J; c += TPB) {
    hr[c] = num<T>::from_d(-h[2 * c]);
    hi[c] = num<T>::from_d(-h[2 * c + 1]);
    hni[c] = num<T>::from_d(h[2 * c + 1]);
  }
  __syncthreads();
  const int64_t e0 = (int64_t)blockIdx.x * (CHUNK / 2) + threadIdx.x;
  A ar[UC], ai[UC];
#pragma unroll
  for (int u = 0; u < UC; ++u) {
    const int64_t r = 2 * (e0 + (int64_t)u * TPB);
    acc_set(ar[u], (r < n) ? w[r] : num<T>::zero());
    acc_set(ai[u], (r < n) ? w[r + 1] : num<T>::zero());
  }
  // (-h)(v) = (-hr vr + hi vi) + i (-hr vi - hi vr) with hr, hi the parts of h
  for (int c = 0; c < J; ++c) {
    const T *col = V + (int64_t)c * ldv;
    T vr[UC], vi[UC];
#pragma unroll
    for (int u = 0; u < UC; ++u) {
      const int64_t r = 2 * (e0 + (int64_t)u * TPB);
      vr[u] = (r < n) ? ldg(col + r) : num<T>::zero();
      vi[u] = (r < n) ? ldg(col + r + 1) : num<T>::zero();
    }
    const T a = hr[c], b = hi[c], nb = hni[c];
#pragma unroll
    for (int u = 0; u < UC; ++u) {
      acc_add_prod(ar[u], a, vr[u]);
      acc_add_prod(ar[u], nb, vi[u]);
      acc_add_prod(ai[u], a, vi[u]);
      acc_add_prod(ai[u], b, vr[u]);
    }
  }
  A nrm;
  acc_set(nrm, num<T>::zero());
#pragma unroll
  for (int u = 0; u < UC; ++u) {
    const int64_t r = 2 * (e0 + (int64_t)u * TPB);
    if (r < n) {
      const T xr = acc_get(ar[u]), xi = acc_get(ai[u]);
      w[r] = xr;
      w[r + 1] = xi;
      acc_add_prod(nrm, xr, xr);
      acc_add_prod(nrm, xi, xi);
    }
  }
  if (partials) {
    const double sum = block_reduce_to_d(acc_get(nrm), red);
    if (threadIdx.x == 0) partials[blockIdx.x] = sum;
  }
}

// x = V z (x += V z with accumulate), z complex, FP64 output
template <typename T>
__global__ void __launch_bounds__(TPB) k_reconstruct_c(const T *__restrict__ V, int64_t ldv, int m,
                                                       const double *__restrict__ z, double *__restrict__ x,
                                                       int64_t n, int accumulate) {
  pdl_wait();
  pdl_trigger();
  using A = typename acc_of<T>::type;
  extern __shared__ unsigned char smem_raw[];
  T *zr = reinterpret_cast<T *>(smem_raw);
  T *zi = zr + m;
  T *zni = zi + m;
  for (int c = threadIdx.x; c < m; c += TPB) {
    zr[c] = num<T>::from_d(z[2 * c]);
    zi[c] = num<T>::from_d(z[2 * c + 1]);
    zni[c] = num<T>::from_d(-z[2 * c + 1]);
  }
  __syncthreads();
  const int64_t e0 = (int64_t)blockIdx.x * (CHUNK / 2) + threadIdx.x;
  A ar[UC], ai[UC];
#pragma unroll
  for (int u = 0; u < UC; ++u) {
    acc_set(ar[u], num<T>::zero());
    acc_set(ai[u], num<T>::zero());
  }
  for (int c = 0; c < m; ++c) {
    const T *col = V + (int64_t)c * ldv;
    const T a = zr[c], b = zi[c], nb = zni[c];
#pragma unroll
    for (int u = 0; u < UC; ++u) {
      const int64_t r = 2 * (e0 + (int64_t)u * TPB);
      if (r < n) {
        const T vr = ldg(col + r), vi = ldg(col + r + 1);
        acc_add_prod(ar[u], a, vr);
        acc_add_prod(ar[u], nb, vi);
        acc_add_prod(ai[u], a, vi);
        acc_add_prod(ai[u], b, vr);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < UC; ++u) {
    const int64_t r = 2 * (e0 + (int64_t)u * TPB);
    if (r < n) {
      const double pr = accumulate ? x[r] : 0.0, pi = accumulate ? x[r + 1] : 0.0;
      x[r] = pr + num<T>::to_d(acc_get(ar[u]));
      x[r + 1] = pi + num<T>::to_d(acc_get(ai[u]));
    }
  }
}

// out = (cr + i ci) in
template <typename T>
__global__ void __launch_bounds__(TPB) k_scale_c(const T *__restrict__ in, T *__restrict__ out, int64_t n,
                                                 double cr, double ci) {
  pdl_wait();
  pdl_trigger();
  using A = typename acc_of<T>::type;
  const T a = num<T>::from_d(cr), b = num<T>::from_d(ci), nb = num<T>::from_d(-ci);
  const int64_t e0 = (int64_t)blockIdx.x * (CHUNK / 2) + threadIdx.x;
#pragma unroll
  for (int u = 0; u < UC; ++u) {
    const int64_t r = 2 * (e0 + (int64_t)u * TPB);
    if (r < n) {
      const T xr = ldg(in + r), xi = ldg(in + r + 1);
      A yr, yi;
      acc_set_prod(yr, a, xr);
      acc_add_prod(yr, nb, xi);
      acc_set_prod(yi, a, xi);
      acc_add_prod(yi, b, xr);
      out[r] = acc_get(yr);
      out[r + 1] = acc_get(yi);
    }
  }
}


// ---- Arnoldi with delayed reorthogonalization (opts.orth = PP_ORTH_DCGS2) ----
//
// Step j holds the final basis columns V_0..V_{j-1} and, in column j, the
// candidate u_j = w_{j-1} - V h1 left by the previous step's single
// Gram-Schmidt pass (unnormalized); y = A q(A)^2 u_j is applied to it before
// it is reorthogonalized.  One sweep forms s = V^T u, t = V^T y, a = u.u,
// g = u.y; a one-block kernel turns them into v_j = (u - V s)/beta, beta^2 =
// a - s.s (the second CGS pass of column j-1, whose h is h1 + s), and the
// first-pass coefficients of A q(A)^2 v_j = (y - V H s)/beta (linearity and
// the Arnoldi relation of the earlier columns); a second sweep writes v_j
// and the next candidate u_{j+1} = y/beta - V d - e u.  Two sweeps over V
// per step instead of the three of CGS2 plus the normalization pass.

// partials[chunk*(2J+2) + c]: c < J: V_c.u, J + c: V_c.y, 2J: u.u, 2J+1: u.y

template <typename T>
__global__ void __launch_bounds__(TPB, sizeof(T) == 4 ? 3 : 2) k_dot2(const T *__restrict__ V, int64_t ldv, int J, const T *__restrict__ u,
                                              const T *__restrict__ y, int64_t n, double *__restrict__ partials) {
  pdl_wait();
  pdl_trigger();
  using A = typename acc_of<T>::type;
  static_assert(CG == 8, "the reduce-scatter takes 2 x 8 column sums");
  __shared__ double red[2 * CG + 2][TPB / 32];
  const int c0 = blockIdx.y * CG;
  const int ncol = max(0, min(CG, J - c0));
  const int64_t base = (int64_t)blockIdx.x * CHUNK + threadIdx.x;
  const int64_t stride = 2 * (int64_t)J + 2;
  T uv[U], yv[U];
#pragma unroll
  for (int k = 0; k < U; ++k) {
    const int64_t r = base + (int64_t)k * TPB;
    uv[k] = (r < n) ? ldg(u + r) : num<T>::zero();
    yv[k] = (r < n) ? ldg(y + r) : num<T>::zero();
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (blockIdx.y == 0) {  // u.u and u.y
    A aa, ag;
    acc_set(aa, num<T>::zero());
    acc_set(ag, num<T>::zero());
#pragma unroll
    for (int k = 0; k < U; ++k) {
      acc_add_prod(aa, uv[k], uv[k]);
      acc_add_prod(ag, uv[k], yv[k]);
    }
    const T sa = warp_reduce_d(acc_get(aa)), sg = warp_reduce_d(acc_get(ag));
    if (lane == 0) {
      red[2 * CG][wid] = num<T>::to_d(sa);
      red[2 * CG + 1][wid] = num<T>::to_d(sg);
    }
  }
  if (ncol > 0) {
    // the group's column sums stay in registers until one reduce-scatter
    A as[CG], at[CG];
#pragma unroll
    for (int q = 0; q < CG; ++q) {
      acc_set(as[q], num<T>::zero());
      acc_set(at[q], num<T>::zero());
    }
    constexpr int CU = sizeof(T) == 4 ? 4 : 2;
#pragma unroll
    for (int g0 = 0; g0 < CG; g0 += CU) {
      if (g0 < ncol) {  // uniform over the block
        T vals[CU][U];
#pragma unroll
        for (int q = 0; q < CU; ++q) {
          const T *col = V + (int64_t)(c0 + min(g0 + q, ncol - 1)) * ldv;
#pragma unroll
          for (int k = 0; k < U; ++k) {
            const int64_t r = base + (int64_t)k * TPB;
            vals[q][k] = (r < n && g0 + q < ncol) ? ldg(col + r) : num<T>::zero();
          }
        }
#pragma unroll
        for (int q = 0; q < CU; ++q)
          if (g0 + q < ncol) {
#pragma unroll
            for (int k = 0; k < U; ++k) {
              acc_add_prod(as[g0 + q], vals[q][k], uv[k]);
              acc_add_prod(at[g0 + q], vals[q][k], yv[k]);
            }
          }
      }
    }
    T v[16];
#pragma unroll
    for (int q = 0; q < CG; ++q) {
      v[q] = acc_get(as[q]);
      v[CG + q] = acc_get(at[q]);
    }
    const T tot = warp_reduce_scatter<16>(v, lane);
    const int idx = rs_index<16>(lane);  // idx < CG: V_{c0+idx}.u, else V_{c0+idx-CG}.y
    if (rs_writer<16>(lane) && (idx & (CG - 1)) < ncol) red[idx][wid] = num<T>::to_d(tot);
  }
  __syncthreads();
  const int tix = threadIdx.x;
  double sum = 0.0;
  int slot = -1;
  int64_t out = 0;
  if (tix < ncol) {
    slot = tix;
    out = c0 + tix;
  } else if (tix >= CG && tix < CG + ncol) {
    slot = tix;
    out = J + c0 + (tix - CG);
  } else if (blockIdx.y == 0 && (tix == 2 * CG || tix == 2 * CG + 1)) {
    slot = tix;
    out = 2 * J + (tix - 2 * CG);
  }
  if (slot >= 0) {
    for (int q = 0; q < TPB / 32; ++q) sum += red[slot][q];
    partials[(int64_t)blockIdx.x * stride + out] = sum;
  }
}

// u <- (u - V s) / beta (= v_j) and y <- y / beta - V d - e u (= u_{j+1}), in place;
// co = [s_0..s_{J-1}, d_0..d_{J-1}], sc = [1/beta, e]
template <typename T>
__global__ void __launch_bounds__(TPB, sizeof(T) == 4 ? 3 : 2) k_update2(const T *__restrict__ V, int64_t ldv, int J,
                                                 const double *__restrict__ co, const double *__restrict__ sc,
                                                 T *__restrict__ u, T *__restrict__ y, int64_t n) {
  pdl_wait();
  pdl_trigger();
  using A = typename acc_of<T>::type;
  extern __shared__ unsigned char smem_raw[];
  T *ns = reinterpret_cast<T *>(smem_raw);  // -s
  T *nd = ns + J;                            // -d
  for (int c = threadIdx.x; c < J; c += TPB) {
    ns[c] = num<T>::from_d(-co[c]);
    nd[c] = num<T>::from_d(-co[J + c]);
  }
  const T ib = num<T>::from_d(sc[0]), ne = num<T>::from_d(-sc[1]);
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * CHUNK + threadIdx.x;
  A a1[U], a2[U];
#pragma unroll
  for (int k = 0; k < U; ++k) {
    const int64_t r = base + (int64_t)k * TPB;
    const T ur = (r < n) ? u[r] : num<T>::zero();
    const T yr = (r < n) ? y[r] : num<T>::zero();
    acc_set(a1[k], ur);
    acc_set_prod(a2[k], ib, yr);
    acc_add_prod(a2[k], ne, ur);
  }
  constexpr int CU = sizeof(T) == 4 ? 4 : 2;
  int c = 0;
  for (; c + CU <= J; c += CU) {
    T vals[CU][U];
#pragma unroll
    for (int q = 0; q < CU; ++q) {
      const T *col = V + (int64_t)(c + q) * ldv;
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const int64_t r = base + (int64_t)k * TPB;
        vals[q][k] = (r < n) ? ldg(col + r) : num<T>::zero();
      }
    }
#pragma unroll
    for (int q = 0; q < CU; ++q) {
      const T sq = ns[c + q], dq = nd[c + q];
#pragma unroll
      for (int k = 0; k < U; ++k)
        if (base + (int64_t)k * TPB < n) {
          acc_add_prod(a1[k], sq, vals[q][k]);
          acc_add_prod(a2[k], dq, vals[q][k]);
        }
    }
  }
  for (; c < J; ++c) {
    const T *col = V + (int64_t)c * ldv;
    const T sq = ns[c], dq = nd[c];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const int64_t r = base + (int64_t)k * TPB;
      if (r < n) {
        const T vv = ldg(col + r);
        acc_add_prod(a1[k], sq, vv);
        acc_add_prod(a2[k], dq, vv);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < U; ++k) {
    const int64_t r = base + (int64_t)k * TPB;
    if (r < n) {
      A v;
      acc_set_prod(v, ib, acc_get(a1[k]));
      u[r] = acc_get(v);
      y[r] = acc_get(a2[k]);
    }
  }
}

// The step's coefficients, FP64.  Block c of the 2J + 2 blocks sums column c
// of the inner-product sweep's partials (nb chunks x (2J + 2), row-major) in
// a fixed order into R[c]; the last block to finish (a ticket in the status)
// reads R = [s (J), t (J), a, g] and does the algebra with few FP64
// operations (one SM retires only about two FP64 additions per clock).
// h1s = the first-pass coefficients of column J-1 (J values), kept from the
// previous step.  Writes H[0:J, J-1] = h1s + s, H[J, J-1] = beta, the new
// first-pass coefficients h1_new (J + 1 values) into h1s and into
// H[0:J+1, J], co = [s, d], sc = [1/beta, e]; a vanishing or non-finite beta
// sets the status (breakdown at Krylov dimension J, or bad) and zeroes
// 1/beta, d, e.  Dynamic shared memory: 2J + 1 doubles (s and p = H s).
__global__ void __launch_bounds__(256) k_dcgs_coef(const double *__restrict__ part, int nb, int J, double *R,
                                                   double *__restrict__ H, int ldh, double *__restrict__ h1s,
                                                   double *__restrict__ co, double *__restrict__ sc, double rel,
                                                   DevStatus *st) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ double shm[];
  __shared__ double red[32];
  __shared__ int last;
  __shared__ double sh_beta, sh_ok, sh_st;
  const int S = 2 * J + 2, c = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
  {
    double v = 0.0;
    for (int b = tid; b < nb; b += blockDim.x) v += part[(int64_t)b * S + c];
    v = block_sum(v, red);
    if (tid == 0) {
      R[c] = v;
      __threadfence();
      last = atomicAdd(&st->ticket, 1u) == (unsigned)S - 1;
    }
    __syncthreads();
    if (!last) return;
  }
  __threadfence();
  double *s = shm;      // J
  double *p = shm + J;  // J + 1
  for (int i = tid; i < J; i += blockDim.x) s[i] = __ldcg(R + i);
  const double a = __ldcg(R + 2 * J), g = __ldcg(R + 2 * J + 1);
  if (tid < 32) {  // s.s, s.t, |h1s + s|^2 in one warp
    double ss = 0.0, st_ = 0.0, rr = 0.0;
    for (int i = lane; i < J; i += 32) {
      const double si = __ldcg(R + i), ti = __ldcg(R + J + i), hf = h1s[i] + si;
      ss += si * si;
      st_ += si * ti;
      rr += hf * hf;
    }
    ss = warp_sum(ss);
    st_ = warp_sum(st_);
    rr = warp_sum(rr);
    if (lane == 0) {
      st->ticket = 0;
      const double b2 = a - ss;
      const double beta = b2 > 0.0 ? sqrt(b2) : 0.0;
      const bool finite = isfinite(a) && isfinite(ss) && isfinite(g);
      bool bd = !(beta > 0.0) || (J > 0 && beta <= rel * sqrt(rr + beta * beta));
      if (!finite) {
        st->bad = 1;
        bd = true;
      }
      if (bd && !st->breakdown) {
        st->breakdown = 1;
        st->m_bd = J;
      }
      sh_beta = beta;
      sh_ok = bd ? 0.0 : 1.0;
      sh_st = st_;
    }
  }
  __syncthreads();
  const double beta = sh_beta;
  const bool ok = sh_ok != 0.0;
  const double hlast = ok ? beta : 0.0;  // H[J, J-1]
  // row i of p = H[0:J+1, 0:J] s (upper Hessenberg: from column i-1 on); column J-1
  // is h1s + s (rows < J) and beta (row J), the rest is final from earlier steps
  for (int i = tid; i <= J; i += blockDim.x) {
    double v = 0.0;
    int k = i > 0 ? i - 1 : 0;
    for (; k + 8 <= J - 1; k += 8) {
      double hv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) hv[q] = H[(size_t)(k + q) * ldh + i];
#pragma unroll
      for (int q = 0; q < 8; ++q) v += hv[q] * s[k + q];
    }
    for (; k < J - 1; ++k) v += H[(size_t)k * ldh + i] * s[k];
    if (J > 0) {
      const double hc = i < J ? h1s[i] + s[i] : hlast;
      v += hc * s[J - 1];
      H[(size_t)(J - 1) * ldh + i] = hc;
    }
    p[i] = v;
  }
  __syncthreads();
  const double ib = ok ? 1.0 / beta : 0.0;
  const double vy = (g - sh_st) * ib;  // v_j . y
  const double hJ = (vy - p[J]) * ib;
  const double cJ = p[J] * ib + hJ;
  for (int i = tid; i <= J; i += blockDim.x) {
    const double hn = i < J ? (__ldcg(R + J + i) - p[i]) * ib : hJ;
    h1s[i] = ok ? hn : 0.0;
    H[(size_t)J * ldh + i] = ok ? hn : 0.0;
    if (i < J) {
      const double ci = p[i] * ib + hn;
      co[i] = s[i];
      co[J + i] = ok ? ci - cJ * s[i] * ib : 0.0;
    }
  }
  if (tid == 0) {
    sc[0] = ib;
    sc[1] = ok ? cJ * ib : 0.0;
  }
}
}  // namespace

int vec_nchunks(int64_t n) { return (int)nchunks(n); }
int vec_chunk_rows() { return CHUNK; }

template <typename T>
int vec_from_f64(const double *in, T *out, int64_t n, cudaStream_t s) {
  PP_CUDA_TRY(pdl_launch(k_from_f64<T>, dim3(grid_for(n, 256, kMaxGrid)), dim3(256), 0, s, in, out, n));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template <typename T>
int vec_to_f64(const T *in, double *out, int64_t n, cudaStream_t s) {
  PP_CUDA_TRY(pdl_launch(k_to_f64<T>, dim3(grid_for(n, 256, kMaxGrid)), dim3(256), 0, s, in, out, n));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template <typename T>
int vec_fill_hash(T *out, int64_t n, uint64_t seed, cudaStream_t s) {
  PP_CUDA_TRY(pdl_launch(k_fill_hash<T>, dim3(grid_for(n, 256, kMaxGrid)), dim3(256), 0, s, out, n, seed));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template int vec_fill_hash<double>(double *, int64_t, uint64_t, cudaStream_t);
template int vec_fill_hash<dw>(dw *, int64_t, uint64_t, cudaStream_t);

template <typename TI, typename TO>
int vec_convert(const TI *in, TO *out, int64_t n, cudaStream_t s) {
  PP_CUDA_TRY(pdl_launch(k_convert<TI, TO>, dim3(grid_for(n, 256, kMaxGrid)), dim3(256), 0, s, in, out, n));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template int vec_convert<dw, float>(const dw *, float *, int64_t, cudaStream_t);

template <typename T>
int vec_scale(const T *in, T *out, int64_t n, double c, const double *c_dev, cudaStream_t s, const Seg &S) {
  PP_CUDA_TRY(pdl_launch(k_scale<T>, dim3(nchunks(n)), dim3(TPB), 0, s, in, out, n, c, c_dev, S));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
int vec_recip(const double *in, double *out, cudaStream_t s) {
  PP_CUDA_TRY(pdl_launch(k_recip, dim3(1), dim3(32), 0, s, in, out));
  ++pp_launch_count();
  return PP_OK;
}
template <typename T>
int vec_copy(const T *in, T *out, int64_t n, cudaStream_t s) {
  PP_CUDA_TRY(pdl_launch(k_copy<T>, dim3(grid_for(n, 256, kMaxGrid)), dim3(256), 0, s, in, out, n));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template <typename T>
int vec_dot_partials(const T *x, const T *y, int64_t n, double *partials, int, cudaStream_t s, const Seg &S) {
  PP_CUDA_TRY(pdl_launch(k_dot<T>, dim3(nchunks(n)), dim3(TPB), 0, s, x, y, n, partials, S));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template <typename T>
int vec_lanczos_update(T *w, const T *vj, const T *vjm1, int64_t n, const double *alpha,
                       const double *beta_prev, double *partials, int, cudaStream_t s, const Seg &S) {
  PP_CUDA_TRY(pdl_launch(k_lanczos_update<T>, dim3(nchunks(n)), dim3(TPB), 0, s, w, vj, vjm1, n, alpha, beta_prev, partials, S));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template <typename T>
int vec_multi_dot(const T *V, int64_t ldv, int J, const T *w, int64_t n, double *partials, int,
                  cudaStream_t s, const Seg &S) {
  dim3 grd(nchunks(n), (unsigned)((J + CG - 1) / CG));
  PP_CUDA_TRY(pdl_launch(k_multi_dot<T>, grd, dim3(TPB), 0, s, V, ldv, J, w, n, partials, S));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template <typename T>
int vec_multi_update(const T *V, int64_t ldv, int J, const double *h, T *w, int64_t n,
                     double *partials, int, cudaStream_t s, const Seg &S) {
  const size_t sm = (size_t)J * sizeof(T);
  if (sm > 48 * 1024) PP_CUDA_TRY(cudaFuncSetAttribute(k_multi_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  PP_CUDA_TRY(pdl_launch(k_multi_update<T>, dim3(nchunks(n)), dim3(TPB), sm, s, V, ldv, J, h, w, n, partials, S));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template <typename T>
int vec_update_dot(const T *V, int64_t ldv, int J, const double *h, T *w, int64_t n, double *partials,
                   cudaStream_t s, const Seg &S) {
  // measured on GB300 at n = 2M: registers hold the row's columns up to 8
  // (40 us against 65 us for the two sweeps in double-word); wider, the
  // register arrays cut the occupancy, and a shared-memory tile of the
  // columns takes over up to kUpdateDotTileMaxJ
  if (J <= 8) {
    PP_CUDA_TRY(pdl_launch(k_update_dot<T, 8>, dim3(nchunks(n)), dim3(TPB), 0, s, V, ldv, J, h, w, n, partials, S));
    ++pp_launch_count();
    return PP_OK;
  }
  if (J > kUpdateDotTileMaxJ) return PP_ERR_UNSUPPORTED;
  const size_t sm = ((size_t)J + TPB + (size_t)J * TPB) * sizeof(T);
  if (sm > 48 * 1024)
    PP_CUDA_TRY(cudaFuncSetAttribute(k_update_dot_tile<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  PP_CUDA_TRY(pdl_launch(k_update_dot_tile<T>, dim3(nchunks(n)), dim3(TPB), sm, s, V, ldv, J, h, w, n, partials, S));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template <typename T>
int vec_reconstruct(const T *V, int64_t ldv, int m, const double *z, double *x, int64_t n,
                    int accumulate, cudaStream_t s, const Seg &S, const int *m_seg) {
  const size_t sm = (size_t)m * sizeof(T);
  if (sm > 48 * 1024) PP_CUDA_TRY(cudaFuncSetAttribute(k_reconstruct<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  PP_CUDA_TRY(pdl_launch(k_reconstruct<T>, dim3(nchunks(n)), dim3(TPB), sm, s, V, ldv, m, m_seg, z, x, n, accumulate, S));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}

int reduce_cols(const double *partials, int nb, int ncols, int mode, double *out_a, double *out_b,
                cudaStream_t s, const Seg &S) {
  PP_CUDA_TRY(pdl_launch(k_reduce_cols, dim3(ncols, S.nseg), dim3(256), 0, s, partials, nb, ncols, mode, out_a, out_b, S));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}

int norm_finalize(const double *partials, int nb, double *beta_out, double *inv_out,
                  const double *ref, int nref, double rel, int m_here, DevStatus *st,
                  cudaStream_t s, const Seg &S) {
  PP_CUDA_TRY(pdl_launch(k_norm_finalize, dim3(S.nseg), dim3(256), 0, s, partials, nb, beta_out, inv_out, ref, nref, rel, m_here, st, S));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}

template <typename T>
int vec_multi_dot_c(const T *V, int64_t ldv, int J, const T *w, int64_t n, double *partials, cudaStream_t s) {
  PP_CUDA_TRY(pdl_launch(k_multi_dot_c<T>, dim3(nchunks(n), (J + CG - 1) / CG), dim3(TPB), 0, s, V, ldv, J, w, n,
                         partials));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template <typename T>
int vec_multi_update_c(const T *V, int64_t ldv, int J, const double *h, T *w, int64_t n, double *partials,
                       cudaStream_t s) {
  const size_t sm = (size_t)3 * J * sizeof(T);
  if (sm > 48 * 1024)
    PP_CUDA_TRY(cudaFuncSetAttribute(k_multi_update_c<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  PP_CUDA_TRY(pdl_launch(k_multi_update_c<T>, dim3(nchunks(n)), dim3(TPB), sm, s, V, ldv, J, h, w, n, partials));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template <typename T>
int vec_reconstruct_c(const T *V, int64_t ldv, int m, const double *z, double *x, int64_t n, int accumulate,
                      cudaStream_t s) {
  const size_t sm = (size_t)3 * m * sizeof(T);
  if (sm > 48 * 1024)
    PP_CUDA_TRY(cudaFuncSetAttribute(k_reconstruct_c<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  PP_CUDA_TRY(pdl_launch(k_reconstruct_c<T>, dim3(nchunks(n)), dim3(TPB), sm, s, V, ldv, m, z, x, n, accumulate));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template <typename T>
int vec_scale_c(const T *in, T *out, int64_t n, double cr, double ci, cudaStream_t s) {
  PP_CUDA_TRY(pdl_launch(k_scale_c<T>, dim3(nchunks(n)), dim3(TPB), 0, s, in, out, n, cr, ci));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}

template <typename T>
int vec_dot2(const T *V, int64_t ldv, int J, const T *u, const T *y, int64_t n, double *partials, cudaStream_t s) {
  dim3 grd(nchunks(n), (unsigned)std::max(1, (J + CG - 1) / CG));
  PP_CUDA_TRY(pdl_launch(k_dot2<T>, grd, dim3(TPB), 0, s, V, ldv, J, u, y, n, partials));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
template <typename T>
int vec_update2(const T *V, int64_t ldv, int J, const double *co, const double *sc, T *u, T *y, int64_t n,
                cudaStream_t s) {
  const size_t sm = (size_t)2 * std::max(J, 1) * sizeof(T);
  if (sm > 48 * 1024) PP_CUDA_TRY(cudaFuncSetAttribute(k_update2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  PP_CUDA_TRY(pdl_launch(k_update2<T>, dim3(nchunks(n)), dim3(TPB), sm, s, V, ldv, J, co, sc, u, y, n));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
int dcgs_coef(const double *partials, int nb, int J, double *R, double *H, int ldh, double *h1s, double *co,
              double *sc, double rel, DevStatus *st, cudaStream_t s) {
  if (J > kDcgsMaxJ) return pp_set_error(PP_ERR_INVALID_ARG, "delayed reorthogonalization: basis too wide");
  const size_t sm = sizeof(double) * ((size_t)2 * J + 1);
  if (sm > 48 * 1024) PP_CUDA_TRY(cudaFuncSetAttribute(k_dcgs_coef, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  PP_CUDA_TRY(pdl_launch(k_dcgs_coef, dim3(2 * J + 2), dim3(256), sm, s, partials, nb, J, R, H, ldh, h1s, co, sc, rel,
                         st));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}

#define PP_INST(T)                                                                                  \
  template int vec_from_f64<T>(const double *, T *, int64_t, cudaStream_t);                       \
  template int vec_to_f64<T>(const T *, double *, int64_t, cudaStream_t);                         \
  template int vec_scale<T>(const T *, T *, int64_t, double, const double *, cudaStream_t,        \
                            const Seg &);                                                         \
  template int vec_copy<T>(const T *, T *, int64_t, cudaStream_t);                                \
  template int vec_dot_partials<T>(const T *, const T *, int64_t, double *, int, cudaStream_t,    \
                                   const Seg &);                                                  \
  template int vec_lanczos_update<T>(T *, const T *, const T *, int64_t, const double *,          \
                                     const double *, double *, int, cudaStream_t, const Seg &);   \
  template int vec_multi_dot<T>(const T *, int64_t, int, const T *, int64_t, double *, int,       \
                                cudaStream_t, const Seg &);                                       \
  template int vec_multi_update<T>(const T *, int64_t, int, const double *, T *, int64_t, double *, \
                                   int, cudaStream_t, const Seg &);                               \
  template int vec_reconstruct<T>(const T *, int64_t, int, const double *, double *, int64_t, int, \
                                  cudaStream_t, const Seg &, const int *);                        \
  template int vec_update_dot<T>(const T *, int64_t, int, const double *, T *, int64_t, double *,  \
                                 cudaStream_t, const Seg &);                                      \
  template int vec_dot2<T>(const T *, int64_t, int, const T *, const T *, int64_t, double *, cudaStream_t); \
  template int vec_update2<T>(const T *, int64_t, int, const double *, const double *, T *, T *, int64_t,  \
                              cudaStream_t);                                                       \
  template int vec_multi_dot_c<T>(const T *, int64_t, int, const T *, int64_t, double *, cudaStream_t); \
  template int vec_multi_update_c<T>(const T *, int64_t, int, const double *, T *, int64_t, double *, \
                                     cudaStream_t);                                               \
  template int vec_reconstruct_c<T>(const T *, int64_t, int, const double *, double *, int64_t, int, \
                                    cudaStream_t);                                                \
  template int vec_scale_c<T>(const T *, T *, int64_t, double, double, cudaStream_t);
PP_INST(double)
PP_INST(float)
PP_INST(dw)
