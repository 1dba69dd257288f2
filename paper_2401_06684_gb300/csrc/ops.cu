// Operator kernels: one application of A fused with the vector update of a
// step of q(A) v,
//     out = alpha (A x) + beta x  [+ gamma y]  [+ delta v],
// which covers a plain product u = A x (alpha = 1, beta = 0), every Horner
// step of the Newton form w_i = ((A - x_i)/cap) w_{i+1} + a_i v (Sec. 5.2; no
// y term for real nodes), its conjugate-pair steps (gamma = (Im x_i/cap)^2)
// and every step b_i = 2 sigma(A) b_{i+1} - b_{i+2} + c_i v of the matrix
// Clenshaw recurrence (Sec. 5.1, gamma = -1).  The stencil is folded into
// three constants
//     K0 = alpha d + beta, Km = alpha cm, Kp = alpha cp,
// so one pass reads x (with its neighbours) and v, [y,] and writes out: 3
// (4 with y) vectors of HBM traffic per step for the matrix-free operators.
// The arithmetic is that of the vectors: FP64, double-word pairs or FP32.
#include "common.cuh"
#include "internal.h"

namespace {


// One stencil row evaluated as a compensated linear combination
//   K0 x_c + Km (x_w + x_s + x_d) + Kp (x_e + x_n + x_u) [+ Y y] [+ D v].
template <typename T, bool SUB_Y, bool ADD_V>
__device__ __forceinline__ T stencil_row(T xc, T xw, T xe, T xs, T xn, T xd, T xu, T yy, T vv,
                                         const Konst<T> &K) {
  using A = typename acc_of<T>::type;
  A nm, np, r;
  acc_set(nm, xd);
  acc_add(nm, xw);
  acc_add(nm, xs);
  acc_set(np, xu);
  acc_add(np, xe);
  acc_add(np, xn);
  acc_set_prod(r, K.K0, xc);
  acc_add_prod(r, K.Km, acc_raw(nm));
  acc_add_prod(r, K.Kp, acc_raw(np));
  if (SUB_Y) acc_add_prod(r, K.Y, yy);
  if (ADD_V) acc_add_prod(r, K.D, vv);
  return acc_get(r);
}

// P consecutive entries through one vector load / store of P * sizeof(T)
// bytes (4, 8 or 16; the address must be aligned to it).
template <int BYTES>
struct raw_vec;
template <>
struct raw_vec<16> {
  using type = int4;
};
template <>
struct raw_vec<8> {
  using type = int2;
};
template <>
struct raw_vec<4> {
  using type = int;
};

template <typename T, int P>
__device__ __forceinline__ void ld_p(const T *p, T (&r)[P]) {
  using R = typename raw_vec<sizeof(T) * P>::type;
  const R v = __ldg(reinterpret_cast<const R *>(p));
  memcpy(r, &v, sizeof(R));
}

template <typename T, int P>
__device__ __forceinline__ void st_p(T *p, const T (&r)[P]) {
  using R = typename raw_vec<sizeof(T) * P>::type;
  R v;
  memcpy(&v, r, sizeof(R));
  *reinterpret_cast<R *>(p) = v;
}

template <typename T, int P>
__device__ __forceinline__ void zero_p(T (&r)[P]) {
#pragma unroll
  for (int q = 0; q < P; ++q) r[q] = num<T>::zero();
}

constexpr int ST_THREADS = 128;           // threads per block of the stencil kernels (default)
constexpr int kStencilMaxThreads = 512;  // largest block the tile tuner may pick

// Entries [i0, i0 + P) of a row by separate loads, those at or past nx as
// zero (rows of any length and alignment).
template <typename T, int P>
__device__ __forceinline__ void ld_s(const T *p, int cnt, T (&r)[P]) {
#pragma unroll
  for (int q = 0; q < P; ++q) r[q] = q < cnt ? ldg(p + q) : num<T>::zero();
}

// 2D 5-point and 3D 7-point stencils (nz = 1 for 2D): P consecutive x
// entries of one grid row (P = 16 bytes of entries; the threads take two rows
// each through stencil_rows2 below, this one alone for the last row of an
// odd plane).  VEC (nx % P == 0 and 16-byte aligned
// vectors): every load is a coalesced 16-byte load: the row itself, its four
// y/z neighbour rows, y and v.  Otherwise the same P entries come through
// separate loads, masked at the end of the row (several loads in flight per
// thread either way).  The two x neighbours outside the thread's P entries
// are scalar loads.  Neighbour reuse between threads and planes is left to
// L1/L2.
template <typename T, int P, bool VEC, bool SUB_Y, bool ADD_V>
__device__ __forceinline__ void stencil_rows(const T *__restrict__ x, const T *__restrict__ y,
                                             const T *__restrict__ v, T *__restrict__ out, int nx, int ny,
                                             int nz, int i0, int j, int k, const Konst<T> &K) {
  const int64_t plane = (int64_t)nx * ny;
  const int64_t off = (int64_t)k * plane + (int64_t)j * nx + i0;
  const T zero = num<T>::zero();
  const int cnt = nx - i0 < P ? nx - i0 : P;
  T xc[P], xs[P], xn[P], xd[P], xu[P], yy[P], vv[P];
  if constexpr (VEC) {
    ld_p<T, P>(x + off, xc);
    if (j > 0) ld_p<T, P>(x + off - nx, xs); else zero_p<T, P>(xs);
    if (j + 1 < ny) ld_p<T, P>(x + off + nx, xn); else zero_p<T, P>(xn);
    if (k > 0) ld_p<T, P>(x + off - plane, xd); else zero_p<T, P>(xd);
    if (k + 1 < nz) ld_p<T, P>(x + off + plane, xu); else zero_p<T, P>(xu);
    if (SUB_Y) ld_p<T, P>(y + off, yy); else zero_p<T, P>(yy);
    if (ADD_V) ld_p<T, P>(v + off, vv); else zero_p<T, P>(vv);
  } else {
    ld_s<T, P>(x + off, cnt, xc);
    if (j > 0) ld_s<T, P>(x + off - nx, cnt, xs); else zero_p<T, P>(xs);
    if (j + 1 < ny) ld_s<T, P>(x + off + nx, cnt, xn); else zero_p<T, P>(xn);
    if (k > 0) ld_s<T, P>(x + off - plane, cnt, xd); else zero_p<T, P>(xd);
    if (k + 1 < nz) ld_s<T, P>(x + off + plane, cnt, xu); else zero_p<T, P>(xu);
    if (SUB_Y) ld_s<T, P>(y + off, cnt, yy); else zero_p<T, P>(yy);
    if (ADD_V) ld_s<T, P>(v + off, cnt, vv); else zero_p<T, P>(vv);
  }
  const T xw0 = i0 > 0 ? ldg(x + off - 1) : zero;
  const T xeP = i0 + P < nx ? ldg(x + off + P) : zero;
  T o[P];
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const T xw = q == 0 ? xw0 : xc[q - 1];
    const T xe = q == P - 1 ? xeP : xc[q + 1];  // past the row's end: zero (Dirichlet)
    o[q] = stencil_row<T, SUB_Y, ADD_V>(xc[q], xw, xe, xs[q], xn[q], xd[q], xu[q], yy[q], vv[q], K);
  }
  if constexpr (VEC) {
    st_p<T, P>(out + off, o);
  } else {
#pragma unroll
    for (int q = 0; q < P; ++q)
      if (q < cnt) out[off + q] = o[q];
  }
}

// Rows j and j+1 (j + 1 < ny) of the same P columns: each row's centre load
// is the other's y neighbour, and every load of both rows is issued before
// the arithmetic, so each thread keeps twice the bytes in flight.  Measured
// against one row per thread: 128^3 FP32 step 5.69 -> 4.58 us, double-word
// 12.0 -> 10.6 us, 8192^2 FP32 (out of L2) 149.8 -> 128.1 us.
template <typename T, int P, bool VEC, bool SUB_Y, bool ADD_V>
__device__ __forceinline__ void stencil_rows2(const T *__restrict__ x, const T *__restrict__ y,
                                              const T *__restrict__ v, T *__restrict__ out, int nx, int ny,
                                              int nz, int i0, int j, int k, const Konst<T> &K) {
  const int64_t plane = (int64_t)nx * ny;
  const int64_t off = (int64_t)k * plane + (int64_t)j * nx + i0;
  const int64_t off1 = off + nx;
  const T zero = num<T>::zero();
  const int cnt = nx - i0 < P ? nx - i0 : P;
  T c0[P], c1[P], s0[P], n1[P], d0[P], u0[P], d1[P], u1[P], y0[P], y1[P], v0[P], v1[P];
  auto ld = [&](const T *p, T(&r)[P]) {
    if constexpr (VEC)
      ld_p<T, P>(p, r);
    else
      ld_s<T, P>(p, cnt, r);
  };
  ld(x + off, c0);
  ld(x + off1, c1);
  if (j > 0) ld(x + off - nx, s0); else zero_p<T, P>(s0);
  if (j + 2 < ny) ld(x + off1 + nx, n1); else zero_p<T, P>(n1);
  if (k > 0) {
    ld(x + off - plane, d0);
    ld(x + off1 - plane, d1);
  } else {
    zero_p<T, P>(d0);
    zero_p<T, P>(d1);
  }
  if (k + 1 < nz) {
    ld(x + off + plane, u0);
    ld(x + off1 + plane, u1);
  } else {
    zero_p<T, P>(u0);
    zero_p<T, P>(u1);
  }
  if (SUB_Y) {
    ld(y + off, y0);
    ld(y + off1, y1);
  } else {
    zero_p<T, P>(y0);
    zero_p<T, P>(y1);
  }
  if (ADD_V) {
    ld(v + off, v0);
    ld(v + off1, v1);
  } else {
    zero_p<T, P>(v0);
    zero_p<T, P>(v1);
  }
  const T w0 = i0 > 0 ? ldg(x + off - 1) : zero;
  const T e0 = i0 + P < nx ? ldg(x + off + P) : zero;
  const T w1 = i0 > 0 ? ldg(x + off1 - 1) : zero;
  const T e1 = i0 + P < nx ? ldg(x + off1 + P) : zero;
  T o0[P], o1[P];
#pragma unroll
  for (int q = 0; q < P; ++q) {
    o0[q] = stencil_row<T, SUB_Y, ADD_V>(c0[q], q == 0 ? w0 : c0[q - 1], q == P - 1 ? e0 : c0[q + 1], s0[q], c1[q],
                                         d0[q], u0[q], y0[q], v0[q], K);
    o1[q] = stencil_row<T, SUB_Y, ADD_V>(c1[q], q == 0 ? w1 : c1[q - 1], q == P - 1 ? e1 : c1[q + 1], c0[q], n1[q],
                                         d1[q], u1[q], y1[q], v1[q], K);
  }
  if constexpr (VEC) {
    st_p<T, P>(out + off, o0);
    st_p<T, P>(out + off1, o1);
  } else {
#pragma unroll
    for (int q = 0; q < P; ++q)
      if (q < cnt) {
        out[off + q] = o0[q];
        out[off1 + q] = o1[q];
      }
  }
}

// The unit's rows: j and j + 1 together, or j alone at the end of an odd plane.
template <typename T, int P, bool VEC, bool SUB_Y, bool ADD_V>
__device__ __forceinline__ void stencil_unit(const T *__restrict__ x, const T *__restrict__ y,
                                             const T *__restrict__ v, T *__restrict__ out, int nx, int ny, int nz,
                                             int i0, int j, int k, const Konst<T> &K) {
  if (j + 1 < ny)
    stencil_rows2<T, P, VEC, SUB_Y, ADD_V>(x, y, v, out, nx, ny, nz, i0, j, k, K);
  else
    stencil_rows<T, P, VEC, SUB_Y, ADD_V>(x, y, v, out, nx, ny, nz, i0, j, k, K);
}

// Unit u of a grid with txs units per row pair and nyp row pairs per plane
// -> (first entry i0, first row j = 2 * pair, plane k); 32-bit divisions
// where the grid allows them (64-bit ones are emulated).
template <int P>
__device__ __forceinline__ void unit_coords(int64_t u, int64_t units, int txs, int nyp, int *i0, int *j, int *k) {
  if (units <= 0x7fffffff) {
    const unsigned uu = (unsigned)u, r = uu / (unsigned)txs;
    *i0 = (int)(uu - r * (unsigned)txs) * P;
    const unsigned kk = r / (unsigned)nyp;
    *j = 2 * (int)(r - kk * (unsigned)nyp);
    *k = (int)kk;
  } else {
    const int64_t r = u / txs;
    *i0 = (int)(u - r * txs) * P;
    *j = 2 * (int)(r % nyp);
    *k = (int)(r / nyp);
  }
}

// One thread per unit of P consecutive entries of two neighbouring rows.
// FLAT: units numbered x-fastest over the whole grid (txs units per row pair),
// so no thread idles whatever the row length; otherwise (rows that split
// into whole x tiles) a 2D block of blockDim.x units by blockDim.y row pairs
// of one plane, the flat block index running over (x tile, y tile, plane),
// which needs no division per thread.
template <typename T, int P, bool VEC, bool FLAT, bool SUB_Y, bool ADD_V>
__global__ void __launch_bounds__(kStencilMaxThreads) st_step(const T *__restrict__ x, const T *__restrict__ y,
                                                                const T *__restrict__ v, T *__restrict__ out,
                                                                int nx, int ny, int nz, int txs, int64_t units,
                                                                unsigned gx, unsigned gy, Konst<T> K) {
  pdl_wait();
  pdl_trigger();
  int i0, j, k;
  if constexpr (FLAT) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= units) return;
    unit_coords<P>(u, units, txs, (ny + 1) / 2, &i0, &j, &k);
  } else {
    const unsigned blk = blockIdx.x;
    const unsigned bx = blk % gx, rest = blk / gx;
    const unsigned by = rest % gy;
    k = (int)(rest / gy);
    i0 = (int)(bx * blockDim.x + threadIdx.x) * P;
    j = 2 * (int)(by * blockDim.y + threadIdx.y);
    if (i0 >= nx || j >= ny) return;
  }
  stencil_unit<T, P, VEC, SUB_Y, ADD_V>(x, y, v, out, nx, ny, nz, i0, j, k, K);
}

// Batched form: many grids (segments of concatenated vectors) in one launch.
// The flat block index is mapped to its segment by a per-block table (one
// load instead of a binary search over the segments' first blocks, whose
// dependent loads came before any of the block's work); each segment has
// its own geometry, constants and load path
// (16-byte loads where its row length allows them), and its units are mapped
// as in st_step.
template <typename T, int P, bool SUB_Y, bool ADD_V>
__global__ void __launch_bounds__(kStencilMaxThreads) bst_step(const T *__restrict__ x, const T *__restrict__ y,
                                                                 const T *__restrict__ v, T *__restrict__ out,
                                                                 const BatchSeg *__restrict__ segs,
                                                                 const int *__restrict__ blkseg,
                                                                 const Konst<T> *__restrict__ K,
                                                                 const int *__restrict__ active) {
  pdl_wait();
  pdl_trigger();
  const unsigned blk = blockIdx.x;
  const int lo = __ldg(blkseg + blk);
  if (active && !active[lo]) return;
  const BatchSeg g = segs[lo];
  const int64_t u = (int64_t)(blk - g.blk0) * blockDim.x + threadIdx.x;
  if (u >= g.units) return;
  int i0, j, k;
  unit_coords<P>(u, g.units, g.txs, (g.ny + 1) / 2, &i0, &j, &k);
  if (g.vec)
    stencil_unit<T, P, true, SUB_Y, ADD_V>(x + g.off, SUB_Y ? y + g.off : y, ADD_V ? v + g.off : v, out + g.off,
                                           g.nx, g.ny, g.nz, i0, j, k, K[lo]);
  else
    stencil_unit<T, P, false, SUB_Y, ADD_V>(x + g.off, SUB_Y ? y + g.off : y, ADD_V ? v + g.off : v,
                                            out + g.off, g.nx, g.ny, g.nz, i0, j, k, K[lo]);
}

// CSR.  Rows of up to long_len entries: L lanes per row, lane-strided over
// the row, shuffle sum.  Longer rows (the nlong rows listed in long_rows,
// long_len > 0; power-law graphs have a few rows thousands of entries long,
// whose sequential lane loops would otherwise set the kernel's duration):
// one block of 256 threads per row, thread-strided, then a fixed-order block
// sum.  The first nlong blocks take the long rows, the others the short ones.
//
// Accumulation (csr_acc): FP64 and FP32 vectors accumulate by FMA in their
// own arithmetic.  Double-word vectors accumulate every row sum and the
// step's update in a triple-float sum s + (e_hi + e_lo) on the FP32 pipes:
// each product c x of double-word operands is split exactly into its
// leading part (TwoSum into s) and the error-free residuals of its partial
// products (FMA TwoProd), which are added to e with TwoSum; only the
// products' u^2-sized tails go in unsplit.  The sum is then accurate to about
// 2^-72 of the summands, and the result is rounded once to a double-word pair
// (2^-48 of itself).  Rows like those of a graph Laplacian, whose diagonal is
// minus the sum of the other entries, cancel heavily: with the lazy double-
// word accumulator their error was 2^-48 of the summands, above what FP64
// reaches, and on Example 3's graph the square root missed its 1e-7 target;
// FP64 arithmetic in the kernel met it but ran on GB300's narrow FP64 pipe.
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }

template <typename T>
struct csr_acc {
  T s;
  __device__ __forceinline__ void zero() { s = (T)0; }
  __device__ __forceinline__ void add_prod(T c, T x) { s = fma_t(c, x, s); }
  __device__ __forceinline__ void add(const csr_acc &o) { s += o.s; }
  __device__ __forceinline__ csr_acc shfl(int o, int width) const {
    csr_acc r;
    r.s = __shfl_xor_sync(0xffffffffu, s, o, width);
    return r;
  }
  __device__ __forceinline__ T get() const { return s; }
};

template <>
struct csr_acc<dw> {
  // s + (eh + el): s takes the leading parts by TwoSum, eh the rounding
  // errors and residuals by TwoSum (lazily: its own errors go to el)
  float s, eh, el;
  __device__ __forceinline__ void zero() { s = eh = el = 0.f; }
  __device__ __forceinline__ void add_e(float f) {
    const dw t = dw_two_sum(eh, f);
    eh = t.hi;
    el = __fadd_rn(el, t.lo);
  }
  __device__ __forceinline__ void add_lead(float p) {
    const dw t = dw_two_sum(s, p);
    s = t.hi;
    add_e(t.lo);
  }
  // c x for double-word c and x: the FMA TwoProd residual of every partial
  // product is kept; c.lo x.lo (and the residuals of the cross terms, both
  // u^2 |c x|) go to el directly
  __device__ __forceinline__ void add_prod(dw c, dw x) {
    const float p0 = __fmul_rn(c.hi, x.hi), r0 = __fmaf_rn(c.hi, x.hi, -p0);
    const float p1 = __fmul_rn(c.hi, x.lo), r1 = __fmaf_rn(c.hi, x.lo, -p1);
    const float p2 = __fmul_rn(c.lo, x.hi), r2 = __fmaf_rn(c.lo, x.hi, -p2);
    add_lead(p0);
    add_e(r0);
    add_e(__fadd_rn(p1, p2));
    el = __fadd_rn(el, __fadd_rn(__fadd_rn(r1, r2), __fmul_rn(c.lo, x.lo)));
  }
  // c x for a value c exact in FP32 (matrices whose entries all are)
  __device__ __forceinline__ void add_prod(float c, dw x) {
    const float p0 = __fmul_rn(c, x.hi), r0 = __fmaf_rn(c, x.hi, -p0);
    const float p1 = __fmul_rn(c, x.lo), r1 = __fmaf_rn(c, x.lo, -p1);
    add_lead(p0);
    add_e(r0);
    add_e(p1);
    el = __fadd_rn(el, r1);
  }
  __device__ __forceinline__ void add(const csr_acc &o) {
    add_lead(o.s);
    add_e(o.eh);
    el = __fadd_rn(el, o.el);
  }
  __device__ __forceinline__ csr_acc shfl(int o, int width) const {
    csr_acc r;
    r.s = __shfl_xor_sync(0xffffffffu, s, o, width);
    r.eh = __shfl_xor_sync(0xffffffffu, eh, o, width);
    r.el = __shfl_xor_sync(0xffffffffu, el, o, width);
    return r;
  }
  __device__ __forceinline__ dw get() const {
    const dw t = dw_two_sum(s, eh);
    return dw_fast_two_sum(t.hi, __fadd_rn(t.lo, el));
  }
};

// out = alpha sum + beta x [+ gamma y] [+ delta v] in the accumulator
template <typename T, bool SUB_Y, bool ADD_V>
__device__ __forceinline__ T csr_finish(const csr_acc<T> &sum, T alpha, T beta, T gamma, T delta, T xr, T yr,
                                        T vr) {
  csr_acc<T> r;
  r.zero();
  r.add_prod(alpha, sum.get());
  r.add_prod(beta, xr);
  if (SUB_Y) r.add_prod(gamma, yr);
  if (ADD_V) r.add_prod(delta, vr);
  return r.get();
}

// acc += sum over p = p0, p0 + stride, ... < p1 of val[p] x[col[p]], U entries
// per round with all their loads issued before the first product (the
// dependent col -> x gathers of a round overlap); the products are added in
// the order of the plain loop, so the sum is bit for bit the same.
template <typename T, typename VT, int U>
__device__ __forceinline__ void csr_row_sum(csr_acc<T> &acc, const int32_t *__restrict__ col,
                                            const VT *__restrict__ val, const T *__restrict__ x, int64_t p0,
                                            int64_t p1, int64_t stride) {
  int64_t p = p0;
  for (; p + (U - 1) * stride < p1; p += U * stride) {
    int32_t c[U];
    VT a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      c[u] = __ldg(col + p + u * stride);
      a[u] = ldg(val + p + u * stride);
    }
    T xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = ldg(x + c[u]);
#pragma unroll
    for (int u = 0; u < U; ++u) acc.add_prod(a[u], xv[u]);
  }
  for (; p < p1; p += stride) acc.add_prod(ldg(val + p), ldg(x + __ldg(col + p)));
}

template <typename T, typename VT, int L, bool SUB_Y, bool ADD_V>
__global__ void __launch_bounds__(256) csr_step(const int64_t *__restrict__ rowptr,
                                                const int32_t *__restrict__ col, const VT *__restrict__ val,
                                                const T *__restrict__ x, const T *__restrict__ y,
                                                const T *__restrict__ v, T *__restrict__ out, int64_t n, T alpha,
                                                T beta, T gamma, T delta, const int32_t *__restrict__ long_rows,
                                                int nlong, int nwarp, int64_t long_len,
                                                const int32_t *__restrict__ perm, int64_t nshort) {
  pdl_wait();
  pdl_trigger();
  auto finish = [&](int64_t row, const csr_acc<T> &sum) {
    out[row] = csr_finish<T, SUB_Y, ADD_V>(sum, alpha, beta, gamma, delta, ldg(x + row),
                                           SUB_Y ? ldg(y + row) : num<T>::zero(),
                                           ADD_V ? ldg(v + row) : num<T>::zero());
  };
  csr_acc<T> acc;
  acc.zero();
  if ((int)blockIdx.x < nlong) {
    __shared__ csr_acc<T> red[8];
    const int64_t row = __ldg(long_rows + blockIdx.x);
    const int64_t p1 = __ldg(rowptr + row + 1);
    csr_row_sum<T, VT, 4>(acc, col, val, x, __ldg(rowptr + row) + threadIdx.x, p1, blockDim.x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc.add(acc.shfl(o, 32));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      csr_acc<T> tot = red[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) tot.add(red[w]);
      finish(row, tot);
    }
    return;
  }
  const int nwb = (nwarp + 7) / 8;  // blocks of 8 warps, a warp per medium row
  if ((int)blockIdx.x < nlong + nwb) {
    const int wi = ((int)blockIdx.x - nlong) * 8 + (int)(threadIdx.x >> 5), ln = threadIdx.x & 31;
    if (wi >= nwarp) return;
    const int64_t row = __ldg(long_rows + nlong + wi);
    const int64_t p1 = __ldg(rowptr + row + 1);
    csr_row_sum<T, VT, 4>(acc, col, val, x, __ldg(rowptr + row) + ln, p1, 32);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc.add(acc.shfl(o, 32));
    if (ln == 0) finish(row, acc);
    return;
  }
  const int64_t t = (int64_t)(blockIdx.x - nlong - nwb) * blockDim.x + threadIdx.x;
  const int64_t slot = t / L;
  const int lane = (int)(t % L);
  bool mine = slot < (perm ? nshort : n);
  int64_t row = slot;
  if (mine) {
    if (perm) row = __ldg(perm + slot);
    const int64_t p0 = __ldg(rowptr + row), p1 = __ldg(rowptr + row + 1);
    if (long_len > 0 && p1 - p0 > long_len)
      mine = false;  // a long row: its own block or warp computes it
    else
      for (int64_t p = p0 + lane; p < p1; p += L) acc.add_prod(ldg(val + p), ldg(x + __ldg(col + p)));
  }
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) acc.add(acc.shfl(o, L));
  if (mine && lane == 0) finish(row, acc);
}

// Block form for r right-hand sides of one matrix (block SpMM): the r
// vectors of a group are the segments x + s * sstride, s < r <= kCsrMaxRhs.
// Each lane group reads a row's (col, val) once and applies it to every
// active segment (active[s] != 0, read once per thread into a bit mask), so
// the matrix costs one pass per step for all r processes instead of r.  The
// lane-strided accumulation and the shuffle order per segment are those of
// csr_step, so every segment's result equals the single-vector step's bit
// for bit.
template <typename T, typename VT, int L, bool SUB_Y, bool ADD_V>
__global__ void __launch_bounds__(256) csr_step_multi(const int64_t *__restrict__ rowptr,
                                                      const int32_t *__restrict__ col, const VT *__restrict__ val,
                                                      const T *__restrict__ x, const T *__restrict__ y,
                                                      const T *__restrict__ v, T *__restrict__ out, int64_t n,
                                                      int64_t sstride, int r, const int *__restrict__ active,
                                                      T alpha, T beta, T gamma, T delta,
                                                      const int32_t *__restrict__ long_rows, int nlong,
                                                      int nwarp, int64_t long_len,
                                                      const int32_t *__restrict__ perm, int64_t nshort) {
  pdl_wait();
  pdl_trigger();
  unsigned mask = 0;
  for (int q = 0; q < r; ++q)
    if (!active || __ldg(active + q)) mask |= 1u << q;
  auto finish = [&](int q, int64_t row, const csr_acc<T> &sum) {
    const int64_t o = (int64_t)q * sstride + row;
    out[o] = csr_finish<T, SUB_Y, ADD_V>(sum, alpha, beta, gamma, delta, ldg(x + o),
                                         SUB_Y ? ldg(y + o) : num<T>::zero(), ADD_V ? ldg(v + o) : num<T>::zero());
  };
  csr_acc<T> acc[kCsrMaxRhs];
#pragma unroll
  for (int q = 0; q < kCsrMaxRhs; ++q) acc[q].zero();
  if ((int)blockIdx.x < nlong) {
    __shared__ csr_acc<T> red[8][kCsrMaxRhs];
    const int64_t row = __ldg(long_rows + blockIdx.x);
    const int64_t p1 = __ldg(rowptr + row + 1);
    for (int64_t p = __ldg(rowptr + row) + threadIdx.x; p < p1; p += blockDim.x) {
      const VT a = ldg(val + p);
      const int64_t cc = __ldg(col + p);
#pragma unroll
      for (int q = 0; q < kCsrMaxRhs; ++q)
        if (mask >> q & 1u) acc[q].add_prod(a, ldg(x + (int64_t)q * sstride + cc));
    }
#pragma unroll
    for (int q = 0; q < kCsrMaxRhs; ++q) {
      if (!(mask >> q & 1u)) continue;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[q].add(acc[q].shfl(o, 32));
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][q] = acc[q];
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int q = 0; q < r; ++q) {
        if (!(mask >> q & 1u)) continue;
        csr_acc<T> tot = red[0][q];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) tot.add(red[w][q]);
        finish(q, row, tot);
      }
    return;
  }
  const int nwb = (nwarp + 7) / 8;  // blocks of 8 warps, a warp per medium row
  if ((int)blockIdx.x < nlong + nwb) {
    const int wi = ((int)blockIdx.x - nlong) * 8 + (int)(threadIdx.x >> 5), ln = threadIdx.x & 31;
    if (wi >= nwarp) return;
    const int64_t row = __ldg(long_rows + nlong + wi);
    const int64_t p1 = __ldg(rowptr + row + 1);
    for (int64_t p = __ldg(rowptr + row) + ln; p < p1; p += 32) {
      const VT a = ldg(val + p);
      const int64_t cc = __ldg(col + p);
#pragma unroll
      for (int q = 0; q < kCsrMaxRhs; ++q)
        if (mask >> q & 1u) acc[q].add_prod(a, ldg(x + (int64_t)q * sstride + cc));
    }
#pragma unroll
    for (int q = 0; q < kCsrMaxRhs; ++q) {
      if (!(mask >> q & 1u)) continue;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[q].add(acc[q].shfl(o, 32));
      if (ln == 0) finish(q, row, acc[q]);
    }
    return;
  }
  const int64_t t = (int64_t)(blockIdx.x - nlong - nwb) * blockDim.x + threadIdx.x;
  const int64_t slot = t / L;
  const int lane = (int)(t % L);
  bool mine = slot < (perm ? nshort : n);
  int64_t row = slot;
  if (mine) {
    if (perm) row = __ldg(perm + slot);
    const int64_t p0 = __ldg(rowptr + row), p1 = __ldg(rowptr + row + 1);
    if (long_len > 0 && p1 - p0 > long_len) {
      mine = false;  // a long row: its own block or warp computes it
    } else {
      for (int64_t p = p0 + lane; p < p1; p += L) {
        const VT a = ldg(val + p);
        const int64_t cc = __ldg(col + p);
#pragma unroll
        for (int q = 0; q < kCsrMaxRhs; ++q)
          if (mask >> q & 1u) acc[q].add_prod(a, ldg(x + (int64_t)q * sstride + cc));
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kCsrMaxRhs; ++q) {
    if (!(mask >> q & 1u)) continue;
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) acc[q].add(acc[q].shfl(o, L));
    if (mine && lane == 0) finish(q, row, acc[q]);
  }
}

template <typename T>
T host_const(double v);
template <>
double host_const<double>(double v) {
  return v;
}
template <>
float host_const<float>(double v) {
  return (float)v;
}
template <>
dw host_const<dw>(double v) {
  return dw_split_host(v);
}

template <typename T, bool SY, bool AV>
int launch_step(const OpDesc &op, const T *x, const T *y, const T *v, T *out, const StepCoef &c,
                cudaStream_t s) {
  if (op.kind == OPK_CSR) {
    const int L = 4;
    const int64_t threads = (op.perm ? op.nshort : op.n) * L;
    const int bs = 256;
    const int64_t nb = (threads + bs - 1) / bs + (op.long_len > 0 ? op.nlong + (op.nwarp + 7) / 8 : 0);
    if (nb > 0x7fffffffll) return pp_set_error(PP_ERR_INVALID_ARG, "CSR grid too large for one launch");
    bool done = false;
    if constexpr (std::is_same<T, dw>::value) {
      if (op.val_f32) {  // values exact in FP32: read as float
        PP_CUDA_TRY(pdl_launch(csr_step<T, float, L, SY, AV>, dim3((unsigned)nb), dim3(bs), 0, s, op.rowptr,
                               op.col, (const float *)op.val, x, y, v, out, op.n, host_const<T>(c.alpha),
                               host_const<T>(c.beta), host_const<T>(c.gamma), host_const<T>(c.delta),
                               op.long_rows, op.long_len > 0 ? op.nlong : 0, op.long_len > 0 ? op.nwarp : 0,
                               op.long_len, op.perm, op.nshort));
        done = true;
      }
    }
    if (!done)
      PP_CUDA_TRY(pdl_launch(csr_step<T, T, L, SY, AV>, dim3((unsigned)nb), dim3(bs), 0, s, op.rowptr, op.col,
                             (const T *)op.val, x, y, v, out, op.n, host_const<T>(c.alpha), host_const<T>(c.beta),
                             host_const<T>(c.gamma), host_const<T>(c.delta), op.long_rows,
                             op.long_len > 0 ? op.nlong : 0, op.long_len > 0 ? op.nwarp : 0, op.long_len, op.perm,
                             op.nshort));
  } else {
    Konst<T> K;
    K.K0 = host_const<T>(c.alpha * op.d + c.beta);
    K.Km = host_const<T>(c.alpha * op.cm);
    K.Kp = host_const<T>(c.alpha * op.cp);
    K.D = host_const<T>(c.delta);
    K.Y = host_const<T>(c.gamma);
    const int nz = op.kind == OPK_ST2D ? 1 : (int)op.nz;
    // widest vector access the row length and every pointer allow
    constexpr int PW = 16 / (int)sizeof(T);
    const size_t align = (size_t)PW * sizeof(T);
    auto ok = [&](const void *p) { return p == nullptr || ((uintptr_t)p % align) == 0; };
    const bool vec = op.nx % PW == 0 && ok(x) && ok(out) && (!SY || ok(y)) && (!AV || ok(v));
    constexpr int P = PW;
    const int txs = (int)((op.nx + P - 1) / P);
    const int64_t units = (int64_t)txs * ((op.ny + 1) / 2) * nz;  // units of P entries x 2 rows
    int bs = ST_THREADS;
    if (op.tile_bdx >= 64 && op.tile_bdx <= kStencilMaxThreads && (op.tile_bdx & (op.tile_bdx - 1)) == 0)
      bs = op.tile_bdx;
    // 2D blocks (bdx units by bs / bdx rows) when a row splits into whole x
    // tiles of 64, 32, 16 or 8 units, else the flat mapping
    int bdx = 0;
    for (int c : {64, 32, 16, 8})
      if (bdx == 0 && c <= bs && txs % c == 0) bdx = c;
    const bool flat = bdx == 0;
    const int bdy = flat ? 1 : bs / bdx;
    const unsigned gx = flat ? 1u : (unsigned)(txs / bdx);
    const unsigned gy = flat ? 1u : (unsigned)(((op.ny + 1) / 2 + bdy - 1) / bdy);
    const int64_t nblk = flat ? (units + bs - 1) / bs : (int64_t)gx * gy * nz;
    if (nblk > 0x7fffffffll) return pp_set_error(PP_ERR_INVALID_ARG, "grid too large for one launch");
    const dim3 blk = flat ? dim3(bs) : dim3(bdx, bdy);
#define PP_ST(V, F)                                                                                       \
  PP_CUDA_TRY(pdl_launch(st_step<T, PW, V, F, SY, AV>, dim3((unsigned)nblk), blk, 0, s, x, y, v, out,      \
                         (int)op.nx, (int)op.ny, nz, txs, units, gx, gy, K))
    if (vec && flat)
      PP_ST(true, true);
    else if (vec)
      PP_ST(true, false);
    else if (flat)
      PP_ST(false, true);
    else
      PP_ST(false, false);
#undef PP_ST
  }
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}

}  // namespace

template <typename T>
int op_step(const OpDesc &op, const T *x, const T *y, const T *v, T *out, const StepCoef &c,
            cudaStream_t s) {
  if (op.kind == OPK_WILSON) return wilson_op_step<T>(op, x, y, v, out, c, s);
  if (c.sub_y && c.add_v) return launch_step<T, true, true>(op, x, y, v, out, c, s);
  if (c.sub_y) return launch_step<T, true, false>(op, x, y, v, out, c, s);
  if (c.add_v) return launch_step<T, false, true>(op, x, y, v, out, c, s);
  return launch_step<T, false, false>(op, x, y, v, out, c, s);
}

template <typename T>
int op_step_csr_multi(const OpDesc &op, int64_t sstride, int r, const int *active, const T *x, const T *y,
                      const T *v, T *out, const StepCoef &c, cudaStream_t s) {
  if (op.kind != OPK_CSR || r < 1 || r > kCsrMaxRhs) return pp_set_error(PP_ERR_INVALID_ARG, "bad CSR block step");
  constexpr int L = 4;
  const int64_t threads = (op.perm ? op.nshort : op.n) * L;
  const int bs = 256;
  const int64_t nb = (threads + bs - 1) / bs + (op.long_len > 0 ? op.nlong + (op.nwarp + 7) / 8 : 0);
  if (nb > 0x7fffffffll) return pp_set_error(PP_ERR_INVALID_ARG, "CSR grid too large for one launch");
  cudaError_t e = cudaSuccess;
  bool vf = false;  // values exact in FP32: read as float (double-word vectors)
  if constexpr (std::is_same<T, dw>::value) vf = op.val_f32 != 0;
#define PP_CSRM_T(VT, SY, AV)                                                                                  \
  e = pdl_launch(csr_step_multi<T, VT, L, SY, AV>, dim3((unsigned)nb), dim3(bs), 0, s, op.rowptr, op.col,      \
                 (const VT *)op.val, x, y, v, out, op.n, sstride, r, active, host_const<T>(c.alpha),          \
                 host_const<T>(c.beta), host_const<T>(c.gamma), host_const<T>(c.delta), op.long_rows,        \
                 op.long_len > 0 ? op.nlong : 0, op.long_len > 0 ? op.nwarp : 0, op.long_len, op.perm, op.nshort)
#define PP_CSRM(SY, AV)                       \
  do {                                        \
    if constexpr (std::is_same<T, dw>::value) \
      if (vf) {                               \
        PP_CSRM_T(float, SY, AV);             \
        break;                                \
      }                                       \
    PP_CSRM_T(T, SY, AV);                     \
  } while (0)
  if (c.sub_y && c.add_v) PP_CSRM(true, true);
  else if (c.sub_y) PP_CSRM(true, false);
  else if (c.add_v) PP_CSRM(false, true);
  else PP_CSRM(false, false);
#undef PP_CSRM
#undef PP_CSRM_T
  PP_CUDA_TRY(e);
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}

template <typename T>
void batch_konst(const double *d, const double *cm, const double *cp, const StepCoef *c, int nseg,
                 Konst<T> *out) {
  for (int i = 0; i < nseg; ++i) {
    out[i].K0 = host_const<T>(c[i].alpha * d[i] + c[i].beta);
    out[i].Km = host_const<T>(c[i].alpha * cm[i]);
    out[i].Kp = host_const<T>(c[i].alpha * cp[i]);
    out[i].D = host_const<T>(c[i].delta);
    out[i].Y = host_const<T>(c[i].gamma);
  }
}

template <typename T>
int op_step_batch(const BatchSeg *segs, const int *blkseg, unsigned nblk, int P, const Konst<T> *K,
                  const int *active, const T *x, const T *y, const T *v, T *out, bool sub_y, bool add_v,
                  cudaStream_t s) {
  constexpr int PW = 16 / (int)sizeof(T);
  const dim3 blk(ST_THREADS);
#define PP_BST(PP, SY, AV) \
  e = pdl_launch(bst_step<T, PP, SY, AV>, dim3(nblk), blk, 0, s, x, y, v, out, segs, blkseg, K, active)
  cudaError_t e;
  (void)P;  // always PW entries per thread; each segment picks its load path
  if (sub_y && add_v) PP_BST(PW, true, true);
  else if (sub_y) PP_BST(PW, true, false);
  else if (add_v) PP_BST(PW, false, true);
  else PP_BST(PW, false, false);
#undef PP_BST
  PP_CUDA_TRY(e);
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}

#define PP_BINST(T)                                                                                   \
  template void batch_konst<T>(const double *, const double *, const double *, const StepCoef *, int, \
                               Konst<T> *);                                                          \
  template int op_step_batch<T>(const BatchSeg *, const int *, unsigned, int, const Konst<T> *, const int *, \
                                const T *, const T *, const T *, T *, bool, bool, cudaStream_t); \
  template int op_step_csr_multi<T>(const OpDesc &, int64_t, int, const int *, const T *, const T *, const T *, \
                                    T *, const StepCoef &, cudaStream_t);
PP_BINST(double)
PP_BINST(float)
PP_BINST(dw)

template int op_step<double>(const OpDesc &, const double *, const double *, const double *, double *,
                             const StepCoef &, cudaStream_t);
template int op_step<float>(const OpDesc &, const float *, const float *, const float *, float *,
                            const StepCoef &, cudaStream_t);
template int op_step<dw>(const OpDesc &, const dw *, const dw *, const dw *, dw *, const StepCoef &,
                         cudaStream_t);
