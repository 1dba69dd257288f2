// Wilson-type lattice operator for A = D^H D (a Hermitian positive definite
// stand-in for the lattice QCD kernel of Sec. 6, Example 2):
//
//   (D psi)(x) = (4 + m0) psi(x)
//                - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x)        psi(x + mu)
//                             + (1 + gamma_mu) U_mu(x - mu)^H psi(x - mu) ]
//
// on a periodic L0 x L1 x L2 x L3 lattice (site s = ((x3 L2 + x2) L1 + x1) L0
// + x0), 12 complex components per site (index spin * 3 + colour, real and
// imaginary parts interleaved), links U_mu(s) as complex64 3 x 3 matrices at
// links[((s * 4 + mu) * 3 + a) * 3 + b].  The gamma matrices are the Euclidean
// chiral representation gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
// gamma_4 = [[0, 1], [1, 0]].  D^H is the same operator with the two
// projectors exchanged.
//
// Each hop is done on a half spinor: (1 + S gamma_mu) has rank 2, so the
// neighbour spinor is projected to two spin rows h0, h1 (3 colours each),
// multiplied by the link, and the two lower rows are rebuilt from the upper
// ones with the constant factors of the projector.  The vector arithmetic is
// FP64, double-word pairs or FP32 (the link entries are exact in all three).
//
// Two threads (adjacent lanes) share a site: the thread of parity `half`
// forms h_half only (it reads the two neighbour spin rows that feed it),
// accumulates its upper output row (spin half) and partial sums of both
// lower rows, and the pair exchanges the partial lower rows once at the end
// (one shuffle per entry).  The two threads run the same instructions (the
// projector's signs and row choices are runtime values of `half`), and each
// holds a third fewer accumulators than a thread owning the whole site
// (double-word: 139 -> about 90 registers, so more warps per SM hide the
// latency of the dependent double-word operations).
//
// A Clenshaw step out = alpha A x + beta x - y + delta v takes two launches:
// t = D x, then out = alpha D^H t + beta x - y + delta v.
//
// A = Q^2 with Q = Gamma_5 D(m_w, mu) (Sec. 6, Example 2): the same D with
// mass m_w and chemical potential mu, whose hop to x + 3 (direction 3, gamma_4)
// carries e^{mu} and whose hop to x - 3 carries e^{-mu}; Gamma_5 =
// diag(1, 1, -1, -1) on spin.  A step is t = Q x, then out = alpha Q t +
// beta x + delta v with complex alpha, beta, delta (a q with complex
// coefficients); Q is non-Hermitian for mu != 0.
#include "common.cuh"
#include "internal.h"

namespace {

template <typename T>
struct cx {
  T re, im;
};

template <typename T>
__device__ __forceinline__ T from_f(float f);
template <>
__device__ __forceinline__ double from_f<double>(float f) {
  return (double)f;
}
template <>
__device__ __forceinline__ float from_f<float>(float f) {
  return f;
}

// a + S b and a + S i b for S = +1 / -1
template <int S, typename T>
__device__ __forceinline__ cx<T> add_s(const cx<T> &a, const cx<T> &b) {
  if (S > 0) return {a.re + b.re, a.im + b.im};
  return {a.re - b.re, a.im - b.im};
}
template <int S, typename T>
__device__ __forceinline__ cx<T> add_si(const cx<T> &a, const cx<T> &b) {
  // S i (br + i bi) = -S bi + i S br
  if (S > 0) return {a.re - b.im, a.im + b.re};
  return {a.re + b.im, a.im - b.re};
}

template <typename T>
__device__ __forceinline__ cx<T> ld_c(const T *p, int k) {
  return {ldg(p + 2 * k), ldg(p + 2 * k + 1)};
}

// The arithmetic a link entry enters the products in: FP32 for double-word
// vectors (the entries are floats; a dw x float product is one FMA
// shorter), the vector arithmetic otherwise.
template <typename T>
struct link_arith {
  using type = T;
};
template <>
struct link_arith<dw> {
  using type = float;
};

// chi[a] = sum_b M_ab h[b] with M = U (ADJ = false) or U^H (ADJ = true)
template <bool ADJ, typename T>
__device__ __forceinline__ void color_mul(const float2 (&u)[9], const cx<T> (&h)[3], cx<T> (&chi)[3]) {
  using A = typename acc_of<T>::type;
  using C = typename link_arith<T>::type;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    A re, im;
    acc_set(re, num<T>::zero());
    acc_set(im, num<T>::zero());
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float2 m = ADJ ? u[b * 3 + a] : u[a * 3 + b];
      const C mr = from_f<C>(m.x);
      const C mi = from_f<C>(ADJ ? -m.y : m.y);
      const C nmi = from_f<C>(ADJ ? m.y : -m.y);
      // (mr + i mi)(hr + i hi) = (mr hr - mi hi) + i (mr hi + mi hr)
      acc_add_prod(re, mr, h[b].re);
      acc_add_prod(re, nmi, h[b].im);
      acc_add_prod(im, mr, h[b].im);
      acc_add_prod(im, mi, h[b].re);
    }
    chi[a] = {acc_get(re), acc_get(im)};
  }
}

// (neg ? -a : a) by flipping sign bits (integer pipe, no floating-point
// operation and no select between two computed values)
__device__ __forceinline__ float neg_if(float a, bool neg) {
  return __int_as_float(__float_as_int(a) ^ (neg ? 0x80000000u : 0u));
}
__device__ __forceinline__ double neg_if(double a, bool neg) {
  const unsigned long long m = neg ? 0x8000000000000000ull : 0ull;
  return __longlong_as_double((long long)((unsigned long long)__double_as_longlong(a) ^ m));
}
__device__ __forceinline__ dw neg_if(dw a, bool neg) {
  const unsigned m = neg ? 0x80000000u : 0u;
  return {__int_as_float(__float_as_int(a.hi) ^ m), __int_as_float(__float_as_int(a.lo) ^ m)};
}

// The rows the thread of parity `half` owns, [colour * 2 + {re, im}]: u the
// upper row (spin half), p the lower row 2 + half, x the lower row 3 - half
// (partial: its sum goes to the partner thread).
template <typename A>
struct Rows {
  A u[6], p[6], x[6];
};

// dst += (neg ? -1 : 1) (IM ? i : 1) c
template <bool IM, typename A, typename T>
__device__ __forceinline__ void acc_c(A *dst, const cx<T> (&c)[3], bool neg) {
#pragma unroll
  for (int col = 0; col < 3; ++col) {
    const T re = IM ? -c[col].im : c[col].re;  // i (re + i im) = -im + i re
    const T im = IM ? c[col].re : c[col].im;
    acc_add(dst[2 * col], neg_if(re, neg));
    acc_add(dst[2 * col + 1], neg_if(im, neg));
  }
}

// One hop in direction MU, the thread's half: with the projector
// (1 + S gamma_MU) the half spinor is h_half = p_half + sg (i) p_lo of the
// neighbour (MU 0: h0 = p0 - S i p3, h1 = p1 - S i p2; MU 1: h0 = p0 - S p3,
// h1 = p1 + S p2; MU 2: h0 = p0 - S i p2, h1 = p1 + S i p3; MU 3: h0 = p0 +
// S p2, h1 = p1 + S p3), chi = M h_half (M = U or U^H, times f when SCALE)
// goes to the upper row, and the projector's lower rows get (MU 0: row 3 +=
// S i chi0, row 2 += S i chi1; MU 1: row 3 -= S chi0, row 2 += S chi1; MU 2:
// row 2 += S i chi0, row 3 -= S i chi1; MU 3: row 2 += S chi0, row 3 += S chi1).
template <int MU, int S, bool ADJ, bool SCALE, typename A, typename T>
__device__ __forceinline__ void hop_body(Rows<A> &R, const T *__restrict__ psi, const float2 (&u)[9], T f,
                                         int half) {
  constexpr bool IM = MU == 0 || MU == 2;
  const int lo = MU <= 1 ? 3 - half : 2 + half;
  const bool nsg = MU == 0 ? (S > 0) : MU == 3 ? (S < 0) : (half ? S < 0 : S > 0);
  cx<T> h[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cx<T> pu = ld_c(psi, half * 3 + c), pl = ld_c(psi, lo * 3 + c);
    const T are = IM ? -pl.im : pl.re, aim = IM ? pl.re : pl.im;
    h[c] = {pu.re + neg_if(are, nsg), pu.im + neg_if(aim, nsg)};
  }
  cx<T> chi[3];
  color_mul<ADJ>(u, h, chi);
  if constexpr (SCALE) {
#pragma unroll
    for (int c = 0; c < 3; ++c) chi[c] = {chi[c].re * f, chi[c].im * f};
  }
  acc_c<false>(R.u, chi, false);
  const bool ntg = MU == 0 ? (S < 0) : MU == 3 ? (S < 0) : MU == 1 ? (half ? S < 0 : S > 0) : (half ? S > 0 : S < 0);
  if (MU <= 1)
    acc_c<IM>(R.x, chi, ntg);
  else
    acc_c<IM>(R.p, chi, ntg);
}

// The thread's half of a hop (thread pair per site).
template <int MU, int S, bool ADJ, bool SCALE, typename A, typename T>
__device__ __forceinline__ void hop(Rows<A> &R, const T *__restrict__ psi, const float2 *__restrict__ link, T f,
                                    int half) {
  float2 u[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) u[k] = __ldg(link + k);
  hop_body<MU, S, ADJ, SCALE>(R, psi, u, f, half);
}

// Both halves of a hop in one thread (the link loaded once).
template <int MU, int S, bool ADJ, bool SCALE, typename A, typename T>
__device__ __forceinline__ void hop2(Rows<A> &R0, Rows<A> &R1, const T *__restrict__ psi,
                                     const float2 *__restrict__ link, T f) {
  float2 u[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) u[k] = __ldg(link + k);
  hop_body<MU, S, ADJ, SCALE>(R0, psi, u, f, 0);
  hop_body<MU, S, ADJ, SCALE>(R1, psi, u, f, 1);
}

template <typename T>
__device__ __forceinline__ T shfl_partner(T v) {
  return __shfl_xor_sync(0xffffffffu, v, 1);
}
template <>
__device__ __forceinline__ dw shfl_partner<dw>(dw v) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, 1), __shfl_xor_sync(0xffffffffu, v.lo, 1)};
}

// Double-word and FP32 sites take a thread pair; FP64 (bound by the narrow
// FP64 pipe, where the pair measured slower: 0.69 against 0.57 ms per D^H D
// at 16^3 x 32) keeps one thread per site doing both halves (0.58 ms).
template <typename T>
constexpr bool kPairSites = !std::is_same<T, double>::value;

template <typename T, typename A>
__device__ __forceinline__ void rows_zero(Rows<A> &R) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    acc_set(R.u[k], num<T>::zero());
    acc_set(R.p[k], num<T>::zero());
    acc_set(R.x[k], num<T>::zero());
  }
}

// One thread with both halves: row 2 = R0.p + R1.x, row 3 = R1.p + R0.x.
template <typename T, typename A>
__device__ __forceinline__ void rows_merge(Rows<A> &R0, Rows<A> &R1) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const T a = acc_get(R1.x[k]), b = acc_get(R0.x[k]);
    acc_add(R0.p[k], a);
    acc_add(R1.p[k], b);
  }
}

// p += the partner's x: both lower rows complete (every lane of the warp
// takes part)
template <typename T, typename A>
__device__ __forceinline__ void pair_exchange(Rows<A> &R) {
#pragma unroll
  for (int k = 0; k < 6; ++k) acc_add(R.p[k], shfl_partner<T>(acc_get(R.x[k])));
}

struct Lat {
  int L[4];
  int64_t st[4];  // site strides
  int64_t V;
};

// CHEM: the direction-3 hops carry ef (forward) and eb (backward).
template <int MU, bool DAG, bool CHEM, typename A, typename T>
__device__ __forceinline__ void hop_pair(Rows<A> &R, const T *__restrict__ in, const float2 *__restrict__ U,
                                         const Lat &lat, int64_t s, int coord, T ef, T eb, int half) {
  const int L = lat.L[MU];
  const int64_t st = lat.st[MU];
  const int64_t fwd = s + (coord + 1 == L ? -(int64_t)(L - 1) * st : st);
  const int64_t bwd = s + (coord == 0 ? (int64_t)(L - 1) * st : -st);
  constexpr bool SC = CHEM && MU == 3;
  // D: forward (1 - gamma), backward (1 + gamma); D^H: exchanged
  hop<MU, DAG ? 1 : -1, false, SC>(R, in + fwd * 24, U + (s * 4 + MU) * 9, ef, half);
  hop<MU, DAG ? -1 : 1, true, SC>(R, in + bwd * 24, U + (bwd * 4 + MU) * 9, eb, half);
}

// hop_pair for one thread doing both halves of the site.
template <int MU, bool DAG, bool CHEM, typename A, typename T>
__device__ __forceinline__ void hop_pair2(Rows<A> &R0, Rows<A> &R1, const T *__restrict__ in,
                                          const float2 *__restrict__ U, const Lat &lat, int64_t s, int coord, T ef,
                                          T eb) {
  const int L = lat.L[MU];
  const int64_t st = lat.st[MU];
  const int64_t fwd = s + (coord + 1 == L ? -(int64_t)(L - 1) * st : st);
  const int64_t bwd = s + (coord == 0 ? (int64_t)(L - 1) * st : -st);
  constexpr bool SC = CHEM && MU == 3;
  hop2<MU, DAG ? 1 : -1, false, SC>(R0, R1, in + fwd * 24, U + (s * 4 + MU) * 9, ef);
  hop2<MU, DAG ? -1 : 1, true, SC>(R0, R1, in + bwd * 24, U + (bwd * 4 + MU) * 9, eb);
}

// Lattice coordinates of site s.
__device__ __forceinline__ void site_coords(const Lat &lat, int64_t s, int *c) {
  int64_t r = s;
  c[0] = (int)(r % lat.L[0]);
  r /= lat.L[0];
  c[1] = (int)(r % lat.L[1]);
  r /= lat.L[1];
  c[2] = (int)(r % lat.L[2]);
  c[3] = (int)(r / lat.L[2]);
}

// out = Kd in + Kh (hop sum of in) [+ Kb x] [+ Ky y] [+ Kv v], two threads
// per site (thread 2 s + half writes spin rows half and 2 + half).
template <typename T, bool DAG, bool ADD_X, bool SUB_Y, bool ADD_V>
__global__ void __launch_bounds__(128) wilson_step(const T *__restrict__ in, const T *__restrict__ x,
                                                   const T *__restrict__ y, const T *__restrict__ v,
                                                   T *__restrict__ out, const float2 *__restrict__ U,
                                                   Lat lat, T Kd, T Kh, T Kb, T Ky, T Kv) {
  pdl_wait();
  pdl_trigger();
  using A = typename acc_of<T>::type;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const T one = num<T>::from_d(1.0);
  // rows half and 2 + half of site s from R (u: upper, p: lower)
  auto epi = [&](const Rows<A> &R, int64_t s, int half) {
    const int64_t o = s * 24;
#pragma unroll
    for (int k = 0; k < 12; ++k) {  // the upper row's 6 entries, then the lower row's
      const int64_t g = o + (k < 6 ? 6 * half + k : 12 + 6 * half + (k - 6));
      A res;
      acc_set_prod(res, Kd, ldg(in + g));
      acc_add_prod(res, Kh, acc_raw(k < 6 ? R.u[k] : R.p[k - 6]));
      if (ADD_X) acc_add_prod(res, Kb, ldg(x + g));
      if (SUB_Y) acc_add_prod(res, Ky, ldg(y + g));
      if (ADD_V) acc_add_prod(res, Kv, ldg(v + g));
      out[g] = acc_get(res);
    }
  };
  if constexpr (kPairSites<T>) {
    const int half = (int)(tid & 1);
    const bool valid = (tid >> 1) < lat.V;
    const int64_t s = valid ? (tid >> 1) : lat.V - 1;  // lanes past the end compute a site, store nothing
    int c[4];
    site_coords(lat, s, c);
    Rows<A> R;
    rows_zero<T>(R);
    hop_pair<0, DAG, false>(R, in, U, lat, s, c[0], one, one, half);
    hop_pair<1, DAG, false>(R, in, U, lat, s, c[1], one, one, half);
    hop_pair<2, DAG, false>(R, in, U, lat, s, c[2], one, one, half);
    hop_pair<3, DAG, false>(R, in, U, lat, s, c[3], one, one, half);
    pair_exchange<T>(R);
    if (valid) epi(R, s, half);
  } else {  // one thread, both halves (compile-time signs)
    const int64_t s = tid;
    if (s >= lat.V) return;
    int c[4];
    site_coords(lat, s, c);
    Rows<A> R0, R1;
    rows_zero<T>(R0);
    rows_zero<T>(R1);
    hop_pair2<0, DAG, false>(R0, R1, in, U, lat, s, c[0], one, one);
    hop_pair2<1, DAG, false>(R0, R1, in, U, lat, s, c[1], one, one);
    hop_pair2<2, DAG, false>(R0, R1, in, U, lat, s, c[2], one, one);
    hop_pair2<3, DAG, false>(R0, R1, in, U, lat, s, c[3], one, one);
    rows_merge<T>(R0, R1);
    epi(R0, s, 0);
    epi(R1, s, 1);
  }
}

// Complex coefficients of a Q^2 step, with the negated imaginary parts the
// products need.
template <typename T>
struct QCoef {
  T ar, ai, nai, br, bi, nbi, dr, di, ndi;
};

// Output rows half and 2 + half of site s for wilson_q_step.
template <typename T, bool EPI, bool AX, bool AV, typename A>
__device__ __forceinline__ void q_epi(const Rows<A> &R, int64_t s, int half, const T *__restrict__ in,
                                      const T *__restrict__ x, const T *__restrict__ v, T *__restrict__ out, T Kd,
                                      T Kh, const QCoef<T> &k) {
  const int64_t o = s * 24;
#pragma unroll
  for (int q = 0; q < 6; ++q) {  // (re, im) pairs: 3 of the upper row, 3 of the lower row
    const bool lower = q >= 3;
    const int col = lower ? q - 3 : q;
    const int64_t g = o + (lower ? 12 : 0) + 6 * half + 2 * col;
    A tr, ti;
    acc_set_prod(tr, Kd, ldg(in + g));
    acc_add_prod(tr, Kh, acc_raw(lower ? R.p[2 * col] : R.u[2 * col]));
    acc_set_prod(ti, Kd, ldg(in + g + 1));
    acc_add_prod(ti, Kh, acc_raw(lower ? R.p[2 * col + 1] : R.u[2 * col + 1]));
    T dr = acc_get(tr), di = acc_get(ti);
    if (lower) {  // Gamma_5: spins 2 and 3 change sign
      dr = -dr;
      di = -di;
    }
    if constexpr (!EPI) {
      out[g] = dr;
      out[g + 1] = di;
    } else {
      A rr, ri;
      acc_set_prod(rr, k.ar, dr);
      acc_add_prod(rr, k.nai, di);
      acc_set_prod(ri, k.ar, di);
      acc_add_prod(ri, k.ai, dr);
      if constexpr (AX) {
        const T xr = ldg(x + g), xi = ldg(x + g + 1);
        acc_add_prod(rr, k.br, xr);
        acc_add_prod(rr, k.nbi, xi);
        acc_add_prod(ri, k.br, xi);
        acc_add_prod(ri, k.bi, xr);
      }
      if constexpr (AV) {
        const T vr = ldg(v + g), vi = ldg(v + g + 1);
        acc_add_prod(rr, k.dr, vr);
        acc_add_prod(rr, k.ndi, vi);
        acc_add_prod(ri, k.dr, vi);
        acc_add_prod(ri, k.di, vr);
      }
      out[g] = acc_get(rr);
      out[g + 1] = acc_get(ri);
    }
  }
}

// Q = Gamma_5 D(m_w, mu): EPI = false: out = Q in; EPI: out = alpha (Q in)
// [+ beta x] [+ delta v] with complex alpha, beta, delta.  Two threads per
// site as in wilson_step.
template <typename T, bool EPI, bool AX, bool AV>
__global__ void __launch_bounds__(128) wilson_q_step(const T *__restrict__ in, const T *__restrict__ x,
                                                     const T *__restrict__ v, T *__restrict__ out,
                                                     const float2 *__restrict__ U, Lat lat, T Kd, T Kh, T ef,
                                                     T eb, QCoef<T> k) {
  pdl_wait();
  pdl_trigger();
  using A = typename acc_of<T>::type;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if constexpr (kPairSites<T>) {
    const int half = (int)(tid & 1);
    const bool valid = (tid >> 1) < lat.V;
    const int64_t s = valid ? (tid >> 1) : lat.V - 1;
    int c[4];
    site_coords(lat, s, c);
    Rows<A> R;
    rows_zero<T>(R);
    hop_pair<0, false, true>(R, in, U, lat, s, c[0], ef, eb, half);
    hop_pair<1, false, true>(R, in, U, lat, s, c[1], ef, eb, half);
    hop_pair<2, false, true>(R, in, U, lat, s, c[2], ef, eb, half);
    hop_pair<3, false, true>(R, in, U, lat, s, c[3], ef, eb, half);
    pair_exchange<T>(R);
    if (valid) q_epi<T, EPI, AX, AV>(R, s, half, in, x, v, out, Kd, Kh, k);
  } else {
    const int64_t s = tid;
    if (s >= lat.V) return;
    int c[4];
    site_coords(lat, s, c);
    Rows<A> R0, R1;
    rows_zero<T>(R0);
    rows_zero<T>(R1);
    hop_pair2<0, false, true>(R0, R1, in, U, lat, s, c[0], ef, eb);
    hop_pair2<1, false, true>(R0, R1, in, U, lat, s, c[1], ef, eb);
    hop_pair2<2, false, true>(R0, R1, in, U, lat, s, c[2], ef, eb);
    hop_pair2<3, false, true>(R0, R1, in, U, lat, s, c[3], ef, eb);
    rows_merge<T>(R0, R1);
    q_epi<T, EPI, AX, AV>(R0, s, 0, in, x, v, out, Kd, Kh, k);
    q_epi<T, EPI, AX, AV>(R1, s, 1, in, x, v, out, Kd, Kh, k);
  }
}

template <typename T>
T host_c(double v);
template <>
double host_c<double>(double v) {
  return v;
}
template <>
float host_c<float>(double v) {
  return (float)v;
}
template <>
dw host_c<dw>(double v) {
  return dw_split_host(v);
}

template <typename T, bool DAG, bool AX, bool SY, bool AV>
int launch(const T *in, const T *x, const T *y, const T *v, T *out, const float2 *U, const Lat &lat,
           double kd, double kh, double kb, double ky, double kv, cudaStream_t s) {
  const int bs = 128;
  const int64_t nb = ((kPairSites<T> ? 2 : 1) * lat.V + bs - 1) / bs;  // threads per site
  PP_CUDA_TRY(pdl_launch(wilson_step<T, DAG, AX, SY, AV>, dim3((unsigned)nb), dim3(bs), 0, s, in, x, y, v, out, U, lat, host_c<T>(kd),
                                                             host_c<T>(kh), host_c<T>(kb), host_c<T>(ky),
                                                             host_c<T>(kv)));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}

Lat make_lat(const OpDesc &op) {
  Lat lat;
  lat.V = 1;
  for (int d = 0; d < 4; ++d) {
    lat.L[d] = (int)op.L[d];
    lat.st[d] = lat.V;
    lat.V *= op.L[d];
  }
  return lat;
}

template <typename T, bool EPI, bool AX, bool AV>
int launch_q(const OpDesc &op, const T *in, const T *x, const T *v, T *out, const StepCoef &c, cudaStream_t s) {
  const Lat lat = make_lat(op);
  const int bs = 128;
  const int64_t nb = ((kPairSites<T> ? 2 : 1) * lat.V + bs - 1) / bs;  // threads per site
  QCoef<T> k;
  k.ar = host_c<T>(c.alpha);
  k.ai = host_c<T>(c.alpha_im);
  k.nai = host_c<T>(-c.alpha_im);
  k.br = host_c<T>(c.beta);
  k.bi = host_c<T>(c.beta_im);
  k.nbi = host_c<T>(-c.beta_im);
  k.dr = host_c<T>(c.delta);
  k.di = host_c<T>(c.delta_im);
  k.ndi = host_c<T>(-c.delta_im);
  PP_CUDA_TRY(pdl_launch(wilson_q_step<T, EPI, AX, AV>, dim3((unsigned)nb), dim3(bs), 0, s, in, x, v, out,
                         (const float2 *)op.links, lat, host_c<T>(4.0 + op.mass), host_c<T>(-0.5),
                         host_c<T>(std::exp(op.mu_c)), host_c<T>(std::exp(-op.mu_c)), k));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}

// t = Q x, then out = alpha Q t [+ beta x] [+ delta v] (complex coefficients)
template <typename T>
int wilson_q2_step(const OpDesc &op, const T *x, const T *v, T *out, const StepCoef &c, cudaStream_t s) {
  if (c.sub_y) return pp_set_error(PP_ERR_UNSUPPORTED, "Q^2 step with a y term");
  T *t = (T *)op.tmp;
  int rc = launch_q<T, false, false, false>(op, x, nullptr, nullptr, t, c, s);
  if (rc) return rc;
  const bool ax = c.beta != 0.0 || c.beta_im != 0.0;
  if (ax && c.add_v) return launch_q<T, true, true, true>(op, t, x, v, out, c, s);
  if (ax) return launch_q<T, true, true, false>(op, t, x, v, out, c, s);
  if (c.add_v) return launch_q<T, true, false, true>(op, t, x, v, out, c, s);
  return launch_q<T, true, false, false>(op, t, x, v, out, c, s);
}

}  // namespace

template <typename T>
int wilson_q_apply(const OpDesc &op, const T *x, T *out, cudaStream_t s) {
  const StepCoef c{1.0, 0.0, 0.0, false, false};
  return launch_q<T, false, false, false>(op, x, nullptr, nullptr, out, c, s);
}
template int wilson_q_apply<double>(const OpDesc &, const double *, double *, cudaStream_t);
template int wilson_q_apply<float>(const OpDesc &, const float *, float *, cudaStream_t);
template int wilson_q_apply<dw>(const OpDesc &, const dw *, dw *, cudaStream_t);

template <typename T>
int wilson_op_step(const OpDesc &op, const T *x, const T *y, const T *v, T *out, const StepCoef &c,
                   cudaStream_t s) {
  if (op.q2) return wilson_q2_step<T>(op, x, v, out, c, s);
  const Lat lat = make_lat(op);
  const float2 *U = (const float2 *)op.links;
  T *t = (T *)op.tmp;
  const double md = 4.0 + op.mass;
  // t = D x
  int rc = launch<T, false, false, false, false>(x, nullptr, nullptr, nullptr, t, U, lat, md, -0.5, 0.0,
                                                 0.0, 0.0, s);
  if (rc) return rc;
  // out = alpha D^H t + beta x [+ gamma y] [+ delta v]
  const double kd = c.alpha * md, kh = -0.5 * c.alpha;
  const bool ax = c.beta != 0.0;
  if (!ax && !c.sub_y && !c.add_v)
    return launch<T, true, false, false, false>(t, x, y, v, out, U, lat, kd, kh, 0.0, c.gamma, 0.0, s);
  if (ax && !c.sub_y && !c.add_v)
    return launch<T, true, true, false, false>(t, x, y, v, out, U, lat, kd, kh, c.beta, c.gamma, 0.0, s);
  if (ax && !c.sub_y && c.add_v)
    return launch<T, true, true, false, true>(t, x, y, v, out, U, lat, kd, kh, c.beta, c.gamma, c.delta, s);
  if (ax && c.sub_y && c.add_v)
    return launch<T, true, true, true, true>(t, x, y, v, out, U, lat, kd, kh, c.beta, c.gamma, c.delta, s);
  if (ax && c.sub_y && !c.add_v)
    return launch<T, true, true, true, false>(t, x, y, v, out, U, lat, kd, kh, c.beta, c.gamma, 0.0, s);
  if (!ax && c.add_v && !c.sub_y)
    return launch<T, true, false, false, true>(t, x, y, v, out, U, lat, kd, kh, 0.0, c.gamma, c.delta, s);
  if (!ax && c.sub_y && c.add_v)
    return launch<T, true, false, true, true>(t, x, y, v, out, U, lat, kd, kh, 0.0, c.gamma, c.delta, s);
  return launch<T, true, false, true, false>(t, x, y, v, out, U, lat, kd, kh, 0.0, c.gamma, 0.0, s);
}

template int wilson_op_step<double>(const OpDesc &, const double *, const double *, const double *, double *,
                                    const StepCoef &, cudaStream_t);
template int wilson_op_step<float>(const OpDesc &, const float *, const float *, const float *, float *,
                                   const StepCoef &, cudaStream_t);
template int wilson_op_step<dw>(const OpDesc &, const dw *, const dw *, const dw *, dw *, const StepCoef &,
                                cudaStream_t);
