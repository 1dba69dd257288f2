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
template <>
__device__ __forceinline__ dw from_f<dw>(float f) {
  return {f, 0.f};
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

// hs[(row * 3 + col) * 2 + {0, 1}] += f * chi[col], f in {1, -1, i, -i} = (FI ? i : 1) * FS
template <int FS, bool FI, typename A, typename T>
__device__ __forceinline__ void acc_row(A *hs, int row, const cx<T> (&chi)[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    A &r = hs[(row * 3 + c) * 2 + 0];
    A &i = hs[(row * 3 + c) * 2 + 1];
    if (!FI) {
      if (FS > 0) {
        acc_add(r, chi[c].re);
        acc_add(i, chi[c].im);
      } else {
        acc_sub(r, chi[c].re);
        acc_sub(i, chi[c].im);
      }
    } else {  // FS i (re + i im) = -FS im + i FS re
      if (FS > 0) {
        acc_sub(r, chi[c].im);
        acc_add(i, chi[c].re);
      } else {
        acc_add(r, chi[c].im);
        acc_sub(i, chi[c].re);
      }
    }
  }
}

// chi[a] = sum_b M_ab h[b] with M = U (ADJ = false) or U^H (ADJ = true)
template <bool ADJ, typename T>
__device__ __forceinline__ void color_mul(const float2 (&u)[9], const cx<T> (&h)[3], cx<T> (&chi)[3]) {
  using A = typename acc_of<T>::type;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    A re, im;
    acc_set(re, num<T>::zero());
    acc_set(im, num<T>::zero());
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float2 m = ADJ ? u[b * 3 + a] : u[a * 3 + b];
      const T mr = from_f<T>(m.x);
      const T mi = from_f<T>(ADJ ? -m.y : m.y);
      const T nmi = from_f<T>(ADJ ? m.y : -m.y);
      // (mr + i mi)(hr + i hi) = (mr hr - mi hi) + i (mr hi + mi hr)
      acc_add_prod(re, mr, h[b].re);
      acc_add_prod(re, nmi, h[b].im);
      acc_add_prod(im, mr, h[b].im);
      acc_add_prod(im, mi, h[b].re);
    }
    chi[a] = {acc_get(re), acc_get(im)};
  }
}

// One hop in direction MU: hs += (1 + S gamma_MU) M psi_nb, M = U or U^H,
// times f when SCALE (the chemical-potential factor).
template <int MU, int S, bool ADJ, bool SCALE, typename A, typename T>
__device__ __forceinline__ void hop(A *hs, const T *__restrict__ psi, const float2 *__restrict__ link, T f) {
  float2 u[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) u[k] = __ldg(link + k);
  cx<T> h0[3], h1[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cx<T> p0 = ld_c(psi, 0 * 3 + c), p1 = ld_c(psi, 1 * 3 + c);
    const cx<T> p2 = ld_c(psi, 2 * 3 + c), p3 = ld_c(psi, 3 * 3 + c);
    if (MU == 0) {  // h0 = p0 - S i p3, h1 = p1 - S i p2
      h0[c] = add_si<-S>(p0, p3);
      h1[c] = add_si<-S>(p1, p2);
    } else if (MU == 1) {  // h0 = p0 - S p3, h1 = p1 + S p2
      h0[c] = add_s<-S>(p0, p3);
      h1[c] = add_s<S>(p1, p2);
    } else if (MU == 2) {  // h0 = p0 - S i p2, h1 = p1 + S i p3
      h0[c] = add_si<-S>(p0, p2);
      h1[c] = add_si<S>(p1, p3);
    } else {  // h0 = p0 + S p2, h1 = p1 + S p3
      h0[c] = add_s<S>(p0, p2);
      h1[c] = add_s<S>(p1, p3);
    }
  }
  cx<T> c0[3], c1[3];
  color_mul<ADJ>(u, h0, c0);
  color_mul<ADJ>(u, h1, c1);
  if constexpr (SCALE) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      c0[c] = {c0[c].re * f, c0[c].im * f};
      c1[c] = {c1[c].re * f, c1[c].im * f};
    }
  }
  acc_row<1, false>(hs, 0, c0);
  acc_row<1, false>(hs, 1, c1);
  if (MU == 0) {  // row2 = S i chi1, row3 = S i chi0
    acc_row<S, true>(hs, 2, c1);
    acc_row<S, true>(hs, 3, c0);
  } else if (MU == 1) {  // row2 = S chi1, row3 = -S chi0
    acc_row<S, false>(hs, 2, c1);
    acc_row<-S, false>(hs, 3, c0);
  } else if (MU == 2) {  // row2 = S i chi0, row3 = -S i chi1
    acc_row<S, true>(hs, 2, c0);
    acc_row<-S, true>(hs, 3, c1);
  } else {  // row2 = S chi0, row3 = S chi1
    acc_row<S, false>(hs, 2, c0);
    acc_row<S, false>(hs, 3, c1);
  }
}

struct Lat {
  int L[4];
  int64_t st[4];  // site strides
  int64_t V;
};

// CHEM: the direction-3 hops carry ef (forward) and eb (backward).
template <int MU, bool DAG, bool CHEM, typename A, typename T>
__device__ __forceinline__ void hop_pair(A *hs, const T *__restrict__ in, const float2 *__restrict__ U,
                                         const Lat &lat, int64_t s, int coord, T ef, T eb) {
  const int L = lat.L[MU];
  const int64_t st = lat.st[MU];
  const int64_t fwd = s + (coord + 1 == L ? -(int64_t)(L - 1) * st : st);
  const int64_t bwd = s + (coord == 0 ? (int64_t)(L - 1) * st : -st);
  constexpr bool SC = CHEM && MU == 3;
  // D: forward (1 - gamma), backward (1 + gamma); D^H: exchanged
  hop<MU, DAG ? 1 : -1, false, SC>(hs, in + fwd * 24, U + (s * 4 + MU) * 9, ef);
  hop<MU, DAG ? -1 : 1, true, SC>(hs, in + bwd * 24, U + (bwd * 4 + MU) * 9, eb);
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

// out = Kd in + Kh (hop sum of in) [+ Kb x] [+ Ky y] [+ Kv v], one thread per site
template <typename T, bool DAG, bool ADD_X, bool SUB_Y, bool ADD_V>
__global__ void __launch_bounds__(128) wilson_step(const T *__restrict__ in, const T *__restrict__ x,
                                                   const T *__restrict__ y, const T *__restrict__ v,
                                                   T *__restrict__ out, const float2 *__restrict__ U,
                                                   Lat lat, T Kd, T Kh, T Kb, T Ky, T Kv) {
  pdl_wait();
  pdl_trigger();
  using A = typename acc_of<T>::type;
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= lat.V) return;
  int64_t r = s;
  const int c0 = (int)(r % lat.L[0]);
  r /= lat.L[0];
  const int c1 = (int)(r % lat.L[1]);
  r /= lat.L[1];
  const int c2 = (int)(r % lat.L[2]);
  const int c3 = (int)(r / lat.L[2]);
  A hs[24];
#pragma unroll
  for (int k = 0; k < 24; ++k) acc_set(hs[k], num<T>::zero());
  const T one = num<T>::from_d(1.0);
  hop_pair<0, DAG, false>(hs, in, U, lat, s, c0, one, one);
  hop_pair<1, DAG, false>(hs, in, U, lat, s, c1, one, one);
  hop_pair<2, DAG, false>(hs, in, U, lat, s, c2, one, one);
  hop_pair<3, DAG, false>(hs, in, U, lat, s, c3, one, one);
  const int64_t o = s * 24;
#pragma unroll
  for (int k = 0; k < 24; ++k) {
    A res;
    acc_set_prod(res, Kd, ldg(in + o + k));
    acc_add_prod(res, Kh, acc_raw(hs[k]));
    if (ADD_X) acc_add_prod(res, Kb, ldg(x + o + k));
    if (SUB_Y) acc_add_prod(res, Ky, ldg(y + o + k));
    if (ADD_V) acc_add_prod(res, Kv, ldg(v + o + k));
    out[o + k] = acc_get(res);
  }
}

// Complex coefficients of a Q^2 step, with the negated imaginary parts the
// products need.
template <typename T>
struct QCoef {
  T ar, ai, nai, br, bi, nbi, dr, di, ndi;
};

// Q = Gamma_5 D(m_w, mu): EPI = false: out = Q in; EPI: out = alpha (Q in)
// [+ beta x] [+ delta v] with complex alpha, beta, delta.  One thread per site.
template <typename T, bool EPI, bool AX, bool AV>
__global__ void __launch_bounds__(128) wilson_q_step(const T *__restrict__ in, const T *__restrict__ x,
                                                     const T *__restrict__ v, T *__restrict__ out,
                                                     const float2 *__restrict__ U, Lat lat, T Kd, T Kh, T ef,
                                                     T eb, QCoef<T> k) {
  pdl_wait();
  pdl_trigger();
  using A = typename acc_of<T>::type;
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= lat.V) return;
  int c[4];
  site_coords(lat, s, c);
  A hs[24];
#pragma unroll
  for (int q = 0; q < 24; ++q) acc_set(hs[q], num<T>::zero());
  hop_pair<0, false, true>(hs, in, U, lat, s, c[0], ef, eb);
  hop_pair<1, false, true>(hs, in, U, lat, s, c[1], ef, eb);
  hop_pair<2, false, true>(hs, in, U, lat, s, c[2], ef, eb);
  hop_pair<3, false, true>(hs, in, U, lat, s, c[3], ef, eb);
  const int64_t o = s * 24;
#pragma unroll
  for (int q = 0; q < 12; ++q) {  // complex component q = spin * 3 + colour
    A tr, ti;
    acc_set_prod(tr, Kd, ldg(in + o + 2 * q));
    acc_add_prod(tr, Kh, acc_raw(hs[2 * q]));
    acc_set_prod(ti, Kd, ldg(in + o + 2 * q + 1));
    acc_add_prod(ti, Kh, acc_raw(hs[2 * q + 1]));
    T dr = acc_get(tr), di = acc_get(ti);
    if (q >= 6) {  // Gamma_5: spins 2 and 3 change sign
      dr = -dr;
      di = -di;
    }
    if constexpr (!EPI) {
      out[o + 2 * q] = dr;
      out[o + 2 * q + 1] = di;
    } else {
      A rr, ri;
      acc_set_prod(rr, k.ar, dr);
      acc_add_prod(rr, k.nai, di);
      acc_set_prod(ri, k.ar, di);
      acc_add_prod(ri, k.ai, dr);
      if constexpr (AX) {
        const T xr = ldg(x + o + 2 * q), xi = ldg(x + o + 2 * q + 1);
        acc_add_prod(rr, k.br, xr);
        acc_add_prod(rr, k.nbi, xi);
        acc_add_prod(ri, k.br, xi);
        acc_add_prod(ri, k.bi, xr);
      }
      if constexpr (AV) {
        const T vr = ldg(v + o + 2 * q), vi = ldg(v + o + 2 * q + 1);
        acc_add_prod(rr, k.dr, vr);
        acc_add_prod(rr, k.ndi, vi);
        acc_add_prod(ri, k.dr, vi);
        acc_add_prod(ri, k.di, vr);
      }
      out[o + 2 * q] = acc_get(rr);
      out[o + 2 * q + 1] = acc_get(ri);
    }
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
  const int64_t nb = (lat.V + bs - 1) / bs;
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
  const int64_t nb = (lat.V + bs - 1) / bs;
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
