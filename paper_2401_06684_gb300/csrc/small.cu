// Small projected solve z = beta0 H_m^{-1/2} e_1 (the final step of Algorithm 1) on
// the device, in FP64.
//
// The paper forms H_m^{1/2} by a blocked Schur method and solves a linear
// system (Sec. 3.1).  Schur iterations are sequential and GB300's FP64 pipe is
// narrow, so here the function is split into independent shifted solves that
// run in parallel:
//     z^{-1/2} = (2/pi) int_0^inf (t^2 + z)^{-1} dt,   t = e^u,
// discretised by the trapezoid rule in u (nodes s_k = e^{2 u_k}, weights
// w_k = (2h/pi) e^{u_k}; constructed on the host), so
//     H^{-1/2} e_1 ~= sum_k w_k (H + s_k I)^{-1} e_1.
// Every shifted matrix has its spectrum in the right half-plane shifted by
// s_k > 0, so each solve is well posed.  One CTA (Hessenberg: Givens QR) or
// one thread (symmetric tridiagonal: LDL^T recurrence) per node; a final
// single-CTA pass sums the nodes in a fixed order and forms the stopping
// estimate ||f_m - f_{m-k}|| / ||f_m|| from the coefficient vectors alone,
// valid because V_m is orthonormal (Sec. 3.1, after Algorithm 2).
#include "common.cuh"
#include "internal.h"

namespace {

// Symmetric tridiagonal T = tridiag(beta, alpha, beta) read from the Lanczos
// Hessenberg storage: alpha_i = H[i,i], beta_i = H[i+1,i].
__global__ void k_tri_quad(const double *__restrict__ H, int ldh, int m, const double *__restrict__ sig,
                           const double *__restrict__ wt, int K, double *__restrict__ X,
                           double *__restrict__ scratch, Seg S) {
  pdl_wait();
  pdl_trigger();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int seg = blockIdx.y;
  if (k >= K || (S.active && !S.active[seg])) return;
  const int64_t so = seg * S.dstride;
  H += so;
  sig += so;
  wt += so;
  X += so;
  scratch += so;
  const double s = sig[k];
  double *cp = scratch + (int64_t)k * m;  // modified super-diagonal
  double *x = X + (int64_t)k * m;         // modified rhs, then solution
  // forward elimination of (T + sI) x = e_1 (one FP64 division per row)
  double iden = 1.0 / (H[0] + s);
  double cprev = (m > 1) ? H[1] * iden : 0.0;
  double dprev = iden;
  cp[0] = cprev;
  x[0] = dprev;
  for (int i = 1; i < m; ++i) {
    const double bsub = H[(int64_t)(i - 1) * ldh + i];  // beta_{i-1}
    iden = 1.0 / ((H[(int64_t)i * ldh + i] + s) - bsub * cprev);
    const double bsup = (i + 1 < m) ? H[(int64_t)i * ldh + i + 1] : 0.0;
    cprev = bsup * iden;
    dprev = (-bsub * dprev) * iden;
    cp[i] = cprev;
    x[i] = dprev;
  }
  // back substitution, scaled by the weight
  double xn = x[m - 1];
  const double w = wt[k];
  x[m - 1] = w * xn;
  for (int i = m - 2; i >= 0; --i) {
    xn = x[i] - cp[i] * xn;
    x[i] = w * xn;
  }
}

// Upper Hessenberg: Givens QR of (H + sI) column by column, rotations applied
// to the right-hand side e_1, then back substitution.  The working matrix is
// column-major with leading dimension m+1 (odd strides avoid smem bank
// conflicts), in dynamic shared memory or, for large m, in global scratch.
__global__ void __launch_bounds__(128) k_hess_quad(const double *__restrict__ H, int ldh, int m,
                                                   const double *__restrict__ sig,
                                                   const double *__restrict__ wt,
                                                   double *__restrict__ X, double *__restrict__ gscratch,
                                                   int use_smem, Seg S) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ double sm[];
  const int k = blockIdx.x;
  const int seg = blockIdx.y;
  if (S.active && !S.active[seg]) return;
  const int64_t so = seg * S.dstride;
  H += so;
  sig += so;
  wt += so;
  X += so;
  const int ld = m + 1;
  double *M = use_smem ? sm
                       : gscratch + ((int64_t)seg * gridDim.x + k) * ((int64_t)ld * m + 2 * m);
  double *g = M + (int64_t)ld * m;  // rhs / solution, m entries
  const double s = sig[k];
  // one flat loop over the m x m entries (loads issued back to back, not one
  // column at a time)
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int c = idx / m, r = idx - c * m;
    double v = (r <= c + 1) ? H[(int64_t)c * ldh + r] : 0.0;
    if (r == c) v += s;
    M[(int64_t)c * ld + r] = v;
  }
  for (int r = threadIdx.x; r < m; r += blockDim.x) g[r] = (r == 0) ? 1.0 : 0.0;
  __syncthreads();
  for (int c = 0; c + 1 < m; ++c) {
    const double a = M[(int64_t)c * ld + c];
    const double b = M[(int64_t)c * ld + c + 1];
    const bool nz = a != 0.0 || b != 0.0;
    const double ir = nz ? rhypot(a, b) : 0.0;  // 1 / sqrt(a^2 + b^2) in one call
    const double cs = nz ? a * ir : 1.0;
    const double sn = b * ir;
    __syncthreads();  // everyone has read the pivot pair
    for (int cc = c + threadIdx.x; cc < m; cc += blockDim.x) {
      const double t1 = M[(int64_t)cc * ld + c];
      const double t2 = M[(int64_t)cc * ld + c + 1];
      M[(int64_t)cc * ld + c] = cs * t1 + sn * t2;
      M[(int64_t)cc * ld + c + 1] = -sn * t1 + cs * t2;
    }
    if (threadIdx.x == 0) {
      const double g1 = g[c], g2 = g[c + 1];
      g[c] = cs * g1 + sn * g2;
      g[c + 1] = -sn * g1 + cs * g2;
    }
    __syncthreads();
  }
  // back substitution R x = g, column oriented; the diagonal's reciprocals
  // first, in parallel, so that the sequential steps only multiply
  double *rd = g + m;
  for (int c = threadIdx.x; c < m; c += blockDim.x) rd[c] = 1.0 / M[(int64_t)c * ld + c];
  __syncthreads();
  for (int c = m - 1; c >= 0; --c) {
    if (threadIdx.x == 0) g[c] = g[c] * rd[c];
    __syncthreads();
    const double xc = g[c];
    for (int r = threadIdx.x; r < c; r += blockDim.x) g[r] -= M[(int64_t)c * ld + r] * xc;
    __syncthreads();
  }
  const double w = wt[k];
  for (int r = threadIdx.x; r < m; r += blockDim.x) X[(int64_t)k * m + r] = w * g[r];
}

// Warp-per-node variant for m <= 64: lanes own columns (rotations) and rows
// (back substitution); warp-synchronous, several nodes per block.
__global__ void __launch_bounds__(256) k_hess_quad_warp(const double *__restrict__ H, int ldh, int m,
                                                        const double *__restrict__ sig,
                                                        const double *__restrict__ wt, int K,
                                                        double *__restrict__ X, Seg S) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ double sm[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int k = blockIdx.x * (blockDim.x >> 5) + wid;
  const int seg = blockIdx.y;
  if (k >= K || (S.active && !S.active[seg])) return;  // whole warp leaves together
  const int64_t so = seg * S.dstride;
  H += so;
  sig += so;
  wt += so;
  X += so;
  const int ld = m + 1;
  double *M = sm + (int64_t)wid * ((int64_t)ld * m + 2 * m);
  double *g = M + (int64_t)ld * m;
  double *rd = g + m;
  const double s = sig[k];
  for (int idx = lane; idx < m * m; idx += 32) {
    const int c = idx / m, r = idx - c * m;
    double v = (r <= c + 1) ? H[(int64_t)c * ldh + r] : 0.0;
    if (r == c) v += s;
    M[(int64_t)c * ld + r] = v;
  }
  for (int r = lane; r < m; r += 32) g[r] = (r == 0) ? 1.0 : 0.0;
  __syncwarp();
  for (int c = 0; c + 1 < m; ++c) {
    const double a = M[(int64_t)c * ld + c];
    const double b = M[(int64_t)c * ld + c + 1];
    const bool nz = a != 0.0 || b != 0.0;
    const double ir = nz ? rhypot(a, b) : 0.0;
    const double cs = nz ? a * ir : 1.0;
    const double sn = b * ir;
    __syncwarp();
    for (int cc = c + lane; cc < m; cc += 32) {
      const double t1 = M[(int64_t)cc * ld + c];
      const double t2 = M[(int64_t)cc * ld + c + 1];
      M[(int64_t)cc * ld + c] = cs * t1 + sn * t2;
      M[(int64_t)cc * ld + c + 1] = -sn * t1 + cs * t2;
    }
    if (lane == 0) {
      const double g1 = g[c], g2 = g[c + 1];
      g[c] = cs * g1 + sn * g2;
      g[c + 1] = -sn * g1 + cs * g2;
    }
    __syncwarp();
  }
  for (int c = lane; c < m; c += 32) rd[c] = 1.0 / M[(int64_t)c * ld + c];
  __syncwarp();
  for (int c = m - 1; c >= 0; --c) {
    const double xc = g[c] * rd[c];
    __syncwarp();
    for (int r = lane; r < c; r += 32) g[r] -= M[(int64_t)c * ld + r] * xc;
    if (lane == 0) g[c] = xc;
    __syncwarp();
  }
  const double w = wt[k];
  for (int r = lane; r < m; r += 32) X[(int64_t)k * m + r] = w * g[r];
}

// z_i = beta0 sum_k X[k][i]: one warp per component (lanes stride over the
// nodes, fixed shuffle tree), then the stopping estimate over the components.
__global__ void __launch_bounds__(1024) k_combine(const double *__restrict__ X, int K, int m, int mprev,
                                                  double *__restrict__ z, double *__restrict__ zprev,
                                                  double tol, DevStatus *st, Seg S) {
  pdl_wait();
  pdl_trigger();
  __shared__ double rd[32], rz[32];
  const int seg = blockIdx.x;
  if (S.active && !S.active[seg]) return;
  const int64_t so = seg * S.dstride;
  X += so;
  z += so;
  zprev += so;
  st += seg;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double beta0 = st->beta0;
  double d2 = 0.0, z2 = 0.0;
  for (int i = wid; i < m; i += 32) {
    double s = 0.0;
    for (int k = lane; k < K; k += 32) s += X[(int64_t)k * m + i];
    s = warp_sum(s) * beta0;
    const double p = (i < mprev) ? zprev[i] : 0.0;
    d2 += (s - p) * (s - p);
    z2 += s * s;
    if (lane == 0) z[i] = s;
  }
  if (lane == 0) {
    rd[wid] = d2;
    rz[wid] = z2;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) zprev[i] = z[i];
  if (threadIdx.x == 0) {
    double D = 0.0, Z = 0.0;
    for (int q = 0; q < 32; ++q) {
      D += rd[q];
      Z += rz[q];
    }
    const double est = (mprev > 0 && Z > 0.0) ? sqrt(D / Z) : INFINITY;
    st->est = est;
    st->znorm = sqrt(Z);
    if (!isfinite(Z)) st->bad = 1;
    st->conv = (est < tol) ? 1 : 0;
  }
}

// ---- complex Hessenberg H (complex operators) ----
struct zc {
  double re, im;
};
__device__ __forceinline__ zc zadd(zc a, zc b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ zc zsub(zc a, zc b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ zc zmul(zc a, zc b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
// conj(a) b
__device__ __forceinline__ zc zcmul(zc a, zc b) { return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re}; }
// a / b by Smith's algorithm (Smith, "Algorithm 116: Complex division",
// CACM 5(8), 1962): scale by the larger part of b to avoid overflow
__device__ __forceinline__ zc zdiv(zc a, zc b) {
  if (fabs(b.re) >= fabs(b.im)) {
    const double r = b.im / b.re, d = b.re + b.im * r;
    return {(a.re + a.im * r) / d, (a.im - a.re * r) / d};
  }
  const double r = b.re / b.im, d = b.re * r + b.im;
  return {(a.re * r + a.im) / d, (a.im * r - a.re) / d};
}

// One CTA per node: (H + s_k I) x = e_1 by complex Givens QR (rotation
// [[conj c, conj s], [-s, c]] with c = a/r, s = b/r, r = sqrt(|a|^2 + |b|^2)),
// then back substitution; the working matrix in shared memory or, for large
// m, in global scratch (column-major, leading dimension m+1).
__global__ void __launch_bounds__(128) k_hess_quad_c(const double *__restrict__ H, int ldh, int m,
                                                     const double *__restrict__ sig, const double *__restrict__ wt,
                                                     double *__restrict__ X, double *__restrict__ gscratch,
                                                     int use_smem) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ double sm[];
  const int k = blockIdx.x;
  const int ld = m + 1;
  zc *M = reinterpret_cast<zc *>(use_smem ? sm : gscratch + (int64_t)k * 2 * ((int64_t)ld * m + 2 * m));
  zc *g = M + (int64_t)ld * m;
  const double s = sig[k];
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int c = idx / m, r = idx - c * m;
    zc v = {0.0, 0.0};
    if (r <= c + 1) v = {H[2 * ((int64_t)c * ldh + r)], H[2 * ((int64_t)c * ldh + r) + 1]};
    if (r == c) v.re += s;
    M[(int64_t)c * ld + r] = v;
  }
  for (int r = threadIdx.x; r < m; r += blockDim.x) g[r] = {r == 0 ? 1.0 : 0.0, 0.0};
  __syncthreads();
  for (int c = 0; c + 1 < m; ++c) {
    const zc a = M[(int64_t)c * ld + c];
    const zc b = M[(int64_t)c * ld + c + 1];
    const bool nz = a.re != 0.0 || a.im != 0.0 || b.re != 0.0 || b.im != 0.0;
    const double ir = nz ? rnorm4d(a.re, a.im, b.re, b.im) : 0.0;
    const zc cs = nz ? zc{a.re * ir, a.im * ir} : zc{1.0, 0.0};
    const zc sn = {b.re * ir, b.im * ir};
    __syncthreads();  // everyone has read the pivot pair
    for (int cc = c + threadIdx.x; cc < m; cc += blockDim.x) {
      const zc t1 = M[(int64_t)cc * ld + c];
      const zc t2 = M[(int64_t)cc * ld + c + 1];
      M[(int64_t)cc * ld + c] = zadd(zcmul(cs, t1), zcmul(sn, t2));
      M[(int64_t)cc * ld + c + 1] = zsub(zmul(cs, t2), zmul(sn, t1));
    }
    if (threadIdx.x == 0) {
      const zc g1 = g[c], g2 = g[c + 1];
      g[c] = zadd(zcmul(cs, g1), zcmul(sn, g2));
      g[c + 1] = zsub(zmul(cs, g2), zmul(sn, g1));
    }
    __syncthreads();
  }
  zc *rd = g + m;  // reciprocals of the diagonal, in parallel first
  for (int c = threadIdx.x; c < m; c += blockDim.x) rd[c] = zdiv(zc{1.0, 0.0}, M[(int64_t)c * ld + c]);
  __syncthreads();
  for (int c = m - 1; c >= 0; --c) {
    if (threadIdx.x == 0) g[c] = zmul(g[c], rd[c]);
    __syncthreads();
    const zc xc = g[c];
    for (int r = threadIdx.x; r < c; r += blockDim.x) g[r] = zsub(g[r], zmul(M[(int64_t)c * ld + r], xc));
    __syncthreads();
  }
  const double w = wt[k];
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    X[2 * ((int64_t)k * m + r)] = w * g[r].re;
    X[2 * ((int64_t)k * m + r) + 1] = w * g[r].im;
  }
}

// z_i = beta0 sum_k X[k][i] (complex), then the stopping estimate, as k_combine.
__global__ void __launch_bounds__(1024) k_combine_c(const double *__restrict__ X, int K, int m, int mprev,
                                                    double *__restrict__ z, double *__restrict__ zprev, double tol,
                                                    DevStatus *st) {
  pdl_wait();
  pdl_trigger();
  __shared__ double rd[32], rz[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const double beta0 = st->beta0;
  double d2 = 0.0, z2 = 0.0;
  for (int i = wid; i < m; i += 32) {
    double sr = 0.0, si = 0.0;
    for (int k = lane; k < K; k += 32) {
      sr += X[2 * ((int64_t)k * m + i)];
      si += X[2 * ((int64_t)k * m + i) + 1];
    }
    sr = warp_sum(sr) * beta0;
    si = warp_sum(si) * beta0;
    const double pr = (i < mprev) ? zprev[2 * i] : 0.0, pi = (i < mprev) ? zprev[2 * i + 1] : 0.0;
    d2 += (sr - pr) * (sr - pr) + (si - pi) * (si - pi);
    z2 += sr * sr + si * si;
    if (lane == 0) {
      z[2 * i] = sr;
      z[2 * i + 1] = si;
    }
  }
  if (lane == 0) {
    rd[wid] = d2;
    rz[wid] = z2;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * m; i += blockDim.x) zprev[i] = z[i];
  if (threadIdx.x == 0) {
    double D = 0.0, Z = 0.0;
    for (int q = 0; q < 32; ++q) {
      D += rd[q];
      Z += rz[q];
    }
    const double est = (mprev > 0 && Z > 0.0) ? sqrt(D / Z) : INFINITY;
    st->est = est;
    st->znorm = sqrt(Z);
    if (!isfinite(Z)) st->bad = 1;
    st->conv = (est < tol) ? 1 : 0;
  }
}

}  // namespace

int small_tridiag_quad(const double *H, int ldh, int m, const double *sig, const double *wt, int K,
                       double *X, double *scratch, cudaStream_t s, const Seg &S) {
  PP_CUDA_TRY(pdl_launch(k_tri_quad, dim3((K + 127) / 128, S.nseg), dim3(128), 0, s, H, ldh, m, sig, wt, K, X, scratch, S));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}

int small_hess_quad(const double *H, int ldh, int m, const double *sig, const double *wt, int K,
                    double *X, double *scratch, cudaStream_t s, const Seg &S) {
  if (m <= 64) {
    const size_t per_warp = ((size_t)(m + 1) * m + 2 * (size_t)m) * sizeof(double);
    // at most 2 nodes per block: the rotations are chains of dependent FP64
    // operations, and GB300's FP64 pipe is narrow, so spreading the nodes over
    // more SMs shortens the launch (8 per block left most SMs idle)
    int wpb = (int)((48 * 1024) / per_warp);
    if (wpb > 2) wpb = 2;
    if (wpb < 1) wpb = 1;
    const unsigned grid = (unsigned)((K + wpb - 1) / wpb);
    PP_CUDA_TRY(pdl_launch(k_hess_quad_warp, dim3(grid, S.nseg), dim3(32 * wpb), per_warp * wpb, s, H, ldh, m, sig, wt, K, X, S));
    ++pp_launch_count();
    PP_CUDA_TRY(cudaGetLastError());
    return PP_OK;
  }
  const size_t bytes = ((size_t)(m + 1) * m + 2 * (size_t)m) * sizeof(double);
  const size_t kSmemMax = 200 * 1024;
  const int use_smem = bytes <= kSmemMax ? 1 : 0;
  if (use_smem && bytes > 48 * 1024)
    PP_CUDA_TRY(cudaFuncSetAttribute(k_hess_quad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  PP_CUDA_TRY(pdl_launch(k_hess_quad, dim3(K, S.nseg), dim3(128), use_smem ? bytes : 0, s, H, ldh, m, sig, wt, X, scratch, use_smem, S));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}

size_t small_hess_scratch_doubles(int m, int K) {
  return (size_t)K * ((size_t)(m + 1) * m + 2 * (size_t)m);
}

int small_combine(const double *X, int K, int m, int mprev, double *z, double *zprev, double tol,
                  DevStatus *st, cudaStream_t s, const Seg &S) {
  PP_CUDA_TRY(pdl_launch(k_combine, dim3(S.nseg), dim3(1024), 0, s, X, K, m, mprev, z, zprev, tol, st, S));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}

int small_hess_quad_c(const double *H, int ldh, int m, const double *sig, const double *wt, int K, double *X,
                      double *scratch, cudaStream_t s) {
  const size_t bytes = ((size_t)(m + 1) * m + 2 * (size_t)m) * 2 * sizeof(double);
  const size_t kSmemMax = 200 * 1024;
  const int use_smem = bytes <= kSmemMax ? 1 : 0;
  if (use_smem && bytes > 48 * 1024)
    PP_CUDA_TRY(cudaFuncSetAttribute(k_hess_quad_c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  PP_CUDA_TRY(pdl_launch(k_hess_quad_c, dim3(K), dim3(128), use_smem ? bytes : 0, s, H, ldh, m, sig, wt, X, scratch,
                         use_smem));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}

size_t small_hess_scratch_doubles_c(int m, int K) {
  return (size_t)K * 2 * ((size_t)(m + 1) * m + 2 * (size_t)m);
}

int small_combine_c(const double *X, int K, int m, int mprev, double *z, double *zprev, double tol, DevStatus *st,
                    cudaStream_t s) {
  PP_CUDA_TRY(pdl_launch(k_combine_c, dim3(1), dim3(1024), 0, s, X, K, m, mprev, z, zprev, tol, st));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}
