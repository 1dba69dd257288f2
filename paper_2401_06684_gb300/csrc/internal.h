// Internal interfaces between the translation units of the library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <functional>
#include <string>
#include <vector>

#include "../../include/pp.h"

enum OpKind { OPK_CSR = 0, OPK_ST2D = 1, OPK_ST3D = 2, OPK_WILSON = 3 };

// Everything a kernel needs to apply A.  Stencil rows are
//   (A x)_c = d x_c + cm * (x at -1 offsets) + cp * (x at +1 offsets).
struct OpDesc {
  int kind;
  int64_t n;
  int64_t nx, ny, nz;
  double d, cm, cp;
  const int64_t *rowptr;
  const int32_t *col;
  const void *val;  // CSR values in the vector arithmetic (double, dw or float)
  // double-word vectors: the values are exact in FP32 and val holds them as
  // float (half the bytes, cheaper exact products)
  int val_f32 = 0;
  // CSR rows longer than long_len entries: long_rows lists first the nlong
  // rows that get a block each, then the nwarp rows that get a warp each;
  // long_len = 0: every row takes the lane path
  const int32_t *long_rows;
  int nlong;
  int64_t long_len;
  int nwarp = 0;
  // the rows of the lane path in the order the lane groups take them (sorted
  // by length within windows, so that the rows of a warp take about as many
  // rounds); NULL: row t for lane group t
  const int32_t *perm = nullptr;
  int64_t nshort = 0;
  // Wilson D^H D: lattice extents, mass shift, complex64 links and one
  // scratch vector (in the vector arithmetic) for the intermediate D x
  int64_t L[4];
  double mass;
  const void *links;
  void *tmp;
  int tile_bdx;  // stencil kernels: threads per block (0 = 128)
  // Wilson Q^2 (q2 = 1): A = Q^2, Q = Gamma_5 D(mass, mu_c), chemical
  // potential mu_c on the direction-3 hops
  int q2 = 0;
  double mu_c = 0.0;
};

// out = alpha * (A x) + beta * x  [+ gamma * y]  [+ delta * v]; sub_y switches
// the y term on (gamma = -1: the Clenshaw step subtracts y).
struct StepCoef {
  double alpha, beta, delta;
  bool sub_y, add_v;
  double gamma = -1.0;
  // imaginary parts of alpha, beta, delta (complex operators only: a step of
  // q(A) v for a q with complex coefficients)
  double alpha_im = 0.0, beta_im = 0.0, delta_im = 0.0;
};

template <typename T>
int op_step(const OpDesc &op, const T *x, const T *y, const T *v, T *out, const StepCoef &c,
            cudaStream_t s);

// Step t (0 .. k-1) of the matrix Clenshaw recurrence for q(A) v with
// q = sum_{i<=k} cf_i T_i(sigma), sigma(A) = (2A - (a+b) I)/(b-a), s1 = 4/(b-a),
// s2 = -2(a+b)/(b-a): b_k = cf_k v is folded into the first step and the
// last step carries the factors 1/2 (q(A) v = (b_0 - b_2)/2 + cf_0 v / 2 ...
// in the operator form out = alpha A x + beta x [- y] [+ delta v]).
inline StepCoef clenshaw_coef(const std::vector<double> &cf, double s1, double s2, int t) {
  const int k = (int)cf.size() - 1;
  if (k == 1) return {0.5 * s1 * cf[1], 0.5 * s2 * cf[1] + cf[0], 0.0, false, false};
  if (t == 0) return {s1 * cf[k], s2 * cf[k] + cf[k - 1], 0.0, false, false};
  if (t == 1 && k == 2) return {0.5 * s1, 0.5 * s2, cf[0] - cf[2], false, true};
  if (t == 1) return {s1, s2, cf[k - 2] - cf[k], false, true};
  if (t == k - 1) return {0.5 * s1, 0.5 * s2, cf[0], true, true};
  return {s1, s2, cf[k - 1 - t], true, true};
}

// Step t (0 .. k-1) of q(A) v for q = sum_{i<=k} b_i R_i in the basis of
// NewtonForm, by the backward recurrence
//   w_k = b_k v,  w_i = ((A - c_i)/cap) w_{i+1} + e_{i+1} w_{i+2} + b_i v,  q(A) v = w_0
// (for real nodes the Horner scheme of the Newton form; the scaling by cap
// keeps coefficients and vectors inside the FP32 range at high degree).  Step
// t computes w_{k-1-t}; the first step folds w_k = b_k v, the second folds
// e_k w_k into the v term, later steps read w_{i+2} (as y) only where
// e_{i+1} != 0.  Real nodes: three vector streams per step, one fewer than
// the Clenshaw step.
inline StepCoef horner_step(const std::vector<double> &b, const std::vector<double> &c,
                            const std::vector<double> &e, double cap, int t) {
  const int k = (int)b.size() - 1;
  const double r = 1.0 / cap;
  if (t == 0) return {b[k] * r, b[k - 1] - c[k - 1] * b[k] * r, 0.0, false, false, 0.0};
  const int i = k - 1 - t;
  if (t == 1) return {r, -c[i] * r, b[i] + e[i + 1] * b[k], false, true, 0.0};
  return {r, -c[i] * r, b[i], e[i + 1] != 0.0, true, e[i + 1]};
}

// Step t of q(A) v for a complex Newton form (complex nodes c_i without
// conjugate symmetry, no e terms): w_k = b_k v, w_i = ((A - c_i)/cap) w_{i+1}
// + b_i v; the first step folds w_k (complex alpha), later steps read x =
// w_{i+1} and v.  bi, ci: imaginary parts of b, c.
inline StepCoef horner_step_cx(const std::vector<double> &b, const std::vector<double> &bi,
                               const std::vector<double> &c, const std::vector<double> &ci, double cap, int t) {
  const int k = (int)b.size() - 1;
  const double r = 1.0 / cap;
  StepCoef s{r, 0.0, 0.0, false, false, 0.0};
  if (t == 0) {
    // alpha = b_k r, beta = b_{k-1} - c_{k-1} b_k r
    s.alpha = b[k] * r;
    s.alpha_im = bi[k] * r;
    s.beta = b[k - 1] - (c[k - 1] * s.alpha - ci[k - 1] * s.alpha_im);
    s.beta_im = bi[k - 1] - (c[k - 1] * s.alpha_im + ci[k - 1] * s.alpha);
    return s;
  }
  const int i = k - 1 - t;
  s.beta = -c[i] * r;
  s.beta_im = -ci[i] * r;
  s.delta = b[i];
  s.delta_im = bi[i];
  s.add_v = true;
  return s;
}

// Constants of one stencil row: K0 x_c + Km (sum of -1 neighbours) + Kp (sum
// of +1 neighbours) [+ Y y] [+ D v], in the vector arithmetic.
template <typename T>
struct Konst {
  T K0, Km, Kp, D, Y;
};

// One grid of a batched stencil launch: rows [off, off + nx ny nz) of the
// concatenated vectors, gx x gy blocks per plane, first flat block blk0.
struct BatchSeg {
  int64_t off;
  int nx, ny, nz;
  int txs;        // units (16 bytes of entries of two rows) per row pair
  int64_t units;  // txs * ceil(ny / 2) * nz
  unsigned blk0;  // first block of the segment (blocks of 128 threads)
  int vec;        // 16-byte loads (nx a multiple of the entries per 16 bytes)
};
// Threads per block of the batched stencil kernel.
constexpr int kBatchBlock = 128;

// Host: Konst of out = alpha A x + beta x [- y] + delta v for every segment
// (stencil diagonal d, neighbour weights cm / cp, coefficients c[i]).
template <typename T>
void batch_konst(const double *d, const double *cm, const double *cp, const StepCoef *c, int nseg,
                 Konst<T> *out);
// Batched stencil step over all segments (P entries per thread: 1, or the
// 16-byte width when every segment's nx allows it); blkseg[b] = the segment
// of block b; inactive segments skipped.
template <typename T>
int op_step_batch(const BatchSeg *segs, const int *blkseg, unsigned nblk, int P, const Konst<T> *K,
                  const int *active, const T *x, const T *y, const T *v, T *out, bool sub_y, bool add_v,
                  cudaStream_t s);

// Block CSR step for r <= kCsrMaxRhs right-hand sides of the same matrix
// (block SpMM): the r vectors of x, y, v, out are segments at s * sstride;
// segments with active[s] == 0 are skipped (active may be NULL).
constexpr int kCsrMaxRhs = 16;
template <typename T>
int op_step_csr_multi(const OpDesc &op, int64_t sstride, int r, const int *active, const T *x, const T *y,
                      const T *v, T *out, const StepCoef &c, cudaStream_t s);

// Wilson D^H D step (wilson.cu): t = D x into op.tmp, then
// out = alpha D^H t + beta x [- y] [+ delta v].  With op.q2: t = Q x, then
// out = alpha Q t + beta x + delta v with complex alpha, beta, delta.
template <typename T>
int wilson_op_step(const OpDesc &op, const T *x, const T *y, const T *v, T *out, const StepCoef &c,
                   cudaStream_t s);
// out = Q x, Q = Gamma_5 D(op.mass, op.mu_c) (one launch; op.q2 handles)
template <typename T>
int wilson_q_apply(const OpDesc &op, const T *x, T *out, cudaStream_t s);

// ---- vector kernels (vec.cu) ----
// A vector may be the concatenation of independent problems ("segments"),
// each padded to whole chunks of vec_chunk_rows() rows (padding zero).
// nseg = 1 (the default) is a single vector.
struct Seg {
  int nseg = 1;
  const int *chunk_seg = nullptr;  // segment of each chunk (device)
  const int *chunk0 = nullptr;     // first chunk of each segment, nseg + 1 entries (device)
  const int *active = nullptr;     // nonzero while the segment iterates (device; NULL = all)
  int64_t dstride = 0;             // doubles between consecutive segments' FP64 scratch
};

// Number of row chunks (= blocks, = partial sums) of the reduction kernels.
int vec_nchunks(int64_t n);
int vec_chunk_rows();
template <typename T>
int vec_from_f64(const double *in, T *out, int64_t n, cudaStream_t s);
template <typename T>
int vec_to_f64(const T *in, double *out, int64_t n, cudaStream_t s);
// out = in * c * c_dev[segment] (c_dev may be NULL)
template <typename T>
int vec_scale(const T *in, T *out, int64_t n, double c, const double *c_dev, cudaStream_t s,
              const Seg &S = Seg());
template <typename T>
int vec_copy(const T *in, T *out, int64_t n, cudaStream_t s);
// out[0] = 1 / in[0] (0 for 0), on the device
int vec_recip(const double *in, double *out, cudaStream_t s);
// partials[chunk] = sum over the chunk of x.y
template <typename T>
int vec_dot_partials(const T *x, const T *y, int64_t n, double *partials, int nb, cudaStream_t s,
                     const Seg &S = Seg());
// w -= alpha v_j + beta v_{j-1} (vjm1 may be NULL); norm^2 partials
template <typename T>
int vec_lanczos_update(T *w, const T *vj, const T *vjm1, int64_t n, const double *alpha,
                       const double *beta_prev, double *partials, int nb, cudaStream_t s,
                       const Seg &S = Seg());
// partials[chunk*J + c] = sum over the chunk of V_c . w
template <typename T>
int vec_multi_dot(const T *V, int64_t ldv, int J, const T *w, int64_t n, double *partials, int nb,
                  cudaStream_t s, const Seg &S = Seg());
// w -= V h  (h on device, J entries per segment); norm^2 partials if partials != NULL
template <typename T>
int vec_multi_update(const T *V, int64_t ldv, int J, const double *h, T *w, int64_t n,
                     double *partials, int nb, cudaStream_t s, const Seg &S = Seg());
// w -= V h, then partials[chunk*J + c] = sum over the chunk of V_c . (new w),
// V read once (J <= 8; PP_ERR_UNSUPPORTED otherwise, nothing launched)
template <typename T>
int vec_update_dot(const T *V, int64_t ldv, int J, const double *h, T *w, int64_t n, double *partials,
                   cudaStream_t s, const Seg &S = Seg());
// x = V z (accumulate = 0) or x += V z (accumulate = 1), FP64 output; with
// m_seg, segment s uses min(m, m_seg[s]) columns
template <typename T>
int vec_reconstruct(const T *V, int64_t ldv, int m, const double *z, double *x, int64_t n,
                    int accumulate, cudaStream_t s, const Seg &S = Seg(), const int *m_seg = nullptr);
// ---- complex vectors: n reals = n/2 complex entries, (re, im) interleaved ----
// partials[chunk*2J + 2c + {0,1}] = sum over the chunk of conj(V_c) w (re, im)
template <typename T>
int vec_multi_dot_c(const T *V, int64_t ldv, int J, const T *w, int64_t n, double *partials, cudaStream_t s);
// w -= V h (h: J complex FP64 values, interleaved); ||w||^2 partials if partials != NULL
template <typename T>
int vec_multi_update_c(const T *V, int64_t ldv, int J, const double *h, T *w, int64_t n, double *partials,
                       cudaStream_t s);
// x = V z or x += V z (z: m complex FP64 values), FP64 output
template <typename T>
int vec_reconstruct_c(const T *V, int64_t ldv, int m, const double *z, double *x, int64_t n, int accumulate,
                      cudaStream_t s);
// out = (cr + i ci) in
template <typename T>
int vec_scale_c(const T *in, T *out, int64_t n, double cr, double ci, cudaStream_t s);
// out[i] = fixed pseudo-random value in [-1, 1) (instantiated for double, dw)
template <typename T>
int vec_fill_hash(T *out, int64_t n, uint64_t seed, cudaStream_t s);
// out = in rounded to the output arithmetic (instantiated for dw -> float)
template <typename TI, typename TO>
int vec_convert(const TI *in, TO *out, int64_t n, cudaStream_t s);

// Reduction of chunk partials per (column, segment):
//   mode 0: out_a[c] = s_c
//   mode 1: out_a[c] = s_c, out_b[c] = s_c
//   mode 2: out_a[c] = s_c, out_b[c] += s_c
int reduce_cols(const double *partials, int nb, int ncols, int mode, double *out_a, double *out_b,
                cudaStream_t s, const Seg &S = Seg());

// Norm finalization: beta = sqrt(sum partials); *beta_out = beta; *inv_out = 1/beta or 0 on
// breakdown, i.e. beta <= rel * ||ref[0..nref)|| (nref = 0: only beta == 0 or non-finite).
// On breakdown sets st->breakdown (first index recorded as m_bd).
struct DevStatus {
  int conv;
  int breakdown;
  int m_bd;
  int bad;  // non-finite value seen
  double est;
  double beta0;
  double znorm;
  unsigned int ticket;  // finished reduction blocks of k_dcgs_coef (its last block resets it)
  int tma_err;          // a paired stencil launch gave up waiting for its TMA loads
};
// Arnoldi with delayed reorthogonalization (vec.cu): the inner products of
// the candidate u and y = A q(A)^2 u with the basis (partials of 2J + 2
// columns: V^T u, V^T y, u.u, u.y), their sums and the step's coefficients
// (FP64; J <= kDcgsMaxJ; R receives the 2J + 2 sums) and the update sweep
// that writes v_j into u's column and the next candidate into y's.
constexpr int kDcgsMaxJ = 4096;

// Two consecutive real-node Horner steps of q(A) v on a stencil grid in one
// launch (halo.cu): w'' = step_b(step_a(w)), both adding delta v; FP32.
// op_pair_ok: the grid and pointers qualify (stencil, nx % 4 == 0, 16-byte
// aligned vectors, the tensor-map encoder available).  *err is set if a
// block's bounded wait on its TMA loads runs out.
bool op_pair_ok(const OpDesc &op, const void *w, const void *v, const void *out);
int op_pair_step(const OpDesc &op, const float *w, const float *v, float *out, const StepCoef &a,
                 const StepCoef &b, int *err, cudaStream_t s);
template <typename T>
int vec_dot2(const T *V, int64_t ldv, int J, const T *u, const T *y, int64_t n, double *partials, cudaStream_t s);
template <typename T>
int vec_update2(const T *V, int64_t ldv, int J, const double *co, const double *sc, T *u, T *y, int64_t n,
                cudaStream_t s);
int dcgs_coef(const double *partials, int nb, int J, double *R, double *H, int ldh, double *h1s, double *co,
              double *sc, double rel, DevStatus *st, cudaStream_t s);
int norm_finalize(const double *partials, int nb, double *beta_out, double *inv_out,
                  const double *ref, int nref, double rel, int m_here, DevStatus *st,
                  cudaStream_t s, const Seg &S = Seg());

// ---- small projected solve (small.cu) ----
// X[k*m + i] = w_k ((H_m + s_k I)^{-1} e_1)_i for the K quadrature nodes.
// With segments, every per-segment array (H, sig, wt, X, scratch, z, zprev)
// sits at base + segment * S.dstride and st at st + segment; the global
// Hessenberg scratch of large m holds nseg * K blocks.
int small_tridiag_quad(const double *H, int ldh, int m, const double *sig, const double *wt, int K,
                       double *X, double *scratch, cudaStream_t s, const Seg &S = Seg());
int small_hess_quad(const double *H, int ldh, int m, const double *sig, const double *wt, int K,
                    double *X, double *scratch, cudaStream_t s, const Seg &S = Seg());
// z = beta0 * sum_k X[k] ; est = ||z - [zprev;0]|| / ||z||; conv = est < tol; zprev <- z
int small_combine(const double *X, int K, int m, int mprev, double *z, double *zprev, double tol,
                  DevStatus *st, cudaStream_t s, const Seg &S = Seg());
// Complex Hessenberg H (column j at H + 2 j ldh, entries (re, im)); X, z and
// zprev complex (2 m doubles per node / vector); one vector (no segments).
int small_hess_quad_c(const double *H, int ldh, int m, const double *sig, const double *wt, int K, double *X,
                      double *scratch, cudaStream_t s);
size_t small_hess_scratch_doubles_c(int m, int K);
int small_combine_c(const double *X, int K, int m, int mprev, double *z, double *zprev, double tol, DevStatus *st,
                    cudaStream_t s);

// ---- host-side construction (poly.cpp) ----
// Chebyshev interpolant of z^{-1/2} at d = degree+1 first-kind nodes of [a,b].
std::vector<double> cheb_interp_coeffs(double a, double b, int degree);
double cheb_eval(const std::vector<double> &c, double a, double b, double z);
// min/max of q over a dense grid of [a,b] and of z q(z)^2
void cheb_scan(const std::vector<double> &c, double a, double b, double *qmin, double *img_lo,
               double *img_hi);
// Interpolant q of z^{-1/2} at real nodes or conjugate pairs (Sec. 5.2) in
// Newton form at the Leja-ordered nodes, written in a real scaled basis:
// R_0 = 1, R_{i+1} = ((z - c_i)/cap) R_i + e_i R_{i-1}, q = sum b_i R_i (for
// real nodes c_i = x_i, e_i = 0: the Newton basis scaled by cap^i; a
// conjugate pair (x_i, conj x_i) has c_i = c_{i+1} = Re x_i, e_{i+1} =
// (Im x_i/cap)^2).
struct NewtonForm {
  std::vector<double> re, im;  // Leja-ordered nodes, a pair as (Im > 0, conjugate)
  double cap = 1.0;            // a quarter of the diameter of the node set
  std::vector<double> b, c, e;
  // complex form (cx): nodes without conjugate symmetry, R_{i+1} = ((z -
  // c_i)/cap) R_i with complex c_i = c + i ci, coefficients b + i bi, e = 0
  bool cx = false;
  std::vector<double> bi, ci;
};
// false for an empty node set, a pair without its conjugate or a non-finite coefficient
bool newton_form(const std::vector<std::complex<double>> &nodes, NewtonForm *F);
// the same for the interpolant of f at the nodes (f(conj z) = conj f(z) for a real q)
bool newton_form_fn(const std::vector<std::complex<double>> &nodes,
                    const std::function<std::complex<double>(std::complex<double>)> &f, NewtonForm *F);
// least-squares polynomial on contour points (Sec. 5.3): basis recurrence H
// (d x (d-1), column-major) and coefficients alpha; its value at z
bool lsq_poly(const std::vector<std::complex<double>> &z, int d, std::vector<std::complex<double>> *H,
              std::vector<std::complex<double>> *alpha);
std::complex<double> lsq_eval(const std::vector<std::complex<double>> &H,
                              const std::vector<std::complex<double>> &alpha, size_t N, std::complex<double> z);
// d points of a conjugation-symmetric set in Leja order (pairs adjacent)
bool leja_select(const std::vector<std::complex<double>> &pts, int d, std::vector<std::complex<double>> *out);
// discretized contour around Ritz values, kept out of |z| < r_min
std::vector<std::complex<double>> lsq_contour(const std::vector<std::complex<double>> &ritz, double r_min, int npts);
// complex nodes of a complex operator (no conjugate symmetry): Newton form of
// the interpolant of z^{-1/2} in reverse Leja order, cx = true
bool newton_form_cx(const std::vector<std::complex<double>> &nodes, NewtonForm *F);
// the same for the interpolant of f at the nodes
bool newton_form_cx_fn(const std::vector<std::complex<double>> &nodes,
                       const std::function<std::complex<double>(std::complex<double>)> &f, NewtonForm *F);
// d points of a set in Leja order, no conjugate pairing (complex operators)
bool leja_select_cx(const std::vector<std::complex<double>> &pts, int d, std::vector<std::complex<double>> *out);
// discretized closed contour around the Ritz values of a complex operator
// (convex hull, no symmetry), kept out of |z| < r_min
std::vector<std::complex<double>> lsq_contour_cx(const std::vector<std::complex<double>> &ritz, double r_min,
                                                 int npts);
std::complex<double> newton_form_eval(const NewtonForm &F, std::complex<double> z);
// min Re q and the extremes of |z q(z)^2| on [lo, hi] (if hi > lo > 0), at
// the nodes and at the extra points
void newton_scan(const NewtonForm &F, double lo, double hi, const std::vector<std::complex<double>> *extra,
                 double *qmin, double *img_lo, double *img_hi);
// eigenvalues of a real upper Hessenberg matrix (row-major); false if not converged
bool hess_eigvals(std::vector<double> H, int n, std::vector<double> *wr, std::vector<double> *wi);
// eigenvalues of a complex upper Hessenberg matrix (row-major); false if not converged
bool zhess_eigvals(std::vector<std::complex<double>> H, int n, std::vector<std::complex<double>> *w);
// f = M^{-*} e_n for a dense complex row-major M; false if singular
bool zsolve_adjoint_last(const std::vector<std::complex<double>> &M, int n, std::vector<std::complex<double>> *f);
// f = M^{-T} e_n for a dense row-major M; false if singular
bool solve_transposed_last(const std::vector<double> &M, int n, std::vector<double> *f);
// Harmonic Ritz values of SPD tridiagonal T (al, be) and beta = h_{m+1,m};
// false if T is not positive definite.
bool harmonic_ritz(const std::vector<double> &al, const std::vector<double> &be, double beta,
                   std::vector<double> *out);
// Trapezoid rule for z^{-1/2} = (2/pi) int_0^inf (t^2 + z)^{-1} dt, t = e^u.
void invsqrt_quadrature(double lo, double hi, double tau, double theta_max, std::vector<double> *sig,
                        std::vector<double> *wt);

int pp_set_error(int status, const std::string &msg);

// Kernels launched by this thread (every launcher increments it).
int64_t &pp_launch_count();
