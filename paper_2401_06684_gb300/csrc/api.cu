// C ABI and the Krylov driver: Algorithm 1 (left) and Algorithm 2 (right)
// polynomially preconditioned Arnoldi/Lanczos for A^{-1/2} b, and A^{1/2} b
// through A^{-1/2}(A b) (Sec. 4).  The host only sequences kernels on the
// handle's stream; all vector work, inner products, the projected matrix
// and the small f(H_m) solve stay on the device.  The host reads back a
// 48-byte status record at each stopping check.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "internal.h"

size_t small_hess_scratch_doubles(int m, int K);

#define RC_(x)                  \
  do {                          \
    int _r = (x);               \
    if (_r != PP_OK) return _r; \
  } while (0)

namespace {
thread_local std::string g_last_error;
thread_local int64_t g_launches = 0;
}

int64_t &pp_launch_count() { return g_launches; }

int pp_set_error(int status, const std::string &msg) {
  g_last_error = msg;
  return status;
}

int pp_cuda_fail(cudaError_t e, const char *what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();  // clear a non-sticky error
  return e == cudaErrorMemoryAllocation ? PP_ERR_OOM : PP_ERR_CUDA;
}

namespace {

constexpr int kMaxDegree = 128;
// CSR rows with more entries than this get a block of their own
constexpr int64_t kLongRow = 64;
// ... and rows with more than this get a whole block (the others a warp)
constexpr int64_t kBlockRow = 1024;
// CSR rows of the lane path are sorted by length within windows of this many
// rows when the variance of their lengths exceeds kPermMinVar
constexpr size_t kPermWindow = 4096;
constexpr double kPermMinVar = 1.0;
constexpr int kMaxM = 4096;
constexpr double kBreakdownRel = 1e-12;
constexpr int kIntervalSteps = 200;

void ws_free(Workspace &w) {
  if (w.V) cudaFree(w.V);
  if (w.Y) cudaFree(w.Y);
  if (w.tmp) cudaFree(w.tmp);
  if (w.dmem) cudaFree(w.dmem);
  if (w.hess) cudaFree(w.hess);
  if (w.st) cudaFree(w.st);
  if (w.st_host) cudaFreeHost(w.st_host);
  if (w.io) cudaFree(w.io);
  if (w.val_dw) cudaFree(w.val_dw);
  if (w.val_f) cudaFree(w.val_f);
  if (w.long_rows) cudaFree(w.long_rows);
  if (w.csr_perm) cudaFree(w.csr_perm);
  if (w.Vf) cudaFree(w.Vf);
  if (w.Yf) cudaFree(w.Yf);
  if (w.ev0) cudaEventDestroy(w.ev0);
  if (w.ev1) cudaEventDestroy(w.ev1);
  w = Workspace();
}

// Profiling brackets a run of consecutive operator launches (one q(A)
// application or one product with A; category 0), the orthogonalization of
// a Krylov step (1) or a stopping check's small solve (2) with a pair of
// events on the handle's stream; the per-launch average of the operator runs
// then includes the short gaps between the launches of a run.
int prof_begin(pp_ctx *c, int cat = 0) {
  if (!c->opts.profile) return PP_OK;
  if (c->prof_used + 2 > c->prof_ev.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      PP_CUDA_TRY(cudaEventCreate(&e));
      c->prof_ev.push_back(e);
    }
  }
  if (c->prof_cat.size() < c->prof_ev.size() / 2) c->prof_cat.resize(c->prof_ev.size() / 2);
  c->prof_cat[c->prof_used / 2] = cat;
  PP_CUDA_TRY(cudaEventRecord(c->prof_ev[c->prof_used], c->stream));
  return PP_OK;
}

int prof_end(pp_ctx *c) {
  if (!c->opts.profile) return PP_OK;
  PP_CUDA_TRY(cudaEventRecord(c->prof_ev[c->prof_used + 1], c->stream));
  c->prof_used += 2;
  return PP_OK;
}

// Algorithmic bytes of one operator step out = alpha A x + beta x [+ gamma y] [+ delta v].
double step_bytes(const pp_ctx *c, const StepCoef &k, double esz) {
  double vecs = 2.0 + (k.sub_y ? 1.0 : 0.0) + (k.add_v ? 1.0 : 0.0);
  double bytes = vecs * esz * (double)c->n;
  if (c->op_kind == OPK_CSR) bytes += (esz + 4.0) * (double)(c->nnz > 0 ? c->nnz : 0) + 8.0 * (double)(c->n + 1);
  if (c->op_kind == OPK_WILSON) {
    // t = D x (read x, write t) and out = alpha D^H t + beta x ...: the second
    // launch reads t and x; both read the links (288 bytes per site)
    const double sites = (double)c->n / 24.0;
    bytes += (2.0 + (k.beta != 0.0 || k.beta_im != 0.0 ? 1.0 : 0.0)) * esz * (double)c->n + 2.0 * 288.0 * sites;
  }
  return bytes;
}

// One operator launch of the chain: counted and its algorithmic bytes added.
template <typename T>
int run_op(pp_ctx *c, const OpDesc &op, const T *x, const T *y, const T *v, T *out, const StepCoef &k) {
  int rc = op_step<T>(op, x, y, v, out, k, c->stream);
  if (rc) return rc;
  c->chain_launches += 1;
  c->chain_bytes += step_bytes(c, k, (double)sizeof(T));
  return PP_OK;
}

// A run of operator launches bracketed for profiling.
template <typename T>
int run_op_timed(pp_ctx *c, const OpDesc &op, const T *x, const T *y, const T *v, T *out,
                 const StepCoef &k) {
  RC_(prof_begin(c));
  RC_(run_op<T>(c, op, x, y, v, out, k));
  return prof_end(c);
}

double prof_ms(pp_ctx *c, int cat = 0) {
  double t = 0.0;
  for (size_t i = 0; i + 1 < c->prof_used; i += 2) {
    if (c->prof_cat[i / 2] != cat) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->prof_ev[i], c->prof_ev[i + 1]) == cudaSuccess) t += ms;
  }
  return t;
}

// Layout of the FP64 scratch (offsets in doubles).
struct DLayout {
  size_t H, h1, part, X, tri, z, zprev, sig, wt, scal, dd, total;
  int ldh, nb, K;
};

// Complex operators keep H, h, the partial sums, X, z and zprev as complex
// (re, im) pairs: twice the doubles.
DLayout dlayout(const pp_ctx *c, int m_cap) {
  DLayout L;
  const size_t cw = c->cplx ? 2 : 1;
  L.ldh = m_cap + 1;
  L.nb = vec_nchunks(c->n);
  L.K = (int)c->qsig.size();
  size_t o = 0;
  L.H = o;
  o += cw * (m_cap + 1) * m_cap;
  L.h1 = o;
  o += cw * (m_cap + 1);
  L.part = o;
  o += 2 * L.nb * (m_cap + 1);  // complex: (re, im) per column; delayed reorthogonalization: 2J + 2 columns
  L.X = o;
  o += cw * L.K * m_cap;
  L.tri = o;
  o += (size_t)L.K * m_cap;
  L.z = o;
  o += cw * m_cap;
  L.zprev = o;
  o += cw * m_cap;
  L.sig = o;
  o += (size_t)L.K;
  L.wt = o;
  o += (size_t)L.K;
  L.scal = o;
  o += 8;
  L.dd = o;  // delayed reorthogonalization: the reduced inner products (2 m + 2) and s, d (2 m)
  o += 4 * ((size_t)m_cap + 2);
  L.total = o;
  return L;
}

// Basis layout requested from ensure_ws.
enum Layout { LAYOUT_KEEP = -1, LAYOUT_FULL = 0, LAYOUT_TWO_PASS = 1 };


int ensure_ws(pp_ctx *c, int prec, int m_cap, bool need_y, int layout = LAYOUT_KEEP) {
  Workspace &w = c->ws;
  const size_t esz = 8;  // double and double-word are both 8 bytes
  const bool two_pass = layout == LAYOUT_KEEP ? w.two_pass : layout == LAYOUT_TWO_PASS;
  if (two_pass) need_y = false;
  if (w.prec != prec || m_cap > w.m_cap || (need_y && !w.has_y) || !w.dmem || w.two_pass != two_pass) {
    if (w.V) cudaFree(w.V), w.V = nullptr;
    if (w.Y) cudaFree(w.Y), w.Y = nullptr;
    if (w.tmp) cudaFree(w.tmp), w.tmp = nullptr;
    if (w.dmem) cudaFree(w.dmem), w.dmem = nullptr;
    if (w.Vf) cudaFree(w.Vf), w.Vf = nullptr;
    if (w.Yf) cudaFree(w.Yf), w.Yf = nullptr;
    const int mc = m_cap > w.m_cap ? m_cap : w.m_cap;
    const int vcols = two_pass ? 4 : mc + 1;
    if (two_pass) w.has_y = false;
    w.ldv = (c->n + 31) / 32 * 32;
    w.esz = esz;
    w.two_pass = two_pass;
    PP_CUDA_TRY(cudaMalloc(&w.V, (size_t)vcols * w.ldv * esz));
    if (need_y || w.has_y) {
      PP_CUDA_TRY(cudaMalloc(&w.Y, (size_t)mc * w.ldv * esz));
      w.has_y = true;
    }
    PP_CUDA_TRY(cudaMalloc(&w.tmp, (size_t)kTmpVecs * w.ldv * esz));
    if (prec == PP_PREC_MIXED) {
      PP_CUDA_TRY(cudaMalloc(&w.Vf, (size_t)vcols * w.ldv * sizeof(float)));
      if (w.has_y) PP_CUDA_TRY(cudaMalloc(&w.Yf, (size_t)mc * w.ldv * sizeof(float)));
    }
    DLayout L = dlayout(c, mc);
    PP_CUDA_TRY(cudaMalloc(&w.dmem, L.total * sizeof(double)));
    w.dmem_n = L.total;
    w.m_cap = mc;
    w.prec = prec;
    c->quad_uploaded = false;
  }
  if (!w.st) {
    PP_CUDA_TRY(cudaMalloc(&w.st, sizeof(DevStatus)));
    PP_CUDA_TRY(cudaMallocHost(&w.st_host, sizeof(DevStatus)));
    PP_CUDA_TRY(cudaEventCreate(&w.ev0));
    PP_CUDA_TRY(cudaEventCreate(&w.ev1));
  }
  if (!c->quad_uploaded) {
    DLayout L = dlayout(c, w.m_cap);
    PP_CUDA_TRY(cudaMemcpyAsync(w.dmem + L.sig, c->qsig.data(), L.K * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    PP_CUDA_TRY(cudaMemcpyAsync(w.dmem + L.wt, c->qwt.data(), L.K * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    c->quad_uploaded = true;
  }
  RC_(csr_prepare(c, prec));
  return PP_OK;
}

// Arithmetic of the vectors: IEEE FP64, double-word pairs, or FP32.
enum Arith { AR_F64 = 0, AR_DW = 1, AR_F32 = 2 };

template <typename T>
constexpr int arith_of() {
  return std::is_same<T, double>::value ? AR_F64 : (std::is_same<T, dw>::value ? AR_DW : AR_F32);
}

OpDesc make_op(const pp_ctx *c, int arith) {
  OpDesc op;
  op.kind = c->op_kind;
  op.n = c->n;
  op.nx = c->dims[0];
  op.ny = c->dims[1];
  op.nz = c->dims[2];
  op.d = c->st_d;
  op.cm = c->st_cm;
  op.cp = c->st_cp;
  op.rowptr = c->rowptr;
  op.col = c->col;
  op.long_rows = c->ws.long_rows;
  const bool scanned = c->ws.nlong > 0 || c->ws.nwarp > 0;
  op.nlong = scanned ? c->ws.nlong : 0;
  op.nwarp = scanned ? c->ws.nwarp : 0;
  op.long_len = scanned ? kLongRow : 0;
  op.perm = c->ws.csr_perm;
  op.nshort = c->ws.nshort;
  op.val_f32 = arith == AR_DW && c->ws.val_exact_f32 == 1 ? 1 : 0;
  op.val = arith == AR_DW ? (op.val_f32 ? c->ws.val_f : c->ws.val_dw)
                          : (arith == AR_F32 ? c->ws.val_f : (const void *)c->val);
  for (int d = 0; d < 4; ++d) op.L[d] = c->dims[d];
  op.mass = c->mass;
  op.links = c->links;
  op.q2 = c->stencil == PP_WILSON4D_Q2 ? 1 : 0;
  op.mu_c = c->mu_c;
  const size_t esz = arith == AR_F32 ? sizeof(float) : sizeof(double);
  op.tmp = c->ws.tmp ? (void *)((char *)c->ws.tmp + (size_t)(kTmpVecs - 1) * c->ws.ldv * esz) : nullptr;
  op.tile_bdx = c->tile_bdx;
  return op;
}

#define RC(x)                \
  do {                       \
    int _r = (x);            \
    if (_r != PP_OK) return _r; \
  } while (0)

// y = q(A) x in deg q operator applications: the Horner scheme of the Newton
// form with its first step folded, or (opts.clenshaw, Chebyshev q) the matrix
// Clenshaw recurrence with the first two steps folded (b_{k+1} = 0, b_k =
// c_k x).  Horner steps read no second previous iterate; the same buffer
// rotation serves both.
// Two Horner steps in one launch (halo.cu), counted as one launch moving
// three vectors (w and v read, the result written).
int run_pair(pp_ctx *c, const OpDesc &op, const float *w, const float *v, float *out, const StepCoef &a,
             const StepCoef &b) {
  RC_(op_pair_step(op, w, v, out, a, b, c->pair_err, c->stream));
  c->chain_launches += 1;
  c->chain_bytes += 3.0 * sizeof(float) * (double)c->n;
  return PP_OK;
}

// q(A) v with the real-node Horner steps after the first taken two at a time
// (opts.halo, FP32, inside a solve).  Only for a q without conjugate-pair
// steps: those read the vector two steps back, which a pair keeps in shared
// memory only.
bool pair_path(const pp_ctx *c, const OpDesc &op, const float *in, const float *out, float *const bufs[3], int k) {
  if (c->opts.halo != 1 || c->pair_err == nullptr || k < 3 || !poly_horner(c) || c->nf.cx || in == out) return false;
  for (int t = 1; t < k; ++t) {
    const StepCoef sc = poly_step_coef(c, t);
    if (sc.sub_y || !sc.add_v) return false;
  }
  return op_pair_ok(op, in, bufs[0], out) && op_pair_ok(op, bufs[1], in, bufs[0]);
}

int poly_apply_pairs(pp_ctx *c, const OpDesc &op, const float *in, float *out, float *bufs[3], int k) {
  float *B[2] = {bufs[0], bufs[1]};
  RC(run_op<float>(c, op, in, nullptr, nullptr, B[0], poly_step_coef(c, 0)));
  const float *cur = B[0];
  int nxt = 1;
  for (int t = 1; t <= k - 1;) {
    const bool two = t + 1 <= k - 1;
    float *dst = (two ? t + 1 : t) == k - 1 ? out : B[nxt];
    if (two)
      RC(run_pair(c, op, cur, in, dst, poly_step_coef(c, t), poly_step_coef(c, t + 1)));
    else
      RC(run_op<float>(c, op, cur, nullptr, in, dst, poly_step_coef(c, t)));
    cur = dst;
    nxt ^= 1;
    t += two ? 2 : 1;
  }
  return PP_OK;
}

template <typename T>
int poly_apply_raw(pp_ctx *c, const OpDesc &op, const T *in, T *out, T *bufs[3]) {
  const int k = (int)c->coef.size() - 1;
  cudaStream_t s = c->stream;
  if constexpr (std::is_same<T, float>::value)
    if (pair_path(c, op, in, out, bufs, k)) return poly_apply_pairs(c, op, in, out, bufs, k);
  if (k == 0) {
    if (c->nf.cx) return vec_scale_c<T>(in, out, c->n, c->nf.b[0], c->nf.bi[0], s);
    return vec_scale<T>(in, out, c->n, poly_const(c), nullptr, s);
  }
  if (k == 1) return run_op<T>(c, op, in, nullptr, nullptr, out, poly_step_coef(c, 0));
  int i2 = 0, i1 = 1, i0 = 2;  // buffer indices of b_{i+2}, b_{i+1}, free
  RC(run_op<T>(c, op, in, nullptr, nullptr, bufs[i2], poly_step_coef(c, 0)));
  if (k == 2) return run_op<T>(c, op, bufs[i2], nullptr, in, out, poly_step_coef(c, 1));
  RC(run_op<T>(c, op, bufs[i2], nullptr, in, bufs[i1], poly_step_coef(c, 1)));
  for (int t = 2; t <= k - 2; ++t) {
    RC(run_op<T>(c, op, bufs[i1], bufs[i2], in, bufs[i0], poly_step_coef(c, t)));
    const int tmp = i2;
    i2 = i1;
    i1 = i0;
    i0 = tmp;
  }
  return run_op<T>(c, op, bufs[i1], bufs[i2], in, out, poly_step_coef(c, k - 1));
}

template <typename T>
int poly_apply_t(pp_ctx *c, const OpDesc &op, const T *in, T *out, T *bufs[3]) {
  if (c->degree == 0) return poly_apply_raw<T>(c, op, in, out, bufs);
  RC_(prof_begin(c));
  RC_(poly_apply_raw<T>(c, op, in, out, bufs));
  return prof_end(c);
}

// FP32 unit roundoff and the safety factor of the precision switch.
constexpr double kU32 = 0x1p-24;
constexpr double kMixedSafety = 4.0;
// Breakdown threshold of FP32 steps: |h_{j+1,j}| at the level of FP32
// rounding of the column means the direction is noise.
constexpr double kBreakdownRelF32 = 4.0 * 0x1p-24;

// State of one pp_apply call shared by the steps of the Krylov loop.
struct Solve {
  pp_ctx *c;
  cudaStream_t s;
  int64_t n, ldv;
  double *H, *h1, *part, *X, *tri, *z, *zprev, *sig, *wt, *scal, *dd;
  int ldh, nb, K;
  bool right, lanczos;
  bool dcgs = false;  // Arnoldi with delayed reorthogonalization (left, real)
  bool plain = false;  // w = A v_j alone (the node run of Sec. 5.2)
  bool cx = false;     // complex Gram-Schmidt, H complex (column j at H + 2 j ldh)
  int deg;
  int64_t mvms, ip;
};

// The orthogonalization of Krylov step j: w (column j + 1 of V) against the
// basis by Lanczos or CGS2 (complex CGS2 for complex operators), h_{j+1,j} =
// ||w|| and v_{j+1} = w / h_{j+1,j}.
template <typename T>
int orth_step(Solve &S, T *V, T *vj, T *wv, int j, double bd_rel) {
  pp_ctx *c = S.c;
  cudaStream_t s = S.s;
  const int64_t n = S.n, ldv = S.ldv;
  const int nb = S.nb;
  if (S.cx) {  // complex CGS2: h = V^* w (conjugated), w -= V h, twice
    double *hc = S.H + (size_t)2 * j * S.ldh;
    const int J = j + 1;
    RC(vec_multi_dot_c<T>(V, ldv, J, wv, n, S.part, s));
    RC(reduce_cols(S.part, nb, 2 * J, 1, S.h1, hc, s));
    RC(vec_multi_update_c<T>(V, ldv, J, S.h1, wv, n, nullptr, s));
    RC(vec_multi_dot_c<T>(V, ldv, J, wv, n, S.part, s));
    RC(reduce_cols(S.part, nb, 2 * J, 2, S.h1, hc, s));
    RC(vec_multi_update_c<T>(V, ldv, J, S.h1, wv, n, S.part, s));
    // h_{j+1,j} = ||w|| (real; its imaginary part stays 0)
    RC(norm_finalize(S.part, nb, hc + 2 * (j + 1), S.scal, hc, 2 * J, bd_rel, J, c->ws.st, s));
    S.ip += 2 * J + 1;
    return vec_scale<T>(wv, wv, n, 1.0, S.scal, s);
  }
  double *hcol = S.H + (size_t)j * S.ldh;
  if (S.lanczos) {
    RC(vec_dot_partials<T>(wv, vj, n, S.part, nb, s));
    RC(reduce_cols(S.part, nb, 1, 0, hcol + j, nullptr, s));
    RC(vec_lanczos_update<T>(wv, vj, j > 0 ? V + (size_t)(j - 1) * ldv : nullptr, n, hcol + j,
                             j > 0 ? S.H + (size_t)(j - 1) * S.ldh + j : nullptr, S.part, nb, s));
    RC(norm_finalize(S.part, nb, hcol + j + 1, S.scal, hcol + j, 1, bd_rel, j + 1, c->ws.st, s));
    S.ip += 2;
  } else {  // CGS2: h = V^* w, w -= V h, twice
    const int J = j + 1;
    RC(vec_multi_dot<T>(V, ldv, J, wv, n, S.part, nb, s));
    RC(reduce_cols(S.part, nb, J, 1, S.h1, hcol, s));
    // first update and second inner products in one pass over V where J allows
    const int rc = vec_update_dot<T>(V, ldv, J, S.h1, wv, n, S.part, s);
    if (rc == PP_ERR_UNSUPPORTED) {
      RC(vec_multi_update<T>(V, ldv, J, S.h1, wv, n, nullptr, nb, s));
      RC(vec_multi_dot<T>(V, ldv, J, wv, n, S.part, nb, s));
    } else if (rc != PP_OK) {
      return rc;
    }
    RC(reduce_cols(S.part, nb, J, 2, S.h1, hcol, s));
    RC(vec_multi_update<T>(V, ldv, J, S.h1, wv, n, S.part, nb, s));
    RC(norm_finalize(S.part, nb, hcol + j + 1, S.scal, hcol, J, bd_rel, J, c->ws.st, s));
    S.ip += 2 * J + 1;
  }
  return vec_scale<T>(wv, wv, n, 1.0, S.scal, s);
}

// Krylov step j in arithmetic T (Algorithm 1 or 2, one pass of the loop):
// w = A q(A)^2 v_j applied in three stages, orthogonalization against the
// stored basis (columns of V in arithmetic T), h_{j+1,j} = ||w|| and
// v_{j+1} = w / h_{j+1,j} in column j+1 of V.
template <typename T>
int krylov_step(Solve &S, const OpDesc &op, T *V, T *Y, T *t[6], int j, double bd_rel) {
  pp_ctx *c = S.c;
  const int64_t ldv = S.ldv;
  T *pb[3] = {t[2], t[3], t[4]};
  T *vj = V + (size_t)j * ldv;
  T *wv = V + (size_t)(j + 1) * ldv;
  if (S.plain) {          // Arnoldi on A itself
    RC(run_op<T>(c, op, vj, nullptr, nullptr, wv, {1.0, 0.0, 0.0, false, false}));
    S.mvms += 1;
  } else if (!S.right) {  // Algorithm 1: u = A v_j, y = q(A) u, w = q(A) y
    RC(run_op_timed<T>(c, op, vj, nullptr, nullptr, t[0], {1.0, 0.0, 0.0, false, false}));
    RC(poly_apply_t<T>(c, op, t[0], t[1], pb));
    RC(poly_apply_t<T>(c, op, t[1], wv, pb));
    S.mvms += 2 * S.deg + 1;
  } else {                // Algorithm 2: y_j = q(A) v_j, u = q(A) y_j, w = A u
    T *yj = Y + (size_t)j * ldv;
    RC(poly_apply_t<T>(c, op, vj, yj, pb));
    RC(poly_apply_t<T>(c, op, yj, t[0], pb));
    RC(run_op_timed<T>(c, op, t[0], nullptr, nullptr, wv, {1.0, 0.0, 0.0, false, false}));
    S.mvms += 2 * S.deg + 1;
  }
  RC_(prof_begin(c, 1));
  RC_(orth_step<T>(S, V, vj, wv, j, bd_rel));
  return prof_end(c);
}

// Step j of Arnoldi with delayed reorthogonalization (opts.orth =
// PP_ORTH_DCGS2; left preconditioning, real arithmetic): column j holds the
// candidate u_j (one Gram-Schmidt pass, unnormalized), y = A q(A)^2 u_j goes
// to column j + 1; one sweep forms the inner products, one block the
// coefficients, and one more sweep leaves v_j in column j and the candidate
// u_{j+1} in column j + 1 (vec.cu, k_dot2 / k_dcgs_coef / k_update2; k_dcgs_coef also
// sums the sweep's per-chunk partials, a block per column).
// Afterwards columns 0..j of V and columns 0..j-1 of H are final.
template <typename T>
int krylov_step_d(Solve &S, const OpDesc &op, T *V, T *t[6], int j, double bd_rel) {
  pp_ctx *c = S.c;
  cudaStream_t s = S.s;
  const int64_t n = S.n, ldv = S.ldv;
  T *pb[3] = {t[2], t[3], t[4]};
  T *u = V + (size_t)j * ldv;
  T *y = V + (size_t)(j + 1) * ldv;
  RC(run_op_timed<T>(c, op, u, nullptr, nullptr, t[0], {1.0, 0.0, 0.0, false, false}));
  RC(poly_apply_t<T>(c, op, t[0], t[1], pb));
  RC(poly_apply_t<T>(c, op, t[1], y, pb));
  S.mvms += 2 * S.deg + 1;
  RC_(prof_begin(c, 1));
  double *R = S.dd, *co = S.dd + 2 * (size_t)(j + 1);
  RC(vec_dot2<T>(V, ldv, j, u, y, n, S.part, s));
  RC(dcgs_coef(S.part, S.nb, j, R, S.H, S.ldh, S.h1, co, S.scal, bd_rel, c->ws.st, s));
  RC(vec_update2<T>(V, ldv, j, co, S.scal, u, y, n, s));
  S.ip += 2 * (int64_t)j + 2;
  return prof_end(c);
}

// Before the stopping check at Krylov dimension m of the delayed scheme: the
// second pass of column m - 1 (H[0:m, m-1] += V_{0:m}^T u_m, u_m in column m).
template <typename T>
int dcgs_finalize(Solve &S, T *V, int m) {
  pp_ctx *c = S.c;
  RC_(prof_begin(c, 1));
  RC(vec_multi_dot<T>(V, S.ldv, m, V + (size_t)m * S.ldv, S.n, S.part, S.nb, S.s));
  RC(reduce_cols(S.part, S.nb, m, 2, S.dd, S.H + (size_t)(m - 1) * S.ldh, S.s));
  S.ip += m;
  return prof_end(c);
}

// Extra factor on a kappa_pre estimated from H_m rather than bounded by an
// image interval.
constexpr double kKappaEstSafety = 4.0;

// Ratio of the extreme moduli of the eigenvalues of H_m (the Ritz values of
// the preconditioned operator A q(A)^2; its extreme eigenvalues are the first
// to converge), read back after a stopping check.  INFINITY if an eigenvalue
// is zero or the QR does not converge.
double tridiag_eig(const std::vector<double> &al, const std::vector<double> &be, int k);
int hm_kappa(const Solve &S, int m, double *kappa) {
  const size_t cw = S.cx ? 2 : 1;
  std::vector<double> h(cw * (size_t)S.ldh * m);
  PP_CUDA_TRY(cudaMemcpyAsync(h.data(), S.H, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, S.s));
  PP_CUDA_TRY(cudaStreamSynchronize(S.s));
  std::vector<double> mod;
  if (S.cx) {
    std::vector<std::complex<double>> Hd((size_t)m * m, 0.0), w;
    for (int j = 0; j < m; ++j)
      for (int i = 0; i <= std::min(j + 1, m - 1); ++i)
        Hd[(size_t)i * m + j] = {h[2 * ((size_t)j * S.ldh + i)], h[2 * ((size_t)j * S.ldh + i) + 1]};
    if (zhess_eigvals(Hd, m, &w))
      for (const auto &z : w) mod.push_back(std::abs(z));
  } else if (S.lanczos) {
    std::vector<double> al(m), be(m > 1 ? m - 1 : 0);
    for (int j = 0; j < m; ++j) {
      al[j] = h[(size_t)j * S.ldh + j];
      if (j + 1 < m) be[j] = h[(size_t)j * S.ldh + j + 1];
    }
    mod.push_back(std::fabs(tridiag_eig(al, be, 0)));
    mod.push_back(std::fabs(tridiag_eig(al, be, m - 1)));
  } else {
    std::vector<double> Hd((size_t)m * m, 0.0), wr, wi;
    for (int j = 0; j < m; ++j)
      for (int i = 0; i <= std::min(j + 1, m - 1); ++i) Hd[(size_t)i * m + j] = h[(size_t)j * S.ldh + i];
    if (hess_eigvals(Hd, m, &wr, &wi))
      for (int k = 0; k < m; ++k) mod.push_back(std::hypot(wr[k], wi[k]));
  }
  double lo = INFINITY, hi = 0.0;
  for (double v : mod) {
    lo = std::fmin(lo, v);
    hi = std::fmax(hi, v);
  }
  *kappa = mod.empty() || !(lo > 0.0) || !std::isfinite(hi) ? INFINITY : hi / lo;
  return PP_OK;
}

// ---- segment graphs ----
// The kernels of the Krylov steps between two stopping checks (and the
// small solve at the check) depend only on the step range, the precision
// phase and the handle's state, not on b or x; their launches are captured
// once as a CUDA graph and replayed by later solves (one graph launch per
// segment instead of hundreds of kernel launches; the host still reads the
// status record at every check).  Direct launches when profiling (the chain
// events) or if a capture ever failed.
void segs_clear(pp_ctx *c) {
  for (auto &kv : c->segs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  c->segs.clear();
}

void segs_destroy(pp_ctx *c) {
  segs_clear(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  c->cap_stream = nullptr;
}

// Everything a captured segment bakes in: workspace pointers, q, options, tol.
void segs_validate(pp_ctx *c, double tol) {
  const Workspace &w = c->ws;
  uint64_t tb;
  memcpy(&tb, &tol, sizeof tb);
  std::vector<uint64_t> sig = {(uint64_t)(uintptr_t)w.V,   (uint64_t)(uintptr_t)w.Y,
                               (uint64_t)(uintptr_t)w.tmp, (uint64_t)(uintptr_t)w.dmem,
                               (uint64_t)(uintptr_t)w.Vf,  (uint64_t)(uintptr_t)w.Yf,
                               (uint64_t)(uintptr_t)w.hess, (uint64_t)(uintptr_t)w.st,
                               (uint64_t)(uintptr_t)w.val_dw, (uint64_t)(uintptr_t)w.val_f,
                               (uint64_t)(uintptr_t)w.long_rows, (uint64_t)(uintptr_t)w.csr_perm,
                               (uint64_t)w.ldv,
                               c->poly_gen, (uint64_t)c->degree, (uint64_t)c->opts.side,
                               (uint64_t)c->opts.precision, (uint64_t)c->opts.orth,
                               (uint64_t)c->opts.check_every, (uint64_t)c->opts.clenshaw,
                               (uint64_t)c->opts.halo, (uint64_t)c->tile_bdx, tb};
  if (sig != c->seg_sig) {
    segs_clear(c);
    c->seg_sig = sig;
  }
}

// Run body() for the segment `key`: replay its graph, or capture it (the
// captured launches run once by launching the new graph), or run directly.
int run_segment(pp_ctx *c, Solve &S, uint64_t key, const std::function<int()> &body) {
  if (c->opts.profile || c->graphs_off) return body();
  cudaStream_t s = c->stream;
  auto it = c->segs.find(key);
  if (it != c->segs.end()) {
    PP_CUDA_TRY(cudaGraphLaunch(it->second.exec, s));
    pp_launch_count() += it->second.launches;
    c->chain_launches += it->second.chain_launches;
    c->chain_bytes += it->second.chain_bytes;
    S.mvms += it->second.mvms;
    S.ip += it->second.ip;
    return PP_OK;
  }
  const int64_t l0 = pp_launch_count(), cl0 = c->chain_launches, mv0 = S.mvms, ip0 = S.ip;
  const double cb0 = c->chain_bytes;
  if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    c->cap_stream = nullptr;
    c->graphs_off = true;
    return body();
  }
  // the segment's launches go to the capture stream while it records
  cudaStream_t cs = c->cap_stream;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    c->graphs_off = true;
    return body();
  }
  c->stream = cs;
  S.s = cs;
  const int rc = body();
  c->stream = s;
  S.s = s;
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cs, &g);
  cudaGraphExec_t exec = nullptr;
  const bool ok = rc == PP_OK && e == cudaSuccess && g && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {  // nothing of the segment ran: undo the counts and run it directly
    cudaGetLastError();
    pp_launch_count() = l0;
    c->chain_launches = cl0;
    c->chain_bytes = cb0;
    S.mvms = mv0;
    S.ip = ip0;
    if (rc != PP_OK) return rc;
    c->graphs_off = true;
    return body();
  }
  SegGraph sg;
  sg.exec = exec;
  sg.launches = pp_launch_count() - l0;
  sg.chain_launches = c->chain_launches - cl0;
  sg.chain_bytes = c->chain_bytes - cb0;
  sg.mvms = S.mvms - mv0;
  sg.ip = S.ip - ip0;
  c->segs[key] = sg;
  PP_CUDA_TRY(cudaGraphLaunch(exec, s));
  return PP_OK;
}

// Scratch of the global-memory Hessenberg solves for m (grows only; a new
// allocation invalidates the captured segments that use the old one).
int ensure_hess(pp_ctx *c, bool cx, int m, int K) {
  Workspace &w = c->ws;
  const size_t need = cx ? small_hess_scratch_doubles_c(m, K) : small_hess_scratch_doubles(m, K);
  const size_t smem_bytes = ((size_t)(m + 1) * m + 2 * (size_t)m) * (cx ? 2 : 1) * sizeof(double);
  if (smem_bytes > 200 * 1024 && w.hess_n < need) {
    segs_clear(c);
    if (w.hess) cudaFree(w.hess);
    w.hess = nullptr;
    w.hess_n = 0;
    PP_CUDA_TRY(cudaMalloc(&w.hess, need * sizeof(double)));
    w.hess_n = need;
  }
  return PP_OK;
}

// Solve in arithmetic T1; with PP_PREC_MIXED (T1 = dw, T2 = float) the loop
// may move to FP32 at a stopping check.  A perturbation of relative size u
// in a later step changes f_m by about u * kappa_pre times the part of the
// solution still to come (inexact Krylov relaxation; kappa_pre = the ratio
// of the ends of the image of z q(z)^2, which bounds how much a small
// eigenvalue's error is amplified in z^{-1/2}).  That remaining part is
// estimated from the stopping estimate est_m and the observed convergence
// rate rho = (est_m / est_{m-k})^{1/k} as est_m rho / (1 - rho), so the
// switch is taken once
//     est_m rho / (1 - rho) * 4 u_32 * kappa_pre <= tol.
// The start vector, the leading basis vectors and the result stay at
// FP64-grade accuracy; H_m, its coefficients and the small solve are FP64
// throughout.  For complex operators, whose q's image is known only at Ritz
// values, kappa_pre is estimated at each check from the eigenvalues of H_m
// (hm_kappa), times kKappaEstSafety.
template <typename T1, typename T2>
int solve(pp_ctx *c, int f, const double *b_dev, int m_max, double tol, double *x_dev, pp_stats *out) {
  const int prec = c->opts.precision;
  const bool mixed = !std::is_same<T1, T2>::value;
  const bool right = c->opts.side == PP_RIGHT;
  RC(ensure_ws(c, prec, m_max, right, LAYOUT_FULL));
  Workspace &w = c->ws;
  cudaStream_t s = c->stream;
  const OpDesc op1 = make_op(c, arith_of<T1>());
  const OpDesc op2 = make_op(c, arith_of<T2>());
  const int64_t n = c->n, ldv = w.ldv;
  const DLayout L = dlayout(c, w.m_cap);
  double *D = w.dmem;
  // paired stencil launches (opts.halo) report a failed TMA wait to the status
  // record, which this solve reads at every stopping check
  struct PairErrScope {
    pp_ctx *c;
    ~PairErrScope() { c->pair_err = nullptr; }
  } pair_scope{c};
  c->pair_err = &w.st->tma_err;
  Solve S;
  S.c = c;
  S.s = s;
  S.n = n;
  S.ldv = ldv;
  S.H = D + L.H;
  S.h1 = D + L.h1;
  S.part = D + L.part;
  S.X = D + L.X;
  S.tri = D + L.tri;
  S.z = D + L.z;
  S.zprev = D + L.zprev;
  S.sig = D + L.sig;
  S.wt = D + L.wt;
  S.scal = D + L.scal;
  S.dd = D + L.dd;
  S.ldh = L.ldh;
  S.nb = L.nb;
  S.K = L.K;
  S.right = right;
  S.lanczos = c->opts.orth == PP_ORTH_LANCZOS || (c->opts.orth == PP_ORTH_AUTO && c->hermitian);
  S.cx = c->cplx;
  S.dcgs = c->opts.orth == PP_ORTH_DCGS2;
  S.deg = c->degree;
  S.mvms = 0;
  S.ip = 0;
  const int ldh = L.ldh, nb = L.nb, K = L.K;
  const size_t cw = S.cx ? 2 : 1;
  T1 *V1 = (T1 *)w.V, *Y1 = (T1 *)w.Y;
  T2 *V2 = (T2 *)(mixed ? w.Vf : w.V), *Y2 = (T2 *)(mixed ? w.Yf : w.Y);
  T1 *t1[6];
  T2 *t2[6];
  for (int i = 0; i < 6; ++i) {
    t1[i] = (T1 *)w.tmp + (size_t)i * ldv;
    t2[i] = (T2 *)w.tmp + (size_t)i * ldv;
  }
  const int deg = c->degree;
  const int kchk = c->opts.check_every > 0 ? c->opts.check_every : (64 / (deg + 1) > 1 ? 64 / (deg + 1) : 1);
  const int64_t launches0 = pp_launch_count();
  c->chain_launches = 0;
  c->chain_bytes = 0.0;
  c->prof_used = 0;

  PP_CUDA_TRY(cudaEventRecord(w.ev0, s));
  PP_CUDA_TRY(cudaMemsetAsync(w.st, 0, sizeof(DevStatus), s));
  PP_CUDA_TRY(cudaMemsetAsync(S.H, 0, sizeof(double) * cw * ldh * w.m_cap, s));

  // right-hand side in the phase-1 arithmetic
  const T1 *rhs;
  if (std::is_same<T1, double>::value) {
    rhs = (const T1 *)b_dev;
  } else {
    RC(vec_from_f64<T1>(b_dev, t1[0], n, s));
    rhs = t1[0];
  }
  if (f == PP_SQRT) {  // Sec. 4: A^{1/2} b = A^{-1/2} (A b)
    RC(run_op_timed<T1>(c, op1, rhs, nullptr, nullptr, t1[1], {1.0, 0.0, 0.0, false, false}));
    rhs = t1[1];
    S.mvms += 1;
  }
  T1 *pb[3] = {t1[2], t1[3], t1[4]};
  if (!right) {  // Algorithm 1: c = q(A) b, v_1 = c / ||c||
    RC(poly_apply_t<T1>(c, op1, rhs, V1, pb));
    S.mvms += deg;
  } else {       // Algorithm 2: v_1 = b / ||b||
    RC(vec_copy<T1>(rhs, V1, n, s));
  }
  RC(vec_dot_partials<T1>(V1, V1, n, S.part, nb, s));
  RC(norm_finalize(S.part, nb, &w.st->beta0, S.scal, nullptr, 0, 0.0, 0, w.st, s));
  RC(vec_scale<T1>(V1, V1, n, 1.0, S.scal, s));
  PP_CUDA_TRY(cudaMemcpyAsync(w.st_host, w.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  PP_CUDA_TRY(cudaStreamSynchronize(s));
  DevStatus hs = *w.st_host;
  if (hs.tma_err) return pp_set_error(PP_ERR_TIMEOUT, "a paired stencil launch gave up waiting for its TMA loads");
  if (hs.bad) return pp_set_error(PP_ERR_INVALID_ARG, "non-finite norm of the start vector");
  if (hs.breakdown) {  // zero start vector: f(A) 0 = 0
    PP_CUDA_TRY(cudaMemsetAsync(x_dev, 0, sizeof(double) * n, s));
    PP_CUDA_TRY(cudaStreamSynchronize(s));
    if (out) {
      memset(out, 0, sizeof(*out));
      out->mvms = S.mvms;
      out->launches = pp_launch_count() - launches0;
    }
    return PP_OK;
  }
  // stop at the device: memset flags that record a breakdown of the start
  PP_CUDA_TRY(cudaMemsetAsync(&w.st->conv, 0, 3 * sizeof(int), s));

  // Precision switch (PP_PREC_MIXED): columns [0, nv1) of V1 (and [0, ny1)
  // of Y1) hold the phase-1 basis; V2 / Y2 hold FP32 copies of them and the
  // FP32 columns after them.
  const double kappa_pre = c->img_lo > 0.0 && !c->image_on_points ? c->img_hi / c->img_lo : INFINITY;
  // Complex operators only: on the real non-normal graph Laplacian the FP32
  // Horner chain of a Ritz interpolant that is huge between its nodes lost
  // its accuracy (a false FP32 breakdown after the switch, error 4e-6), which
  // no eigenvalue estimate of A q(A)^2 sees; those handles stay in double-word.
  const bool kappa_from_hm = mixed && c->image_on_points && c->cplx;
  double amp = kMixedSafety * kU32 * kappa_pre;
  double est_prev = INFINITY;
  int phase = 1, nv1 = 0, ny1 = 0;
  auto switch_phase = [&](int m_now) -> int {
    if constexpr (!std::is_same<T1, T2>::value) {
      // columns 0..m_now are contiguous at stride ldv in both bases: one launch
      RC((vec_convert<T1, T2>(V1, V2, (int64_t)(m_now + 1) * ldv, s)));
      if (right && m_now > 0) RC((vec_convert<T1, T2>(Y1, Y2, (int64_t)m_now * ldv, s)));
      // the leading columns the result takes from the phase-1 basis: 0..m_now,
      // or 0..m_now-1 with delayed reorthogonalization, whose column m_now
      // still holds the candidate (its final form is written in phase 2)
      nv1 = S.dcgs && m_now > 0 ? m_now : m_now + 1;
      ny1 = m_now;
      phase = 2;
    }
    (void)m_now;
    return PP_OK;
  };
  if (mixed && amp <= tol) RC(switch_phase(0));  // FP32 suffices from the start

  int m = 0, mprev = 0, checks = 0, status = PP_ERR_NOT_CONVERGED, switched_at = mixed ? (phase == 2 ? 0 : -1) : 0;
  bool bd = false;
  // Segments of steps [j0, j1) ending at a stopping check (every kchk steps
  // and at m_max), each with the check's small solve.
  for (int j0 = 0; j0 < m_max;) {
    const int j1 = std::min((j0 / kchk + 1) * kchk, m_max);
    if (!S.lanczos) RC(ensure_hess(c, S.cx, j1, K));
    segs_validate(c, tol);
    const int mp = mprev, ph = phase;
    auto body = [&]() -> int {
      for (int j = j0; j < j1; ++j) {
        if (S.dcgs && ph == 1)
          RC(krylov_step_d<T1>(S, op1, V1, t1, j, kBreakdownRel));
        else if (S.dcgs)
          RC(krylov_step_d<T2>(S, op2, V2, t2, j, std::is_same<T2, float>::value ? kBreakdownRelF32 : kBreakdownRel));
        else if (ph == 1)
          RC(krylov_step<T1>(S, op1, V1, Y1, t1, j, kBreakdownRel));
        else
          RC(krylov_step<T2>(S, op2, V2, Y2, t2, j,
                             std::is_same<T2, float>::value ? kBreakdownRelF32 : kBreakdownRel));
      }
      if (S.dcgs) {  // the check's Hessenberg matrix needs column j1 - 1 final
        if (ph == 1)
          RC(dcgs_finalize<T1>(S, V1, j1));
        else
          RC(dcgs_finalize<T2>(S, V2, j1));
      }
      RC(prof_begin(c, 2));
      if (S.cx)  // S.s: the capture stream while a segment records
        RC(small_hess_quad_c(S.H, ldh, j1, S.sig, S.wt, K, S.X, w.hess, S.s));
      else if (S.lanczos)
        RC(small_tridiag_quad(S.H, ldh, j1, S.sig, S.wt, K, S.X, S.tri, S.s));
      else
        RC(small_hess_quad(S.H, ldh, j1, S.sig, S.wt, K, S.X, w.hess, S.s));
      if (S.cx)
        RC(small_combine_c(S.X, K, j1, mp, S.z, S.zprev, tol, w.st, S.s));
      else
        RC(small_combine(S.X, K, j1, mp, S.z, S.zprev, tol, w.st, S.s));
      return prof_end(c);
    };
    RC(run_segment(c, S, ((uint64_t)j0 << 34) | ((uint64_t)j1 << 2) | (uint64_t)ph, body));
    m = j1;
    j0 = j1;
    {
      mprev = m;
      ++checks;
      PP_CUDA_TRY(cudaMemcpyAsync(w.st_host, w.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
      PP_CUDA_TRY(cudaStreamSynchronize(s));
      hs = *w.st_host;
      if (hs.tma_err) return pp_set_error(PP_ERR_TIMEOUT, "a paired stencil launch gave up waiting for its TMA loads");
      if (hs.bad) return pp_set_error(PP_ERR_CUDA, "non-finite values in the Krylov process");
      if (hs.breakdown) {
        bd = true;
        status = PP_OK;
        break;
      }
      if (hs.conv) {
        status = PP_OK;
        break;
      }
      if (mixed && phase == 1 && std::isfinite(est_prev) && std::isfinite(hs.est) && est_prev > 0.0) {
        if (kappa_from_hm) {
          double kap;
          RC(hm_kappa(S, m, &kap));
          amp = kMixedSafety * kKappaEstSafety * kU32 * kap;
        }
        double rho = std::pow(hs.est / est_prev, 1.0 / kchk);
        if (!(rho < 0.999)) rho = 0.999;
        if (hs.est * rho / (1.0 - rho) * amp <= tol) {
          RC(switch_phase(m));
          switched_at = m;
        }
      }
      est_prev = hs.est;
    }
  }
  // f_m = V_m z (left) or Y_m z (right); with a precision switch the leading
  // columns come from the phase-1 basis
  if (S.cx) {
    const int k1 = phase == 1 ? m : std::min(m, right ? ny1 : nv1);
    if (k1 > 0) RC(vec_reconstruct_c<T1>(right ? Y1 : V1, ldv, k1, S.z, x_dev, n, 0, s));
    if (m > k1)
      RC(vec_reconstruct_c<T2>((right ? Y2 : V2) + (size_t)k1 * ldv, ldv, m - k1, S.z + 2 * k1, x_dev, n,
                               k1 > 0 ? 1 : 0, s));
  } else if (phase == 1) {
    RC(vec_reconstruct<T1>(right ? Y1 : V1, ldv, m, S.z, x_dev, n, 0, s));
  } else {
    const int k1 = std::min(m, right ? ny1 : nv1);
    if (k1 > 0) RC(vec_reconstruct<T1>(right ? Y1 : V1, ldv, k1, S.z, x_dev, n, 0, s));
    if (m > k1)
      RC(vec_reconstruct<T2>((right ? Y2 : V2) + (size_t)k1 * ldv, ldv, m - k1, S.z + k1, x_dev, n,
                             k1 > 0 ? 1 : 0, s));
  }
  PP_CUDA_TRY(cudaEventRecord(w.ev1, s));
  PP_CUDA_TRY(cudaEventSynchronize(w.ev1));
  if (out) {
    memset(out, 0, sizeof(*out));
    out->status = status;
    out->iters = bd ? hs.m_bd : m;
    out->checks = checks;
    out->breakdown = bd ? 1 : 0;
    out->mvms = S.mvms;
    out->inner_products = S.ip;
    out->est_err = hs.est;
    out->beta0 = hs.beta0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, w.ev0, w.ev1);
    out->ms_total = ms;
    out->launches = pp_launch_count() - launches0;
    out->chain_launches = c->chain_launches;
    out->chain_bytes = c->chain_bytes;
    out->chain_ms = c->opts.profile ? prof_ms(c) : 0.0;
    out->orth_ms = c->opts.profile ? prof_ms(c, 1) : 0.0;
    out->small_ms = c->opts.profile ? prof_ms(c, 2) : 0.0;
    out->switch_iter = switched_at;
  }
  if (status != PP_OK) pp_set_error(status, "m_max reached before the stopping estimate fell below tol");
  return status;
}

// Two-pass Lanczos (Hermitian A): pass 1 is the Lanczos loop of solve() with
// three rotating basis vectors, keeping H_m and the stopping checks; pass 2
// regenerates v_1 .. v_m from the stored alpha_j, beta_j (the same kernels on
// the same data, so the same vectors bit for bit) and accumulates f_m = V_m z
// (left) or Y_m z (right, y_j = q(A) v_j recomputed in the step) as it goes.
// The precision switch of PP_PREC_MIXED happens at the same step in both
// passes.  Basis storage: columns j mod 3, plus v_1 kept in column 3.
template <typename T1, typename T2>
int solve_two_pass(pp_ctx *c, int f, const double *b_dev, int m_max, double tol, double *x_dev, pp_stats *out) {
  const int prec = c->opts.precision;
  const bool mixed = !std::is_same<T1, T2>::value;
  const bool right = c->opts.side == PP_RIGHT;
  RC(ensure_ws(c, prec, m_max, false, LAYOUT_TWO_PASS));
  Workspace &w = c->ws;
  cudaStream_t s = c->stream;
  const OpDesc op1 = make_op(c, arith_of<T1>());
  const OpDesc op2 = make_op(c, arith_of<T2>());
  const int64_t n = c->n, ldv = w.ldv;
  const DLayout L = dlayout(c, w.m_cap);
  double *D = w.dmem;
  double *H = D + L.H, *part = D + L.part, *X = D + L.X, *tri = D + L.tri, *z = D + L.z, *zprev = D + L.zprev;
  double *sig = D + L.sig, *wt = D + L.wt, *scal = D + L.scal;
  const int ldh = L.ldh, nb = L.nb, K = L.K, deg = c->degree;
  T1 *V1 = (T1 *)w.V;
  T2 *V2 = (T2 *)(mixed ? w.Vf : w.V);
  T1 *t1[6];
  T2 *t2[6];
  for (int i = 0; i < 6; ++i) {
    t1[i] = (T1 *)w.tmp + (size_t)i * ldv;
    t2[i] = (T2 *)w.tmp + (size_t)i * ldv;
  }
  auto col1 = [&](int j) { return V1 + (size_t)(j % 3) * ldv; };
  auto col2 = [&](int j) { return V2 + (size_t)(j % 3) * ldv; };
  const int kchk = c->opts.check_every > 0 ? c->opts.check_every : (64 / (deg + 1) > 1 ? 64 / (deg + 1) : 1);
  const int64_t launches0 = pp_launch_count();
  int64_t mvms = 0, ip = 0;
  c->chain_launches = 0;
  c->chain_bytes = 0.0;
  c->prof_used = 0;
  PP_CUDA_TRY(cudaEventRecord(w.ev0, s));
  PP_CUDA_TRY(cudaMemsetAsync(w.st, 0, sizeof(DevStatus), s));
  PP_CUDA_TRY(cudaMemsetAsync(H, 0, sizeof(double) * (size_t)ldh * w.m_cap, s));
  // w = A q(A)^2 v (three stages; right preconditioning leaves y = q(A) v in ty)
  auto apply_pre = [&](auto tag, const OpDesc &op, auto *v, auto *wv, auto **t, auto *ty) -> int {
    using T = decltype(tag);
    T *pb[3] = {t[2], t[3], t[4]};
    if (!right) {
      RC_(run_op_timed<T>(c, op, v, nullptr, nullptr, t[0], {1.0, 0.0, 0.0, false, false}));
      RC_(poly_apply_t<T>(c, op, t[0], t[1], pb));
      RC_(poly_apply_t<T>(c, op, t[1], wv, pb));
    } else {
      RC_(poly_apply_t<T>(c, op, v, ty, pb));
      RC_(poly_apply_t<T>(c, op, ty, t[0], pb));
      RC_(run_op_timed<T>(c, op, t[0], nullptr, nullptr, wv, {1.0, 0.0, 0.0, false, false}));
    }
    mvms += 2 * deg + 1;
    return PP_OK;
  };
  // start vector (as solve())
  const T1 *rhs;
  if (std::is_same<T1, double>::value) {
    rhs = (const T1 *)b_dev;
  } else {
    RC(vec_from_f64<T1>(b_dev, t1[0], n, s));
    rhs = t1[0];
  }
  if (f == PP_SQRT) {
    RC(run_op_timed<T1>(c, op1, rhs, nullptr, nullptr, t1[1], {1.0, 0.0, 0.0, false, false}));
    rhs = t1[1];
    mvms += 1;
  }
  T1 *v0 = V1 + (size_t)3 * ldv;
  {
    T1 *pb[3] = {t1[2], t1[3], t1[4]};
    if (!right) {
      RC(poly_apply_t<T1>(c, op1, rhs, v0, pb));
      mvms += deg;
    } else {
      RC(vec_copy<T1>(rhs, v0, n, s));
    }
  }
  RC(vec_dot_partials<T1>(v0, v0, n, part, nb, s));
  RC(norm_finalize(part, nb, &w.st->beta0, scal, nullptr, 0, 0.0, 0, w.st, s));
  RC(vec_scale<T1>(v0, v0, n, 1.0, scal, s));
  RC(vec_copy<T1>(v0, col1(0), n, s));
  PP_CUDA_TRY(cudaMemcpyAsync(w.st_host, w.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  PP_CUDA_TRY(cudaStreamSynchronize(s));
  DevStatus hs = *w.st_host;
  if (hs.bad) return pp_set_error(PP_ERR_INVALID_ARG, "non-finite norm of the start vector");
  if (hs.breakdown) {
    PP_CUDA_TRY(cudaMemsetAsync(x_dev, 0, sizeof(double) * n, s));
    PP_CUDA_TRY(cudaStreamSynchronize(s));
    if (out) {
      memset(out, 0, sizeof(*out));
      out->mvms = mvms;
      out->launches = pp_launch_count() - launches0;
    }
    return PP_OK;
  }
  PP_CUDA_TRY(cudaMemsetAsync(&w.st->conv, 0, 3 * sizeof(int), s));
  // Lanczos step j in arithmetic T on the rotating columns; pass 1 forms
  // alpha_j and beta_j, pass 2 (regen) reuses the stored ones
  auto lanczos_step = [&](auto tag, const OpDesc &op, auto *vj, auto *vjm1, auto *wv, auto **t, int j, bool regen,
                          double bd_rel) -> int {
    using T = decltype(tag);
    RC_(apply_pre(tag, op, vj, wv, t, t[5]));
    double *hcol = H + (size_t)j * ldh;
    if (!regen) {
      RC_(vec_dot_partials<T>(wv, vj, n, part, nb, s));
      RC_(reduce_cols(part, nb, 1, 0, hcol + j, nullptr, s));
    }
    RC_(vec_lanczos_update<T>(wv, vj, j > 0 ? vjm1 : nullptr, n, hcol + j, j > 0 ? H + (size_t)(j - 1) * ldh + j : nullptr,
                              part, nb, s));
    if (!regen) {
      RC_(norm_finalize(part, nb, hcol + j + 1, scal, hcol + j, 1, bd_rel, j + 1, w.st, s));
      ip += 2;
    } else {
      RC_(vec_recip(hcol + j + 1, scal, s));
    }
    return vec_scale<T>(wv, wv, n, 1.0, scal, s);
  };
  const double kappa_pre = c->img_lo > 0.0 && !c->image_on_points ? c->img_hi / c->img_lo : INFINITY;
  const double amp = kMixedSafety * kU32 * kappa_pre;
  double est_prev = INFINITY;
  int phase = 1, sw = mixed ? -1 : 0;
  auto convert_live = [&](int m_now) -> int {  // v_{m_now} and v_{m_now - 1} to FP32
    if constexpr (!std::is_same<T1, T2>::value) {
      for (int q = std::max(0, m_now - 1); q <= m_now; ++q) RC_((vec_convert<T1, T2>(col1(q), col2(q), n, s)));
    }
    (void)m_now;
    return PP_OK;
  };
  if (mixed && amp <= tol) {
    RC(convert_live(0));
    phase = 2;
    sw = 0;
  }
  int m = 0, mprev = 0, checks = 0, status = PP_ERR_NOT_CONVERGED;
  bool bd = false;
  for (int j = 0; j < m_max; ++j) {  // pass 1
    if (phase == 1)
      RC(lanczos_step(T1(), op1, col1(j), col1(j + 2), col1(j + 1), t1, j, false, kBreakdownRel));
    else
      RC(lanczos_step(T2(), op2, col2(j), col2(j + 2), col2(j + 1), t2, j, false,
                      std::is_same<T2, float>::value ? kBreakdownRelF32 : kBreakdownRel));
    m = j + 1;
    if (m % kchk == 0 || m == m_max) {
      RC(small_tridiag_quad(H, ldh, m, sig, wt, K, X, tri, s));
      RC(small_combine(X, K, m, mprev, z, zprev, tol, w.st, s));
      mprev = m;
      ++checks;
      PP_CUDA_TRY(cudaMemcpyAsync(w.st_host, w.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
      PP_CUDA_TRY(cudaStreamSynchronize(s));
      hs = *w.st_host;
      if (hs.bad) return pp_set_error(PP_ERR_CUDA, "non-finite values in the Krylov process");
      if (hs.breakdown) {
        bd = true;
        status = PP_OK;
        break;
      }
      if (hs.conv) {
        status = PP_OK;
        break;
      }
      if (mixed && phase == 1 && std::isfinite(est_prev) && std::isfinite(hs.est) && est_prev > 0.0) {
        double rho = std::pow(hs.est / est_prev, 1.0 / kchk);
        if (!(rho < 0.999)) rho = 0.999;
        if (hs.est * rho / (1.0 - rho) * amp <= tol) {
          RC(convert_live(m));
          phase = 2;
          sw = m;
        }
      }
      est_prev = hs.est;
    }
  }
  // pass 2: regenerate the basis and accumulate x (mz columns, the last
  // check's z).  As in solve(), the leading columns 0 .. sw of the
  // reconstruction come from the phase-1 vectors and step j runs in FP32 from
  // j = sw on (sw = the pass-1 switch).
  const int mz = mprev > 0 ? mprev : m;
  RC(vec_copy<T1>(v0, col1(0), n, s));
  for (int j = 0; j < mz; ++j) {
    const bool phase2 = mixed && sw >= 0 && j >= sw;
    if (!right) {
      if (!mixed || sw < 0 || j <= sw)
        RC(vec_reconstruct<T1>(col1(j), ldv, 1, z + j, x_dev, n, j > 0 ? 1 : 0, s));
      else
        RC(vec_reconstruct<T2>(col2(j), ldv, 1, z + j, x_dev, n, 1, s));
    }
    if (mixed && j == sw) RC(convert_live(j));
    if (j + 1 < mz || right) {
      if (!phase2) {
        RC(lanczos_step(T1(), op1, col1(j), col1(j + 2), col1(j + 1), t1, j, true, kBreakdownRel));
        if (right) RC(vec_reconstruct<T1>(t1[5], ldv, 1, z + j, x_dev, n, j > 0 ? 1 : 0, s));
      } else {
        RC(lanczos_step(T2(), op2, col2(j), col2(j + 2), col2(j + 1), t2, j, true,
                        std::is_same<T2, float>::value ? kBreakdownRelF32 : kBreakdownRel));
        if (right) RC(vec_reconstruct<T2>(t2[5], ldv, 1, z + j, x_dev, n, j > 0 ? 1 : 0, s));
      }
    }
  }
  PP_CUDA_TRY(cudaEventRecord(w.ev1, s));
  PP_CUDA_TRY(cudaEventSynchronize(w.ev1));
  if (out) {
    memset(out, 0, sizeof(*out));
    out->status = status;
    out->iters = bd ? hs.m_bd : m;
    out->checks = checks;
    out->breakdown = bd ? 1 : 0;
    out->mvms = mvms;
    out->inner_products = ip;
    out->est_err = hs.est;
    out->beta0 = hs.beta0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, w.ev0, w.ev1);
    out->ms_total = ms;
    out->launches = pp_launch_count() - launches0;
    out->chain_launches = c->chain_launches;
    out->chain_bytes = c->chain_bytes;
    out->chain_ms = c->opts.profile ? prof_ms(c) : 0.0;
    out->switch_iter = sw;
  }
  if (status != PP_OK) pp_set_error(status, "m_max reached before the stopping estimate fell below tol");
  return status;
}

int check_ready(pp_ctx *c) {
  if (!c) return pp_set_error(PP_ERR_INVALID_ARG, "NULL handle");
  if (!c->have_poly) return pp_set_error(PP_ERR_STATE, "pp_build_poly has not been called");
  return PP_OK;
}

template <typename T>
int op_apply_t(pp_ctx *c, const double *x, double *y) {
  RC(ensure_ws(c, c->opts.precision, c->ws.m_cap > 0 ? c->ws.m_cap : 1, false));
  const OpDesc op = make_op(c, arith_of<T>());
  T *t0 = (T *)c->ws.tmp, *t1 = t0 + c->ws.ldv;
  if constexpr (std::is_same<T, double>::value) {
    (void)t0;
    (void)t1;
    return op_step<T>(op, (const T *)x, nullptr, nullptr, (T *)y, {1.0, 0.0, 0.0, false, false}, c->stream);
  } else {
    RC(vec_from_f64<T>(x, t0, c->n, c->stream));
    RC(op_step<T>(op, t0, nullptr, nullptr, t1, {1.0, 0.0, 0.0, false, false}, c->stream));
    return vec_to_f64<T>(t1, y, c->n, c->stream);
  }
}

template <typename T>
int poly_apply_api_t(pp_ctx *c, const double *x, double *y) {
  RC(ensure_ws(c, c->opts.precision, c->ws.m_cap > 0 ? c->ws.m_cap : 1, false));
  const OpDesc op = make_op(c, arith_of<T>());
  T *t[6];
  for (int i = 0; i < 6; ++i) t[i] = (T *)c->ws.tmp + (size_t)i * c->ws.ldv;
  T *pb[3] = {t[2], t[3], t[4]};
  if constexpr (std::is_same<T, double>::value) {
    return poly_apply_t<T>(c, op, (const T *)x, (T *)y, pb);
  } else {
    RC(vec_from_f64<T>(x, t[0], c->n, c->stream));
    RC(poly_apply_t<T>(c, op, t[0], t[1], pb));
    return vec_to_f64<T>(t[1], y, c->n, c->stream);
  }
}

// ---- q(A) x without device allocation (pp_poly_apply_static) ----
//
// Scratch for pp_poly_apply_static: five vectors of PP_STATIC_MAX_N entries
// of 8 bytes (10 MiB), resident on every device that loads the library until
// the process exits.  Host code may not use the symbol as an address: the
// device address is looked up once per device with cudaGetSymbolAddress.
constexpr int kStaticVecs = 5;
constexpr int kStaticMaxDevices = 64;

}  // namespace

int csr_prepare(pp_ctx *c, int prec) {
  if (c->op_kind != OPK_CSR) return PP_OK;
  Workspace &w = c->ws;
  if (c->nnz < 0) {
    int64_t nnz = 0;
    PP_CUDA_TRY(cudaMemcpy(&nnz, c->rowptr + c->n, sizeof(int64_t), cudaMemcpyDeviceToHost));
    c->nnz = nnz;
  }
  if (w.nlong < 0) {
    // rows longer than kLongRow entries, listed once per handle (rowptr read
    // back): those above kBlockRow first (a block each), then the others (a
    // warp each)
    std::vector<int64_t> rp((size_t)c->n + 1);
    PP_CUDA_TRY(cudaMemcpy(rp.data(), c->rowptr, sizeof(int64_t) * rp.size(), cudaMemcpyDeviceToHost));
    std::vector<int32_t> lr, wr;
    for (int64_t i = 0; i < c->n; ++i) {
      const int64_t len = rp[i + 1] - rp[i];
      if (len > kBlockRow)
        lr.push_back((int32_t)i);
      else if (len > kLongRow)
        wr.push_back((int32_t)i);
    }
    const size_t nl = lr.size();
    lr.insert(lr.end(), wr.begin(), wr.end());
    if (!lr.empty()) {
      PP_CUDA_TRY(cudaMalloc(&w.long_rows, sizeof(int32_t) * lr.size()));
      PP_CUDA_TRY(cudaMemcpy(w.long_rows, lr.data(), sizeof(int32_t) * lr.size(), cudaMemcpyHostToDevice));
    }
    w.nlong = (int)nl;
    w.nwarp = (int)wr.size();
    // the lane path's rows sorted by length within windows of kPermWindow
    // rows, where the lengths vary: a warp serves 32 / L rows, and with rows
    // of mixed lengths (a power-law graph) each warp ran as many rounds as
    // its longest row.  The windows keep the rows' accesses local.  The sum
    // of each row is computed exactly as before.
    std::vector<int32_t> sr;
    sr.reserve((size_t)c->n);
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = 0; i < c->n; ++i) {
      const int64_t len = rp[i + 1] - rp[i];
      if (len > kLongRow) continue;
      sr.push_back((int32_t)i);
      s1 += (double)len;
      s2 += (double)len * (double)len;
    }
    const double ns = (double)sr.size();
    if (!sr.empty() && s2 / ns - (s1 / ns) * (s1 / ns) > kPermMinVar) {
      auto len_of = [&](int32_t r) { return rp[(size_t)r + 1] - rp[(size_t)r]; };
      for (size_t w0 = 0; w0 < sr.size(); w0 += kPermWindow) {
        const size_t w1 = std::min(sr.size(), w0 + (size_t)kPermWindow);
        std::stable_sort(sr.begin() + w0, sr.begin() + w1,
                         [&](int32_t a, int32_t b) { return len_of(a) < len_of(b); });
      }
      PP_CUDA_TRY(cudaMalloc(&w.csr_perm, sizeof(int32_t) * sr.size()));
      PP_CUDA_TRY(cudaMemcpy(w.csr_perm, sr.data(), sizeof(int32_t) * sr.size(), cudaMemcpyHostToDevice));
      w.nshort = (int64_t)sr.size();
    }
  }
  if (prec == PP_PREC_DW || prec == PP_PREC_MIXED) {
    if (w.val_exact_f32 < 0) {  // values read back once: are they all exact in FP32?
      std::vector<double> v((size_t)c->nnz);
      if (c->nnz > 0) PP_CUDA_TRY(cudaMemcpy(v.data(), c->val, sizeof(double) * v.size(), cudaMemcpyDeviceToHost));
      int exact = 1;
      for (double x : v)
        if ((double)(float)x != x) {
          exact = 0;
          break;
        }
      w.val_exact_f32 = exact;
    }
    if (w.val_exact_f32 && !w.val_f) {  // the double-word step then reads FP32 values
      PP_CUDA_TRY(cudaMalloc(&w.val_f, (size_t)std::max<int64_t>(c->nnz, 1) * sizeof(float)));
      RC_(vec_from_f64<float>(c->val, (float *)w.val_f, c->nnz, c->stream));
    }
    if (!w.val_exact_f32 && !w.val_dw) {
      PP_CUDA_TRY(cudaMalloc(&w.val_dw, (size_t)std::max<int64_t>(c->nnz, 1) * sizeof(dw)));
      RC_(vec_from_f64<dw>(c->val, (dw *)w.val_dw, c->nnz, c->stream));
    }
  }
  if (prec == PP_PREC_MIXED && !w.val_f) {
    PP_CUDA_TRY(cudaMalloc(&w.val_f, (size_t)std::max<int64_t>(c->nnz, 1) * sizeof(float)));
    RC_(vec_from_f64<float>(c->val, (float *)w.val_f, c->nnz, c->stream));
  }
  return PP_OK;
}

OpDesc handle_op_desc(const pp_ctx *c, int arith) { return make_op(c, arith); }

static __device__ __align__(256) double pp_static_scratch[kStaticVecs * (size_t)PP_STATIC_MAX_N];

namespace {

std::mutex g_static_mu;
void *g_static_addr[kStaticMaxDevices] = {};

// Device address of pp_static_scratch on the handle's device (looked up on
// the first call per device).  The handle's kernels run on the device that
// was current when it was created; the lookup needs that device current, so
// a call from a thread whose current device differs is refused instead of
// handing the kernels another GPU's copy of the array.
int static_scratch_addr(const pp_ctx *c, void **out) {
  int dev = 0;
  PP_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != c->device)
    return pp_set_error(PP_ERR_INVALID_ARG, "the current CUDA device (" + std::to_string(dev) +
                                                ") is not the handle's device (" + std::to_string(c->device) + ")");
  if (dev < 0 || dev >= kStaticMaxDevices) return pp_set_error(PP_ERR_UNSUPPORTED, "device ordinal >= 64");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void *p = nullptr;
    PP_CUDA_TRY(cudaGetSymbolAddress(&p, pp_static_scratch));
    if (!p) return pp_set_error(PP_ERR_CUDA, "cudaGetSymbolAddress returned NULL");
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return PP_OK;
}

template <typename T>
int poly_apply_static_t(pp_ctx *c, const double *x, double *y, void *base) {
  const OpDesc op = make_op(c, arith_of<T>());
  T *t[kStaticVecs];
  for (int i = 0; i < kStaticVecs; ++i) t[i] = (T *)base + (size_t)i * PP_STATIC_MAX_N;
  if (std::is_same<T, double>::value) {
    T *pb[3] = {t[0], t[1], t[2]};
    return poly_apply_raw<T>(c, op, (const T *)x, (T *)y, pb);
  }
  T *pb[3] = {t[2], t[3], t[4]};
  RC(vec_from_f64<T>(x, t[0], c->n, c->stream));
  RC(poly_apply_raw<T>(c, op, t[0], t[1], pb));
  return vec_to_f64<T>(t[1], y, c->n, c->stream);
}

// ---- spectral interval of a Hermitian operator (pp_build_poly without an interval) ----

// Number of eigenvalues of the symmetric tridiagonal T = (al, be) below x:
// the negative pivots of T - x I = L D L^T (Sturm sequence).
int sturm_count(const std::vector<double> &al, const std::vector<double> &be, double x) {
  int cnt = 0;
  double d = 1.0;
  for (size_t i = 0; i < al.size(); ++i) {
    d = (al[i] - x) - (i > 0 ? be[i - 1] * be[i - 1] / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

// k-th smallest eigenvalue (k = 0 .. m-1) by bisection inside the Gershgorin interval.
double tridiag_eig(const std::vector<double> &al, const std::vector<double> &be, int k) {
  double lo = INFINITY, hi = -INFINITY;
  for (size_t i = 0; i < al.size(); ++i) {
    const double r = (i > 0 ? std::fabs(be[i - 1]) : 0.0) + (i + 1 < al.size() ? std::fabs(be[i]) : 0.0);
    lo = std::fmin(lo, al[i] - r);
    hi = std::fmax(hi, al[i] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::fmax(std::fabs(lo), std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count(al, be, mid) > k)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Extreme Ritz values of A after `steps` Lanczos steps from a fixed
// pseudo-random start, in arithmetic T on the device with three rotating
// vectors (no basis is kept); the tridiagonal matrix is read back and its
// extreme eigenvalues found on the host.
template <typename T>
int lanczos_extremes(pp_ctx *c, int steps, double *lo, double *hi) {
  if (c->qsig.empty()) {  // the workspace layout needs a quadrature size
    c->qsig.assign(1, 1.0);
    c->qwt.assign(1, 1.0);
  }
  RC(ensure_ws(c, c->opts.precision, 1, false));
  Workspace &w = c->ws;
  cudaStream_t s = c->stream;
  const OpDesc op = make_op(c, arith_of<T>());
  const int64_t n = c->n, ldv = w.ldv;
  const DLayout L = dlayout(c, w.m_cap);
  double *part = w.dmem + L.part, *scal = w.dmem + L.scal;
  const int nb = L.nb;
  T *t[3];
  for (int i = 0; i < 3; ++i) t[i] = (T *)w.tmp + (size_t)i * ldv;
  double *coef = nullptr;  // alpha_j at [2 j], beta_j at [2 j + 1]
  PP_CUDA_TRY(cudaMalloc(&coef, sizeof(double) * 2 * (size_t)steps));
  auto body = [&]() -> int {
    PP_CUDA_TRY(cudaMemsetAsync(w.st, 0, sizeof(DevStatus), s));
    PP_CUDA_TRY(cudaMemsetAsync(coef, 0, sizeof(double) * 2 * (size_t)steps, s));
    T *vprev = t[1], *vj = t[0], *wv = t[2];
    RC(vec_fill_hash<T>(vj, n, 0x5eedull, s));
    RC(vec_dot_partials<T>(vj, vj, n, part, nb, s));
    RC(norm_finalize(part, nb, &w.st->beta0, scal, nullptr, 0, 0.0, 0, w.st, s));
    RC(vec_scale<T>(vj, vj, n, 1.0, scal, s));
    for (int j = 0; j < steps; ++j) {
      RC(op_step<T>(op, vj, nullptr, nullptr, wv, {1.0, 0.0, 0.0, false, false}, s));
      RC(vec_dot_partials<T>(wv, vj, n, part, nb, s));
      RC(reduce_cols(part, nb, 1, 0, coef + 2 * j, nullptr, s));
      RC(vec_lanczos_update<T>(wv, vj, j > 0 ? vprev : nullptr, n, coef + 2 * j,
                               j > 0 ? coef + 2 * j - 1 : nullptr, part, nb, s));
      RC(norm_finalize(part, nb, coef + 2 * j + 1, scal, coef + 2 * j, 1, kBreakdownRel, j + 1, w.st, s));
      RC(vec_scale<T>(wv, wv, n, 1.0, scal, s));
      T *old = vprev;
      vprev = vj;
      vj = wv;
      wv = old;
    }
    std::vector<double> ch(2 * (size_t)steps);
    PP_CUDA_TRY(cudaMemcpyAsync(ch.data(), coef, sizeof(double) * ch.size(), cudaMemcpyDeviceToHost, s));
    PP_CUDA_TRY(cudaMemcpyAsync(w.st_host, w.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    PP_CUDA_TRY(cudaStreamSynchronize(s));
    if (w.st_host->bad) return pp_set_error(PP_ERR_CUDA, "non-finite values in the interval estimate");
    const int m = w.st_host->breakdown ? std::max(1, w.st_host->m_bd) : steps;
    std::vector<double> al(m), be(m > 1 ? m - 1 : 0);
    for (int j = 0; j < m; ++j) {
      al[j] = ch[2 * (size_t)j];
      if (j + 1 < m) be[j] = ch[2 * (size_t)j + 1];
    }
    *lo = tridiag_eig(al, be, 0);
    *hi = tridiag_eig(al, be, m - 1);
    return PP_OK;
  };
  const int rc = body();
  cudaFree(coef);
  return rc;
}

// Node run of Sec. 5.2: d Arnoldi steps on A (classical Gram-Schmidt twice,
// the kernels of the solve loop) from the fixed pseudo-random start vector,
// in arithmetic T.  Returns the Hessenberg matrix (column j at Hh[j * ldh],
// rows 0 .. j+1) and the number m <= d of steps before the Krylov space
// became invariant.
template <typename T>
int ritz_arnoldi(pp_ctx *c, int d, std::vector<double> *Hh, int *ldh_out, int *m_out) {
  if (c->qsig.empty()) {  // the workspace layout needs a quadrature size
    c->qsig.assign(1, 1.0);
    c->qwt.assign(1, 1.0);
  }
  RC(ensure_ws(c, c->opts.precision, d, false, LAYOUT_FULL));
  Workspace &w = c->ws;
  cudaStream_t s = c->stream;
  const OpDesc op = make_op(c, arith_of<T>());
  const DLayout L = dlayout(c, w.m_cap);
  double *D = w.dmem;
  Solve S;
  S.c = c;
  S.s = s;
  S.n = c->n;
  S.ldv = w.ldv;
  S.H = D + L.H;
  S.h1 = D + L.h1;
  S.part = D + L.part;
  S.X = D + L.X;
  S.tri = D + L.tri;
  S.z = D + L.z;
  S.zprev = D + L.zprev;
  S.sig = D + L.sig;
  S.wt = D + L.wt;
  S.scal = D + L.scal;
  S.ldh = L.ldh;
  S.nb = L.nb;
  S.K = L.K;
  S.right = false;
  S.lanczos = false;
  S.plain = true;
  S.cx = c->cplx;
  S.deg = 0;
  S.mvms = 0;
  S.ip = 0;
  const size_t cw = S.cx ? 2 : 1;
  T *V = (T *)w.V;
  T *t[6];
  for (int i = 0; i < 6; ++i) t[i] = (T *)w.tmp + (size_t)i * w.ldv;
  PP_CUDA_TRY(cudaMemsetAsync(w.st, 0, sizeof(DevStatus), s));
  PP_CUDA_TRY(cudaMemsetAsync(S.H, 0, sizeof(double) * cw * L.ldh * w.m_cap, s));
  RC(vec_fill_hash<T>(V, c->n, 0x5eedull, s));
  RC(vec_dot_partials<T>(V, V, c->n, S.part, S.nb, s));
  RC(norm_finalize(S.part, S.nb, &w.st->beta0, S.scal, nullptr, 0, 0.0, 0, w.st, s));
  RC(vec_scale<T>(V, V, c->n, 1.0, S.scal, s));
  for (int j = 0; j < d; ++j) RC(krylov_step<T>(S, op, V, nullptr, t, j, kBreakdownRel));
  Hh->assign(cw * L.ldh * d, 0.0);  // complex operators: (re, im) pairs
  PP_CUDA_TRY(cudaMemcpyAsync(Hh->data(), S.H, sizeof(double) * Hh->size(), cudaMemcpyDeviceToHost, s));
  PP_CUDA_TRY(cudaMemcpyAsync(w.st_host, w.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  PP_CUDA_TRY(cudaStreamSynchronize(s));
  if (w.st_host->bad) return pp_set_error(PP_ERR_CUDA, "non-finite values in the Ritz value run");
  *m_out = w.st_host->breakdown ? std::max(1, w.st_host->m_bd) : d;
  *ldh_out = L.ldh;
  return PP_OK;
}

// Closed-form spectral interval of the 2D / 3D stencil operators.
bool closed_form_interval(const pp_ctx *c, double *a, double *b) {
  if (c->op_kind == OPK_ST2D) {
    *a = *b = 0.0;
    for (int i = 0; i < 2; ++i) {
      const double N = (double)c->dims[i];
      *a += 2.0 - 2.0 * std::cos(M_PI / (N + 1));
      *b += 2.0 - 2.0 * std::cos(N * M_PI / (N + 1));
    }
    return true;
  }
  if (c->op_kind == OPK_ST3D) {
    // Sec. 6, Example 1 for the Laplacian; convection-diffusion factors are
    // diagonally similar to tridiag(-r, 2+ch, -r), r = sqrt(1+ch)
    const double r = std::sqrt(1.0 + c->ch);
    *a = *b = 0.0;
    for (int i = 0; i < 3; ++i) {
      const double N = (double)c->dims[i];
      *a += (2.0 + c->ch) - 2.0 * r * std::cos(M_PI / (N + 1));
      *b += (2.0 + c->ch) - 2.0 * r * std::cos(N * M_PI / (N + 1));
    }
    return true;
  }
  return false;
}

// Polynomial-independent tail of pp_build_poly: the quadrature of the small
// solve sized by the image [lo, hi] of z q(z)^2, and a fresh device layout.
void finish_poly(pp_ctx *c, double margin = 1e3) {
  // real Ritz values for Hermitian A, |arg| <= pi/3 allowed otherwise (more
  // when q has complex nodes far from the real axis); margins around the image
  double theta = c->hermitian ? 0.0 : M_PI / 3.0;
  if (!c->hermitian)
    for (size_t i = 0; i < c->nf.re.size(); ++i)
      theta = std::fmax(theta, std::fmin(0.45 * M_PI, 1.5 * std::fabs(std::atan2(c->nf.im[i], c->nf.re[i]))));
  invsqrt_quadrature(c->img_lo / margin, c->img_hi * margin, 1e-15, theta, &c->qsig, &c->qwt);
  c->quad_uploaded = false;
  ++c->poly_gen;
  if (c->ws.dmem) {  // K may have changed: re-layout on next use
    cudaFree(c->ws.dmem);
    c->ws.dmem = nullptr;
  }
  c->have_poly = true;
}

int read_nnz(pp_ctx *c) {
  if (c->op_kind == OPK_CSR && c->nnz < 0) {
    int64_t nnz = 0;
    PP_CUDA_TRY(cudaMemcpy(&nnz, c->rowptr + c->n, sizeof(int64_t), cudaMemcpyDeviceToHost));
    c->nnz = nnz;
  }
  return PP_OK;
}

// q = the interpolant of z^{-1/2} at the nodes (real values or conjugate
// pairs with Re > 0), in Newton form at their Leja order (Sec. 5.2); [lo, hi]
// serves the positivity check and the image interval, which also covers the
// nodes.  Host only.
int set_poly_nodes(pp_ctx *c, int kind, const std::vector<std::complex<double>> &nodes, double lo, double hi,
                   const std::vector<std::complex<double>> *check_pts = nullptr) {
  const int d = (int)nodes.size();
  if (d < 1 || d > kMaxDegree + 1) return pp_set_error(PP_ERR_INVALID_ARG, "need 1 .. 129 nodes");
  std::vector<char> used(d, 0);
  for (int i = 0; i < d; ++i) {
    const std::complex<double> z = nodes[i];
    if (!std::isfinite(z.real()) || !std::isfinite(z.imag())) return pp_set_error(PP_ERR_INVALID_ARG, "non-finite node");
    if (!(z.real() > 0.0))
      return pp_set_error(PP_ERR_NONPRIMARY, "a node with Re <= 0 (A q(A)^2 would need a non-principal root)");
    if (z.imag() != 0.0 && c->hermitian) return pp_set_error(PP_ERR_INVALID_ARG, "complex node for a Hermitian operator");
    for (int j = 0; j < i; ++j)
      if (nodes[j] == z) return pp_set_error(PP_ERR_NONPRIMARY, "coincident nodes");
    if (z.imag() > 0.0) {  // its conjugate must be in the set
      int m = -1;
      for (int j = 0; j < d && m < 0; ++j)
        if (!used[j] && nodes[j] == std::conj(z)) m = j;
      if (m < 0) return pp_set_error(PP_ERR_INVALID_ARG, "complex node without its conjugate");
      used[m] = 1;
    }
  }
  for (int i = 0; i < d; ++i)
    if (nodes[i].imag() < 0.0 && !used[i]) return pp_set_error(PP_ERR_INVALID_ARG, "complex node without its conjugate");
  if (!check_pts && (!(lo > 0.0) || !(hi > lo) || !std::isfinite(hi)))
    return pp_set_error(PP_ERR_INVALID_ARG, "need 0 < a < b");
  NewtonForm F;
  if (!newton_form(nodes, &F)) return pp_set_error(PP_ERR_NONPRIMARY, "non-finite Newton coefficient");
  double qmin, img_lo, img_hi;
  newton_scan(F, check_pts ? 0.0 : lo, check_pts ? 0.0 : hi, check_pts, &qmin, &img_lo, &img_hi);
  if (!(qmin > 0.0)) return pp_set_error(PP_ERR_NONPRIMARY, "Re q is not positive on [a,b] or at a node");
  c->poly_kind = kind;
  c->nf = F;
  c->coef.resize(d);
  double p = 1.0;
  for (int i = 0; i < d; ++i) {
    c->coef[i] = F.b[i] / p;
    p *= F.cap;
  }
  c->degree = d - 1;
  c->a = lo;
  c->b = hi;
  c->img_lo = img_lo;
  c->img_hi = img_hi;
  c->image_on_points = check_pts != nullptr;
  finish_poly(c, check_pts ? 1e6 : 1e3);
  return PP_OK;
}

// Complex operators: q = the interpolant of z^{-1/2} at complex nodes with
// Re > 0 and no conjugate symmetry (Sec. 5.2 for a complex non-Hermitian A),
// in Newton form at their Leja order.  Positivity (Re q > 0) is checked at
// the nodes, the check points and, if hi > lo > 0, on [lo, hi].
int set_poly_nodes_cx(pp_ctx *c, int kind, const std::vector<std::complex<double>> &nodes, double lo, double hi,
                      const std::vector<std::complex<double>> *check_pts) {
  const int d = (int)nodes.size();
  if (d < 1 || d > kMaxDegree + 1) return pp_set_error(PP_ERR_INVALID_ARG, "need 1 .. 129 nodes");
  for (int i = 0; i < d; ++i) {
    const std::complex<double> z = nodes[i];
    if (!std::isfinite(z.real()) || !std::isfinite(z.imag())) return pp_set_error(PP_ERR_INVALID_ARG, "non-finite node");
    if (!(z.real() > 0.0))
      return pp_set_error(PP_ERR_NONPRIMARY, "a node with Re <= 0 (A q(A)^2 would need a non-principal root)");
    for (int j = 0; j < i; ++j)
      if (nodes[j] == z) return pp_set_error(PP_ERR_NONPRIMARY, "coincident nodes");
  }
  NewtonForm F;
  if (!newton_form_cx(nodes, &F)) return pp_set_error(PP_ERR_NONPRIMARY, "non-finite Newton coefficient");
  std::vector<std::complex<double>> pts = check_pts ? *check_pts : nodes;
  double qmin, img_lo, img_hi;
  newton_scan(F, lo, hi, &pts, &qmin, &img_lo, &img_hi);
  if (!(qmin > 0.0)) return pp_set_error(PP_ERR_NONPRIMARY, "Re q is not positive at a node or check point");
  c->poly_kind = kind;
  c->nf = F;
  c->coef.resize(d);  // real parts of b_i / cap^i (pp_get_poly)
  double p = 1.0;
  for (int i = 0; i < d; ++i) {
    c->coef[i] = F.b[i] / p;
    p *= F.cap;
  }
  c->degree = d - 1;
  c->a = lo;
  c->b = hi;
  c->img_lo = img_lo;
  c->img_hi = img_hi;
  c->image_on_points = true;
  finish_poly(c, 1e6);
  return PP_OK;
}

// Default check interval of node-based kinds: the closed form of the
// stencils, else the extreme real parts of the reference values lowered by
// 5 % / raised by 1 % (as for the interval estimate).
void node_interval(const pp_ctx *c, const double *ab, const std::vector<std::complex<double>> &ref, double *lo,
                   double *hi) {
  if (ab) {
    *lo = ab[0];
    *hi = ab[1];
    return;
  }
  if (closed_form_interval(c, lo, hi)) return;
  double mn = INFINITY, mx = -INFINITY;
  for (const auto &z : ref) {
    mn = std::fmin(mn, z.real());
    mx = std::fmax(mx, z.real());
  }
  *lo = 0.95 * mn;
  *hi = 1.01 * mx;
  if (!(*hi > *lo)) *hi = *lo * 1.01 + 1e-300;
}

// pp_build_poly for PP_RITZ_LEJA / PP_HARMONIC_RITZ (Sec. 5.2): degree + 1
// Arnoldi steps on A; the nodes are the eigenvalues of H_d, or of H_d +
// h_{d+1,d}^2 H_d^{-T} e_d e_d^T (harmonic).  Hermitian A: H_d read as the
// Lanczos matrix T (diagonal and sub-diagonal), eigenvalues by bisection,
// harmonic ones from the symmetric pencil (T^2 + beta^2 e_d e_d^T, T).
// Non-Hermitian A: the Hessenberg H_d, Francis QR.
int build_ritz(pp_ctx *c, int degree, int kind, const double *ab) {
  RC(read_nnz(c));
  const int d = (int)std::min<int64_t>((int64_t)degree + 1, c->n);
  std::vector<double> H;
  int ldh = 0, m = 0;
  const int rc = c->opts.precision == PP_PREC_F64 ? ritz_arnoldi<double>(c, d, &H, &ldh, &m)
                                                  : ritz_arnoldi<dw>(c, d, &H, &ldh, &m);
  if (rc != PP_OK) return rc;
  if (c->cplx) {  // complex H_d (column j at 2 j ldh): complex QR, no conjugate pairs
    const double beta = m < d ? 0.0 : H[2 * ((size_t)(m - 1) * ldh + m)];
    std::vector<std::complex<double>> Hd((size_t)m * m, 0.0), ritz, nodes;
    for (int j = 0; j < m; ++j)
      for (int i = 0; i <= std::min(j + 1, m - 1); ++i)
        Hd[(size_t)i * m + j] = {H[2 * ((size_t)j * ldh + i)], H[2 * ((size_t)j * ldh + i) + 1]};
    if (!zhess_eigvals(Hd, m, &ritz)) return pp_set_error(PP_ERR_NONPRIMARY, "Hessenberg QR did not converge");
    if (kind == PP_HARMONIC_RITZ) {
      std::vector<std::complex<double>> f;
      if (!zsolve_adjoint_last(Hd, m, &f)) return pp_set_error(PP_ERR_NONPRIMARY, "H_d is singular");
      for (int i = 0; i < m; ++i) Hd[(size_t)i * m + m - 1] += beta * beta * f[i];
      if (!zhess_eigvals(Hd, m, &nodes)) return pp_set_error(PP_ERR_NONPRIMARY, "Hessenberg QR did not converge");
    } else {
      nodes = ritz;
    }
    double lo = 0.0, hi = 0.0;
    if (ab) {
      lo = ab[0];
      hi = ab[1];
    }
    return set_poly_nodes_cx(c, kind, nodes, lo, hi, &ritz);
  }
  const double beta = m < d ? 0.0 : H[(size_t)(m - 1) * ldh + m];  // h_{m+1,m}
  std::vector<std::complex<double>> ritz, nodes;
  if (c->hermitian) {
    std::vector<double> al(m), be(m > 1 ? m - 1 : 0);
    for (int j = 0; j < m; ++j) {
      al[j] = H[(size_t)j * ldh + j];
      if (j + 1 < m) be[j] = H[(size_t)j * ldh + j + 1];
    }
    for (int k = 0; k < m; ++k) ritz.emplace_back(tridiag_eig(al, be, k), 0.0);
    if (kind == PP_HARMONIC_RITZ) {
      std::vector<double> hv;
      if (!harmonic_ritz(al, be, beta, &hv))
        return pp_set_error(PP_ERR_NONPRIMARY, "Lanczos matrix not positive definite: A is not HPD");
      for (double v : hv) nodes.emplace_back(v, 0.0);
    } else {
      nodes = ritz;
    }
  } else {
    std::vector<double> Hd((size_t)m * m, 0.0), wr, wi;
    for (int j = 0; j < m; ++j)
      for (int i = 0; i <= std::min(j + 1, m - 1); ++i) Hd[(size_t)i * m + j] = H[(size_t)j * ldh + i];
    if (!hess_eigvals(Hd, m, &wr, &wi)) return pp_set_error(PP_ERR_NONPRIMARY, "Hessenberg QR did not converge");
    for (int k = 0; k < m; ++k) ritz.emplace_back(wr[k], wi[k]);
    if (kind == PP_HARMONIC_RITZ) {
      std::vector<double> f;
      if (!solve_transposed_last(Hd, m, &f)) return pp_set_error(PP_ERR_NONPRIMARY, "H_d is singular");
      for (int i = 0; i < m; ++i) Hd[(size_t)i * m + m - 1] += beta * beta * f[i];
      if (!hess_eigvals(Hd, m, &wr, &wi)) return pp_set_error(PP_ERR_NONPRIMARY, "Hessenberg QR did not converge");
      for (int k = 0; k < m; ++k) nodes.emplace_back(wr[k], wi[k]);
    } else {
      nodes = ritz;
    }
  }
  double lo, hi;
  if (!c->hermitian && !ab && !closed_form_interval(c, &lo, &hi)) {
    // no spectral interval of a non-normal operator: q is checked at the
    // Ritz values and the nodes, the indication of Sec. 5.2 (between them an
    // interpolant may dip anywhere where A has no eigenvalues), and the
    // quadrature gets a margin of 1e6 around the image of those points
    lo = INFINITY;
    hi = -INFINITY;
    for (const auto &z : ritz) {
      lo = std::fmin(lo, z.real());
      hi = std::fmax(hi, z.real());
    }
    return set_poly_nodes(c, kind, nodes, lo, hi, &ritz);
  }
  node_interval(c, ab, ritz, &lo, &hi);
  return set_poly_nodes(c, kind, nodes, lo, hi);
}

// The spectral interval [a, b] of the Chebyshev and least-squares kinds: the
// given one, the closed form of the stencils, or for other Hermitian handles
// the extreme Ritz values of kIntervalSteps Lanczos steps (a lowered by 5 %,
// b raised by 1 %).  *have = false for a non-Hermitian CSR handle without one.
int spectral_interval(pp_ctx *c, const double *ab, double *a, double *b, bool *have) {
  *have = true;
  if (ab) {
    *a = ab[0];
    *b = ab[1];
    return PP_OK;
  }
  if (closed_form_interval(c, a, b)) return PP_OK;
  if (c->hermitian) {
    RC(read_nnz(c));
    const int steps = (int)std::min<int64_t>(kIntervalSteps, c->n);
    double lo = 0.0, hi = 0.0;
    const int rc = c->opts.precision == PP_PREC_F64 ? lanczos_extremes<double>(c, steps, &lo, &hi)
                                                    : lanczos_extremes<dw>(c, steps, &lo, &hi);
    if (rc != PP_OK) return rc;
    *a = 0.95 * lo;
    *b = 1.01 * hi;
    return PP_OK;
  }
  *have = false;
  return PP_OK;
}

// q = the least-squares approximation of z^{-1/2} of degree `degree` on the
// contour points (Sec. 5.3): orthonormal basis by Arnoldi on diag(z),
// alpha = P^* z^{-1/2}; Re q > 0 required at every point; the device then
// evaluates q in Newton form at degree + 1 Leja points of the contour (the
// same polynomial: it interpolates its own values there), checked to
// reproduce q on all points.
int set_poly_lsq(pp_ctx *c, int degree, const std::vector<std::complex<double>> &pts) {
  using cplx = std::complex<double>;
  const int d = degree + 1;
  const size_t N = pts.size();
  if (degree < 0 || degree > kMaxDegree) return pp_set_error(PP_ERR_INVALID_ARG, "degree out of [0, 128]");
  if (N < (size_t)d) return pp_set_error(PP_ERR_INVALID_ARG, "need at least degree + 1 contour points");
  std::vector<std::pair<double, double>> up, lo;
  double rmin = INFINITY, rmax = -INFINITY;
  for (const cplx &z : pts) {
    if (!std::isfinite(z.real()) || !std::isfinite(z.imag())) return pp_set_error(PP_ERR_INVALID_ARG, "non-finite point");
    if (z.imag() == 0.0 && !(z.real() > 0.0))
      return pp_set_error(PP_ERR_INVALID_ARG, "a contour point on (-inf, 0] (z^{-1/2} has its branch cut there)");
    if (z.imag() != 0.0 && c->hermitian) return pp_set_error(PP_ERR_INVALID_ARG, "complex contour point for a Hermitian operator");
    if (z.imag() > 0.0) up.emplace_back(z.real(), z.imag());
    if (z.imag() < 0.0) lo.emplace_back(z.real(), -z.imag());
    rmin = std::fmin(rmin, z.real());
    rmax = std::fmax(rmax, z.real());
  }
  std::sort(up.begin(), up.end());
  std::sort(lo.begin(), lo.end());
  if (up != lo && !c->cplx)
    return pp_set_error(PP_ERR_UNSUPPORTED,
                        "contour not symmetric about the real axis: q would be complex (no complex vectors for real A)");
  std::vector<cplx> H, alpha;
  if (!lsq_poly(pts, d, &H, &alpha)) return pp_set_error(PP_ERR_INVALID_ARG, "fewer distinct contour points than degree + 1");
  double qmin = INFINITY, img_lo = INFINITY, img_hi = -INFINITY, qmax = 0.0;
  std::vector<cplx> qv(N);
  for (size_t i = 0; i < N; ++i) {
    qv[i] = lsq_eval(H, alpha, N, pts[i]);
    const double p = std::abs(pts[i] * qv[i] * qv[i]);
    qmin = std::fmin(qmin, qv[i].real());
    qmax = std::fmax(qmax, std::abs(qv[i]));
    img_lo = std::fmin(img_lo, p);
    img_hi = std::fmax(img_hi, p);
  }
  if (!(qmin > 0.0)) return pp_set_error(PP_ERR_NONPRIMARY, "Re q is not positive on the contour (Sec. 5.3)");
  std::vector<cplx> nodes;
  if (!(c->cplx ? leja_select_cx(pts, d, &nodes) : leja_select(pts, d, &nodes)))
    return pp_set_error(PP_ERR_INVALID_ARG, "cannot pick interpolation points");
  NewtonForm F;
  const auto qf = [&](cplx z) { return lsq_eval(H, alpha, N, z); };
  if (!(c->cplx ? newton_form_cx_fn(nodes, qf, &F) : newton_form_fn(nodes, qf, &F)))
    return pp_set_error(PP_ERR_NONPRIMARY, "non-finite Newton coefficient");
  double dev = 0.0;
  for (size_t i = 0; i < N; ++i) dev = std::fmax(dev, std::abs(newton_form_eval(F, pts[i]) - qv[i]));
  if (!(dev <= 1e-8 * qmax)) return pp_set_error(PP_ERR_NONPRIMARY, "Newton form does not reproduce q on the contour");
  c->poly_kind = PP_LSQ_CONTOUR;
  c->nf = F;
  c->coef.resize(d);
  double p = 1.0;
  for (int i = 0; i < d; ++i) {
    c->coef[i] = F.b[i] / p;
    p *= F.cap;
  }
  c->degree = degree;
  c->a = rmin;
  c->b = rmax;
  c->img_lo = img_lo;
  c->img_hi = img_hi;
  // a complex operator's contour only indicates its spectrum (as its Ritz
  // values do for PP_RITZ_LEJA): the same wide quadrature and, under
  // PP_PREC_MIXED, kappa_pre from H_m
  c->image_on_points = c->cplx;
  finish_poly(c, c->cplx ? 1e6 : 1e3);
  return PP_OK;
}

// pp_build_poly for PP_LSQ_CONTOUR: the segment [a, b] of a real spectral
// interval, else (non-Hermitian CSR) the contour around the Ritz values of
// max(60, degree + 1) Arnoldi steps (Example 3 uses 60), kept out of
// |z| < half the smallest Ritz modulus; N = max(2000, 20 (degree + 1)) points.
int build_lsq(pp_ctx *c, int degree, const double *ab) {
  double a = 0.0, b = 0.0;
  bool have = false;
  RC(spectral_interval(c, ab, &a, &b, &have));
  const int npts = std::max(2000, 20 * (degree + 1));
  std::vector<std::complex<double>> pts;
  if (c->cplx) {  // complex operator: the closed contour around the complex Ritz values
    const int steps = (int)std::min<int64_t>(std::max(60, degree + 1), c->n / 2);
    std::vector<double> H;
    int ldh = 0, m = 0;
    const int rc = c->opts.precision == PP_PREC_F64 ? ritz_arnoldi<double>(c, steps, &H, &ldh, &m)
                                                    : ritz_arnoldi<dw>(c, steps, &H, &ldh, &m);
    if (rc != PP_OK) return rc;
    std::vector<std::complex<double>> Hd((size_t)m * m, 0.0), ritz;
    for (int j = 0; j < m; ++j)
      for (int i = 0; i <= std::min(j + 1, m - 1); ++i)
        Hd[(size_t)i * m + j] = {H[2 * ((size_t)j * ldh + i)], H[2 * ((size_t)j * ldh + i) + 1]};
    if (!zhess_eigvals(Hd, m, &ritz)) return pp_set_error(PP_ERR_NONPRIMARY, "Hessenberg QR did not converge");
    double rmin = INFINITY;
    for (const auto &z : ritz) {
      if (!(z.real() > 0.0)) return pp_set_error(PP_ERR_NONPRIMARY, "a Ritz value with Re <= 0");
      rmin = std::fmin(rmin, std::abs(z));
    }
    pts = lsq_contour_cx(ritz, 0.5 * rmin, npts);
  } else if (have) {
    if (!(a > 0.0) || !(b > a) || !std::isfinite(b)) return pp_set_error(PP_ERR_INVALID_ARG, "need 0 < a < b");
    for (int i = 0; i < npts; ++i) pts.emplace_back(a + (b - a) * (double)i / (npts - 1), 0.0);
  } else {
    RC(read_nnz(c));
    const int steps = (int)std::min<int64_t>(std::max(60, degree + 1), c->n);
    std::vector<double> H;
    int ldh = 0, m = 0;
    const int rc = c->opts.precision == PP_PREC_F64 ? ritz_arnoldi<double>(c, steps, &H, &ldh, &m)
                                                    : ritz_arnoldi<dw>(c, steps, &H, &ldh, &m);
    if (rc != PP_OK) return rc;
    std::vector<double> Hd((size_t)m * m, 0.0), wr, wi;
    for (int j = 0; j < m; ++j)
      for (int i = 0; i <= std::min(j + 1, m - 1); ++i) Hd[(size_t)i * m + j] = H[(size_t)j * ldh + i];
    if (!hess_eigvals(Hd, m, &wr, &wi)) return pp_set_error(PP_ERR_NONPRIMARY, "Hessenberg QR did not converge");
    // Ritz values within 1e-4 of the largest modulus of zero approximate the
    // null space of a singular A (60 steps bring a graph Laplacian's zero
    // eigenvalue only to about -1e-6 of it; its square root is taken through
    // A^{-1/2}(A b), Sec. 4, whose right-hand side has no component there):
    // left out
    double amax = 0.0;
    for (int k = 0; k < m; ++k) amax = std::fmax(amax, std::abs(std::complex<double>(wr[k], wi[k])));
    std::vector<std::complex<double>> ritz;
    double rmin = INFINITY;
    for (int k = 0; k < m; ++k) {
      const std::complex<double> z(wr[k], wi[k]);
      if (std::abs(z) <= 1e-4 * amax) continue;
      if (!(z.real() > 0.0)) return pp_set_error(PP_ERR_NONPRIMARY, "a Ritz value with Re <= 0");
      ritz.push_back(z);
      rmin = std::fmin(rmin, std::abs(z));
    }
    if (ritz.empty()) return pp_set_error(PP_ERR_NONPRIMARY, "no nonzero Ritz value");
    pts = lsq_contour(ritz, 0.5 * rmin, npts);
  }
  return set_poly_lsq(c, degree, pts);
}

pp_ctx *new_ctx(void *stream) {
  pp_ctx *c = new pp_ctx();
  pp_default_opts(&c->opts);
  c->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&c->device) != cudaSuccess) c->device = 0;
  return c;
}

}  // namespace

extern "C" {

void pp_default_opts(pp_opts *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->side = PP_LEFT;
  o->precision = PP_PREC_F64;
  o->orth = PP_ORTH_AUTO;
  o->check_every = 0;
}

int pp_create_csr(pp_handle *h, int64_t n, const int64_t *rowptr_d, const int32_t *col_d,
                  const void *val_d, int32_t dtype, int32_t is_hermitian, void *cuda_stream) {
  if (!h) return pp_set_error(PP_ERR_INVALID_ARG, "NULL handle pointer");
  *h = nullptr;
  if (n <= 0 || !rowptr_d || !col_d || !val_d) return pp_set_error(PP_ERR_INVALID_ARG, "n <= 0 or NULL CSR array");
  if (dtype != PP_F64) return pp_set_error(PP_ERR_UNSUPPORTED, "CSR values must be PP_F64");
  if (n > INT32_MAX) return pp_set_error(PP_ERR_INVALID_ARG, "n > 2^31 - 1 (column indices are int32)");
  pp_ctx *c = new_ctx(cuda_stream);
  c->op_kind = OPK_CSR;
  c->n = n;
  c->rowptr = rowptr_d;
  c->col = col_d;
  c->val = (const double *)val_d;
  c->hermitian = is_hermitian ? 1 : 0;
  // nnz = rowptr[n] is read lazily (first DW use) to keep creation free of device calls
  c->nnz = -1;
  *h = c;
  return PP_OK;
}

int pp_create_stencil(pp_handle *h, int32_t kind, const int64_t dims[4], const double *params,
                      const void *links_d, int32_t dtype, void *cuda_stream) {
  if (!h) return pp_set_error(PP_ERR_INVALID_ARG, "NULL handle pointer");
  *h = nullptr;
  if (!dims) return pp_set_error(PP_ERR_INVALID_ARG, "NULL dims");
  if (kind == PP_WILSON4D_DHD || kind == PP_WILSON4D_Q2) {
    if (dtype != PP_C128) return pp_set_error(PP_ERR_UNSUPPORTED, "Wilson vectors must be PP_C128");
    if (!links_d) return pp_set_error(PP_ERR_INVALID_ARG, "Wilson operator needs links_d");
    if (!params || !std::isfinite(params[0])) return pp_set_error(PP_ERR_INVALID_ARG, "params[0] = m0 must be finite");
    if (kind == PP_WILSON4D_Q2 && !(std::isfinite(params[1]) && std::fabs(params[1]) <= 20.0))
      return pp_set_error(PP_ERR_INVALID_ARG, "params[1] = mu must be finite, |mu| <= 20");
    int64_t V = 1;
    for (int i = 0; i < 4; ++i) {
      if (dims[i] < 1 || dims[i] > (1 << 16)) return pp_set_error(PP_ERR_INVALID_ARG, "bad 4D dims");
      V *= dims[i];
    }
    if (V > ((int64_t)1 << 28)) return pp_set_error(PP_ERR_INVALID_ARG, "lattice with more than 2^28 sites");
    pp_ctx *c = new_ctx(cuda_stream);
    c->op_kind = OPK_WILSON;
    for (int i = 0; i < 4; ++i) c->dims[i] = dims[i];
    c->links = links_d;
    c->mass = params[0];
    c->hermitian = 1;
    if (kind == PP_WILSON4D_Q2) {  // Q^2 is Hermitian only at mu = 0 (Q = Gamma_5 D(m, 0) is)
      c->mu_c = params[1];
      c->hermitian = params[1] == 0.0 ? 1 : 0;
      c->cplx = params[1] != 0.0;
    }
    c->stencil = kind;
    c->n = 24 * V;  // real view of 12 complex components per site
    *h = c;
    return PP_OK;
  }
  if (dtype != PP_F64) return pp_set_error(PP_ERR_UNSUPPORTED, "stencil vectors must be PP_F64");
  if (links_d) return pp_set_error(PP_ERR_INVALID_ARG, "links_d must be NULL for this stencil kind");
  pp_ctx *c = nullptr;
  if (kind == PP_LAPLACE2D5) {
    if (dims[0] < 1 || dims[1] < 1 || dims[0] > (1 << 24) || dims[1] > (1 << 24))
      return pp_set_error(PP_ERR_INVALID_ARG, "bad 2D dims");
    c = new_ctx(cuda_stream);
    c->op_kind = OPK_ST2D;
    c->dims[0] = dims[0];
    c->dims[1] = dims[1];
    c->dims[2] = 1;
    c->st_d = 4.0;
    c->st_cm = -1.0;
    c->st_cp = -1.0;
    c->hermitian = 1;
  } else if (kind == PP_LAPLACE3D7 || kind == PP_CONVDIFF3D7_UPWIND) {
    for (int i = 0; i < 3; ++i)
      if (dims[i] < 1 || dims[i] > (1 << 20)) return pp_set_error(PP_ERR_INVALID_ARG, "bad 3D dims");
    double ch = 0.0;
    if (kind == PP_CONVDIFF3D7_UPWIND) {
      if (!params || !(params[0] > 0.0) || !std::isfinite(params[0]))
        return pp_set_error(PP_ERR_INVALID_ARG, "convection-diffusion needs params[0] = c*h > 0");
      ch = params[0];
    }
    c = new_ctx(cuda_stream);
    c->op_kind = OPK_ST3D;
    for (int i = 0; i < 3; ++i) c->dims[i] = dims[i];
    c->ch = ch;
    c->st_d = 6.0 + 3.0 * ch;
    c->st_cm = -(1.0 + ch);
    c->st_cp = -1.0;
    c->hermitian = (kind == PP_LAPLACE3D7) ? 1 : 0;
  } else {
    return pp_set_error(PP_ERR_INVALID_ARG, "unknown stencil kind");
  }
  c->stencil = kind;
  c->n = c->dims[0] * c->dims[1] * c->dims[2];
  if (c->n > ((int64_t)1 << 34)) {
    delete c;
    return pp_set_error(PP_ERR_INVALID_ARG, "grid with more than 2^34 points");
  }
  *h = c;
  return PP_OK;
}

int pp_set_opts(pp_handle c, const pp_opts *o) {
  if (!c || !o) return pp_set_error(PP_ERR_INVALID_ARG, "NULL argument");
  if (o->side != PP_LEFT && o->side != PP_RIGHT) return pp_set_error(PP_ERR_INVALID_ARG, "bad side");
  if (o->precision != PP_PREC_F64 && o->precision != PP_PREC_DW && o->precision != PP_PREC_MIXED)
    return pp_set_error(PP_ERR_INVALID_ARG, "bad precision");
  if (o->orth < PP_ORTH_AUTO || o->orth > PP_ORTH_DCGS2) return pp_set_error(PP_ERR_INVALID_ARG, "bad orth");
  if (o->check_every < 0) return pp_set_error(PP_ERR_INVALID_ARG, "check_every < 0");
  if (o->profile != 0 && o->profile != 1) return pp_set_error(PP_ERR_INVALID_ARG, "profile must be 0 or 1");
  if (o->two_pass != 0 && o->two_pass != 1) return pp_set_error(PP_ERR_INVALID_ARG, "two_pass must be 0 or 1");
  if (o->clenshaw != 0 && o->clenshaw != 1) return pp_set_error(PP_ERR_INVALID_ARG, "clenshaw must be 0 or 1");
  if (o->halo != 0 && o->halo != 1) return pp_set_error(PP_ERR_INVALID_ARG, "halo must be 0 or 1");
  c->opts = *o;
  return PP_OK;
}

int pp_build_poly(pp_handle c, int32_t degree, int32_t kind, const double *ab) {
  if (!c) return pp_set_error(PP_ERR_INVALID_ARG, "NULL handle");
  if (kind != PP_CHEBYSHEV && kind != PP_RITZ_LEJA && kind != PP_HARMONIC_RITZ && kind != PP_LSQ_CONTOUR) {
    if (kind == PP_NODES) return pp_set_error(PP_ERR_INVALID_ARG, "PP_NODES is set by pp_set_poly_nodes");
    return pp_set_error(PP_ERR_INVALID_ARG, "unknown polynomial kind");
  }
  if (degree < 0 || degree > kMaxDegree) return pp_set_error(PP_ERR_INVALID_ARG, "degree out of [0, 128]");
  if (ab && (!(ab[0] > 0.0) || !(ab[1] > ab[0]) || !std::isfinite(ab[1])))
    return pp_set_error(PP_ERR_INVALID_ARG, "need 0 < a < b");
  if (kind == PP_LSQ_CONTOUR) return build_lsq(c, degree, ab);
  if (kind != PP_CHEBYSHEV) return build_ritz(c, degree, kind, ab);
  if (c->cplx && !ab) return pp_set_error(PP_ERR_INVALID_ARG, "complex operators need interval_ab for PP_CHEBYSHEV");
  double a, b;
  bool have = false;
  RC(spectral_interval(c, ab, &a, &b, &have));
  if (!have) return pp_set_error(PP_ERR_INVALID_ARG, "non-Hermitian CSR handles need interval_ab");
  if (!(a > 0.0) || !(b > a) || !std::isfinite(b)) return pp_set_error(PP_ERR_INVALID_ARG, "need 0 < a < b");
  std::vector<double> cf = cheb_interp_coeffs(a, b, degree);
  double qmin, lo, hi;
  cheb_scan(cf, a, b, &qmin, &lo, &hi);
  if (!(qmin > 0.0)) return pp_set_error(PP_ERR_NONPRIMARY, "q is not positive on [a,b]");
  {  // the same q in Newton form at its d = degree + 1 first-kind nodes
    const int d = degree + 1;
    std::vector<std::complex<double>> xc(d);
    for (int k = 0; k < d; ++k) xc[k] = 0.5 * (a + b) + 0.5 * (b - a) * std::cos(M_PI * (k + 0.5) / d);
    if (!newton_form(xc, &c->nf)) return pp_set_error(PP_ERR_NONPRIMARY, "non-finite Newton coefficient");
  }
  c->poly_kind = PP_CHEBYSHEV;
  c->coef = cf;
  c->degree = degree;
  // a complex spectrum is not bounded by the image of [a,b]: no FP32 switch
  c->image_on_points = c->cplx;
  c->a = a;
  c->b = b;
  c->img_lo = lo;
  c->img_hi = hi;
  finish_poly(c);
  return PP_OK;
}

int pp_get_poly(pp_handle c, double *coeffs, int32_t cap, int32_t *ncoeffs, double *ab, double *image) {
  if (!c) return pp_set_error(PP_ERR_INVALID_ARG, "NULL handle");
  if (!c->have_poly) return pp_set_error(PP_ERR_STATE, "pp_build_poly has not been called");
  if (ncoeffs) *ncoeffs = (int32_t)c->coef.size();
  if (coeffs)
    for (int i = 0; i < (int)c->coef.size() && i < cap; ++i) coeffs[i] = c->coef[i];
  if (ab) {
    ab[0] = c->a;
    ab[1] = c->b;
  }
  if (image) {
    image[0] = c->img_lo;
    image[1] = c->img_hi;
  }
  return PP_OK;
}

int pp_get_poly_nodes(pp_handle c, int32_t *kind, double *nodes_re, double *nodes_im, int32_t cap,
                      int32_t *nnodes, double *scale) {
  if (!c) return pp_set_error(PP_ERR_INVALID_ARG, "NULL handle");
  if (!c->have_poly) return pp_set_error(PP_ERR_STATE, "pp_build_poly has not been called");
  if (kind) *kind = c->poly_kind;
  const int d = (int)c->nf.re.size();
  if (nnodes) *nnodes = d;
  for (int i = 0; i < d && i < cap; ++i) {
    if (nodes_re) nodes_re[i] = c->nf.re[i];
    if (nodes_im) nodes_im[i] = c->nf.im[i];
  }
  if (scale) *scale = c->nf.cap;
  return PP_OK;
}

int pp_set_poly_lsq(pp_handle c, int32_t degree, const double *pts_re, const double *pts_im, int32_t npts) {
  if (!c) return pp_set_error(PP_ERR_INVALID_ARG, "NULL handle");
  if (!pts_re || npts < 1) return pp_set_error(PP_ERR_INVALID_ARG, "need contour points");
  std::vector<std::complex<double>> z(npts);
  for (int i = 0; i < npts; ++i) z[i] = {pts_re[i], pts_im ? pts_im[i] : 0.0};
  return set_poly_lsq(c, degree, z);
}

int pp_set_poly_nodes(pp_handle c, const double *nodes_re, const double *nodes_im, int32_t count,
                      const double *ab) {
  if (!c) return pp_set_error(PP_ERR_INVALID_ARG, "NULL handle");
  if (!nodes_re || count < 1 || count > kMaxDegree + 1) return pp_set_error(PP_ERR_INVALID_ARG, "need 1 .. 129 nodes");
  if (ab && (!(ab[0] > 0.0) || !(ab[1] > ab[0]) || !std::isfinite(ab[1])))
    return pp_set_error(PP_ERR_INVALID_ARG, "need 0 < a < b");
  std::vector<std::complex<double>> z(count);
  for (int i = 0; i < count; ++i) z[i] = {nodes_re[i], nodes_im ? nodes_im[i] : 0.0};
  if (c->cplx) return set_poly_nodes_cx(c, PP_NODES, z, ab ? ab[0] : 0.0, ab ? ab[1] : 0.0, nullptr);
  double lo, hi;
  node_interval(c, ab, z, &lo, &hi);
  return set_poly_nodes(c, PP_NODES, z, lo, hi);
}

int pp_get_quadrature(pp_handle c, double *sig, double *wt, int32_t cap, int32_t *K) {
  if (!c) return pp_set_error(PP_ERR_INVALID_ARG, "NULL handle");
  if (!c->have_poly) return pp_set_error(PP_ERR_STATE, "pp_build_poly has not been called");
  if (K) *K = (int32_t)c->qsig.size();
  for (int i = 0; i < (int)c->qsig.size() && i < cap; ++i) {
    if (sig) sig[i] = c->qsig[i];
    if (wt) wt[i] = c->qwt[i];
  }
  return PP_OK;
}

int pp_apply(pp_handle c, int32_t f, const void *b_d, int64_t nrhs, int32_t m_max, double tol,
             void *x_d, pp_stats *stats) {
  RC(check_ready(c));
  if (f != PP_SQRT && f != PP_INVSQRT && f != PP_SIGN)
    return pp_set_error(PP_ERR_INVALID_ARG, "f must be PP_SQRT, PP_INVSQRT or PP_SIGN");
  if (f == PP_SIGN && c->stencil != PP_WILSON4D_Q2)
    return pp_set_error(PP_ERR_UNSUPPORTED, "PP_SIGN needs a PP_WILSON4D_Q2 handle");
  if (!b_d || !x_d) return pp_set_error(PP_ERR_INVALID_ARG, "NULL vector");
  if (b_d == x_d) return pp_set_error(PP_ERR_INVALID_ARG, "x_d aliases b_d");
  if (nrhs < 1) return pp_set_error(PP_ERR_INVALID_ARG, "nrhs < 1");
  if (c->cplx) {
    if (c->opts.orth == PP_ORTH_LANCZOS || c->opts.two_pass)
      return pp_set_error(PP_ERR_INVALID_ARG, "a non-Hermitian complex operator needs Arnoldi (CGS2)");
  }
  if (c->opts.orth == PP_ORTH_DCGS2 && (c->cplx || c->opts.side == PP_RIGHT))
    return pp_set_error(PP_ERR_UNSUPPORTED,
                        "delayed reorthogonalization is implemented for left preconditioning of real operators");
  if (nrhs > 1 && c->op_kind == OPK_WILSON) {
    // Wilson handles: the columns one after another on the handle
    // (the later ones replay the captured segment graphs)
    const size_t esz = c->op_kind == OPK_WILSON ? 16 : 8;  // complex128 / float64 entries per row
    const int64_t rows = c->op_kind == OPK_WILSON ? c->n / 2 : c->n;
    pp_stats tot;
    memset(&tot, 0, sizeof tot);
    int worst = PP_OK;
    for (int64_t r = 0; r < nrhs; ++r) {
      pp_stats st;
      const int rc = pp_apply(c, f, (const char *)b_d + (size_t)r * rows * esz, 1, m_max, tol,
                              (char *)x_d + (size_t)r * rows * esz, &st);
      if (rc != PP_OK && rc != PP_ERR_NOT_CONVERGED) return rc;
      if (rc != PP_OK) worst = rc;
      tot.iters = std::max(tot.iters, st.iters);
      tot.checks += st.checks;
      tot.breakdown |= st.breakdown;
      tot.mvms += st.mvms;
      tot.inner_products += st.inner_products;
      tot.est_err = std::max(tot.est_err, st.est_err);
      tot.beta0 = std::max(tot.beta0, st.beta0);
      tot.ms_total += st.ms_total;
      tot.launches += st.launches;
      tot.chain_launches += st.chain_launches;
      tot.chain_bytes += st.chain_bytes;
      tot.chain_ms += st.chain_ms;
      tot.switch_iter = r == 0 ? st.switch_iter : std::max(tot.switch_iter, st.switch_iter);
    }
    tot.status = worst;
    if (stats) *stats = tot;
    if (worst != PP_OK) pp_set_error(worst, "m_max reached before the stopping estimate fell below tol");
    return worst;
  }
  if (f == PP_SIGN) {  // sign(Q) b = Q (Q^2)^{-1/2} b (Sec. 6, Example 2)
    // (Q^2)^{-1/2} b into x_d, then x_d -> scratch, Q scratch -> x_d (FP64)
    const int rc = pp_apply(c, PP_INVSQRT, b_d, 1, m_max, tol, x_d, stats);
    if (rc != PP_OK && rc != PP_ERR_NOT_CONVERGED) return rc;
    double *tmp = (double *)c->ws.tmp;  // kTmpVecs scratch vectors of 8-byte entries, free after the solve
    PP_CUDA_TRY(cudaMemcpyAsync(tmp, x_d, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->stream));
    const OpDesc op = make_op(c, AR_F64);
    RC(wilson_q_apply<double>(op, tmp, (double *)x_d, c->stream));
    PP_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (rc != PP_OK) pp_set_error(rc, "m_max reached before the stopping estimate fell below tol");
    return rc;
  }
  if (nrhs > 1) {
    pp_handle hs[1] = {c};
    const int32_t fs[1] = {f};
    const void *bs[1] = {b_d};
    void *xs[1] = {x_d};
    const int64_t rs[1] = {nrhs};
    return pp_apply_batch(hs, 1, fs, bs, rs, xs, m_max, tol, c->stream, stats);
  }
  if (m_max < 1 || m_max > kMaxM) return pp_set_error(PP_ERR_INVALID_ARG, "m_max out of [1, 4096]");
  if (!(tol >= 0.0)) return pp_set_error(PP_ERR_INVALID_ARG, "tol < 0");
  if (c->op_kind == OPK_CSR && c->nnz < 0) {
    int64_t nnz = 0;
    PP_CUDA_TRY(cudaMemcpy(&nnz, c->rowptr + c->n, sizeof(int64_t), cudaMemcpyDeviceToHost));
    c->nnz = nnz;
  }
  if (c->opts.two_pass) {
    const bool lanczos = c->opts.orth == PP_ORTH_LANCZOS || (c->opts.orth == PP_ORTH_AUTO && c->hermitian);
    if (!lanczos) return pp_set_error(PP_ERR_INVALID_ARG, "two-pass needs the Lanczos recurrence (Hermitian A)");
    if (c->opts.precision == PP_PREC_MIXED)
      return solve_two_pass<dw, float>(c, f, (const double *)b_d, m_max, tol, (double *)x_d, stats);
    if (c->opts.precision == PP_PREC_DW)
      return solve_two_pass<dw, dw>(c, f, (const double *)b_d, m_max, tol, (double *)x_d, stats);
    return solve_two_pass<double, double>(c, f, (const double *)b_d, m_max, tol, (double *)x_d, stats);
  }
  if (c->opts.precision == PP_PREC_MIXED)
    return solve<dw, float>(c, f, (const double *)b_d, m_max, tol, (double *)x_d, stats);
  if (c->opts.precision == PP_PREC_DW) return solve<dw, dw>(c, f, (const double *)b_d, m_max, tol, (double *)x_d, stats);
  return solve<double, double>(c, f, (const double *)b_d, m_max, tol, (double *)x_d, stats);
}

int pp_apply_host(pp_handle c, int32_t f, const double *b_h, int64_t nrhs, int32_t m_max, double tol,
                  double *x_h, pp_stats *stats) {
  RC(check_ready(c));
  if (!b_h || !x_h) return pp_set_error(PP_ERR_INVALID_ARG, "NULL vector");
  if (nrhs != 1) return pp_set_error(PP_ERR_UNSUPPORTED, "pp_apply_host takes nrhs = 1");
  if (!c->ws.io) PP_CUDA_TRY(cudaMalloc(&c->ws.io, 2 * sizeof(double) * (size_t)c->n));
  double *bd = c->ws.io, *xd = c->ws.io + c->n;
  PP_CUDA_TRY(cudaMemcpyAsync(bd, b_h, sizeof(double) * c->n, cudaMemcpyHostToDevice, c->stream));
  int rc = pp_apply(c, f, bd, nrhs, m_max, tol, xd, stats);
  if (rc != PP_OK && rc != PP_ERR_NOT_CONVERGED) return rc;
  PP_CUDA_TRY(cudaMemcpyAsync(x_h, xd, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->stream));
  PP_CUDA_TRY(cudaStreamSynchronize(c->stream));
  return rc;
}

int pp_op_apply(pp_handle c, const void *x_d, void *y_d) {
  if (!c || !x_d || !y_d || x_d == y_d) return pp_set_error(PP_ERR_INVALID_ARG, "bad arguments");
  if (c->op_kind == OPK_CSR && c->nnz < 0) {
    int64_t nnz = 0;
    PP_CUDA_TRY(cudaMemcpy(&nnz, c->rowptr + c->n, sizeof(int64_t), cudaMemcpyDeviceToHost));
    c->nnz = nnz;
  }
  if (!c->have_poly) {  // the workspace layout needs a quadrature size; use a trivial one
    c->qsig.assign(1, 1.0);
    c->qwt.assign(1, 1.0);
  }
  if (c->opts.precision == PP_PREC_MIXED) return op_apply_t<float>(c, (const double *)x_d, (double *)y_d);
  if (c->opts.precision == PP_PREC_DW) return op_apply_t<dw>(c, (const double *)x_d, (double *)y_d);
  return op_apply_t<double>(c, (const double *)x_d, (double *)y_d);
}

int pp_poly_apply(pp_handle c, const void *x_d, void *y_d) {
  RC(check_ready(c));
  if (!x_d || !y_d || x_d == y_d) return pp_set_error(PP_ERR_INVALID_ARG, "bad arguments");
  if (c->op_kind == OPK_CSR && c->nnz < 0) {
    int64_t nnz = 0;
    PP_CUDA_TRY(cudaMemcpy(&nnz, c->rowptr + c->n, sizeof(int64_t), cudaMemcpyDeviceToHost));
    c->nnz = nnz;
  }
  if (c->opts.precision == PP_PREC_MIXED) return poly_apply_api_t<float>(c, (const double *)x_d, (double *)y_d);
  if (c->opts.precision == PP_PREC_DW) return poly_apply_api_t<dw>(c, (const double *)x_d, (double *)y_d);
  return poly_apply_api_t<double>(c, (const double *)x_d, (double *)y_d);
}

int pp_autotune(pp_handle c, double tol, int32_t max_degree, int32_t *degree_out) {
  if (!c) return pp_set_error(PP_ERR_INVALID_ARG, "NULL handle");
  if (!(tol > 0.0) || !(tol < 1.0)) return pp_set_error(PP_ERR_INVALID_ARG, "tol out of (0, 1)");
  if (max_degree < 0 || max_degree > kMaxDegree) return pp_set_error(PP_ERR_INVALID_ARG, "max_degree out of [0, 128]");
  // the interval: from an earlier pp_build_poly, else as pp_build_poly would take it
  if (!c->have_poly) RC(pp_build_poly(c, 0, PP_CHEBYSHEV, nullptr));
  const double a = c->a, b = c->b;
  const bool lanczos = c->opts.orth == PP_ORTH_LANCZOS || (c->opts.orth == PP_ORTH_AUTO && c->hermitian);
  // operator pass cost in vector passes: Horner step 3 / Clenshaw step 4
  // (matrix-free), plus the matrix bytes in vector units (CSR), 2 for the
  // Wilson pair of launches more
  double op_cost = c->opts.clenshaw ? 4.0 : 3.0;
  if (c->op_kind == OPK_CSR && c->nnz > 0) op_cost += (12.0 * (double)c->nnz) / (8.0 * (double)c->n);
  if (c->op_kind == OPK_WILSON) op_cost += 6.0;
  static const int cand[] = {0, 1, 2, 3, 4, 6, 8, 12, 16, 20, 24, 32, 40, 48, 64, 80, 96, 128};
  // model constants: sustained HBM bandwidth, launch-plus-gap time, cost of a check
  constexpr double kBW = 6.0e12, kLaunchS = 3.0e-6, kCheckS = 40.0e-6;
  const double esz = c->opts.precision == PP_PREC_MIXED ? 6.0 : 8.0;  // FP32 / double-word mix
  const double t_pass = esz * (double)c->n / kBW;
  int best = 0;
  double best_cost = INFINITY;
  for (int d : cand) {
    if (d > max_degree) break;
    const std::vector<double> cf = cheb_interp_coeffs(a, b, d);
    double qmin, lo, hi;
    cheb_scan(cf, a, b, &qmin, &lo, &hi);
    if (!(qmin > 0.0) || !(lo > 0.0)) continue;
    // Chebyshev bound on the image interval: error ~ 2 ((sqrt(k) - 1) / (sqrt(k) + 1))^m
    const double kap = hi / lo, sk = std::sqrt(kap);
    const double rate = std::log((sk + 1.0) / std::fmax(sk - 1.0, 1e-300));
    const double m = std::ceil(std::log(2.0 / tol) / std::fmax(rate, 1e-300));
    const double orth = lanczos ? 6.0 : 4.0 * (0.5 * m) + 8.0;
    // time: vector passes at HBM speed plus a fixed cost per launch and per
    // stopping check (small solve and host synchronisation)
    const double launches = (2.0 * d + 1.0) * (c->op_kind == OPK_WILSON ? 2.0 : 1.0) + (lanczos ? 5.0 : 9.0);
    const int kchk = std::max(1, 64 / (d + 1));
    const double cost = m * (t_pass * (op_cost * (2.0 * d + 1.0) + orth) + kLaunchS * launches) +
                        (m / kchk) * kCheckS + d * (t_pass * op_cost + kLaunchS);
    if (cost < best_cost) {
      best_cost = cost;
      best = d;
    }
  }
  const double ab[2] = {a, b};
  RC(pp_build_poly(c, best, PP_CHEBYSHEV, ab));
  if (degree_out) *degree_out = best;
  // tile shape of the stencil step: time each block x-size on the handle's buffers
  if ((c->op_kind == OPK_ST2D || c->op_kind == OPK_ST3D) && c->opts.precision != PP_PREC_F64) {
    RC(ensure_ws(c, c->opts.precision, c->ws.m_cap > 0 ? c->ws.m_cap : 1, false));
    const bool f32 = c->opts.precision == PP_PREC_MIXED;
    cudaEvent_t e0 = c->ws.ev0, e1 = c->ws.ev1;
    float best_ms = INFINITY;
    int best_bdx = 0;
    for (int bdx : {64, 128, 256, 512}) {
      c->tile_bdx = bdx;
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {  // first pass warms up
        PP_CUDA_TRY(cudaEventRecord(e0, c->stream));
        for (int it = 0; it < 5; ++it) {
          int rc;
          if (f32) {
            const OpDesc op = make_op(c, AR_F32);
            float *t = (float *)c->ws.tmp;
            rc = op_step<float>(op, t, t + c->ws.ldv, t + 2 * c->ws.ldv, t + 3 * c->ws.ldv, {1.0, 0.5, 0.25, true, true},
                                c->stream);
          } else {
            const OpDesc op = make_op(c, AR_DW);
            dw *t = (dw *)c->ws.tmp;
            rc = op_step<dw>(op, t, t + c->ws.ldv, t + 2 * c->ws.ldv, t + 3 * c->ws.ldv, {1.0, 0.5, 0.25, true, true},
                             c->stream);
          }
          if (rc) return rc;
        }
        PP_CUDA_TRY(cudaEventRecord(e1, c->stream));
        PP_CUDA_TRY(cudaEventSynchronize(e1));
        PP_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
      }
      if (ms < best_ms) {
        best_ms = ms;
        best_bdx = bdx;
      }
    }
    c->tile_bdx = best_bdx;
  }
  return PP_OK;
}

int pp_poly_apply_static(pp_handle c, const void *x_d, void *y_d) {
  RC(check_ready(c));
  if (!x_d || !y_d || x_d == y_d) return pp_set_error(PP_ERR_INVALID_ARG, "bad arguments");
  if (c->n > PP_STATIC_MAX_N)
    return pp_set_error(PP_ERR_INVALID_ARG, "n = " + std::to_string(c->n) +
                                                " exceeds PP_STATIC_MAX_N = " + std::to_string((long long)PP_STATIC_MAX_N));
  if (c->op_kind == OPK_WILSON)
    return pp_set_error(PP_ERR_UNSUPPORTED, "the Wilson operator needs a sixth scratch vector; use pp_poly_apply");
  if (c->op_kind == OPK_CSR && c->opts.precision != PP_PREC_F64)
    return pp_set_error(PP_ERR_UNSUPPORTED,
                        "CSR handles in PP_PREC_DW / PP_PREC_MIXED need a converted copy of the values; use PP_PREC_F64");
  // (no read-back of a CSR handle's nnz here: it only feeds the byte
  // statistics, and a blocking copy would synchronise the device)
  void *base = nullptr;
  RC(static_scratch_addr(c, &base));
  if (c->opts.precision == PP_PREC_MIXED) return poly_apply_static_t<float>(c, (const double *)x_d, (double *)y_d, base);
  if (c->opts.precision == PP_PREC_DW) return poly_apply_static_t<dw>(c, (const double *)x_d, (double *)y_d, base);
  return poly_apply_static_t<double>(c, (const double *)x_d, (double *)y_d, base);
}

void pp_destroy(pp_handle c) {
  if (!c) return;
  segs_destroy(c);
  for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
  ws_free(c->ws);
  delete c;
}

const char *pp_strerror(int32_t s) {
  switch (s) {
    case PP_OK: return "PP_OK";
    case PP_ERR_INVALID_ARG: return "PP_ERR_INVALID_ARG";
    case PP_ERR_NOT_CONVERGED: return "PP_ERR_NOT_CONVERGED";
    case PP_ERR_NONPRIMARY: return "PP_ERR_NONPRIMARY";
    case PP_ERR_SINGULAR: return "PP_ERR_SINGULAR";
    case PP_ERR_OOM: return "PP_ERR_OOM";
    case PP_ERR_CUDA: return "PP_ERR_CUDA";
    case PP_ERR_TIMEOUT: return "PP_ERR_TIMEOUT";
    case PP_ERR_STATE: return "PP_ERR_STATE";
    case PP_ERR_UNSUPPORTED: return "PP_ERR_UNSUPPORTED";
    default: return "PP_ERR_UNKNOWN";
  }
}

const char *pp_last_error(void) { return g_last_error.c_str(); }

int32_t pp_version(void) { return 100; }

}  // extern "C"
