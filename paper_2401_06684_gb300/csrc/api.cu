// C ABI and the Krylov driver: Algorithm 1 (left) and Algorithm 2 (right)
// polynomially preconditioned Arnoldi/Lanczos for A^{-1/2} b, and A^{1/2} b
// through A^{-1/2}(A b) (Sec. 4).  The host only sequences kernels on the
// handle's stream; all vector work, inner products, the projected matrix
// and the small f(H_m) solve stay on the device.  The host reads back a
// 48-byte status record at each stopping check.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "common.cuh"
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
constexpr int kMaxM = 4096;
constexpr double kBreakdownRel = 1e-12;

struct Workspace {
  int prec = -1;
  int m_cap = 0;
  bool has_y = false;
  int64_t ldv = 0;
  size_t esz = 0;
  void *V = nullptr;
  void *Y = nullptr;
  void *tmp = nullptr;  // 6 vectors
  double *dmem = nullptr;
  size_t dmem_n = 0;
  double *hess = nullptr;
  size_t hess_n = 0;
  DevStatus *st = nullptr;
  DevStatus *st_host = nullptr;
  double *io = nullptr;  // 2 n doubles for pp_apply_host
  void *val_dw = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

}  // namespace

struct pp_ctx {
  int op_kind = OPK_CSR;
  int stencil = -1;
  int64_t n = 0;
  int64_t dims[4] = {0, 0, 0, 0};
  double st_d = 0, st_cm = 0, st_cp = 0, ch = 0;
  const int64_t *rowptr = nullptr;
  const int32_t *col = nullptr;
  const double *val = nullptr;
  int64_t nnz = 0;
  int hermitian = 0;
  cudaStream_t stream = nullptr;
  pp_opts opts;
  bool have_poly = false;
  int degree = 0;
  std::vector<double> coef;
  double a = 0, b = 0, img_lo = 0, img_hi = 0;
  std::vector<double> qsig, qwt;
  bool quad_uploaded = false;
  Workspace ws;
  // operator-launch accounting of the current call (pp_stats.chain_*)
  int64_t chain_launches = 0;
  double chain_bytes = 0.0;
  std::vector<cudaEvent_t> prof_ev;  // start/stop pairs, grown on demand
  size_t prof_used = 0;
};

namespace {


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
  if (w.ev0) cudaEventDestroy(w.ev0);
  if (w.ev1) cudaEventDestroy(w.ev1);
  w = Workspace();
}

// Profiling brackets a run of consecutive operator launches (one q(A)
// application or one product with A) with a pair of events on the handle's
// stream; the per-launch average then includes the short gaps between the
// launches of a run.
int prof_begin(pp_ctx *c) {
  if (!c->opts.profile) return PP_OK;
  if (c->prof_used + 2 > c->prof_ev.size()) {
    for (int i = 0; i < 64; ++i) {
      cudaEvent_t e;
      PP_CUDA_TRY(cudaEventCreate(&e));
      c->prof_ev.push_back(e);
    }
  }
  PP_CUDA_TRY(cudaEventRecord(c->prof_ev[c->prof_used], c->stream));
  return PP_OK;
}

int prof_end(pp_ctx *c) {
  if (!c->opts.profile) return PP_OK;
  PP_CUDA_TRY(cudaEventRecord(c->prof_ev[c->prof_used + 1], c->stream));
  c->prof_used += 2;
  return PP_OK;
}

// One operator launch of the chain: counted and its algorithmic bytes added.
template <typename T>
int run_op(pp_ctx *c, const OpDesc &op, const T *x, const T *y, const T *v, T *out, const StepCoef &k) {
  int rc = op_step<T>(op, x, y, v, out, k, c->stream);
  if (rc) return rc;
  c->chain_launches += 1;
  double vecs = 2.0 + (k.sub_y ? 1.0 : 0.0) + (k.add_v ? 1.0 : 0.0);
  double bytes = vecs * 8.0 * (double)c->n;
  if (c->op_kind == OPK_CSR) bytes += 12.0 * (double)c->nnz + 8.0 * (double)(c->n + 1);
  c->chain_bytes += bytes;
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

double prof_ms(pp_ctx *c) {
  double t = 0.0;
  for (size_t i = 0; i + 1 < c->prof_used; i += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->prof_ev[i], c->prof_ev[i + 1]) == cudaSuccess) t += ms;
  }
  return t;
}

// Layout of the FP64 scratch (offsets in doubles).
struct DLayout {
  size_t H, h1, part, X, tri, z, zprev, sig, wt, scal, total;
  int ldh, nb, K;
};

DLayout dlayout(const pp_ctx *c, int m_cap) {
  DLayout L;
  L.ldh = m_cap + 1;
  L.nb = vec_nchunks(c->n);
  L.K = (int)c->qsig.size();
  size_t o = 0;
  L.H = o;
  o += (size_t)(m_cap + 1) * m_cap;
  L.h1 = o;
  o += (size_t)m_cap + 1;
  L.part = o;
  o += (size_t)L.nb * (m_cap + 1);
  L.X = o;
  o += (size_t)L.K * m_cap;
  L.tri = o;
  o += (size_t)L.K * m_cap;
  L.z = o;
  o += (size_t)m_cap;
  L.zprev = o;
  o += (size_t)m_cap;
  L.sig = o;
  o += (size_t)L.K;
  L.wt = o;
  o += (size_t)L.K;
  L.scal = o;
  o += 8;
  L.total = o;
  return L;
}

int ensure_ws(pp_ctx *c, int prec, int m_cap, bool need_y) {
  Workspace &w = c->ws;
  const size_t esz = 8;  // double and double-word are both 8 bytes
  if (w.prec != prec || m_cap > w.m_cap || (need_y && !w.has_y) || !w.dmem) {
    if (w.V) cudaFree(w.V), w.V = nullptr;
    if (w.Y) cudaFree(w.Y), w.Y = nullptr;
    if (w.tmp) cudaFree(w.tmp), w.tmp = nullptr;
    if (w.dmem) cudaFree(w.dmem), w.dmem = nullptr;
    const int mc = m_cap > w.m_cap ? m_cap : w.m_cap;
    w.ldv = (c->n + 31) / 32 * 32;
    w.esz = esz;
    PP_CUDA_TRY(cudaMalloc(&w.V, (size_t)(mc + 1) * w.ldv * esz));
    if (need_y || w.has_y) {
      PP_CUDA_TRY(cudaMalloc(&w.Y, (size_t)mc * w.ldv * esz));
      w.has_y = true;
    }
    PP_CUDA_TRY(cudaMalloc(&w.tmp, (size_t)6 * w.ldv * esz));
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
  if (prec == PP_PREC_DW && c->op_kind == OPK_CSR && !w.val_dw) {
    PP_CUDA_TRY(cudaMalloc(&w.val_dw, (size_t)c->nnz * sizeof(dw)));
    int rc = vec_from_f64<dw>(c->val, (dw *)w.val_dw, c->nnz, c->stream);
    if (rc) return rc;
  }
  return PP_OK;
}

OpDesc make_op(const pp_ctx *c, int prec) {
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
  op.val = (prec == PP_PREC_DW) ? c->ws.val_dw : (const void *)c->val;
  return op;
}

#define RC(x)                \
  do {                       \
    int _r = (x);            \
    if (_r != PP_OK) return _r; \
  } while (0)

// y = q(A) x by the matrix Clenshaw recurrence with the first two steps
// folded (b_{k+1} = 0, b_k = c_k x): deg q operator applications.
template <typename T>
int poly_apply_raw(pp_ctx *c, const OpDesc &op, const T *in, T *out, T *bufs[3]) {
  const std::vector<double> &cf = c->coef;
  const int k = (int)cf.size() - 1;
  const double s1 = 4.0 / (c->b - c->a), s2 = -2.0 * (c->a + c->b) / (c->b - c->a);
  cudaStream_t s = c->stream;
  if (k == 0) return vec_scale<T>(in, out, c->n, cf[0], nullptr, s);
  if (k == 1) return run_op<T>(c, op, in, nullptr, nullptr, out, {0.5 * s1 * cf[1], 0.5 * s2 * cf[1] + cf[0], 0.0, false, false});
  int i2 = 0, i1 = 1, i0 = 2;  // buffer indices of b_{i+2}, b_{i+1}, free
  RC(run_op<T>(c, op, in, nullptr, nullptr, bufs[i2], {s1 * cf[k], s2 * cf[k] + cf[k - 1], 0.0, false, false}));
  if (k == 2) return run_op<T>(c, op, bufs[i2], nullptr, in, out, {0.5 * s1, 0.5 * s2, cf[0] - cf[2], false, true});
  RC(run_op<T>(c, op, bufs[i2], nullptr, in, bufs[i1], {s1, s2, cf[k - 2] - cf[k], false, true}));
  for (int i = k - 3; i >= 1; --i) {
    RC(run_op<T>(c, op, bufs[i1], bufs[i2], in, bufs[i0], {s1, s2, cf[i], true, true}));
    const int t = i2;
    i2 = i1;
    i1 = i0;
    i0 = t;
  }
  return run_op<T>(c, op, bufs[i1], bufs[i2], in, out, {0.5 * s1, 0.5 * s2, cf[0], true, true});
}

template <typename T>
int poly_apply_t(pp_ctx *c, const OpDesc &op, const T *in, T *out, T *bufs[3]) {
  if (c->degree == 0) return poly_apply_raw<T>(c, op, in, out, bufs);
  RC_(prof_begin(c));
  RC_(poly_apply_raw<T>(c, op, in, out, bufs));
  return prof_end(c);
}

template <typename T>
int solve(pp_ctx *c, int f, const double *b_dev, int m_max, double tol, double *x_dev, pp_stats *out) {
  const int prec = c->opts.precision;
  const bool right = c->opts.side == PP_RIGHT;
  RC(ensure_ws(c, prec, m_max, right));
  Workspace &w = c->ws;
  cudaStream_t s = c->stream;
  const OpDesc op = make_op(c, prec);
  const int64_t n = c->n, ldv = w.ldv;
  const DLayout L = dlayout(c, w.m_cap);
  double *D = w.dmem;
  double *H = D + L.H, *h1 = D + L.h1, *part = D + L.part, *X = D + L.X, *tri = D + L.tri;
  double *z = D + L.z, *zprev = D + L.zprev, *sig = D + L.sig, *wt = D + L.wt, *scal = D + L.scal;
  const int ldh = L.ldh, nb = L.nb, K = L.K;
  T *V = (T *)w.V, *Y = (T *)w.Y;
  T *t[6];
  for (int i = 0; i < 6; ++i) t[i] = (T *)w.tmp + (size_t)i * ldv;
  const int deg = c->degree;
  const bool lanczos = c->opts.orth == PP_ORTH_LANCZOS || (c->opts.orth == PP_ORTH_AUTO && c->hermitian);
  const int kchk = c->opts.check_every > 0 ? c->opts.check_every : (64 / (deg + 1) > 1 ? 64 / (deg + 1) : 1);
  int64_t mvms = 0, ip = 0;
  const int64_t launches0 = pp_launch_count();
  c->chain_launches = 0;
  c->chain_bytes = 0.0;
  c->prof_used = 0;

  PP_CUDA_TRY(cudaEventRecord(w.ev0, s));
  PP_CUDA_TRY(cudaMemsetAsync(w.st, 0, sizeof(DevStatus), s));
  PP_CUDA_TRY(cudaMemsetAsync(H, 0, sizeof(double) * (size_t)ldh * w.m_cap, s));

  // right-hand side in the vector arithmetic
  const T *rhs;
  if (std::is_same<T, double>::value) {
    rhs = (const T *)b_dev;
  } else {
    RC(vec_from_f64<T>(b_dev, t[0], n, s));
    rhs = t[0];
  }
  if (f == PP_SQRT) {  // Sec. 4: A^{1/2} b = A^{-1/2} (A b)
    RC(run_op_timed<T>(c, op, rhs, nullptr, nullptr, t[1], {1.0, 0.0, 0.0, false, false}));
    rhs = t[1];
    mvms += 1;
  }
  T *pb[3] = {t[2], t[3], t[4]};
  if (!right) {  // Algorithm 1: c = q(A) b, v_1 = c / ||c||
    RC(poly_apply_t<T>(c, op, rhs, V, pb));
    mvms += deg;
  } else {       // Algorithm 2: v_1 = b / ||b||
    RC(vec_copy<T>(rhs, V, n, s));
  }
  RC(vec_dot_partials<T>(V, V, n, part, nb, s));
  RC(norm_finalize(part, nb, &w.st->beta0, scal, nullptr, 0, 0.0, 0, w.st, s));
  RC(vec_scale<T>(V, V, n, 1.0, scal, s));
  PP_CUDA_TRY(cudaMemcpyAsync(w.st_host, w.st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
  PP_CUDA_TRY(cudaStreamSynchronize(s));
  DevStatus hs = *w.st_host;
  if (hs.bad) return pp_set_error(PP_ERR_INVALID_ARG, "non-finite norm of the start vector");
  if (hs.breakdown) {  // zero start vector: f(A) 0 = 0
    PP_CUDA_TRY(cudaMemsetAsync(x_dev, 0, sizeof(double) * n, s));
    PP_CUDA_TRY(cudaStreamSynchronize(s));
    if (out) {
      memset(out, 0, sizeof(*out));
      out->mvms = mvms;
      out->launches = pp_launch_count() - launches0;
    }
    return PP_OK;
  }
  // stop at the device: memset flags that record a breakdown of the start
  PP_CUDA_TRY(cudaMemsetAsync(&w.st->conv, 0, 3 * sizeof(int), s));

  int m = 0, mprev = 0, checks = 0, status = PP_ERR_NOT_CONVERGED;
  bool bd = false;
  for (int j = 0; j < m_max; ++j) {
    T *vj = V + (size_t)j * ldv;
    T *wv = V + (size_t)(j + 1) * ldv;
    if (!right) {  // Algorithm 1, line 4: u = A v_j, y = q(A) u, w = q(A) y
      RC(run_op_timed<T>(c, op, vj, nullptr, nullptr, t[0], {1.0, 0.0, 0.0, false, false}));
      RC(poly_apply_t<T>(c, op, t[0], t[1], pb));
      RC(poly_apply_t<T>(c, op, t[1], wv, pb));
    } else {       // Algorithm 2, line 4: y_j = q(A) v_j, u = q(A) y_j, w = A u
      T *yj = Y + (size_t)j * ldv;
      RC(poly_apply_t<T>(c, op, vj, yj, pb));
      RC(poly_apply_t<T>(c, op, yj, t[0], pb));
      RC(run_op_timed<T>(c, op, t[0], nullptr, nullptr, wv, {1.0, 0.0, 0.0, false, false}));
    }
    mvms += 2 * deg + 1;
    double *hcol = H + (size_t)j * ldh;
    if (lanczos) {
      RC(vec_dot_partials<T>(wv, vj, n, part, nb, s));
      RC(reduce_cols(part, nb, 1, 0, hcol + j, nullptr, s));
      RC(vec_lanczos_update<T>(wv, vj, j > 0 ? V + (size_t)(j - 1) * ldv : nullptr, n, hcol + j,
                               j > 0 ? H + (size_t)(j - 1) * ldh + j : nullptr, part, nb, s));
      RC(norm_finalize(part, nb, hcol + j + 1, scal, hcol + j, 1, kBreakdownRel, j + 1, w.st, s));
      ip += 2;
    } else {  // CGS2: h = V^* w, w -= V h, twice
      const int J = j + 1;
      RC(vec_multi_dot<T>(V, ldv, J, wv, n, part, nb, s));
      RC(reduce_cols(part, nb, J, 1, h1, hcol, s));
      RC(vec_multi_update<T>(V, ldv, J, h1, wv, n, nullptr, nb, s));
      RC(vec_multi_dot<T>(V, ldv, J, wv, n, part, nb, s));
      RC(reduce_cols(part, nb, J, 2, h1, hcol, s));
      RC(vec_multi_update<T>(V, ldv, J, h1, wv, n, part, nb, s));
      RC(norm_finalize(part, nb, hcol + j + 1, scal, hcol, J, kBreakdownRel, J, w.st, s));
      ip += 2 * J + 1;
    }
    RC(vec_scale<T>(wv, wv, n, 1.0, scal, s));
    m = j + 1;
    if (m % kchk == 0 || m == m_max) {
      if (lanczos)
        RC(small_tridiag_quad(H, ldh, m, sig, wt, K, X, tri, s));
      else {
        const size_t need = small_hess_scratch_doubles(m, K);
        const size_t smem_bytes = ((size_t)(m + 1) * m + 2 * (size_t)m) * sizeof(double);
        if (smem_bytes > 200 * 1024 && w.hess_n < need) {
          if (w.hess) cudaFree(w.hess);
          w.hess = nullptr;
          w.hess_n = 0;
          PP_CUDA_TRY(cudaMalloc(&w.hess, need * sizeof(double)));
          w.hess_n = need;
        }
        RC(small_hess_quad(H, ldh, m, sig, wt, K, X, w.hess, s));
      }
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
    }
  }
  // f_m = V_m z (left) or Y_m z (right)
  RC(vec_reconstruct<T>(right ? Y : V, ldv, m, z, x_dev, n, s));
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
  const OpDesc op = make_op(c, c->opts.precision);
  T *t0 = (T *)c->ws.tmp, *t1 = t0 + c->ws.ldv;
  if (std::is_same<T, double>::value)
    return op_step<T>(op, (const T *)x, nullptr, nullptr, (T *)y, {1.0, 0.0, 0.0, false, false}, c->stream);
  RC(vec_from_f64<T>(x, t0, c->n, c->stream));
  RC(op_step<T>(op, t0, nullptr, nullptr, t1, {1.0, 0.0, 0.0, false, false}, c->stream));
  return vec_to_f64<T>(t1, y, c->n, c->stream);
}

template <typename T>
int poly_apply_api_t(pp_ctx *c, const double *x, double *y) {
  RC(ensure_ws(c, c->opts.precision, c->ws.m_cap > 0 ? c->ws.m_cap : 1, false));
  const OpDesc op = make_op(c, c->opts.precision);
  T *t[6];
  for (int i = 0; i < 6; ++i) t[i] = (T *)c->ws.tmp + (size_t)i * c->ws.ldv;
  T *pb[3] = {t[2], t[3], t[4]};
  if (std::is_same<T, double>::value) return poly_apply_t<T>(c, op, (const T *)x, (T *)y, pb);
  RC(vec_from_f64<T>(x, t[0], c->n, c->stream));
  RC(poly_apply_t<T>(c, op, t[0], t[1], pb));
  return vec_to_f64<T>(t[1], y, c->n, c->stream);
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

static __device__ __align__(256) double pp_static_scratch[kStaticVecs * (size_t)PP_STATIC_MAX_N];

namespace {

std::mutex g_static_mu;
void *g_static_addr[kStaticMaxDevices] = {};

// Device address of pp_static_scratch on the current device (looked up on the
// first call per device).
int static_scratch_addr(void **out) {
  int dev = 0;
  PP_CUDA_TRY(cudaGetDevice(&dev));
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
  const OpDesc op = make_op(c, c->opts.precision);
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

pp_ctx *new_ctx(void *stream) {
  pp_ctx *c = new pp_ctx();
  pp_default_opts(&c->opts);
  c->stream = (cudaStream_t)stream;
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
  if (dtype != PP_F64) return pp_set_error(PP_ERR_UNSUPPORTED, "CSR values must be PP_F64 in this build");
  if (n > (int64_t)1 << 40) return pp_set_error(PP_ERR_INVALID_ARG, "n too large");
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
  if (dtype != PP_F64) return pp_set_error(PP_ERR_UNSUPPORTED, "stencil vectors must be PP_F64 in this build");
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
  } else if (kind == PP_WILSON4D_DHD) {
    return pp_set_error(PP_ERR_UNSUPPORTED, "Wilson operator not in this build");
  } else {
    return pp_set_error(PP_ERR_INVALID_ARG, "unknown stencil kind");
  }
  c->stencil = kind;
  c->n = c->dims[0] * c->dims[1] * c->dims[2];
  *h = c;
  return PP_OK;
}

int pp_set_opts(pp_handle c, const pp_opts *o) {
  if (!c || !o) return pp_set_error(PP_ERR_INVALID_ARG, "NULL argument");
  if (o->side != PP_LEFT && o->side != PP_RIGHT) return pp_set_error(PP_ERR_INVALID_ARG, "bad side");
  if (o->precision != PP_PREC_F64 && o->precision != PP_PREC_DW) {
    if (o->precision == PP_PREC_MIXED) return pp_set_error(PP_ERR_UNSUPPORTED, "mixed precision not in this build");
    return pp_set_error(PP_ERR_INVALID_ARG, "bad precision");
  }
  if (o->orth < PP_ORTH_AUTO || o->orth > PP_ORTH_CGS2) return pp_set_error(PP_ERR_INVALID_ARG, "bad orth");
  if (o->check_every < 0) return pp_set_error(PP_ERR_INVALID_ARG, "check_every < 0");
  if (o->profile != 0 && o->profile != 1) return pp_set_error(PP_ERR_INVALID_ARG, "profile must be 0 or 1");
  c->opts = *o;
  return PP_OK;
}

int pp_build_poly(pp_handle c, int32_t degree, int32_t kind, const double *ab) {
  if (!c) return pp_set_error(PP_ERR_INVALID_ARG, "NULL handle");
  if (kind != PP_CHEBYSHEV) {
    if (kind >= PP_RITZ_LEJA && kind <= PP_LSQ_CONTOUR) return pp_set_error(PP_ERR_UNSUPPORTED, "polynomial kind not in this build");
    return pp_set_error(PP_ERR_INVALID_ARG, "unknown polynomial kind");
  }
  if (degree < 0 || degree > kMaxDegree) return pp_set_error(PP_ERR_INVALID_ARG, "degree out of [0, 128]");
  double a, b;
  if (ab) {
    a = ab[0];
    b = ab[1];
  } else if (c->op_kind == OPK_ST2D) {
    a = b = 0.0;
    for (int i = 0; i < 2; ++i) {
      const double N = (double)c->dims[i];
      a += 2.0 - 2.0 * std::cos(M_PI / (N + 1));
      b += 2.0 - 2.0 * std::cos(N * M_PI / (N + 1));
    }
  } else if (c->op_kind == OPK_ST3D) {
    // Sec. 6, Example 1 for the Laplacian; convection-diffusion factors are
    // diagonally similar to tridiag(-r, 2+ch, -r), r = sqrt(1+ch)
    const double r = std::sqrt(1.0 + c->ch);
    a = b = 0.0;
    for (int i = 0; i < 3; ++i) {
      const double N = (double)c->dims[i];
      a += (2.0 + c->ch) - 2.0 * r * std::cos(M_PI / (N + 1));
      b += (2.0 + c->ch) - 2.0 * r * std::cos(N * M_PI / (N + 1));
    }
  } else {
    return pp_set_error(PP_ERR_INVALID_ARG, "CSR handles need interval_ab");
  }
  if (!(a > 0.0) || !(b > a) || !std::isfinite(b)) return pp_set_error(PP_ERR_INVALID_ARG, "need 0 < a < b");
  std::vector<double> cf = cheb_interp_coeffs(a, b, degree);
  double qmin, lo, hi;
  cheb_scan(cf, a, b, &qmin, &lo, &hi);
  if (!(qmin > 0.0)) return pp_set_error(PP_ERR_NONPRIMARY, "q is not positive on [a,b]");
  c->coef = cf;
  c->degree = degree;
  c->a = a;
  c->b = b;
  c->img_lo = lo;
  c->img_hi = hi;
  // quadrature for the small solve: real Ritz values for Hermitian A,
  // |arg| <= pi/3 allowed otherwise; generous margins around the image
  const double theta = c->hermitian ? 0.0 : M_PI / 3.0;
  invsqrt_quadrature(lo * 1e-3, hi * 1e3, 1e-15, theta, &c->qsig, &c->qwt);
  c->quad_uploaded = false;
  if (c->ws.dmem) {  // K may have changed: re-layout on next use
    cudaFree(c->ws.dmem);
    c->ws.dmem = nullptr;
  }
  c->have_poly = true;
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
  if (f != PP_SQRT && f != PP_INVSQRT) return pp_set_error(PP_ERR_INVALID_ARG, "f must be PP_SQRT or PP_INVSQRT");
  if (!b_d || !x_d) return pp_set_error(PP_ERR_INVALID_ARG, "NULL vector");
  if (b_d == x_d) return pp_set_error(PP_ERR_INVALID_ARG, "x_d aliases b_d");
  if (nrhs != 1) return pp_set_error(PP_ERR_UNSUPPORTED, "nrhs != 1 not in this build");
  if (m_max < 1 || m_max > kMaxM) return pp_set_error(PP_ERR_INVALID_ARG, "m_max out of [1, 4096]");
  if (!(tol >= 0.0)) return pp_set_error(PP_ERR_INVALID_ARG, "tol < 0");
  if (c->op_kind == OPK_CSR && c->nnz < 0) {
    int64_t nnz = 0;
    PP_CUDA_TRY(cudaMemcpy(&nnz, c->rowptr + c->n, sizeof(int64_t), cudaMemcpyDeviceToHost));
    c->nnz = nnz;
  }
  if (c->opts.precision == PP_PREC_DW) return solve<dw>(c, f, (const double *)b_d, m_max, tol, (double *)x_d, stats);
  return solve<double>(c, f, (const double *)b_d, m_max, tol, (double *)x_d, stats);
}

int pp_apply_host(pp_handle c, int32_t f, const double *b_h, int64_t nrhs, int32_t m_max, double tol,
                  double *x_h, pp_stats *stats) {
  RC(check_ready(c));
  if (!b_h || !x_h) return pp_set_error(PP_ERR_INVALID_ARG, "NULL vector");
  if (nrhs != 1) return pp_set_error(PP_ERR_UNSUPPORTED, "nrhs != 1 not in this build");
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
  if (c->opts.precision == PP_PREC_DW) return poly_apply_api_t<dw>(c, (const double *)x_d, (double *)y_d);
  return poly_apply_api_t<double>(c, (const double *)x_d, (double *)y_d);
}

int pp_poly_apply_static(pp_handle c, const void *x_d, void *y_d) {
  RC(check_ready(c));
  if (!x_d || !y_d || x_d == y_d) return pp_set_error(PP_ERR_INVALID_ARG, "bad arguments");
  if (c->n > PP_STATIC_MAX_N)
    return pp_set_error(PP_ERR_INVALID_ARG, "n = " + std::to_string(c->n) +
                                                " exceeds PP_STATIC_MAX_N = " + std::to_string((long long)PP_STATIC_MAX_N));
  if (c->op_kind == OPK_CSR && c->opts.precision == PP_PREC_DW)
    return pp_set_error(PP_ERR_UNSUPPORTED,
                        "CSR handles in PP_PREC_DW need a converted copy of the values; use PP_PREC_F64");
  if (c->op_kind == OPK_CSR && c->nnz < 0) {
    int64_t nnz = 0;
    PP_CUDA_TRY(cudaMemcpy(&nnz, c->rowptr + c->n, sizeof(int64_t), cudaMemcpyDeviceToHost));
    c->nnz = nnz;
  }
  void *base = nullptr;
  RC(static_scratch_addr(&base));
  if (c->opts.precision == PP_PREC_DW) return poly_apply_static_t<dw>(c, (const double *)x_d, (double *)y_d, base);
  return poly_apply_static_t<double>(c, (const double *)x_d, (double *)y_d, base);
}

void pp_destroy(pp_handle c) {
  if (!c) return;
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
