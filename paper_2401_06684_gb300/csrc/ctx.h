// Handle state shared by the translation units of the C ABI (api.cu, batch.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <vector>

#include "internal.h"

// Scratch vectors of the workspace: 6 for the driver and q(A), a 7th for
// the intermediate D x of the Wilson operator.
constexpr int kTmpVecs = 7;

struct Workspace {
  int prec = -1;
  int m_cap = 0;
  bool two_pass = false;  // basis of 4 columns (two-pass Lanczos) instead of m_cap + 1
  bool has_y = false;
  int64_t ldv = 0;
  size_t esz = 0;
  void *V = nullptr;
  void *Y = nullptr;
  void *tmp = nullptr;  // kTmpVecs vectors
  double *dmem = nullptr;
  size_t dmem_n = 0;
  double *hess = nullptr;
  size_t hess_n = 0;
  DevStatus *st = nullptr;
  DevStatus *st_host = nullptr;
  double *io = nullptr;  // 2 n doubles for pp_apply_host
  void *val_dw = nullptr;  // double-word CSR values (PP_PREC_DW, PP_PREC_MIXED)
  int val_exact_f32 = -1;  // every CSR value exact in FP32 (-1: not checked yet)
  void *val_f = nullptr;  // FP32 CSR values (PP_PREC_MIXED)
  int32_t *long_rows = nullptr;  // CSR rows longer than kLongRow entries: block rows, then warp rows
  int nlong = -1;                // rows with a block each (-1: not scanned yet)
  int nwarp = 0;                 // rows with a warp each
  // CSR rows of the lane path sorted by length within windows of rows, where
  // the lengths vary (NULL: rows in their own order)
  int32_t *csr_perm = nullptr;
  int64_t nshort = 0;
  void *Vf = nullptr;     // FP32 basis of the second phase (PP_PREC_MIXED)
  void *Yf = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

// A captured run of Krylov steps up to a stopping check (CUDA graph) and
// the counters its launches add.
struct SegGraph {
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0, chain_launches = 0, mvms = 0, ip = 0;
  double chain_bytes = 0.0;
};

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
  const void *links = nullptr;  // Wilson: complex64 links (caller-owned)
  double mass = 0.0;
  double mu_c = 0.0;  // Wilson Q^2: chemical potential
  int hermitian = 0;
  // complex non-Hermitian operator (Wilson Q^2 with mu_c != 0): complex
  // Arnoldi coefficients, complex H_m, a complex q
  bool cplx = false;
  cudaStream_t stream = nullptr;
  int device = 0;  // the CUDA device current when the handle was created
  pp_opts opts;
  bool have_poly = false;
  int degree = 0;
  int poly_kind = 0;          // pp_poly_kind of q
  std::vector<double> coef;   // as read back: Chebyshev coefficients, or b_i / cap^i (other kinds)
  NewtonForm nf;              // q at its Leja-ordered nodes, the form the device chain evaluates
  double a = 0, b = 0, img_lo = 0, img_hi = 0;
  // the image was taken at Ritz values only (no spectral interval of a
  // non-normal operator): it does not bound the FP32 amplification, so
  // PP_PREC_MIXED stays in double-word (complex operators estimate that
  // amplification from H_m at each check instead)
  bool image_on_points = false;
  std::vector<double> qsig, qwt;
  int tile_bdx = 0;  // stencil threads per block chosen by pp_autotune (0 = default)
  bool quad_uploaded = false;
  Workspace ws;
  // operator-launch accounting of the current call (pp_stats.chain_*)
  int64_t chain_launches = 0;
  double chain_bytes = 0.0;
  // set by a solve while it runs: the status word that paired stencil launches
  // (opts.halo) report a failed TMA wait to, read at every stopping check
  int *pair_err = nullptr;
  std::vector<cudaEvent_t> prof_ev;  // start/stop pairs, grown on demand
  size_t prof_used = 0;
  std::vector<int> prof_cat;  // category of each pair: 0 operator chain, 1 orthogonalization, 2 small solve
  // segment graphs of pp_apply, keyed by (first step, end step, phase); valid
  // while seg_sig (workspace pointers, q, options, tol) is unchanged
  std::map<uint64_t, SegGraph> segs;
  std::vector<uint64_t> seg_sig;
  uint64_t poly_gen = 0;    // bumped whenever q or its quadrature changes
  bool graphs_off = false;  // capture failed once: direct launches
  // private stream the segments are captured on (capture is not allowed on
  // the legacy default stream a handle may run on); the graphs are launched
  // on the handle's stream
  cudaStream_t cap_stream = nullptr;
};

// q(A) v by the Horner scheme of the Newton form (every kind of q unless
// opts.clenshaw asks for the matrix Clenshaw recurrence of a Chebyshev q;
// always for complex operators).
inline bool poly_horner(const pp_ctx *c) { return c->poly_kind != 0 || !c->opts.clenshaw || c->cplx; }

// Coefficients of step t (0 .. degree-1) of q(A) v.
inline StepCoef poly_step_coef(const pp_ctx *c, int t) {
  if (c->nf.cx) return horner_step_cx(c->nf.b, c->nf.bi, c->nf.c, c->nf.ci, c->nf.cap, t);
  if (poly_horner(c)) return horner_step(c->nf.b, c->nf.c, c->nf.e, c->nf.cap, t);
  const double s1 = 4.0 / (c->b - c->a), s2 = -2.0 * (c->a + c->b) / (c->b - c->a);
  return clenshaw_coef(c->coef, s1, s2, t);
}

// Constant q of degree 0.
inline double poly_const(const pp_ctx *c) { return poly_horner(c) ? c->nf.b[0] : c->coef[0]; }

// CSR handles: read nnz back, list the rows longer than the block-per-row
// threshold (once per handle), and make the double-word copy of the values
// (PP_PREC_DW, PP_PREC_MIXED) and the FP32 one (PP_PREC_MIXED).  Synchronous
// host work; no-op for other handles.
int csr_prepare(pp_ctx *c, int prec);
// The operator description of a handle for vectors in arithmetic `arith`
// (0 FP64, 1 double-word, 2 FP32).
OpDesc handle_op_desc(const pp_ctx *c, int arith);

