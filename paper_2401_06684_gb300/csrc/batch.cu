// Batched solves (pp_apply_batch): many independent problems and right-hand
// sides of the matrix-free stencil operators advance in lockstep, so every
// kernel launch covers all of them and the launch count of a batch is that
// of one solve.  The right-hand sides of one CSR matrix form groups of up to
// kCsrMaxRhs segments whose operator steps are one block SpMM launch (the
// matrix read once per step for all of them).
//
// Every (handle, right-hand side) pair is a segment.  Segments are grouped by
// polynomial degree, evaluation scheme of q (Horner or Clenshaw) and
// orthogonalization (Lanczos or CGS2); a group's
// vectors are the concatenation of its segments, each padded to whole
// reduction chunks (padding stays zero), so the vector kernels find a
// block's segment from a chunk table and read per-segment scalars from
// per-segment FP64 scratch blocks (Seg in internal.h).  The stencil steps use
// a per-segment geometry table and per-segment step constants (Horner or
// Clenshaw steps of q), uploaded
// once per call.  A segment that meets its stopping estimate (or breaks down)
// is masked out of all later launches and keeps its iterate.  Groups run on
// their own streams from their own host threads, concurrently.
//
// The method per segment is that of pp_apply (Algorithm 1 or 2, Sec. 4 for
// the square root, the stopping rule of Sec. 6, Example 1); with
// PP_PREC_MIXED a group moves to FP32 when every active segment satisfies the
// switching rule of pp_apply.
#include <algorithm>
#include <cmath>
#include <functional>
#include <map>
#include <memory>
#include <cstring>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "internal.h"

size_t small_hess_scratch_doubles(int m, int K);

#define BRC(x)                  \
  do {                          \
    int _r = (x);               \
    if (_r != PP_OK) return _r; \
  } while (0)

namespace {

constexpr double kBdRel = 1e-12;
constexpr double kBdRelF32 = 4.0 * 0x1p-24;
constexpr double kU32 = 0x1p-24;
constexpr double kMixedSafety = 4.0;
constexpr int kMaxBatchM = 1024;

struct SegIn {
  pp_ctx *c;
  int member;
  int f;
  const double *b;  // device, this right-hand side
  double *x;        // device, this solution
};

struct SegOut {
  int status = PP_ERR_NOT_CONVERGED, iters = 0, breakdown = 0, switch_iter = 0;
  int64_t mvms = 0, ip = 0;
  double est = INFINITY, beta0 = 0.0;
};

// Per-segment FP64 scratch (offsets in doubles).
struct BLayout {
  size_t H, h1, X, tri, z, zprev, sig, wt, scal, qc0, total;
  int ldh;
};

BLayout blayout(int m_cap, int K) {
  BLayout L;
  L.ldh = m_cap + 1;
  size_t o = 0;
  L.H = o;
  o += (size_t)(m_cap + 1) * m_cap;
  L.h1 = o;
  o += (size_t)m_cap + 1;
  L.X = o;
  o += (size_t)K * m_cap;
  L.tri = o;
  o += (size_t)K * m_cap;
  L.z = o;
  o += (size_t)m_cap;
  L.zprev = o;
  o += (size_t)m_cap;
  L.sig = o;
  o += (size_t)K;
  L.wt = o;
  o += (size_t)K;
  L.scal = o;
  o += 8;
  L.qc0 = o;
  o += 8;
  L.total = (o + 31) / 32 * 32;
  return L;
}

// dst[r] = src[seg][r - off[seg]] inside the segment, 0 in its padding
__global__ void k_gather(const double *const *__restrict__ src, const int64_t *__restrict__ off,
                         const int64_t *__restrict__ len, const int *__restrict__ chunk_seg, int chunk,
                         double *__restrict__ dst, int64_t N) {
  pdl_wait();
  pdl_trigger();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x) {
    const int s = chunk_seg[r / chunk];
    const int64_t i = r - off[s];
    dst[r] = i < len[s] ? src[s][i] : 0.0;
  }
}

// dst[seg][r - off[seg]] = src[r] inside the segment
__global__ void k_scatter(double *const *__restrict__ dst, const int64_t *__restrict__ off,
                          const int64_t *__restrict__ len, const int *__restrict__ chunk_seg, int chunk,
                          const double *__restrict__ src, int64_t N) {
  pdl_wait();
  pdl_trigger();
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N; r += (int64_t)gridDim.x * blockDim.x) {
    const int s = chunk_seg[r / chunk];
    const int64_t i = r - off[s];
    if (i < len[s]) dst[s][i] = src[r];
  }
}

// dst[s * dstride + i] = src[i], i < K, for every segment s
__global__ void k_broadcast(const double *__restrict__ src, int K, double *__restrict__ dst, int64_t dstride) {
  pdl_wait();
  pdl_trigger();
  const int s = blockIdx.x;
  for (int i = threadIdx.x; i < K; i += blockDim.x) dst[s * dstride + i] = src[i];
}

// clear the stopping flags (keep beta0)
__global__ void k_clear_flags(DevStatus *st, int nseg) {
  pdl_wait();
  pdl_trigger();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < nseg) {
    st[s].conv = 0;
    st[s].breakdown = 0;
    st[s].m_bd = 0;
  }
}

// A basis of columns of N entries that grows on demand (doubling, up to a
// cap); the first `used` columns are copied when it moves.
template <typename T>
struct GrowCols {
  T *p = nullptr;
  int cap = 0, cap_max = 0;
  int64_t N = 0;
  ~GrowCols() {
    if (p) cudaFree(p);
  }
  int init(int64_t n, int first, int maxc, cudaStream_t s) {
    N = n;
    cap_max = maxc;
    cap = std::min(first, maxc);
    PP_CUDA_TRY(cudaMalloc(&p, sizeof(T) * (size_t)cap * N));
    PP_CUDA_TRY(cudaMemsetAsync(p, 0, sizeof(T) * (size_t)cap * N, s));
    return PP_OK;
  }
  int ensure(int need, cudaStream_t s) {
    if (need <= cap) return PP_OK;
    const int nc = std::min(cap_max, std::max(need, 2 * cap));
    T *q = nullptr;
    PP_CUDA_TRY(cudaMalloc(&q, sizeof(T) * (size_t)nc * N));
    PP_CUDA_TRY(cudaMemcpyAsync(q, p, sizeof(T) * (size_t)cap * N, cudaMemcpyDeviceToDevice, s));
    PP_CUDA_TRY(cudaMemsetAsync(q + (size_t)cap * N, 0, sizeof(T) * (size_t)(nc - cap) * N, s));
    PP_CUDA_TRY(cudaStreamSynchronize(s));
    cudaFree(p);
    p = q;
    cap = nc;
    return PP_OK;
  }
};
constexpr int kFirstCols = 32;

// Device allocations of one group, freed together.
struct Allocs {
  std::vector<void *> p;
  ~Allocs() {
    for (void *q : p) cudaFree(q);
  }
  template <typename X>
  int get(X **out, size_t bytes) {
    void *q = nullptr;
    PP_CUDA_TRY(cudaMalloc(&q, bytes > 0 ? bytes : 16));
    p.push_back(q);
    *out = (X *)q;
    return PP_OK;
  }
};

// Everything a group's kernels need for one arithmetic.
template <typename T>
struct ArithTabs {
  const BatchSeg *bseg = nullptr;  // geometry table
  const int *blkseg = nullptr;     // segment of every block
  unsigned nblk = 0;
  int P = 1;
  const Konst<T> *K = nullptr;     // (deg + 1) x nseg: [0] = A, [1 + t] = step t of q
  // CSR group (every segment a right-hand side of the same matrix)
  bool csr = false;
  OpDesc op{};
  const pp_ctx *c = nullptr;       // the handle: its q's step coefficients
  int64_t sstride = 0;             // entries between consecutive segments
};

struct GroupCtx {
  int nseg = 0, deg = 0, nb = 0, K = 0;
  int64_t N = 0;
  BLayout L;
  bool lanczos = true, right = false;
  bool horner = false;      // q by the backward recurrence of its Newton form
  std::vector<char> ystep;  // step t of q reads w_{t-2} (any segment needs its y term)
  cudaStream_t s = nullptr;
  double *dmem = nullptr, *part = nullptr, *hess = nullptr;
  size_t hess_n = 0;
  DevStatus *st = nullptr;
  int *active = nullptr, *sqrt_mask = nullptr, *chunk_seg = nullptr, *chunk0 = nullptr;
  Allocs *alloc = nullptr;
  // operator-launch accounting (pp_stats.chain_*): launches, algorithmic bytes
  // over the unconverged processes, and with profiling CUDA events around
  // every run of operator launches
  bool profile = false;
  double active_rows = 0.0;
  double csr_nnz = -1.0, csr_rows = 0.0;  // CSR: the matrix, read once per launch
  int64_t chain_launches = 0;
  double chain_bytes = 0.0;
  // the same accounting split into vector bytes per active row and matrix
  // bytes (a replayed segment graph adds its recorded parts)
  double vec_units = 0.0, mat_bytes = 0.0;
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
  ~GroupCtx() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
  int prof_begin() {
    if (!profile) return PP_OK;
    if (ev_used + 2 > ev.size())
      for (int i = 0; i < 64; ++i) {
        cudaEvent_t e;
        PP_CUDA_TRY(cudaEventCreate(&e));
        ev.push_back(e);
      }
    PP_CUDA_TRY(cudaEventRecord(ev[ev_used], s));
    return PP_OK;
  }
  int prof_end() {
    if (!profile) return PP_OK;
    PP_CUDA_TRY(cudaEventRecord(ev[ev_used + 1], s));
    ev_used += 2;
    return PP_OK;
  }
  double prof_ms() const {
    double t = 0.0;
    for (size_t i = 0; i + 1 < ev_used; i += 2) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) t += ms;
    }
    return t;
  }
  template <typename T>
  void count(bool sy, bool av) {
    chain_launches += 1;
    const double units = (2.0 + (sy ? 1.0 : 0.0) + (av ? 1.0 : 0.0)) * (double)sizeof(T);
    chain_bytes += units * active_rows;
    vec_units += units;
    // CSR values (double-word or FP64: 8 bytes; FP32: 4), int32 columns, int64 row pointers
    if (csr_nnz >= 0.0) {
      const double mb = (sizeof(T) == 4 ? 8.0 : 12.0) * csr_nnz + 8.0 * (csr_rows + 1.0);
      chain_bytes += mb;
      mat_bytes += mb;
    }
  }
  Seg seg(bool with_active) const {
    Seg S;
    S.nseg = nseg;
    S.chunk_seg = chunk_seg;
    S.chunk0 = chunk0;
    S.active = with_active ? active : nullptr;
    S.dstride = (int64_t)L.total;
    return S;
  }
};

// y = q(A) x for every active segment (deg operator launches, or a scaled copy for deg 0)
template <typename T>
int poly_batch(GroupCtx &G, const ArithTabs<T> &A, const T *in, T *out, T *bufs[3]) {
  const int k = G.deg;
  const int ns = G.nseg;
  cudaStream_t s = G.s;
  auto step = [&](int t, const T *x, const T *y, const T *v, T *o, bool sy, bool av) {
    G.count<T>(sy, av);
    if (A.csr) return op_step_csr_multi<T>(A.op, A.sstride, ns, G.active, x, y, v, o, poly_step_coef(A.c, t), s);
    return op_step_batch<T>(A.bseg, A.blkseg, A.nblk, A.P, A.K + (size_t)(1 + t) * ns, G.active, x, y, v, o, sy, av,
                            s);
  };
  if (k == 0) return vec_scale<T>(in, out, G.N, 1.0, G.dmem + G.L.qc0, s, G.seg(true));
  if (k == 1) return step(0, in, nullptr, nullptr, out, false, false);
  int i2 = 0, i1 = 1, i0 = 2;
  BRC(step(0, in, nullptr, nullptr, bufs[i2], false, false));
  if (k == 2) return step(1, bufs[i2], nullptr, in, out, false, true);
  BRC(step(1, bufs[i2], nullptr, in, bufs[i1], false, true));
  for (int t = 2; t <= k - 2; ++t) {
    BRC(step(t, bufs[i1], bufs[i2], in, bufs[i0], G.ystep[t] != 0, true));
    const int tmp = i2;
    i2 = i1;
    i1 = i0;
    i0 = tmp;
  }
  return step(k - 1, bufs[i1], bufs[i2], in, out, G.ystep[k - 1] != 0, true);
}

template <typename T>
int aop_batch(GroupCtx &G, const ArithTabs<T> &A, const int *mask, const T *x, T *out) {
  G.count<T>(false, false);
  BRC(G.prof_begin());
  if (A.csr)
    BRC(op_step_csr_multi<T>(A.op, A.sstride, G.nseg, mask, x, nullptr, nullptr, out, {1.0, 0.0, 0.0, false, false},
                             G.s));
  else
    BRC(op_step_batch<T>(A.bseg, A.blkseg, A.nblk, A.P, A.K, mask, x, nullptr, nullptr, out, false, false, G.s));
  return G.prof_end();
}

template <typename T>
int poly_batch_timed(GroupCtx &G, const ArithTabs<T> &A, const T *in, T *out, T *bufs[3]) {
  BRC(G.prof_begin());
  BRC(poly_batch<T>(G, A, in, out, bufs));
  return G.prof_end();
}

// One lockstep Krylov step j in arithmetic T (the step of pp_apply for every segment).
template <typename T>
int krylov_step_batch(GroupCtx &G, const ArithTabs<T> &A, T *V, T *Y, T *t[6], int j, double bd_rel,
                      int64_t *ip) {
  cudaStream_t s = G.s;
  const int64_t N = G.N;
  T *pb[3] = {t[2], t[3], t[4]};
  T *vj = V + (size_t)j * N;
  T *wv = V + (size_t)(j + 1) * N;
  if (!G.right) {
    BRC(aop_batch<T>(G, A, G.active, vj, t[0]));
    BRC(poly_batch_timed<T>(G, A, t[0], t[1], pb));
    BRC(poly_batch_timed<T>(G, A, t[1], wv, pb));
  } else {
    T *yj = Y + (size_t)j * N;
    BRC(poly_batch_timed<T>(G, A, vj, yj, pb));
    BRC(poly_batch_timed<T>(G, A, yj, t[0], pb));
    BRC(aop_batch<T>(G, A, G.active, t[0], wv));
  }
  const Seg S = G.seg(true);
  const BLayout &L = G.L;
  double *H = G.dmem + L.H;
  double *hcol = H + (size_t)j * L.ldh;
  double *scal = G.dmem + L.scal;
  if (G.lanczos) {
    BRC(vec_dot_partials<T>(wv, vj, N, G.part, G.nb, s, S));
    BRC(reduce_cols(G.part, G.nb, 1, 0, hcol + j, nullptr, s, S));
    BRC(vec_lanczos_update<T>(wv, vj, j > 0 ? vj - N : nullptr, N, hcol + j,
                              j > 0 ? H + (size_t)(j - 1) * L.ldh + j : nullptr, G.part, G.nb, s, S));
    BRC(norm_finalize(G.part, G.nb, hcol + j + 1, scal, hcol + j, 1, bd_rel, j + 1, G.st, s, S));
    *ip += 2;
  } else {
    const int J = j + 1;
    double *h1 = G.dmem + L.h1;
    BRC(vec_multi_dot<T>(V, N, J, wv, N, G.part, G.nb, s, S));
    BRC(reduce_cols(G.part, G.nb, J, 1, h1, hcol, s, S));
    const int rc = vec_update_dot<T>(V, N, J, h1, wv, N, G.part, s, S);
    if (rc == PP_ERR_UNSUPPORTED) {
      BRC(vec_multi_update<T>(V, N, J, h1, wv, N, nullptr, G.nb, s, S));
      BRC(vec_multi_dot<T>(V, N, J, wv, N, G.part, G.nb, s, S));
    } else if (rc != PP_OK) {
      return rc;
    }
    BRC(reduce_cols(G.part, G.nb, J, 2, h1, hcol, s, S));
    BRC(vec_multi_update<T>(V, N, J, h1, wv, N, G.part, G.nb, s, S));
    BRC(norm_finalize(G.part, G.nb, hcol + j + 1, scal, hcol, J, bd_rel, J, G.st, s, S));
    *ip += 2 * J + 1;
  }
  return vec_scale<T>(wv, wv, N, 1.0, scal, s, S);
}

// Geometry and constants of one arithmetic, uploaded to the group's allocations.
template <typename T>
int build_tabs(GroupCtx &G, const std::vector<SegIn> &segs, const std::vector<int64_t> &off, ArithTabs<T> *out) {
  const int ns = G.nseg;
  if (segs[0].c->op_kind == OPK_CSR) {  // one matrix: the block SpMM step, no per-segment tables
    out->csr = true;
    out->c = segs[0].c;
    out->op = handle_op_desc(segs[0].c, std::is_same<T, float>::value ? 2 : (std::is_same<T, dw>::value ? 1 : 0));
    out->sstride = ns > 1 ? off[1] - off[0] : 0;
    return PP_OK;
  }
  constexpr int PW = 16 / (int)sizeof(T);
  const int P = PW;  // entries per thread; each segment has its own load path
  std::vector<BatchSeg> g(ns);
  uint64_t nblk = 0;
  for (int i = 0; i < ns; ++i) {
    const pp_ctx *c = segs[i].c;
    g[i].off = off[i];
    g[i].nx = (int)c->dims[0];
    g[i].ny = (int)c->dims[1];
    g[i].nz = c->op_kind == OPK_ST2D ? 1 : (int)c->dims[2];
    g[i].txs = (g[i].nx + P - 1) / P;
    g[i].units = (int64_t)g[i].txs * ((g[i].ny + 1) / 2) * g[i].nz;  // P entries x 2 rows each
    g[i].vec = g[i].nx % P == 0 ? 1 : 0;
    g[i].blk0 = (unsigned)nblk;
    nblk += (uint64_t)((g[i].units + kBatchBlock - 1) / kBatchBlock);
  }
  if (nblk > 0x7fffffffull) return pp_set_error(PP_ERR_INVALID_ARG, "batch too large for one launch");
  // constants: [0] = A, [1 + t] = step t of q (Clenshaw or Horner)
  const int nt = G.deg + 1;
  std::vector<Konst<T>> Kh((size_t)nt * ns);
  std::vector<double> d(ns), cm(ns), cp(ns);
  std::vector<StepCoef> coefs(ns);
  for (int i = 0; i < ns; ++i) {
    d[i] = segs[i].c->st_d;
    cm[i] = segs[i].c->st_cm;
    cp[i] = segs[i].c->st_cp;
  }
  for (int t = 0; t < nt; ++t) {
    for (int i = 0; i < ns; ++i) {
      const pp_ctx *c = segs[i].c;
      if (t == 0) {
        coefs[i] = {1.0, 0.0, 0.0, false, false};
      } else {
        coefs[i] = poly_step_coef(c, t - 1);
      }
    }
    batch_konst<T>(d.data(), cm.data(), cp.data(), coefs.data(), ns, Kh.data() + (size_t)t * ns);
  }
  std::vector<int> bs((size_t)nblk);
  for (int i = 0; i < ns; ++i) {
    const unsigned e = i + 1 < ns ? g[i + 1].blk0 : (unsigned)nblk;
    for (unsigned b = g[i].blk0; b < e; ++b) bs[b] = i;
  }
  BatchSeg *gd = nullptr;
  Konst<T> *Kd = nullptr;
  int *bsd = nullptr;
  BRC(G.alloc->get(&gd, sizeof(BatchSeg) * ns));
  BRC(G.alloc->get(&Kd, sizeof(Konst<T>) * Kh.size()));
  BRC(G.alloc->get(&bsd, sizeof(int) * std::max<size_t>(bs.size(), 1)));
  PP_CUDA_TRY(cudaMemcpyAsync(gd, g.data(), sizeof(BatchSeg) * ns, cudaMemcpyHostToDevice, G.s));
  PP_CUDA_TRY(cudaMemcpyAsync(Kd, Kh.data(), sizeof(Konst<T>) * Kh.size(), cudaMemcpyHostToDevice, G.s));
  if (!bs.empty()) PP_CUDA_TRY(cudaMemcpyAsync(bsd, bs.data(), sizeof(int) * bs.size(), cudaMemcpyHostToDevice, G.s));
  out->bseg = gd;
  out->blkseg = bsd;
  out->nblk = (unsigned)nblk;
  out->P = P;
  out->K = Kd;
  return PP_OK;
}

// One group of a batch plan: every allocation, table and the segment graphs
// are made once (pp_batch_create) and reused by every solve (pp_batch_apply);
// T1 = phase-1 arithmetic, T2 = FP32 for PP_PREC_MIXED (else T2 = T1).
struct ChainOut {
  int64_t launches = 0;
  double bytes = 0.0, ms = 0.0;
};

struct GroupBase {
  std::vector<SegIn> segs;  // the b / x pointers are set before every solve
  cudaStream_t s = nullptr;
  bool graphs_off = false;  // launch every segment directly
  virtual ~GroupBase() {}
  virtual int run(double tol, bool profile, std::vector<SegOut> &res, int64_t *launches_out, ChainOut *chain) = 0;
};

// A captured segment: the Krylov steps [j0, j1) and the check's small solve.
struct BatchGraph {
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0, chain_launches = 0, ip = 0;
  double vec_units = 0.0, mat_bytes = 0.0;
};

template <typename T1, typename T2>
struct GroupPlan : GroupBase {
  static constexpr bool mixed = !std::is_same<T1, T2>::value;
  int ns = 0, deg = 0, kchk = 1, m_max = 1, CH = 0;
  bool lanczos = true, right = false;
  Allocs al;
  GroupCtx G;
  GrowCols<T1> V1g, Y1g;
  GrowCols<float> V2g, Y2g;
  void *tmp = nullptr;
  double *bcat = nullptr, *xcat = nullptr, *qsd = nullptr;
  int *mseg = nullptr, *mseg2 = nullptr;
  int64_t *offd = nullptr, *lend = nullptr;
  const double **srcd = nullptr;
  double **dstd = nullptr;
  std::vector<int64_t> off, len;
  ArithTabs<T1> A1;
  ArithTabs<T2> A2;
  double amp = INFINITY;
  std::map<uint64_t, BatchGraph> graphs;
  std::vector<const void *> graph_ptrs;  // buffers the captured graphs use

  ~GroupPlan() override { clear_graphs(); }
  void clear_graphs() {
    for (auto &kv : graphs)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    graphs.clear();
  }
  // drop the graphs when a buffer they use has moved
  void validate_graphs() {
    std::vector<const void *> p = {V1g.p, Y1g.p, V2g.p, Y2g.p, G.hess};
    if (p != graph_ptrs) {
      clear_graphs();
      graph_ptrs = p;
    }
  }

  int setup(const std::vector<SegIn> &sg, int deg_, bool lanczos_, bool right_, int kchk_, int m_max_,
            cudaStream_t st) {
    segs = sg;
    s = st;
    ns = (int)segs.size();
    deg = deg_;
    lanczos = lanczos_;
    right = right_;
    kchk = kchk_;
    m_max = m_max_;
    CH = vec_chunk_rows();
    G.alloc = &al;
    G.nseg = ns;
    G.deg = deg;
    G.lanczos = lanczos;
    G.horner = poly_horner(segs[0].c);
    G.ystep.assign(std::max(deg, 1), 0);
    for (int t = 0; t < deg; ++t)
      for (const SegIn &q : segs) G.ystep[t] |= poly_step_coef(q.c, t).sub_y ? 1 : 0;
    G.right = right;
    G.s = s;
    // concatenated layout
    off.assign(ns, 0);
    len.assign(ns, 0);
    std::vector<int> cseg, c0(ns + 1);
    int64_t N = 0;
    for (int i = 0; i < ns; ++i) {
      len[i] = segs[i].c->n;
      off[i] = N;
      c0[i] = (int)(N / CH);
      const int64_t padded = (len[i] + CH - 1) / CH * CH;
      for (int64_t q = 0; q < padded / CH; ++q) cseg.push_back(i);
      N += padded;
    }
    c0[ns] = (int)(N / CH);
    G.N = N;
    G.nb = (int)(N / CH);
    // one quadrature for the group, valid on the union of the segments' images
    double lo = INFINITY, hi = 0.0;
    bool herm = true;
    for (const SegIn &q : segs) {
      lo = std::fmin(lo, q.c->img_lo);
      hi = std::fmax(hi, q.c->img_hi);
      herm = herm && q.c->hermitian;
    }
    std::vector<double> qs, qw;
    const bool csr = segs[0].c->op_kind == OPK_CSR;
    if (csr) {  // one handle: its own rule, as in pp_apply
      qs = segs[0].c->qsig;
      qw = segs[0].c->qwt;
      BRC(csr_prepare(segs[0].c, segs[0].c->opts.precision));
      G.csr_nnz = (double)segs[0].c->nnz;
      G.csr_rows = (double)segs[0].c->n;
    } else {
      invsqrt_quadrature(lo * 1e-3, hi * 1e3, 1e-15, herm ? 0.0 : M_PI / 3.0, &qs, &qw);
    }
    G.K = (int)qs.size();
    G.L = blayout(m_max, G.K);
    const BLayout &L = G.L;
    BRC(V1g.init(N, kFirstCols, m_max + 1, s));
    if (right) BRC(Y1g.init(N, kFirstCols, m_max, s));
    BRC(al.get(&tmp, 8 * (size_t)6 * N));
    BRC(al.get(&G.dmem, sizeof(double) * L.total * ns));
    BRC(al.get(&G.part, sizeof(double) * (size_t)G.nb * (m_max + 1)));
    BRC(al.get(&G.st, sizeof(DevStatus) * ns));
    BRC(al.get(&G.active, sizeof(int) * ns));
    BRC(al.get(&G.sqrt_mask, sizeof(int) * ns));
    BRC(al.get(&mseg, sizeof(int) * ns));
    BRC(al.get(&mseg2, sizeof(int) * ns));
    BRC(al.get(&G.chunk_seg, sizeof(int) * cseg.size()));
    BRC(al.get(&G.chunk0, sizeof(int) * (ns + 1)));
    BRC(al.get(&bcat, sizeof(double) * N));
    BRC(al.get(&xcat, sizeof(double) * N));
    BRC(al.get(&qsd, sizeof(double) * 2 * G.K));
    BRC(al.get(&offd, sizeof(int64_t) * ns));
    BRC(al.get(&lend, sizeof(int64_t) * ns));
    BRC(al.get(&srcd, sizeof(double *) * ns));
    BRC(al.get(&dstd, sizeof(double *) * ns));
    PP_CUDA_TRY(cudaMemsetAsync(tmp, 0, 8 * (size_t)6 * N, s));
    PP_CUDA_TRY(cudaMemsetAsync(G.dmem, 0, sizeof(double) * L.total * ns, s));
    std::vector<int> sq(ns);
    std::vector<double> cf0(ns);
    for (int i = 0; i < ns; ++i) {
      sq[i] = segs[i].f == PP_SQRT ? 1 : 0;
      cf0[i] = poly_const(segs[i].c);
    }
    // the group's constant tables (pageable sources: the copies complete before the call returns)
    PP_CUDA_TRY(cudaMemcpyAsync(G.sqrt_mask, sq.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
    PP_CUDA_TRY(cudaMemcpyAsync(G.chunk_seg, cseg.data(), sizeof(int) * cseg.size(), cudaMemcpyHostToDevice, s));
    PP_CUDA_TRY(cudaMemcpyAsync(G.chunk0, c0.data(), sizeof(int) * (ns + 1), cudaMemcpyHostToDevice, s));
    PP_CUDA_TRY(cudaMemcpyAsync(offd, off.data(), sizeof(int64_t) * ns, cudaMemcpyHostToDevice, s));
    PP_CUDA_TRY(cudaMemcpyAsync(lend, len.data(), sizeof(int64_t) * ns, cudaMemcpyHostToDevice, s));
    PP_CUDA_TRY(cudaMemcpyAsync(qsd, qs.data(), sizeof(double) * G.K, cudaMemcpyHostToDevice, s));
    PP_CUDA_TRY(cudaMemcpyAsync(qsd + G.K, qw.data(), sizeof(double) * G.K, cudaMemcpyHostToDevice, s));
    PP_CUDA_TRY(cudaMemcpy2DAsync(G.dmem + L.qc0, sizeof(double) * L.total, cf0.data(), sizeof(double),
                                  sizeof(double), ns, cudaMemcpyHostToDevice, s));
    // per-segment quadrature nodes / weights
    PP_CUDA_TRY(pdl_launch(k_broadcast, dim3(ns), dim3(128), 0, s, qsd, G.K, G.dmem + L.sig, (int64_t)L.total));
    PP_CUDA_TRY(pdl_launch(k_broadcast, dim3(ns), dim3(128), 0, s, qsd + G.K, G.K, G.dmem + L.wt, (int64_t)L.total));
    pp_launch_count() += 2;
    PP_CUDA_TRY(cudaGetLastError());
    BRC(build_tabs<T1>(G, segs, off, &A1));
    if (mixed) BRC(build_tabs<T2>(G, segs, off, &A2));
    double kappa = 0.0;
    for (const SegIn &q : segs)
      kappa = std::fmax(kappa, q.c->img_lo > 0 && !(q.c->image_on_points && !q.c->cplx) ? q.c->img_hi / q.c->img_lo
                                                                                        : INFINITY);
    amp = kMixedSafety * kU32 * kappa;
    PP_CUDA_TRY(cudaStreamSynchronize(s));
    return PP_OK;
  }

  // Run body() for a segment: replay its graph, capture it (the captured
  // launches then run once through the new graph), or run it directly.
  int run_segment(uint64_t key, bool direct, int64_t *ip, const std::function<int()> &body) {
    if (direct || graphs_off) return body();
    auto it = graphs.find(key);
    if (it != graphs.end()) {
      PP_CUDA_TRY(cudaGraphLaunch(it->second.exec, s));
      pp_launch_count() += it->second.launches;
      G.chain_launches += it->second.chain_launches;
      G.chain_bytes += it->second.vec_units * G.active_rows + it->second.mat_bytes;
      G.vec_units += it->second.vec_units;
      G.mat_bytes += it->second.mat_bytes;
      *ip += it->second.ip;
      return PP_OK;
    }
    const int64_t l0 = pp_launch_count(), cl0 = G.chain_launches, ip0 = *ip;
    const double cb0 = G.chain_bytes, vu0 = G.vec_units, mb0 = G.mat_bytes;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      graphs_off = true;
      return body();
    }
    const int rc = body();
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    cudaGraphExec_t exec = nullptr;
    const bool ok = rc == PP_OK && e == cudaSuccess && g && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {  // nothing of the segment ran: undo the counts and run it directly
      cudaGetLastError();
      pp_launch_count() = l0;
      G.chain_launches = cl0;
      G.chain_bytes = cb0;
      G.vec_units = vu0;
      G.mat_bytes = mb0;
      *ip = ip0;
      if (rc != PP_OK) return rc;
      graphs_off = true;
      return body();
    }
    BatchGraph bg;
    bg.exec = exec;
    bg.launches = pp_launch_count() - l0;
    bg.chain_launches = G.chain_launches - cl0;
    bg.vec_units = G.vec_units - vu0;
    bg.mat_bytes = G.mat_bytes - mb0;
    bg.ip = *ip - ip0;
    graphs[key] = bg;
    PP_CUDA_TRY(cudaGraphLaunch(exec, s));
    return PP_OK;
  }

  int run(double tol, bool profile, std::vector<SegOut> &res, int64_t *launches_out, ChainOut *chain) override {
    const int64_t launches0 = pp_launch_count();
    const BLayout &L = G.L;
    const int64_t N = G.N;
    G.profile = profile;
    G.ev_used = 0;
    G.chain_launches = 0;
    G.chain_bytes = 0.0;
    G.vec_units = 0.0;
    G.mat_bytes = 0.0;
    res.assign(ns, SegOut());
    std::vector<const double *> src(ns);
    std::vector<double *> dst(ns);
    for (int i = 0; i < ns; ++i) {
      src[i] = segs[i].b;
      dst[i] = segs[i].x;
    }
    std::vector<int> ones(ns, 1), zeros(ns, 0);
    PP_CUDA_TRY(cudaMemsetAsync(G.st, 0, sizeof(DevStatus) * ns, s));
    PP_CUDA_TRY(cudaMemcpyAsync(G.active, ones.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
    PP_CUDA_TRY(cudaMemcpyAsync(mseg, zeros.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
    PP_CUDA_TRY(cudaMemcpyAsync(srcd, src.data(), sizeof(double *) * ns, cudaMemcpyHostToDevice, s));
    PP_CUDA_TRY(cudaMemcpyAsync(dstd, dst.data(), sizeof(double *) * ns, cudaMemcpyHostToDevice, s));
    T1 *t1[6];
    T2 *t2[6];
    for (int i = 0; i < 6; ++i) {
      t1[i] = (T1 *)tmp + (size_t)i * N;
      t2[i] = (T2 *)tmp + (size_t)i * N;
    }
    const Seg Sall = G.seg(false);
    G.active_rows = 0.0;
    for (int i = 0; i < ns; ++i) G.active_rows += (double)len[i];
    // right-hand sides, A b for the square roots (Sec. 4), start vectors
    PP_CUDA_TRY(pdl_launch(k_gather, dim3(1024), dim3(256), 0, s, srcd, offd, lend, G.chunk_seg, CH, bcat, N));
    ++pp_launch_count();
    PP_CUDA_TRY(cudaGetLastError());
    BRC(vec_from_f64<T1>(bcat, t1[0], N, s));
    BRC(vec_copy<T1>(t1[0], t1[1], N, s));
    BRC(aop_batch<T1>(G, A1, G.sqrt_mask, t1[0], t1[1]));
    T1 *pb[3] = {t1[2], t1[3], t1[4]};
    if (!right)
      BRC(poly_batch<T1>(G, A1, t1[1], V1g.p, pb));
    else
      BRC(vec_copy<T1>(t1[1], V1g.p, N, s));
    BRC(vec_dot_partials<T1>(V1g.p, V1g.p, N, G.part, G.nb, s, Sall));
    // beta0 of every segment into its status record (stride of DevStatus in doubles)
    BRC(norm_finalize(G.part, G.nb, G.dmem + L.scal + 1, G.dmem + L.scal, nullptr, 0, 0.0, 0, G.st, s, Sall));
    BRC(vec_scale<T1>(V1g.p, V1g.p, N, 1.0, G.dmem + L.scal, s, Sall));
    std::vector<DevStatus> hs(ns);
    std::vector<double> beta0(ns);
    PP_CUDA_TRY(cudaMemcpyAsync(hs.data(), G.st, sizeof(DevStatus) * ns, cudaMemcpyDeviceToHost, s));
    PP_CUDA_TRY(cudaMemcpy2DAsync(beta0.data(), sizeof(double), G.dmem + L.scal + 1, sizeof(double) * L.total,
                                  sizeof(double), ns, cudaMemcpyDeviceToHost, s));
    PP_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<int> act(ns, 1), m_of(ns, 0);
    int nact = ns;
    for (int i = 0; i < ns; ++i) {
      res[i].beta0 = beta0[i];
      res[i].mvms = (segs[i].f == PP_SQRT ? 1 : 0) + (right ? 0 : deg);
      if (hs[i].bad) return pp_set_error(PP_ERR_INVALID_ARG, "non-finite norm of a start vector");
      if (hs[i].breakdown) {  // zero right-hand side: x = 0
        act[i] = 0;
        --nact;
        res[i].status = PP_OK;
        res[i].iters = 0;
      }
    }
    auto update_rows = [&]() {
      G.active_rows = 0.0;
      for (int i = 0; i < ns; ++i)
        if (act[i]) G.active_rows += (double)len[i];
    };
    // beta0 is read by the small solves from the status record
    for (int i = 0; i < ns; ++i) hs[i].beta0 = beta0[i];
    PP_CUDA_TRY(cudaMemcpyAsync(G.st, hs.data(), sizeof(DevStatus) * ns, cudaMemcpyHostToDevice, s));
    PP_CUDA_TRY(pdl_launch(k_clear_flags, dim3((ns + 127) / 128), dim3(128), 0, s, G.st, ns));
    ++pp_launch_count();
    PP_CUDA_TRY(cudaMemcpyAsync(G.active, act.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
    update_rows();
    const Seg S = G.seg(true);
    std::vector<double> est_prev(ns, INFINITY);
    int phase = 1, nv1 = 0, ny1 = 0, switched_at = mixed ? -1 : 0;
    auto switch_phase = [&](int m_now) -> int {
      if constexpr (mixed) {
        if (!V2g.p) BRC(V2g.init(N, std::max(kFirstCols, 2 * (m_now + 1)), m_max + 1, s));
        if (right && !Y2g.p) BRC(Y2g.init(N, std::max(kFirstCols, 2 * (m_now + 1)), m_max, s));
        BRC(V2g.ensure(m_now + 1, s));
        if (right) BRC(Y2g.ensure(std::max(m_now, 1), s));
        // columns 0..m_now are contiguous at stride N in both bases: one launch
        BRC((vec_convert<T1, T2>(V1g.p, (T2 *)V2g.p, (int64_t)(m_now + 1) * N, s)));
        if (right && m_now > 0) BRC((vec_convert<T1, T2>(Y1g.p, (T2 *)Y2g.p, (int64_t)m_now * N, s)));
        nv1 = m_now + 1;
        ny1 = m_now;
        phase = 2;
      }
      (void)m_now;
      return PP_OK;
    };
    if (mixed && amp <= tol) {
      BRC(switch_phase(0));
      switched_at = 0;
    }
    int64_t ip = 0;
    int m = 0;
    for (int j0 = 0; j0 < m_max && nact > 0;) {
      const int j1 = std::min((j0 / kchk + 1) * kchk, m_max);
      // buffers of the segment, before any capture
      if (phase == 1) {
        BRC(V1g.ensure(j1 + 1, s));
        if (right) BRC(Y1g.ensure(j1, s));
      } else {
        BRC(V2g.ensure(j1 + 1, s));
        if (right) BRC(Y2g.ensure(j1, s));
      }
      if (!lanczos) {
        const size_t per = small_hess_scratch_doubles(j1, G.K);
        const size_t smem_bytes = ((size_t)(j1 + 1) * j1 + 2 * (size_t)j1) * sizeof(double);
        if (smem_bytes > 200 * 1024 && G.hess_n < per * ns) {
          BRC(al.get(&G.hess, sizeof(double) * per * ns));
          G.hess_n = per * ns;
        }
      }
      validate_graphs();
      const int ph = phase, mp = j0;
      auto body = [&]() -> int {
        for (int j = j0; j < j1; ++j) {
          if (ph == 1)
            BRC(krylov_step_batch<T1>(G, A1, V1g.p, Y1g.p, t1, j, kBdRel, &ip));
          else
            BRC(krylov_step_batch<T2>(G, A2, (T2 *)V2g.p, (T2 *)Y2g.p, t2, j,
                                      std::is_same<T2, float>::value ? kBdRelF32 : kBdRel, &ip));
        }
        double *H = G.dmem + L.H;
        if (lanczos)
          BRC(small_tridiag_quad(H, L.ldh, j1, G.dmem + L.sig, G.dmem + L.wt, G.K, G.dmem + L.X, G.dmem + L.tri, s, S));
        else
          BRC(small_hess_quad(H, L.ldh, j1, G.dmem + L.sig, G.dmem + L.wt, G.K, G.dmem + L.X, G.hess, s, S));
        return small_combine(G.dmem + L.X, G.K, j1, mp, G.dmem + L.z, G.dmem + L.zprev, tol, G.st, s, S);
      };
      BRC(run_segment(((uint64_t)j0 << 34) | ((uint64_t)j1 << 2) | (uint64_t)ph, profile, &ip, body));
      for (int i = 0; i < ns; ++i)
        if (act[i]) res[i].mvms += (int64_t)(j1 - j0) * (2 * deg + 1);
      m = j1;
      j0 = j1;
      PP_CUDA_TRY(cudaMemcpyAsync(hs.data(), G.st, sizeof(DevStatus) * ns, cudaMemcpyDeviceToHost, s));
      PP_CUDA_TRY(cudaStreamSynchronize(s));
      bool all_relaxed = true;
      for (int i = 0; i < ns; ++i) {
        if (!act[i]) continue;
        if (hs[i].bad) return pp_set_error(PP_ERR_CUDA, "non-finite values in a batched Krylov process");
        res[i].est = hs[i].est;
        if (hs[i].breakdown || hs[i].conv) {
          act[i] = 0;
          --nact;
          res[i].status = PP_OK;
          res[i].breakdown = hs[i].breakdown;
          res[i].iters = hs[i].breakdown ? hs[i].m_bd : m;
          m_of[i] = m;
          continue;
        }
        bool relaxed = false;
        if (std::isfinite(est_prev[i]) && std::isfinite(hs[i].est) && est_prev[i] > 0.0) {
          double rho = std::pow(hs[i].est / est_prev[i], 1.0 / kchk);
          if (!(rho < 0.999)) rho = 0.999;
          relaxed = hs[i].est * rho / (1.0 - rho) * amp <= tol;
        }
        all_relaxed = all_relaxed && relaxed;
        est_prev[i] = hs[i].est;
      }
      PP_CUDA_TRY(cudaMemcpyAsync(G.active, act.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
      update_rows();
      if (mixed && phase == 1 && nact > 0 && all_relaxed) {
        BRC(switch_phase(m));
        switched_at = m;
      }
    }
    for (int i = 0; i < ns; ++i) {
      if (act[i]) {
        res[i].iters = m;
        m_of[i] = m;
      }
      res[i].ip = ip;
      res[i].switch_iter = switched_at;
    }
    // f_m = V_m z (left) or Y_m z (right) per segment, then scattered to the callers' x
    PP_CUDA_TRY(cudaMemcpyAsync(mseg, m_of.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
    const Seg Sr = G.seg(false);
    T1 *B1 = right ? Y1g.p : V1g.p;
    if (phase == 1) {
      BRC(vec_reconstruct<T1>(B1, N, std::max(m, 1), G.dmem + L.z, xcat, N, 0, s, Sr, mseg));
    } else {
      const int k1 = right ? ny1 : nv1;
      std::vector<int> m2(ns);
      for (int i = 0; i < ns; ++i) m2[i] = std::max(0, m_of[i] - k1);
      PP_CUDA_TRY(cudaMemcpyAsync(mseg2, m2.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
      BRC(vec_reconstruct<T1>(B1, N, std::max(k1, 1), G.dmem + L.z, xcat, N, 0, s, Sr, mseg));
      if (m > k1)
        BRC(vec_reconstruct<T2>((right ? (T2 *)Y2g.p : (T2 *)V2g.p) + (size_t)k1 * N, N, m - k1, G.dmem + L.z + k1,
                                xcat, N, 1, s, Sr, mseg2));
    }
    PP_CUDA_TRY(pdl_launch(k_scatter, dim3(1024), dim3(256), 0, s, dstd, offd, lend, G.chunk_seg, CH, xcat, N));
    ++pp_launch_count();
    PP_CUDA_TRY(cudaGetLastError());
    PP_CUDA_TRY(cudaStreamSynchronize(s));
    *launches_out += pp_launch_count() - launches0;
    chain->launches = G.chain_launches;
    chain->bytes = G.chain_bytes;
    chain->ms = G.prof_ms();
    return PP_OK;
  }
};

}  // namespace

// A batch plan (pp_batch_create): the grouping of the processes, every
// group's device state and its captured segment graphs.
struct pp_batch_ctx {
  struct Key {
    int deg;
    bool horner;
    bool lanczos;
    const pp_ctx *csr;  // CSR: the matrix; its right-hand sides in blocks of kCsrMaxRhs
    int64_t block;
  };
  std::vector<pp_ctx *> handles;
  std::vector<int32_t> f;
  std::vector<int64_t> nrhs;
  std::vector<std::vector<uint64_t>> sig;  // per handle: what the plan baked in
  int m_max = 1, prec = 0, side = 0, dev = 0;
  cudaStream_t caller = nullptr;
  std::vector<Key> keys;
  std::vector<std::unique_ptr<GroupBase>> groups;
  std::vector<std::vector<std::pair<int, int>>> where;  // (member, rhs) per segment
  std::vector<cudaStream_t> streams;
  ~pp_batch_ctx() {
    groups.clear();
    for (cudaStream_t st : streams)
      if (st) cudaStreamDestroy(st);
  }
};

namespace {

std::vector<uint64_t> handle_sig(const pp_ctx *c) {
  return {c->poly_gen, (uint64_t)c->degree, (uint64_t)c->opts.precision, (uint64_t)c->opts.side,
          (uint64_t)c->opts.orth, (uint64_t)c->opts.check_every, (uint64_t)c->opts.clenshaw, (uint64_t)c->tile_bdx,
          (uint64_t)c->have_poly};
}

int batch_check(const pp_handle *handles, int32_t count, const int32_t *f, const int64_t *nrhs, int32_t m_max,
                int *prec_out, int *side_out) {
  if (!handles || count < 1 || !f || !nrhs) return pp_set_error(PP_ERR_INVALID_ARG, "NULL argument or count < 1");
  if (m_max < 1 || m_max > kMaxBatchM) return pp_set_error(PP_ERR_INVALID_ARG, "m_max out of [1, 1024]");
  int prec = -1, side = -1;
  for (int i = 0; i < count; ++i) {
    pp_ctx *c = handles[i];
    if (!c) return pp_set_error(PP_ERR_INVALID_ARG, "NULL handle");
    if (!c->have_poly) return pp_set_error(PP_ERR_STATE, "pp_build_poly has not been called on every handle");
    if (c->op_kind != OPK_ST2D && c->op_kind != OPK_ST3D && c->op_kind != OPK_CSR)
      return pp_set_error(PP_ERR_UNSUPPORTED, "batched solves take the 2D/3D stencil and CSR operators only");
    if (f[i] != PP_SQRT && f[i] != PP_INVSQRT) return pp_set_error(PP_ERR_INVALID_ARG, "f must be PP_SQRT or PP_INVSQRT");
    if (nrhs[i] < 1) return pp_set_error(PP_ERR_INVALID_ARG, "nrhs < 1");
    if (prec < 0) prec = c->opts.precision, side = c->opts.side;
    if (c->opts.precision != prec || c->opts.side != side)
      return pp_set_error(PP_ERR_INVALID_ARG, "all handles of a batch need the same precision and side");
  }
  *prec_out = prec;
  *side_out = side;
  return PP_OK;
}

}  // namespace

extern "C" int pp_batch_create(pp_batch *out, const pp_handle *handles, int32_t count, const int32_t *f,
                               const int64_t *nrhs, int32_t m_max, void *cuda_stream) {
  if (!out) return pp_set_error(PP_ERR_INVALID_ARG, "NULL output");
  *out = nullptr;
  int prec = 0, side = 0;
  BRC(batch_check(handles, count, f, nrhs, m_max, &prec, &side));
  std::unique_ptr<pp_batch_ctx> B(new pp_batch_ctx());
  B->handles.assign(handles, handles + count);
  B->f.assign(f, f + count);
  B->nrhs.assign(nrhs, nrhs + count);
  B->m_max = m_max;
  B->prec = prec;
  B->side = side;
  B->caller = (cudaStream_t)cuda_stream;
  PP_CUDA_TRY(cudaGetDevice(&B->dev));
  std::vector<std::vector<SegIn>> gsegs;
  for (int i = 0; i < count; ++i) {
    pp_ctx *c = handles[i];
    B->sig.push_back(handle_sig(c));
    const bool lz = c->opts.orth == PP_ORTH_LANCZOS || (c->opts.orth == PP_ORTH_AUTO && c->hermitian);
    const bool hz = poly_horner(c);
    const pp_ctx *mat = c->op_kind == OPK_CSR ? c : nullptr;
    for (int64_t r = 0; r < nrhs[i]; ++r) {
      const int64_t blk = mat ? r / kCsrMaxRhs : 0;
      int g = -1;
      for (size_t q = 0; q < B->keys.size(); ++q) {
        const pp_batch_ctx::Key &k = B->keys[q];
        if (k.deg == c->degree && k.horner == hz && k.lanczos == lz && k.csr == mat && k.block == blk) g = (int)q;
      }
      if (g < 0) {
        B->keys.push_back({c->degree, hz, lz, mat, blk});
        gsegs.emplace_back();
        B->where.emplace_back();
        g = (int)B->keys.size() - 1;
      }
      SegIn q;
      q.c = c;
      q.member = i;
      q.f = f[i];
      q.b = nullptr;
      q.x = nullptr;
      gsegs[g].push_back(q);
      B->where[g].push_back({i, (int)r});
    }
  }
  const size_t ng = gsegs.size();
  B->streams.assign(ng, nullptr);
  for (size_t g = 0; g < ng; ++g) {
    PP_CUDA_TRY(cudaStreamCreateWithFlags(&B->streams[g], cudaStreamNonBlocking));
    const pp_ctx *c0 = gsegs[g][0].c;
    const int deg = B->keys[g].deg;
    const int kchk = c0->opts.check_every > 0 ? c0->opts.check_every : std::max(1, 64 / (deg + 1));
    GroupBase *gp;
    int rc;
    if (prec == PP_PREC_MIXED) {
      auto *q = new GroupPlan<dw, float>();
      gp = q;
      B->groups.emplace_back(gp);
      rc = q->setup(gsegs[g], deg, B->keys[g].lanczos, side == PP_RIGHT, kchk, m_max, B->streams[g]);
    } else if (prec == PP_PREC_DW) {
      auto *q = new GroupPlan<dw, dw>();
      gp = q;
      B->groups.emplace_back(gp);
      rc = q->setup(gsegs[g], deg, B->keys[g].lanczos, side == PP_RIGHT, kchk, m_max, B->streams[g]);
    } else {
      auto *q = new GroupPlan<double, double>();
      gp = q;
      B->groups.emplace_back(gp);
      rc = q->setup(gsegs[g], deg, B->keys[g].lanczos, side == PP_RIGHT, kchk, m_max, B->streams[g]);
    }
    if (rc != PP_OK) return rc;
  }
  *out = B.release();
  return PP_OK;
}

extern "C" int pp_batch_apply(pp_batch B, const void *const *b_d, void *const *x_d, double tol, pp_stats *stats) {
  if (!B || !b_d || !x_d) return pp_set_error(PP_ERR_INVALID_ARG, "NULL argument");
  if (!(tol >= 0.0)) return pp_set_error(PP_ERR_INVALID_ARG, "tol < 0");
  const int count = (int)B->handles.size();
  for (int i = 0; i < count; ++i) {
    if (!b_d[i] || !x_d[i] || b_d[i] == (const void *)x_d[i])
      return pp_set_error(PP_ERR_INVALID_ARG, "bad vector pointers");
    if (handle_sig(B->handles[i]) != B->sig[i])
      return pp_set_error(PP_ERR_STATE, "a handle of the batch changed its q or options after pp_batch_create");
  }
  const size_t ng = B->groups.size();
  for (size_t g = 0; g < ng; ++g) {
    GroupBase &gp = *B->groups[g];
    for (size_t q = 0; q < gp.segs.size(); ++q) {
      const int i = B->where[g][q].first, r = B->where[g][q].second;
      gp.segs[q].b = (const double *)b_d[i] + (int64_t)r * gp.segs[q].c->n;
      gp.segs[q].x = (double *)x_d[i] + (int64_t)r * gp.segs[q].c->n;
    }
  }
  const bool profile = B->handles[0]->opts.profile != 0;
  cudaStream_t caller = B->caller;
  cudaEvent_t e0, e1, start;
  PP_CUDA_TRY(cudaEventCreateWithFlags(&e0, cudaEventDisableTiming));
  PP_CUDA_TRY(cudaEventCreate(&start));
  PP_CUDA_TRY(cudaEventCreate(&e1));
  PP_CUDA_TRY(cudaEventRecord(start, caller));
  PP_CUDA_TRY(cudaEventRecord(e0, caller));
  for (size_t g = 0; g < ng; ++g) PP_CUDA_TRY(cudaStreamWaitEvent(B->streams[g], e0, 0));
  std::vector<std::vector<SegOut>> outs(ng);
  std::vector<int> rcs(ng, PP_OK);
  std::vector<std::string> errs(ng);
  std::vector<int64_t> launches(ng, 0);
  std::vector<ChainOut> chains(ng);
  const int dev = B->dev;
  auto work = [&](size_t g) {
    cudaSetDevice(dev);
    const int rc = B->groups[g]->run(tol, profile, outs[g], &launches[g], &chains[g]);
    rcs[g] = rc;
    if (rc != PP_OK) errs[g] = pp_last_error();
  };
  if (profile || ng == 1) {  // profiling: groups one after another, so the timed launches do not overlap
    for (size_t g = 0; g < ng; ++g) {
      work(g);
      cudaStreamSynchronize(B->streams[g]);
    }
  } else {
    std::vector<std::thread> th;
    for (size_t g = 1; g < ng; ++g) th.emplace_back(work, g);
    work(0);
    for (std::thread &t : th) t.join();
  }
  int rc = PP_OK;
  for (size_t g = 0; g < ng; ++g) {
    cudaEvent_t eg;
    if (cudaEventCreateWithFlags(&eg, cudaEventDisableTiming) == cudaSuccess) {
      cudaEventRecord(eg, B->streams[g]);
      cudaStreamWaitEvent(caller, eg, 0);
      cudaEventDestroy(eg);
    }
    if (rcs[g] != PP_OK && rc == PP_OK) {
      rc = rcs[g];
      pp_set_error(rc, errs[g]);
    }
  }
  cudaEventRecord(e1, caller);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, start, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(start);
  if (rc != PP_OK) return rc;
  int64_t total_launches = 0;
  ChainOut chain_total;
  for (int64_t l : launches) total_launches += l;
  for (const ChainOut &q : chains) {
    chain_total.launches += q.launches;
    chain_total.bytes += q.bytes;
    chain_total.ms += q.ms;
  }
  int worst = PP_OK;
  if (stats) {
    for (int i = 0; i < count; ++i) {
      memset(&stats[i], 0, sizeof(pp_stats));
      stats[i].status = PP_OK;
      stats[i].est_err = 0.0;
      stats[i].ms_total = ms;
      stats[i].launches = total_launches;
      stats[i].chain_launches = chain_total.launches;
      stats[i].chain_bytes = chain_total.bytes;
      stats[i].chain_ms = chain_total.ms;
    }
  }
  for (size_t g = 0; g < ng; ++g) {
    for (size_t q = 0; q < B->groups[g]->segs.size(); ++q) {
      const SegOut &o = outs[g][q];
      const int i = B->where[g][q].first;
      if (o.status != PP_OK) worst = o.status;
      if (!stats) continue;
      pp_stats &st = stats[i];
      if (o.status != PP_OK) st.status = o.status;
      st.iters = std::max(st.iters, o.iters);
      st.breakdown |= o.breakdown;
      st.mvms += o.mvms;
      st.inner_products += o.ip;
      st.est_err = std::fmax(st.est_err, o.est);
      if (B->where[g][q].second == 0) st.beta0 = o.beta0;
      st.switch_iter = o.switch_iter;
    }
  }
  if (worst != PP_OK) pp_set_error(worst, "m_max reached before every stopping estimate fell below tol");
  return worst;
}

extern "C" void pp_batch_destroy(pp_batch B) { delete B; }

extern "C" int pp_apply_batch(const pp_handle *handles, int32_t count, const int32_t *f, const void *const *b_d,
                              const int64_t *nrhs, void *const *x_d, int32_t m_max, double tol,
                              void *cuda_stream, pp_stats *stats) {
  if (!b_d || !x_d) return pp_set_error(PP_ERR_INVALID_ARG, "NULL argument or count < 1");
  if (!(tol >= 0.0)) return pp_set_error(PP_ERR_INVALID_ARG, "tol < 0");
  pp_batch B = nullptr;
  BRC(pp_batch_create(&B, handles, count, f, nrhs, m_max, cuda_stream));
  // a one-shot plan launches its segments directly (no graph would be replayed)
  for (auto &g : B->groups) g->graphs_off = true;
  const int rc = pp_batch_apply(B, b_d, x_d, tol, stats);
  pp_batch_destroy(B);
  return rc;
}
