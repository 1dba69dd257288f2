// Two consecutive Horner steps of q(A) v on a matrix-free stencil in one
// launch, through halo tiles staged in shared memory by the tensor memory
// accelerator (TMA).
//
// The Newton-form Horner scheme (Sec. 5.2) for real nodes runs steps
//     w' = r A w + beta w + delta v
// (no y term).  A pair of them, w'' = step_b(step_a(w)), needs w' only on the
// output tile plus a one-point halo, and w on the tile plus a two-point halo.
// Each block
//   1. loads the box of w (tile + 2-point halo) and the box of v (tile +
//      1-point halo) with one cp.async.bulk.tensor each, completing on one
//      mbarrier; boxes that reach over the grid edge read zeros, which is the
//      Dirichlet boundary of the stencil operators;
//   2. evaluates step a on the tile + 1-point halo into shared memory (zero
//      outside the grid, as the next step's neighbours there are);
//   3. evaluates step b on the tile and writes it.
// Both steps use the expression order of the single-step kernel (ops.cu,
// stencil_row in FP32), so a pair is bit for bit two single steps.
//
// Traffic per pair: w, v read and w'' written once (3 vectors instead of 6);
// step a's work grows by the halo (about 2.3x on the 32 x 8 x 4 tile).  Each
// thread takes 16-byte segments of 4 entries (16-byte shared-memory loads, one
// index decode per segment, 16-byte stores).  FP32
// only: the double-word step is bound by its arithmetic, where the halo's
// extra work costs more than the traffic saved.
//
// TMA rules kept: a box's x start is a multiple of 16 bytes (the halo's start
// is rounded down to 4 floats and the box widened), the row pitch of the grid
// is a multiple of 16 bytes (nx % 4 == 0; the launcher refuses otherwise),
// the base address is 16-byte aligned, shared-memory destinations are
// 128-byte aligned.  Loads only, from this GPU's memory, no multicast.  The
// wait on the mbarrier is bounded: a block that gives up records the failure
// in *err (the solve reports it at its next stopping check) and skips its
// output.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr int kAx = 4;          // floats per 16 bytes: the x alignment of a box start
constexpr int kPairThreads = 256;
constexpr long kTmaSpinMax = 1l << 22;  // try_wait rounds before a block gives up

template <bool D3>
struct PairGeom {
  static constexpr int TX = D3 ? 32 : 64, TY = D3 ? 8 : 16, TZ = D3 ? 4 : 1;
  // w box: the tile + 2-point halo, x start rounded down to kAx
  static constexpr int XBX = TX + 2 * kAx, XBY = TY + 4, XBZ = D3 ? TZ + 4 : 1;
  // v box: the tile + 1-point halo (same x rounding)
  static constexpr int VBX = TX + 2 * kAx, VBY = TY + 2, VBZ = D3 ? TZ + 2 : 1;
  // step a's result: the tile + 1-point halo in y and z; in x the boxes' range
  // (whole 16-byte segments, the outer three entries on each side unused)
  static constexpr int TBX = XBX, TBY = TY + 2, TBZ = D3 ? TZ + 2 : 1;
  static constexpr int SEG = XBX / 4;  // 16-byte segments per row of the boxes and of T
  static constexpr int XN = XBX * XBY * XBZ, VN = VBX * VBY * VBZ, TN = TBX * TBY * TBZ;
  static constexpr int XOFF = 0;                                 // bytes, 128-aligned
  static constexpr int VOFF = ((XN * 4 + 127) / 128) * 128;      // 128-aligned
  static constexpr int TOFF = VOFF + ((VN * 4 + 127) / 128) * 128;
  static constexpr int BAROFF = TOFF + ((TN * 4 + 15) / 16) * 16;
  static constexpr int SMEM = BAROFF + 16 + 128;  // + slack to align the base to 128
  static constexpr unsigned TX_BYTES = (unsigned)(XN + VN) * 4u;
};

struct PairK {
  float K0, Km, Kp, D;
};

__device__ __forceinline__ float pair_row(float xc, float xw, float xe, float xs, float xn, float xd, float xu,
                                          float v, const PairK &K) {
  // the order of stencil_row<float, false, true>
  float nm = xd;
  nm = __fadd_rn(nm, xw);
  nm = __fadd_rn(nm, xs);
  float np = xu;
  np = __fadd_rn(np, xe);
  np = __fadd_rn(np, xn);
  float r = __fmul_rn(K.K0, xc);
  r = __fmaf_rn(K.Km, nm, r);
  r = __fmaf_rn(K.Kp, np, r);
  r = __fmaf_rn(K.D, v, r);
  return r;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}

template <bool D3>
__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                         uint32_t bar) {
  if constexpr (D3)
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
        "%4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
  else
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
        "%3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

template <bool D3>
__global__ void __launch_bounds__(kPairThreads) st_pair_tma(const __grid_constant__ CUtensorMap wmap,
                                                            const __grid_constant__ CUtensorMap vmap,
                                                            float *__restrict__ out, int nx, int ny, int nz,
                                                            PairK Ka, PairK Kb, int *err) {
  using G = PairGeom<D3>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  float *X = reinterpret_cast<float *>(base + G::XOFF);
  float *V = reinterpret_cast<float *>(base + G::VOFF);
  float *Tt = reinterpret_cast<float *>(base + G::TOFF);
  const uint32_t bar = smem_u32(base + G::BAROFF);
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * G::TX, y0 = blockIdx.y * G::TY, z0 = blockIdx.z * G::TZ;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  pdl_wait();  // w and v come from earlier grids
  pdl_trigger();
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(G::TX_BYTES) : "memory");
    tma_load<D3>(smem_u32(X), &wmap, x0 - kAx, y0 - 2, z0 - 2, bar);
    tma_load<D3>(smem_u32(V), &vmap, x0 - kAx, y0 - 1, z0 - 1, bar);
  }
  bool done = false;
  for (long it = 0; it < kTmaSpinMax && !done; ++it) done = mbar_try_wait(bar, 0);
  if (!__syncthreads_and(done)) {
    if (tid == 0) {
      atomicExch(err, 1);
      // the copies may still land: wait for them (bounded) before the block's
      // shared memory is released
      for (long it = 0; it < kTmaSpinMax && !mbar_try_wait(bar, 0); ++it) {
      }
    }
    return;
  }
  // step a on the tile + 1-point halo (zero outside the grid), 4 entries per
  // task: a 16-byte segment lies wholly inside or outside the grid in x
  // (nx % 4 == 0), its x neighbours come from the adjacent segments (the box
  // reads zeros beyond the grid; the unused outer entries take zeros there too)
  const float4 *X4 = reinterpret_cast<const float4 *>(X);
  const float4 *V4 = reinterpret_cast<const float4 *>(V);
  float4 *T4 = reinterpret_cast<float4 *>(Tt);
  constexpr int RA = G::TBY * G::SEG;
  for (int q = tid; q < G::TBZ * RA; q += kPairThreads) {
    const int tz = q / RA;
    const int rem = q - tz * RA;
    const int ty = rem / G::SEG, sg = rem - ty * G::SEG;
    const int gx = x0 - kAx + 4 * sg, gy = y0 - 1 + ty, gz = D3 ? z0 - 1 + tz : 0;
    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz) {
      const int row = ((D3 ? tz + 1 : 0) * G::XBY + ty + 1) * G::SEG;  // X box row of (gy, gz)
      const float4 c = X4[row + sg];
      const float xw0 = sg > 0 ? X4[row + sg - 1].w : 0.f;
      const float xe3 = sg + 1 < G::SEG ? X4[row + sg + 1].x : 0.f;
      const float4 so = X4[row - G::SEG + sg], no = X4[row + G::SEG + sg];
      float4 dn = make_float4(0.f, 0.f, 0.f, 0.f), up = dn;
      if constexpr (D3) {
        dn = X4[row - G::XBY * G::SEG + sg];
        up = X4[row + G::XBY * G::SEG + sg];
      }
      const float4 v = V4[(tz * G::VBY + ty) * G::SEG + sg];
      t.x = pair_row(c.x, xw0, c.y, so.x, no.x, dn.x, up.x, v.x, Ka);
      t.y = pair_row(c.y, c.x, c.z, so.y, no.y, dn.y, up.y, v.y, Ka);
      t.z = pair_row(c.z, c.y, c.w, so.z, no.z, dn.z, up.z, v.z, Ka);
      t.w = pair_row(c.w, c.z, xe3, so.w, no.w, dn.w, up.w, v.w, Ka);
    }
    T4[q] = t;
  }
  __syncthreads();
  // step b on the tile, 4 entries per task (segment sg + 1 of the T rows)
  constexpr int SB = G::TX / 4, RB = G::TY * SB;
  for (int q = tid; q < G::TZ * RB; q += kPairThreads) {
    const int tz = q / RB;
    const int rem = q - tz * RB;
    const int ty = rem / SB, sg = rem - ty * SB;
    const int gx = x0 + 4 * sg, gy = y0 + ty, gz = z0 + tz;
    if (gx >= nx || gy >= ny || gz >= nz) continue;
    const int row = ((D3 ? tz + 1 : 0) * G::TBY + ty + 1) * G::SEG;
    const int sc = sg + 1;
    const float4 c = T4[row + sc];
    const float xw0 = T4[row + sc - 1].w, xe3 = T4[row + sc + 1].x;
    const float4 so = T4[row - G::SEG + sc], no = T4[row + G::SEG + sc];
    float4 dn = make_float4(0.f, 0.f, 0.f, 0.f), up = dn;
    if constexpr (D3) {
      dn = T4[row - G::TBY * G::SEG + sc];
      up = T4[row + G::TBY * G::SEG + sc];
    }
    const float4 v = V4[((D3 ? tz + 1 : 0) * G::VBY + ty + 1) * G::SEG + sc];
    float4 o;
    o.x = pair_row(c.x, xw0, c.y, so.x, no.x, dn.x, up.x, v.x, Kb);
    o.y = pair_row(c.y, c.x, c.z, so.y, no.y, dn.y, up.y, v.y, Kb);
    o.z = pair_row(c.z, c.y, c.w, so.z, no.z, dn.z, up.z, v.z, Kb);
    o.w = pair_row(c.w, c.z, xe3, so.w, no.w, dn.w, up.w, v.w, Kb);
    *reinterpret_cast<float4 *>(out + ((int64_t)gz * ny + gy) * nx + gx) = o;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

template <bool D3>
int encode_box(CUtensorMap *map, const float *p, const OpDesc &op, int bx, int by, int bz) {
  const int rank = D3 ? 3 : 2;
  const cuuint64_t dims[3] = {(cuuint64_t)op.nx, (cuuint64_t)op.ny, (cuuint64_t)(D3 ? op.nz : 1)};
  const cuuint64_t strides[2] = {(cuuint64_t)op.nx * 4u, (cuuint64_t)op.nx * (cuuint64_t)op.ny * 4u};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = encoder()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<float *>(p), dims, strides,
                               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? PP_OK : pp_set_error(PP_ERR_CUDA, "tensor map encoding failed");
}

PairK pair_konst(const OpDesc &op, const StepCoef &c) {
  return {(float)(c.alpha * op.d + c.beta), (float)(c.alpha * op.cm), (float)(c.alpha * op.cp), (float)c.delta};
}

template <bool D3>
int launch_pair(const OpDesc &op, const float *w, const float *v, float *out, const StepCoef &a, const StepCoef &b,
                int *err, cudaStream_t s) {
  using G = PairGeom<D3>;
  CUtensorMap wm, vm;
  int rc = encode_box<D3>(&wm, w, op, G::XBX, G::XBY, G::XBZ);
  if (rc == PP_OK) rc = encode_box<D3>(&vm, v, op, G::VBX, G::VBY, G::VBZ);
  if (rc != PP_OK) return rc;
  static_assert(G::SMEM <= 48 * 1024, "the pair kernel's shared memory fits the default limit");
  const dim3 grid((unsigned)((op.nx + G::TX - 1) / G::TX), (unsigned)((op.ny + G::TY - 1) / G::TY),
                  (unsigned)(D3 ? (op.nz + G::TZ - 1) / G::TZ : 1));
  PP_CUDA_TRY(pdl_launch(st_pair_tma<D3>, grid, dim3(kPairThreads), (size_t)G::SMEM, s, wm, vm, out, (int)op.nx,
                         (int)op.ny, (int)(D3 ? op.nz : 1), pair_konst(op, a), pair_konst(op, b), err));
  ++pp_launch_count();
  PP_CUDA_TRY(cudaGetLastError());
  return PP_OK;
}

}  // namespace

bool op_pair_ok(const OpDesc &op, const void *w, const void *v, const void *out) {
  if (op.kind != OPK_ST2D && op.kind != OPK_ST3D) return false;
  if (op.nx % kAx != 0 || op.nx > 0x7fffffff || op.ny > 0x7fffffff || op.nz > 0x7fffffff) return false;
  if (op.ny > 65535ll * PairGeom<true>::TY || op.nz > 65535ll * PairGeom<true>::TZ) return false;
  auto al = [](const void *p) { return ((uintptr_t)p % 16) == 0; };
  if (!al(w) || !al(v) || !al(out)) return false;
  return encoder() != nullptr;
}

int op_pair_step(const OpDesc &op, const float *w, const float *v, float *out, const StepCoef &a,
                 const StepCoef &b, int *err, cudaStream_t s) {
  if (!op_pair_ok(op, w, v, out) || a.sub_y || b.sub_y || !a.add_v || !b.add_v || err == nullptr)
    return pp_set_error(PP_ERR_UNSUPPORTED, "paired stencil steps need a real-node Horner pair on a stencil grid "
                                            "with nx % 4 == 0 and 16-byte aligned vectors");
  if (op.kind == OPK_ST3D) return launch_pair<true>(op, w, v, out, a, b, err, s);
  return launch_pair<false>(op, w, v, out, a, b, err, s);
}
