// One dual evaluation of the ridge-regularised matching dual on sm_103a.
//
// For a dual point mu (renumbered destinations), every source i projects its
// scores r_e = -(c_e + a_e mu_j) onto {x >= 0, sum x <= 1} in the metric of
// the ridge term (Section 3.1: x* = Pi_C(-(A^T mu + c) / gamma); Section 3.2,
// Eqs. 4-5), then y = A x is accumulated per destination and the objective
// partials sum c x and sum w x^2 are reduced (Section 6: the local objective
// value and regularisation penalty).  The J-length epilogue forms
// grad = A x - b, g(mu) (Eq. 2) and ||(A x - b)_+|| (Appendix A).
//
// Kernel design (GB300-first, not the paper's bucketed padded slabs):
//  * one persistent CTA per SM walks "tiles" (runs of whole sources holding
//    at most a stage's edges and kTileSources sources): a single problem's
//    tiles are taken in grabs of DUALIP_GRAB from a counter shared by all
//    CTAs (balanced ends), a batched pass's in a contiguous range.  Warp 0
//    streams each tile's offsets, destinations and (c, a) into a
//    kStages-deep shared-memory ring with cp.async.bulk + mbarrier
//    transaction counts; the other warps project;
//  * consumer warps claim batches of eight sources of a staged tile through a
//    per-stage shared counter; the span of a source picks how many lanes
//    share it (4, 8, 16 or 32, up to 16 or 20 edges per lane in registers);
//  * the common case at small gamma is a saturated source with a single
//    candidate (its second score is more than gamma below the first): it gets
//    x = 1 exactly.  Everything else (unsaturated sources, near-ties, spans
//    over 512, the primal output) is projected by a whole warp in several
//    passes over the staged tile, with scores as an unevaluated FP32 pair
//    (hi + lo = -(c + a mu) to about 2^-48 relative) shifted by the block
//    maximum (exact by Sterbenz's lemma near the top), so the threshold and x
//    keep FP32 accuracy relative to gamma; Michelot's finite iteration starts
//    from a set that contains the active set.  A source larger than a tile is
//    projected by one warp from global memory;
//  * y = A x accumulates in 64-bit two's-complement fixed point (scale
//    2^exp_y chosen at create so that no sum can overflow): every add is
//    exact, so A x does not depend on the order of the adds.  Hot
//    destinations (ids renumbered by in-degree) accumulate in shared memory
//    and are flushed once per CTA; the rest go to global atomics;
//  * objective partials are per-lane FP32 TwoSum accumulators and FP32
//    double-float pairs through the warp and CTA trees; batches go to warps
//    dynamically, so their last bits may differ from run to run;
//  * the pass may be launched before the preceding kernel of its stream has
//    finished (programmatic dependent launch): until the consumers have waited
//    for that kernel, the producer reads only the problem's immutable arrays
//    and the schedule counter (rewound by the previous pass, which finished
//    before that kernel began).
#include <cuda_bf16.h>
#include <math_constants.h>

#include "internal.h"

namespace dualip {
namespace {

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per wait

// ---------------------------------------------------------------- PTX ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// explicit shared-space accesses on 32-bit shared addresses
__device__ __forceinline__ float lds_f32(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ int lds_s32(uint32_t a) {
  int v;
  asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ float2 lds_f32x2(uint32_t a) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ int4 lds_s32x4(uint32_t a) {
  int4 v;
  asm volatile("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(a));
  return v;
}
__device__ __forceinline__ float4 lds_f32x4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a));
  return v;
}
__device__ __forceinline__ uint32_t atoms_add_u32(uint32_t a, uint32_t v) {
  uint32_t old;
  asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(a), "r"(v));
  return old;
}
__device__ __forceinline__ void reds_add_u32(uint32_t a, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(v));
}
__device__ __forceinline__ void reds_add_u64(uint32_t a, unsigned long long v) {
  asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(a), "l"(v));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// try_wait, optionally with a suspend-time hint (ns): a warp whose phase has
// not completed may be suspended instead of spinning.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  if (kWaitHintNs > 0) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"((uint32_t)kWaitHintNs)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  }
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait on an mbarrier phase.  Gives up after kWaitLimitNs, when
// another thread has raised `abort`, or when the host has set abort_req in
// the status word, recording the site.
__device__ bool wait_phase(uint64_t* bar, uint32_t parity, volatile int* abort,
                           DeviceStatus* st, int site) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 0) {
      if (*abort) return false;
      if (*reinterpret_cast<volatile int*>(&st->abort_req) ||
          globaltimer() - t0 > kWaitLimitNs) {
        *abort = 1;
        atomicOr(&st->err, kErrTimeout);
        atomicCAS(&st->where, 0, site);
        return false;
      }
    }
  }
}

// ------------------------------------------------------- FP32 helpers ----
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// exact error of s = fl(u + v) (Knuth's TwoSum)
__device__ __forceinline__ float two_sum_err(float u, float v, float s) {
  const float bp = __fsub_rn(s, u);
  return __fadd_rn(__fsub_rn(u, __fsub_rn(s, bp)), __fsub_rn(v, bp));
}
// r = -(c + a m) as a normalised pair hi + lo with hi = fl(r): TwoProduct by
// FMA, TwoSum, then a final TwoSum so that |lo| <= ulp(hi) / 2 even when
// c and a m cancel.
__device__ __forceinline__ void score(float c, float a, float m, float& hi, float& lo) {
  const float p = __fmul_rn(a, m);
  const float pe = __fmaf_rn(a, m, -p);
  const float s = __fadd_rn(c, p);
  const float se = two_sum_err(c, p, s);
  const float h0 = -s, l0 = -__fadd_rn(se, pe);
  hi = __fadd_rn(h0, l0);
  lo = two_sum_err(h0, l0, hi);
}

// Fixed-point accumulation: v * 2^S is exact in FP32 (a power-of-two scale)
// and is rounded once to a 64-bit integer; integer adds are exact and
// independent of their order, so A x is reproducible bit for bit.  The scale
// is chosen at create so that no sum can exceed 2^61.
__device__ __forceinline__ long long to_fixed(float v, float scale) {
  return __float2ll_rn(__fmul_rn(v, scale));
}

// --------------------------------------------------------- smem layout ----
struct alignas(16) StageInfo {
  int64_t s0, s1;  // sources [s0, s1)
  int64_t e0, e1;  // edges [e0, e1)
  int64_t a0;      // first staged edge (multiple of 4)
  int64_t o0;      // first staged offset (a multiple of 4)
  int32_t big;     // single source larger than a stage: read from global
  int32_t slot;    // batched pass: the slot whose problem the tile belongs to
};

template <bool BF16>
struct Layout {
  static constexpr size_t kOffBytes = sizeof(uint32_t) * kStageOffSlots;
  static constexpr int kTile = BF16 ? kTileEdgesBF16 : kTileEdges;  // edges of a tile
  static constexpr int kSlots = kTile + kStageSlack;
  static constexpr size_t kEdgeArr = sizeof(uint32_t) * kSlots;
  // dst carries kDstPad extra slots: a group's aligned window (at most 512
  // slots) never leaves it, and every slot holds a valid destination id
  // (zeroed at start, then earlier tiles' ids), so window slots outside the
  // source need no index masking
  static constexpr size_t kDstArr = sizeof(uint32_t) * (kSlots + kDstPad);
  static constexpr size_t kStageBytes = kOffBytes + kDstArr + kEdgeArr * (BF16 ? 1 : 2);
  static constexpr size_t kMu = kStages * kStageBytes;
  static constexpr size_t kY = kMu + sizeof(float) * kMaxCachedDests;
  static constexpr size_t kBars = kY + sizeof(unsigned long long) * kMaxPrivDests;
  // full[kStages], empty[kStages], and two consumer barriers (batched pass)
  static constexpr size_t kInfo = kBars + sizeof(uint64_t) * (2 * kStages + 2);
  static constexpr size_t kMisc = kInfo + sizeof(StageInfo) * kStages;
  // [kMisc + 512, kMisc + 1024): FP64 block reductions (weighted block class)
  static constexpr size_t kTotal = kMisc + 1024;
  static_assert(kOffBytes % 16 == 0 && kEdgeArr % 16 == 0 && kDstArr % 16 == 0,
                "16-byte staging");
  static_assert(kTotal <= 227 * 1024, "shared memory budget");
  static_assert(kMisc % 16 == 0, "float4 reduction slots at kMisc + 16");
  static_assert(16 + 16 * (kThreads / 32) <= 320, "reduction slots end before the claim counters");
  static_assert(24 * kConsumerWarps <= 512, "FP64 reduction slots");
};

// Stage layout: offsets | dst (4 B per slot, padded) | c, a (8 B per slot:
// FP32 pairs, or 4 B: packed bf16 pair c | a << 16).  Addresses are 32-bit
// shared-space addresses, read with ld.shared.
template <bool BF16>
struct StageView {
  uint32_t off_a, dst_a, ca_a;
  // low 32 bits of a staged source offset (differences within a tile are exact)
  __device__ __forceinline__ uint32_t off(int k) const { return lds_u32(off_a + 4u * k); }
  __device__ __forceinline__ void edge(int k, int& j, float& cv, float& av) const {
    j = lds_s32(dst_a + 4u * k);
    if (BF16) {
      const uint32_t u = lds_u32(ca_a + 4u * k);
      cv = __uint_as_float(u << 16);
      av = __uint_as_float(u & 0xffff0000u);
    } else {
      const float2 v = lds_f32x2(ca_a + 8u * k);
      cv = v.x;
      av = v.y;
    }
  }
};

template <bool BF16>
__device__ __forceinline__ StageView<BF16> stage_view(unsigned char* smem, int s) {
  using L = Layout<BF16>;
  const uint32_t base = smem_u32(smem) + (uint32_t)((size_t)s * L::kStageBytes);
  StageView<BF16> v;
  v.off_a = base;
  v.dst_a = base + (uint32_t)L::kOffBytes;
  v.ca_a = base + (uint32_t)(L::kOffBytes + L::kDstArr);
  return v;
}

// global edge reader (sources too large for a stage)
template <bool BF16>
struct GlobalView {
  const int32_t* dst;
  const float2* ca2;
  const uint32_t* ca;
  __device__ __forceinline__ void edge(int64_t k, int& j, float& cv, float& av) const {
    j = __ldg(dst + k);
    if (BF16) {
      const uint32_t u = __ldg(ca + k);
      cv = __uint_as_float(u << 16);
      av = __uint_as_float(u & 0xffff0000u);
    } else {
      const float2 v = __ldg(ca2 + k);
      cv = v.x;
      av = v.y;
    }
  }
};

// ------------------------------------------------------ per-thread state ----
// Read-only context of a pass.  Shared arrays are addressed by 32-bit
// shared-space addresses.
struct Ctx {
  uint32_t mu_a;  // shared mu cache (h_mu floats)
  const float* mu_g;
  int h_mu;
  uint32_t y_a;   // shared fixed-point bins (h_y x 8 bytes)
  int h_y;
  unsigned long long* y;
  float gamma, inv_gamma;
  float sy;  // 2^ey: fixed-point scale of A x
  float sc, sw;     // 2^ec, 2^ew: fixed-point scales of sum c x and sum w x^2
  long long one_w;  // 2^ew (exact: ew >= 0 whenever the weights are all 1)
  float* x_out;
  // edge arrays in global memory (sources larger than a stage)
  const int32_t* dst_g;
  const float2* ca2_g;
  const uint32_t* ca_g;

  __device__ __forceinline__ float mu_smem(int j) const { return lds_f32(mu_a + 4u * j); }
  __device__ __forceinline__ float mu(int j) const {
    return j < h_mu ? mu_smem(j) : __ldg(mu_g + j);
  }
  // y_j += v in fixed point.  A shared bin is a little-endian (low, high)
  // pair of 32-bit words: the low word takes a returning 32-bit atomic add,
  // its carry goes into the high word, so the 64-bit total stays exact
  // without 64-bit shared-memory atomics.  Global bins use 64-bit reductions.
  __device__ __forceinline__ void scatter(int j, float v) const {
    const long long q = to_fixed(v, sy);
    if (j < h_y) {
      const uint32_t w = y_a + 8u * j;
      if (kSmemRed64) {
        reds_add_u64(w, (unsigned long long)q);
      } else {
        const unsigned lo = (unsigned)q;
        const unsigned old = atoms_add_u32(w, lo);
        const unsigned hi = (unsigned)(q >> 32) + (old + lo < old ? 1u : 0u);
        if (hi) reds_add_u32(w + 4u, hi);
      }
    } else {
      atomicAdd(y + j, (unsigned long long)q);
    }
  }
};

template <bool W>
__device__ __forceinline__ float edge_w(float a) {
  return W ? (a != 0.f ? __fmul_rn(a, a) : 1.f) : 1.f;
}
template <bool W>
__device__ __forceinline__ float edge_alpha(const Ctx& cx, float w) {
  return W ? __frcp_rn(__fmul_rn(cx.gamma, w)) : cx.inv_gamma;
}

// Per-lane objective partials sum c x and sum w x^2 in 64-bit fixed point
// (scales 2^ec and 2^ew, chosen at create so that neither total can reach
// 2^61): each term is rounded once to the grid, and the integer adds are
// exact, so every partial, and the scalars made from them, are the same
// whichever warp or CTA took which source.
struct Sums {
  long long cx = 0, wxx = 0;
  __device__ __forceinline__ void account(const Ctx& c, int j, float cv, float a, float w,
                                          float x) {
    c.scatter(j, __fmul_rn(a, x));
    cx += to_fixed(__fmul_rn(cv, x), c.sc);
    wxx += to_fixed(__fmul_rn(w, __fmul_rn(x, x)), c.sw);
  }
  // a lone unweighted candidate: x = 1, so c x = c and w x^2 = 1 (one_w = 2^ew)
  __device__ __forceinline__ void lone(const Ctx& c, float cv) {
    cx += to_fixed(cv, c.sc);
    wxx += c.one_w;
  }
};

// Double-float (hi + lo) arithmetic for the reductions.  FP64 issues at a
// small fraction of the FP32 rate on this part, so the J-length rows and the
// block/warp trees stay in FP32 pairs and only the final scalars are FP64.
__device__ __forceinline__ void pair_add(float& h, float& l, float v) {
  const float t = __fadd_rn(h, v);
  l = __fadd_rn(l, two_sum_err(h, v, t));
  h = t;
}
__device__ __forceinline__ void pair_addp(float& h, float& l, float h2, float l2) {
  const float t = __fadd_rn(h, h2);
  l = __fadd_rn(__fadd_rn(l, l2), two_sum_err(h, h2, t));
  h = t;
}
// xor-shuffle tree over the warp (fixed order: every lane ends with the sum)
__device__ __forceinline__ void warp_pair_sum(float& h, float& l) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, h, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, l, o);
    pair_addp(h, l, h2, l2);
  }
}
__device__ __forceinline__ double pair_value(float h, float l) { return (double)h + (double)l; }
__device__ __forceinline__ double warp_dmax(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_dsum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------- group projection, registers ----
// G lanes own one source (32/G sources per warp), each lane holds up to K of
// its edges.  Every lane executes every shuffle (full mask; xor offsets stay
// inside a group).
template <int G>
__device__ __forceinline__ float group_max(float v) {
#pragma unroll
  for (int o = G / 2; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <int G>
__device__ __forceinline__ void group_sum2(float& u, float& v) {
#pragma unroll
  for (int o = G / 2; o; o >>= 1) {
    u += __shfl_xor_sync(0xffffffffu, u, o);
    v += __shfl_xor_sync(0xffffffffu, v, o);
  }
}

template <int G>
__device__ __forceinline__ int group_isum(int v) {
#pragma unroll
  for (int o = G / 2; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Four consecutive staged edges from a 16-byte-aligned stage index e.
template <bool BF16>
__device__ __forceinline__ void load4(const StageView<BF16>& sv, int e, int (&j)[4],
                                      float (&c)[4], float (&a)[4]) {
  const int4 jv = lds_s32x4(sv.dst_a + 4u * e);
  j[0] = jv.x;
  j[1] = jv.y;
  j[2] = jv.z;
  j[3] = jv.w;
  if (BF16) {
    const int4 u = lds_s32x4(sv.ca_a + 4u * e);
    const unsigned uu[4] = {(unsigned)u.x, (unsigned)u.y, (unsigned)u.z, (unsigned)u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      c[i] = __uint_as_float(uu[i] << 16);
      a[i] = __uint_as_float(uu[i] & 0xffff0000u);
    }
  } else {
    const float4 p0 = lds_f32x4(sv.ca_a + 8u * e);
    const float4 p1 = lds_f32x4(sv.ca_a + 8u * e + 16u);
    c[0] = p0.x;
    a[0] = p0.y;
    c[1] = p0.z;
    a[1] = p0.w;
    c[2] = p1.x;
    a[2] = p1.y;
    c[3] = p1.z;
    a[3] = p1.w;
  }
}

// The hot path: 32/G sources per warp, G lanes per source.  A source's edges
// are covered by a window aligned down to a multiple of 4 stage slots; each
// lane reads S runs of 4 consecutive edges with 128-bit shared loads (window
// 4 G S slots; the caller guarantees (base mod 4) + degree fits).  Plain FP32
// scores (FMA); the group reduction keeps the two largest scores (and, with
// primal scaling, the saturation sum and the weighted bound).  A saturated
// source whose second score is below the candidate bound has a single
// candidate, which takes x = 1 exactly.  Each lane passes its group's source
// as (stage slot of the first edge, degree; 0 = no source).  Returns, per
// group, whether the source is unsaturated or has near-ties at the top: those
// take the general path.
// SAFE: window slots outside the source may hold ids of another problem
// (batched pass), so they read mu of id 0 instead.
template <int G, int S, bool BF16, bool W, bool MU_SMEM, bool SAFE>
__device__ __forceinline__ bool project_lean(const StageView<BF16>& sv, int base, int d,
                                             int lane, const Ctx& cx, Sums& acc) {
  constexpr int K = 4 * S;
  const int l = lane % G;
  const bool gvalid = d > 0;
  const int ws = base & ~3;
  float rf[K];
  float m1 = -CUDART_INF_F, m2 = -CUDART_INF_F, s0 = 0.f, mb = -CUDART_INF_F;
  int kb = 0;
#pragma unroll
  for (int st = 0; st < S; ++st) {
    const int e = ws + 4 * (l + G * st);
    int jv[4];
    float cv[4], av[4];
    load4<BF16>(sv, e, jv, cv, av);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = 4 * st + i;
      const bool v = (unsigned)(e + i - base) < (unsigned)d;
      // a valid id even outside the source (see Layout), unless SAFE
      const int j = SAFE ? (v ? jv[i] : 0) : jv[i];
      const float m = MU_SMEM ? cx.mu_smem(j) : cx.mu(j);
      const float r = v ? -__fmaf_rn(av[i], m, cv[i]) : -CUDART_INF_F;
      rf[k] = r;
      if (W) {
        const float w = edge_w<W>(av[i]);
        s0 += r > 0.f ? __fmul_rn(edge_alpha<W>(cx, w), r) : 0.f;
        mb = fmaxf(mb, __fsub_rn(r, __fmul_rn(cx.gamma, w)));
      } else {
        m2 = fmaxf(m2, fminf(m1, r));
        kb = r > m1 ? k : kb;
      }
      m1 = fmaxf(m1, r);
    }
  }
  const float lm1 = m1;  // this lane's own maximum
#pragma unroll
  for (int o = G / 2; o; o >>= 1) {
    const float p1 = __shfl_xor_sync(0xffffffffu, m1, o);
    if (W) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      mb = fmaxf(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    } else {
      const float p2 = __shfl_xor_sync(0xffffffffu, m2, o);
      m2 = fmaxf(fmaxf(m2, p2), fminf(m1, p1));
    }
    m1 = fmaxf(m1, p1);
  }
  const float rmax = m1;
  int mode;
  float lb;
  bool lone = false;
  if (W) {
    mode = rmax <= 0.f ? 0 : (s0 <= 1.f ? 1 : 2);
    lb = fminf(__fsub_rn(mb, rmax), 0.f) - __fmul_rn(fabsf(rmax), 0x1p-20f);
    int lc = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (__fsub_rn(rf[k], rmax) > lb) {
        ++lc;
        kb = k;
      }
    }
    if (mode != 2) lc = 0;
    const int cnt = group_isum<G>(lc);
    lone = mode == 2 && cnt == 1;
    if (lc != 1) kb = -1;  // the owner is the lane holding the candidate
  } else {
    // rmax > gamma alone makes sum r_+ / gamma > 1: saturated.  Otherwise
    // (rare) the saturation sum decides.
    mode = rmax <= 0.f ? 0 : 2;
    if (__any_sync(0xffffffffu, gvalid && rmax > 0.f && rmax <= cx.gamma)) {
      float t0 = 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k) t0 += fmaxf(rf[k], 0.f);
#pragma unroll
      for (int o = G / 2; o; o >>= 1) t0 += __shfl_xor_sync(0xffffffffu, t0, o);
      if (rmax > 0.f && __fmul_rn(t0, cx.inv_gamma) <= 1.f) mode = 1;
    }
    lb = -cx.gamma - __fmul_rn(fabsf(rmax), 0x1p-20f);
    lone = mode == 2 && __fsub_rn(m2, rmax) <= lb;
    if (lm1 != rmax) kb = -1;  // the owner holds the group maximum
  }
  if (lone && kb >= 0) {
    // the only candidate is the only active edge: x = 1 exactly
    float c, a;
    int j;
    sv.edge(ws + 4 * (l + G * (kb >> 2)) + (kb & 3), j, c, a);
    if (W) {
      acc.account(cx, j, c, a, edge_w<W>(a), 1.f);
    } else {
      cx.scatter(j, a);
      acc.lone(cx, c);
    }
  }
  if constexpr (G == 1 && !W) {
    // One lane holds the whole source (at most 16 edges): it projects it
    // exactly on its own, as the multi-pass path would (exact pair scores
    // shifted by r_max, Michelot from the bound lb), instead of handing the
    // source to a whole warp.  (Weighted sources take the multi-pass path,
    // whose rounds are FP64.)
    if (gvalid && (mode == 1 || (mode == 2 && !lone))) {
      // rolled loops over a per-lane array (local memory): the path is rare,
      // and its code must stay small beside the hot loop's
      float dl[K];
      const int k0 = base - ws, k1 = k0 + d;
#pragma unroll 4
      for (int k = k0; k < k1; ++k) {
        int j;
        float c, a, hi, lo;
        sv.edge(ws + k, j, c, a);
        score(c, a, MU_SMEM ? cx.mu_smem(j) : cx.mu(j), hi, lo);
        dl[k] = mode == 2 ? __fadd_rn(__fsub_rn(hi, rmax), lo) : __fadd_rn(hi, lo);
      }
      float t = 0.f;
      if (mode == 2) {
        float theta = lb, nprev = -1.f;
        t = lb;
#pragma unroll 1
        for (int it = 0; it <= K; ++it) {
          float sr = 0.f, n = 0.f;
#pragma unroll 4
          for (int k = k0; k < k1; ++k) {
            if (dl[k] > theta) {
              sr += dl[k];
              n += 1.f;
            }
          }
          if (n == nprev) break;
          t = __fdiv_rn(sr - cx.gamma, n);
          nprev = n;
          theta = fmaxf(theta, t);
        }
      }
#pragma unroll 1
      for (int k = k0; k < k1; ++k) {
        const float x = mode == 2 ? (dl[k] > t ? __fmul_rn(cx.inv_gamma, __fsub_rn(dl[k], t)) : 0.f)
                                  : (dl[k] > 0.f ? __fmul_rn(cx.inv_gamma, dl[k]) : 0.f);
        if (x > 0.f) {
          int j;
          float c, a;
          sv.edge(ws + k, j, c, a);
          acc.account(cx, j, c, a, 1.f, x);
        }
      }
      return false;
    }
  }
  return gvalid && (mode == 1 || (mode == 2 && !lone));
}

// Projects the batch sources selected by `mask` (bit q = source q of the
// batch), 32/G at a time: group g takes the g-th remaining set bit.  bq / dq
// are held by lane q: the stage slot of source q's first edge and its degree.
// Returns the mask of sources that need the general path.
template <int G, int S, bool BF16, bool W, bool MU_SMEM, bool SAFE>
__device__ __forceinline__ unsigned lean_over(const StageView<BF16>& sv, unsigned mask, int bq,
                                              int dq, int lane, const Ctx& cx, Sums& acc) {
  unsigned needm = 0u;
  const int g = lane / G;
  while (mask) {
    int q;
    if ((mask & (mask + 1u)) == 0u) {  // 0...01...1: group g takes source g
      q = (mask >> g) & 1u ? g : -1;
    } else {
      unsigned m = mask;
      for (int r = 0; r < g; ++r) m &= m - 1u;
      q = m ? __ffs(m) - 1 : -1;
    }
    const int qs = q < 0 ? 0 : q;
    const int b = __shfl_sync(0xffffffffu, bq, qs);
    const int dd = __shfl_sync(0xffffffffu, dq, qs);
    const bool nd =
        project_lean<G, S, BF16, W, MU_SMEM, SAFE>(sv, b, q >= 0 ? dd : 0, lane, cx, acc);
    needm |= __reduce_or_sync(0xffffffffu, ((lane % G) == 0 && nd && q >= 0) ? (1u << q) : 0u);
#pragma unroll
    for (int r = 0; r < 32 / G; ++r) mask &= mask - 1u;
  }
  return needm;
}

// ------------------------- multi-pass projection (any degree, any group) ----
// One warp reads a staged tile or global memory; scores are recomputed on
// every pass instead of being stored.
struct WarpGroup {
  int lane;
  __device__ __forceinline__ int rank() const { return lane; }
  __device__ __forceinline__ int size() const { return 32; }
  __device__ __forceinline__ float sum(float v) const { return warp_sum(v); }
  __device__ __forceinline__ float max(float v) const { return warp_max(v); }
};
template <bool BF16, bool W, class View>
__device__ __forceinline__ void project_multipass(const View& v, int64_t base, int64_t d,
                                                  int64_t e_glob, int lane, const Ctx& cx,
                                                  Sums& acc) {
  const WarpGroup g{lane};
  auto load = [&](int64_t k, int& j, float& c, float& a, float& hi, float& lo) {
    v.edge(base + k, j, c, a);
    score(c, a, cx.mu(j), hi, lo);
  };
  // one pass: the maximum score, the saturation sum and (weighted) the
  // maximum of r - gamma w, whose shift by the maximum bounds the active set
  float rmax = -CUDART_INF_F, s0 = 0.f, mb = -CUDART_INF_F;
  for (int64_t k = g.rank(); k < d; k += g.size()) {
    int j;
    float c, a, hi, lo;
    load(k, j, c, a, hi, lo);
    const float rf = __fadd_rn(hi, lo);
    rmax = fmaxf(rmax, rf);
    if (rf > 0.f) s0 += __fmul_rn(edge_alpha<W>(cx, edge_w<W>(a)), rf);
    if (W) mb = fmaxf(mb, __fsub_rn(rf, __fmul_rn(cx.gamma, edge_w<W>(a))));
  }
  rmax = g.max(rmax);
  s0 = g.sum(s0);
  int mode = rmax <= 0.f ? 0 : (s0 <= 1.f ? 1 : 2);
  float t = 0.f;
  double td = 0.0;
  if (W && mode == 2) {
    // Weighted: x = alpha (d - t) cancels when the weights of one source
    // spread widely (an edge with a large alpha is active with d - t of order
    // 1 / alpha, far below |t|), so d, the sums, t and x are formed in FP64
    // from the exact pair; the bound is as below.
    const float slack = __fmul_rn(fabsf(rmax), 0x1p-20f);
    const double lb = (double)__fsub_rn(fminf(__fsub_rn(g.max(mb), rmax), 0.f), slack);
    double theta = lb;
    float nprev = -1.f;
    td = lb;
    for (int64_t it = 0; it <= d; ++it) {
      double sr = 0.0, sa = 0.0;
      float n = 0.f;
      for (int64_t k = g.rank(); k < d; k += g.size()) {
        int j;
        float c, a, hi, lo;
        load(k, j, c, a, hi, lo);
        const double dd = ((double)hi - (double)rmax) + (double)lo;
        if (dd > theta) {
          const double al = (double)edge_alpha<W>(cx, edge_w<W>(a));
          sr += al * dd;
          sa += al;
          n += 1.f;
        }
      }
      sr = warp_dsum(sr);
      sa = warp_dsum(sa);
      n = g.sum(n);
      if (n == nprev) break;
      td = (sr - 1.0) / sa;
      nprev = n;
      theta = theta > td ? theta : td;
    }
  } else if (mode == 2) {
    // a lower bound of max_e (d_e - gamma w_e), lowered by the FP32 rounding of
    // the scores, so that {d_e > lb} contains the active set (unweighted: the
    // top edge has d = 0, so the bound is -gamma)
    const float slack = __fmul_rn(fabsf(rmax), 0x1p-20f);
    const float lb = W ? __fsub_rn(fminf(__fsub_rn(g.max(mb), rmax), 0.f), slack)
                       : __fsub_rn(-cx.gamma, slack);
    float theta = lb, nprev = -1.f;
    t = lb;
    for (int64_t it = 0; it <= d; ++it) {
      float sr = 0.f, sa = 0.f, n = 0.f;
      for (int64_t k = g.rank(); k < d; k += g.size()) {
        int j;
        float c, a, hi, lo;
        load(k, j, c, a, hi, lo);
        const float dk = __fadd_rn(__fsub_rn(hi, rmax), lo);
        if (dk > theta) {
          const float al = edge_alpha<W>(cx, edge_w<W>(a));
          sr += W ? __fmul_rn(al, dk) : dk;
          sa += W ? al : 0.f;
          n += 1.f;
        }
      }
      sr = g.sum(sr);
      n = g.sum(n);
      if (W) sa = g.sum(sa);
      if (n == nprev) break;
      t = W ? __fdiv_rn(sr - 1.f, sa) : __fdiv_rn(sr - cx.gamma, n);
      nprev = n;
      theta = fmaxf(theta, t);
    }
  }
  for (int64_t k = g.rank(); k < d; k += g.size()) {
    int j;
    float c, a, hi, lo;
    load(k, j, c, a, hi, lo);
    const float w = edge_w<W>(a);
    const float al = edge_alpha<W>(cx, w);
    float x = 0.f;
    if (mode == 1) {
      const float rf = __fadd_rn(hi, lo);
      x = rf > 0.f ? __fmul_rn(al, rf) : 0.f;
    } else if (W && mode == 2) {
      const double dd = ((double)hi - (double)rmax) + (double)lo;
      x = dd > td ? (float)((double)al * (dd - td)) : 0.f;
    } else if (mode == 2) {
      const float dk = __fadd_rn(__fsub_rn(hi, rmax), lo);
      x = dk > t ? __fmul_rn(al, __fsub_rn(dk, t)) : 0.f;
    }
    if (x > 0.f) acc.account(cx, j, c, a, w, x);
    if (cx.x_out != nullptr) cx.x_out[e_glob + k] = x;
  }
}

// ---------------------------------------------- block class (big sources) ----
// A source larger than a stage is projected by every consumer warp of the CTA
// together, straight from global memory: each pass is strided over the
// kConsumerWarps * 32 consumer threads and ends in a block reduction.  The
// reductions combine the per-warp partials in a fixed order, so every thread
// gets the same values and the result does not depend on timing.  sm holds
// 3 floats per consumer warp; barrier 2 is the consumers' named barrier.
__device__ __forceinline__ void consumer_bar() {
  asm volatile("bar.sync 2, %0;" ::"r"(kConsumerWarps * 32) : "memory");
}
template <bool MAX0, bool MAX2>
__device__ __forceinline__ float3 block_reduce3(float a, float b, float c, float* sm, int cw,
                                                int lane) {
  a = MAX0 ? warp_max(a) : warp_sum(a);
  b = warp_sum(b);
  c = MAX2 ? warp_max(c) : warp_sum(c);
  if (lane == 0) {
    sm[3 * cw] = a;
    sm[3 * cw + 1] = b;
    sm[3 * cw + 2] = c;
  }
  consumer_bar();
  float ra = MAX0 ? -CUDART_INF_F : 0.f, rb = 0.f, rc = MAX2 ? -CUDART_INF_F : 0.f;
  for (int w = 0; w < kConsumerWarps; ++w) {
    ra = MAX0 ? fmaxf(ra, sm[3 * w]) : ra + sm[3 * w];
    rb += sm[3 * w + 1];
    rc = MAX2 ? fmaxf(rc, sm[3 * w + 2]) : rc + sm[3 * w + 2];
  }
  consumer_bar();  // sm is free again
  return make_float3(ra, rb, rc);
}

// The same in FP64 for two sums and a count (the weighted block class); smd
// holds 3 doubles per consumer warp.
__device__ __forceinline__ void block_reduce_d(double& a, double& b, float& c, double* smd, int cw,
                                               int lane) {
  a = warp_dsum(a);
  b = warp_dsum(b);
  c = warp_sum(c);
  if (lane == 0) {
    smd[3 * cw] = a;
    smd[3 * cw + 1] = b;
    smd[3 * cw + 2] = (double)c;
  }
  consumer_bar();
  double ra = 0.0, rb = 0.0, rc = 0.0;
  for (int w = 0; w < kConsumerWarps; ++w) {
    ra += smd[3 * w];
    rb += smd[3 * w + 1];
    rc += smd[3 * w + 2];
  }
  consumer_bar();  // smd is free again
  a = ra;
  b = rb;
  c = (float)rc;
}

// The projection of a source larger than a stage by every consumer thread
// ct = 0 .. NT - 1 (NT = kConsumerWarps * 32), thread ct taking edges ct,
// ct + NT, ... (a fixed assignment, so every sum is the same from run to run).
// Each pass loads kBlockUnroll edges per thread before using them.
//   pass 1: r_max, the saturation sum and max(r - gamma w) (block reductions);
//   pass 2 (sum constraint binding): each thread keeps the shifted scores d of
//     its candidate edges (d > lb, a set that holds the active set; at most
//     kBlockCand per thread) in registers; Michelot's rounds then run on the
//     registers alone, and x goes out for the candidates only.  A thread with
//     more candidates sends the source to full passes (the multi-pass
//     arithmetic) for the rounds and x;
//   unsaturated sum constraint: x = alpha r_+ on one more pass.
template <bool BF16, bool W>
__device__ __forceinline__ void project_block_body(const GlobalView<BF16>& v, int64_t base,
                                                   int64_t d, int64_t e_glob, int ct, int cw,
                                                   int lane, const Ctx& cx, Sums& acc, float* sm);
// Out of line, with its inputs by value and its objective partials returned:
// it is rare, and its registers (edges in flight, candidates) must not weigh
// on the hot loop's allocation.
template <bool BF16, bool W>
__device__ __noinline__ longlong2 project_block(const GlobalView<BF16> v, int64_t base, int64_t d,
                                                int64_t e_glob, int ct, int cw, int lane,
                                                const Ctx cx, float* sm) {
  Sums acc;
  project_block_body<BF16, W>(v, base, d, e_glob, ct, cw, lane, cx, acc, sm);
  return make_longlong2(acc.cx, acc.wxx);
}
template <bool BF16, bool W>
__device__ __forceinline__ void project_block_body(const GlobalView<BF16>& v, int64_t base,
                                                   int64_t d, int64_t e_glob, int ct, int cw,
                                                   int lane, const Ctx& cx, Sums& acc, float* sm) {
  constexpr int NT = kConsumerWarps * 32;
  constexpr int U = kBlockUnroll;
  constexpr int NC = kBlockCand;
  auto load = [&](int64_t k, int& j, float& c, float& a, float& hi, float& lo) {
    v.edge(base + k, j, c, a);
    score(c, a, cx.mu(j), hi, lo);
  };
  float rmax = -CUDART_INF_F, s0 = 0.f, mb = -CUDART_INF_F;
  for (int64_t k0 = ct; k0 < d; k0 += (int64_t)U * NT) {
    int j[U];
    float c[U], a[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {  // the loads first
      const int64_t k = k0 + (int64_t)u * NT;
      if (k < d) v.edge(base + k, j[u], c[u], a[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (k0 + (int64_t)u * NT >= d) break;
      float hi, lo;
      score(c[u], a[u], cx.mu(j[u]), hi, lo);
      const float rf = __fadd_rn(hi, lo);
      rmax = fmaxf(rmax, rf);
      if (rf > 0.f) s0 += __fmul_rn(edge_alpha<W>(cx, edge_w<W>(a[u])), rf);
      if (W) mb = fmaxf(mb, __fsub_rn(rf, __fmul_rn(cx.gamma, edge_w<W>(a[u]))));
    }
  }
  const float3 r1 = block_reduce3<true, true>(rmax, s0, mb, sm, cw, lane);
  rmax = r1.x;
  s0 = r1.y;
  const int mode = rmax <= 0.f ? 0 : (s0 <= 1.f ? 1 : 2);
  if (mode == 0 && cx.x_out == nullptr) return;  // every x is 0
  if (W && mode == 2) {
    // weighted, sum constraint binding: full passes with d, the sums, t and x
    // in FP64 (see the multi-pass path: widely spread weights cancel in FP32)
    double* smd = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(sm) + 496);
    const float slack = __fmul_rn(fabsf(rmax), 0x1p-20f);
    const double lb = (double)__fsub_rn(fminf(__fsub_rn(r1.z, rmax), 0.f), slack);
    double theta = lb, td = lb;
    float nprev = -1.f;
    for (int64_t it = 0; it <= d; ++it) {
      double sr = 0.0, sa = 0.0;
      float n = 0.f;
      for (int64_t k = ct; k < d; k += NT) {
        int j;
        float c, a, hi, lo;
        load(k, j, c, a, hi, lo);
        const double dd = ((double)hi - (double)rmax) + (double)lo;
        if (dd > theta) {
          const double al = (double)edge_alpha<W>(cx, edge_w<W>(a));
          sr += al * dd;
          sa += al;
          n += 1.f;
        }
      }
      block_reduce_d(sr, sa, n, smd, cw, lane);
      if (n == nprev) break;
      td = (sr - 1.0) / sa;
      nprev = n;
      theta = theta > td ? theta : td;
    }
    for (int64_t k = ct; k < d; k += NT) {
      int j;
      float c, a, hi, lo;
      load(k, j, c, a, hi, lo);
      const float w = edge_w<W>(a);
      const double dd = ((double)hi - (double)rmax) + (double)lo;
      const float x = dd > td ? (float)((double)edge_alpha<W>(cx, w) * (dd - td)) : 0.f;
      if (x > 0.f) acc.account(cx, j, c, a, w, x);
      if (cx.x_out != nullptr) cx.x_out[e_glob + k] = x;
    }
    return;
  }
  float t = 0.f;
  if (mode == 2) {
    const float slack = __fmul_rn(fabsf(rmax), 0x1p-20f);
    const float lb = W ? __fsub_rn(fminf(__fsub_rn(r1.z, rmax), 0.f), slack)
                       : __fsub_rn(-cx.gamma, slack);
    // pass 2: the candidates of this thread, in registers
    int64_t ck[NC];
    float cd[NC], ca[NC];
    int nc = 0;
    for (int64_t k0 = ct; k0 < d; k0 += (int64_t)U * NT) {
      int j[U];
      float c[U], a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t k = k0 + (int64_t)u * NT;
        if (k < d) v.edge(base + k, j[u], c[u], a[u]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t k = k0 + (int64_t)u * NT;
        if (k >= d) break;
        float hi, lo;
        score(c[u], a[u], cx.mu(j[u]), hi, lo);
        const float dk = __fadd_rn(__fsub_rn(hi, rmax), lo);
        if (dk > lb) {
#pragma unroll
          for (int q = 0; q < NC; ++q)
            if (q == nc) {
              ck[q] = k;
              cd[q] = dk;
              ca[q] = edge_alpha<W>(cx, edge_w<W>(a[u]));
            }
          ++nc;
        }
      }
    }
    const float3 ov = block_reduce3<true, false>(nc > NC ? 1.f : 0.f, 0.f, 0.f, sm, cw, lane);
    if (ov.x == 0.f) {
      // Michelot's rounds on the registers
      float theta = lb, nprev = -1.f;
      t = lb;
      for (int it = 0; it <= NC * NT; ++it) {
        float sr = 0.f, sa = 0.f, n = 0.f;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          if (q < nc && cd[q] > theta) {
            sr += W ? __fmul_rn(ca[q], cd[q]) : cd[q];
            sa += W ? ca[q] : 0.f;
            n += 1.f;
          }
        }
        const float3 r = block_reduce3<false, false>(sr, sa, n, sm, cw, lane);
        if (r.z == nprev) break;
        t = W ? __fdiv_rn(r.x - 1.f, r.y) : __fdiv_rn(r.x - cx.gamma, r.z);
        nprev = r.z;
        theta = fmaxf(theta, t);
      }
      // x of the candidates (every other edge has x = 0)
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        if (q < nc && cd[q] > t) {
          int j;
          float c, a;
          v.edge(base + ck[q], j, c, a);
          acc.account(cx, j, c, a, edge_w<W>(a), __fmul_rn(ca[q], __fsub_rn(cd[q], t)));
        }
      }
      if (cx.x_out != nullptr) {
        for (int64_t k = ct; k < d; k += NT) {
          float x = 0.f;
#pragma unroll
          for (int q = 0; q < NC; ++q)
            if (q < nc && ck[q] == k && cd[q] > t) x = __fmul_rn(ca[q], __fsub_rn(cd[q], t));
          cx.x_out[e_glob + k] = x;
        }
      }
      return;
    }
    // too many candidates on some thread: full passes
    float theta = lb, nprev = -1.f;
    t = lb;
    for (int64_t it = 0; it <= d; ++it) {
      float sr = 0.f, sa = 0.f, n = 0.f;
      for (int64_t k = ct; k < d; k += NT) {
        int j;
        float c, a, hi, lo;
        load(k, j, c, a, hi, lo);
        const float dk = __fadd_rn(__fsub_rn(hi, rmax), lo);
        if (dk > theta) {
          const float al = edge_alpha<W>(cx, edge_w<W>(a));
          sr += W ? __fmul_rn(al, dk) : dk;
          sa += W ? al : 0.f;
          n += 1.f;
        }
      }
      const float3 r = block_reduce3<false, false>(sr, sa, n, sm, cw, lane);
      if (r.z == nprev) break;
      t = W ? __fdiv_rn(r.x - 1.f, r.y) : __fdiv_rn(r.x - cx.gamma, r.z);
      nprev = r.z;
      theta = fmaxf(theta, t);
    }
  }
  for (int64_t k = ct; k < d; k += NT) {
    int j;
    float c, a, hi, lo;
    load(k, j, c, a, hi, lo);
    const float w = edge_w<W>(a);
    const float al = edge_alpha<W>(cx, w);
    float x = 0.f;
    if (mode == 1) {
      const float rf = __fadd_rn(hi, lo);
      x = rf > 0.f ? __fmul_rn(al, rf) : 0.f;
    } else if (mode == 2) {
      const float dk = __fadd_rn(__fsub_rn(hi, rmax), lo);
      x = dk > t ? __fmul_rn(al, __fsub_rn(dk, t)) : 0.f;
    }
    if (x > 0.f) acc.account(cx, j, c, a, w, x);
    if (cx.x_out != nullptr) cx.x_out[e_glob + k] = x;
  }
}

// Unweighted sources of at most 512 edges that the lane groups leave
// (unsaturated, or several edges within gamma of the top).  One pass over the
// staged source keeps each lane's FP32 scores r = -(c + a mu) (which equal the
// high word of the exact pair) in registers and finds r_max and the saturation
// sum.  The candidate edges, r > 0 when the sum constraint is slack and
// r - r_max > lb otherwise (a set that holds the active set), are marked in a
// bit mask, and only they are revisited: Michelot's rounds recompute their
// exact shifted scores d = (hi - r_max) + lo, as the multi-pass path does,
// and x = (d - t) / gamma goes out.  Near-ties have two or three candidates,
// so the rounds cost little, and the code exists once, keeping the kernel's
// instruction footprint small.  Returns false, having accounted nothing, if
// the rounds have not settled after kCandRounds (the multi-pass path then
// projects the source).
template <bool BF16, bool MU_SMEM, int K = 16>  // K: edges per lane (spans up to 32 K)
__device__ __forceinline__ bool project_warp_cand(const StageView<BF16>& sv, int base, int d,
                                                  int lane, const Ctx& cx, Sums& acc) {
  float rf[K];
  float rmax = -CUDART_INF_F, s0 = 0.f;
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const int k = lane + 32 * i;
    float r = -CUDART_INF_F;
    if (k < d) {
      int j;
      float c, a;
      sv.edge(base + k, j, c, a);
      r = -__fmaf_rn(a, MU_SMEM ? cx.mu_smem(j) : cx.mu(j), c);
    }
    rf[i] = r;
    rmax = fmaxf(rmax, r);
    s0 += fmaxf(r, 0.f);
  }
  rmax = warp_max(rmax);
  s0 = warp_sum(s0);
  const int mode = rmax <= 0.f ? 0 : (__fmul_rn(s0, cx.inv_gamma) <= 1.f ? 1 : 2);
  if (mode == 0) return true;  // every x is 0
  const float lb = __fsub_rn(-cx.gamma, __fmul_rn(fabsf(rmax), 0x1p-20f));
  unsigned cm = 0u;
#pragma unroll
  for (int i = 0; i < K; ++i)
    cm |= (mode == 1 ? rf[i] > 0.f : __fsub_rn(rf[i], rmax) > lb) ? (1u << i) : 0u;
  auto shifted = [&](int k, int& j, float& c, float& a) {
    float hi, lo;
    sv.edge(base + k, j, c, a);
    score(c, a, MU_SMEM ? cx.mu_smem(j) : cx.mu(j), hi, lo);
    return __fadd_rn(__fsub_rn(hi, rmax), lo);
  };
  float t = 0.f;
  if (mode == 2) {
    float theta = lb, nprev = -1.f;
    bool settled = false;
    for (int it = 0; it < kCandRounds; ++it) {
      float sr = 0.f, n = 0.f;
      for (unsigned m = cm; m; m &= m - 1u) {
        int j;
        float c, a;
        const float dk = shifted(lane + 32 * (__ffs(m) - 1), j, c, a);
        if (dk > theta) {
          sr += dk;
          n += 1.f;
        }
      }
      sr = warp_sum(sr);
      n = warp_sum(n);
      if (n == nprev) {
        settled = true;
        break;
      }
      t = __fdiv_rn(sr - cx.gamma, n);
      nprev = n;
      theta = fmaxf(theta, t);
    }
    if (!settled) return false;
  }
  for (unsigned m = cm; m; m &= m - 1u) {
    const int k = lane + 32 * (__ffs(m) - 1);
    int j;
    float c, a, x;
    if (mode == 1) {
      sv.edge(base + k, j, c, a);
      const float r = -__fmaf_rn(a, MU_SMEM ? cx.mu_smem(j) : cx.mu(j), c);
      x = __fmul_rn(cx.inv_gamma, r);  // r > 0 for a candidate
    } else {
      const float dk = shifted(k, j, c, a);
      x = dk > t ? __fmul_rn(cx.inv_gamma, __fsub_rn(dk, t)) : 0.f;
    }
    if (x > 0.f) acc.account(cx, j, c, a, 1.f, x);
  }
  return true;
}

// The unit-box projection (Section 6's clamp map, x_e in [0, 1] with no sum
// constraint): the block problem separates by edge, and its minimiser is
// x = clamp(alpha r, 0, 1), alpha = 1 / (gamma w), r = -(c + a mu) formed by one
// FMA (a single rounding), so x carries FP32 accuracy.  Edges [e0, e1) of the
// view, edge e0 + first + k stride for k = 0, 1, ...; x_out (WX) at
// e_glob0 + (k - e0).
template <bool BF16, bool W, bool WX, class View>
__device__ __forceinline__ void project_box(const View& v, int64_t e0, int64_t e1,
                                            int64_t e_glob0, int first, int stride, const Ctx& cx,
                                            Sums& acc) {
  for (int64_t k = e0 + first; k < e1; k += stride) {
    int j;
    float c, a;
    v.edge(k, j, c, a);
    const float r = -__fmaf_rn(a, cx.mu(j), c);
    const float w = edge_w<W>(a);
    const float x = fminf(fmaxf(__fmul_rn(edge_alpha<W>(cx, w), r), 0.f), 1.f);
    if (x > 0.f) acc.account(cx, j, c, a, w, x);
    if (WX) cx.x_out[e_glob0 + (k - e0)] = x;
  }
}

// J-length epilogue rows: (A x)_j from the fixed-point accumulator (which is
// reset to zero for the next evaluation), grad = D (A x - b) in the caller's
// numbering, and the partials lambda^T (A x - b) and ||(A x - b)_+||^2 as FP32
// pairs.  The accumulator converts exactly to a pair (its high part is an
// integer-valued float, the remainder fits 40 bits) and the scale is a power of
// two, so g = A x - b is formed with one rounding in its low word.
struct EpiAcc {
  float mh = 0.f, ml = 0.f;  // lambda^T g
  float nh = 0.f, nl = 0.f;  // ||g_+||^2
};
__device__ __forceinline__ void epi_rows(const EpiParams& q, int64_t j0, int64_t stride,
                                         EpiAcc& r) {
  // eight rows per round, every load issued before any use
  constexpr int U = 8;
  for (int64_t r0 = j0; r0 < q.J; r0 += U * stride) {
    long long yv[U];
    float bv[U], mv[U], dv[U];
    int jo[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t jr = r0 + u * stride;
      const int64_t jc = jr < q.J ? jr : 0;
      yv[u] = (long long)__ldcg(q.y + jc);
      bv[u] = q.b_r[jc];
      mv[u] = q.mu_r[jc];
      jo[u] = q.orig_of ? q.orig_of[jc] : (int)jc;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) dv[u] = q.D ? q.D[jo[u]] : 1.f;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t jr = r0 + u * stride;
      if (jr >= q.J) continue;
      q.y[jr] = 0ull;
      const float fh = __ll2float_rn(yv[u]);
      const float fl = __ll2float_rn(yv[u] - __float2ll_rn(fh));
      const float ah = __fmul_rn(fh, q.sy), al = __fmul_rn(fl, q.sy);
      const float t = __fsub_rn(ah, bv[u]);
      const float e = __fadd_rn(two_sum_err(ah, -bv[u], t), al);
      const float g = __fadd_rn(t, e);
      const float gl = two_sum_err(t, e, g);
      const float m = mv[u];
      const float pm = __fmul_rn(m, g);
      pair_add(r.mh, r.ml, pm);
      r.ml = __fadd_rn(r.ml, __fmaf_rn(m, gl, __fmaf_rn(m, g, -pm)));
      if (g > 0.f) {
        const float sq = __fmul_rn(g, g);
        pair_add(r.nh, r.nl, sq);
        r.nl = __fadd_rn(r.nl, __fmaf_rn(2.f * g, gl, __fmaf_rn(g, g, -sq)));
      }
      q.grad[jo[u]] = q.D ? __fmaf_rn(dv[u], g, __fmul_rn(dv[u], gl)) : __fadd_rn(g, gl);
    }
  }
}
__device__ __forceinline__ void epi_write(const EpiParams& q, double cxs, double wxx, double mug,
                                          double inf) {
  const double gamma = q.gamma_dev ? (double)*q.gamma_dev : q.gamma;
  const double reg = 0.5 * gamma * wxx;
  q.eval_out[0] = cxs + reg + mug;
  q.eval_out[1] = cxs;
  q.eval_out[2] = reg;
  q.eval_out[3] = sqrt(inf);
  q.eval_out[4] = mug;
}

__device__ __forceinline__ long long warp_isum64(long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// A warp's objective partials of one problem, added to its slot's fixed-point
// sums (batched pass; two integer atomics per warp and slot, exact in any order).
__device__ __forceinline__ void flush_sums(const Sums& acc, long long* dst, int lane) {
  const long long c = warp_isum64(acc.cx), w = warp_isum64(acc.wxx);
  if (lane == 0) {
    if (c) atomicAdd(reinterpret_cast<unsigned long long*>(dst), (unsigned long long)c);
    if (w) atomicAdd(reinterpret_cast<unsigned long long*>(dst) + 1, (unsigned long long)w);
  }
}

// ------------------------------------- multi-block class (hub sources) ----
// A source of at least mb_min edges is projected by the whole grid before the
// pass (whose producer skips its tile).  Its edges are cut into chunks of
// kHubChunk, each CTA takes a contiguous range of chunks, and each warp of it
// a unit of kHubUnit edges of the chunk.  Reading its unit once, a warp
//   * finds the unit's r_max, saturation sum s0 = sum_{r > 0} alpha r and
//     m_u = max (r - gamma w);
//   * appends the unit's candidates (hi, lo, alpha, k) to the source's list:
//     the edges with r > m_u less a rounding margin.  With the sum constraint
//     binding, every active edge has r_e > tau* >= r - gamma w for every edge
//     of the source (x <= 1 in Eq. 5), so r_e > m_u; where the unit alone
//     leaves the constraint slack, every r > 0 joins (the whole source may be
//     slack, and then every edge with r > 0 is active).
// Warps never wait for one another inside a source.  At the end of its run of
// a source's chunks a CTA takes a ticket for them; the CTA whose ticket
// completes the source combines the unit statistics in unit order, runs
// Michelot's rounds on the candidate list and accounts x for the active edges.
// The rounds' sums are 64-bit fixed point, exact in any order, so the result
// does not depend on the order in which the warps appended their candidates.
// No CTA waits for another.
constexpr int kHubWarps = kHubThreads / 32;
constexpr int kHubUnit = kHubChunk / kHubWarps;  // edges of a warp's unit
constexpr int kHubU = kHubUnit / 32;             // edges per lane
constexpr int kHubCtasPerSm = 2;                 // resident hub CTAs per SM (registers, staging)
static_assert(kHubU * 32 * kHubWarps == kHubChunk, "a chunk is one unit per warp");

struct HubParams {
  const int32_t* dst;
  const float2* ca2;
  const uint32_t* ca;
  const float* mu_r;
  const float* gamma_dev;
  float gamma;
  unsigned long long* y;
  int ey, ec, ew;
  float* x_out;
  const HubDesc* hubs;
  const int32_t* chunk_hub;
  int64_t nchunks;
  HubUnitStat* stat;  // [nchunks * kHubWarps]
  float4* cand;
  unsigned* cnt;    // [2 nhub]: candidates appended, chunks completed
  longlong2* part;  // [nhub] fixed-point objective partials
  DeviceStatus* status;
};

// Shared scratch of the solve's fixed-order block reductions.
struct HubRed {
  float f[2][kHubWarps];
  double d[kHubWarps], e[kHubWarps];
  long long q[3][kHubWarps];
  int last;
};

// Scale exponent s with n * m * 2^s < 2^61: n terms of magnitude at most m
// then sum exactly in a 64-bit integer.
__device__ __forceinline__ int hub_fixed_exp(unsigned n, double m) {
  if (n == 0u || !(m > 0.0)) return 0;
  int ex;
  frexp((double)n * m, &ex);
  const int s = 61 - ex;
  return s > 100 ? 100 : (s < -100 ? -100 : s);
}

template <bool BF16, bool W, bool WX>
__device__ __noinline__ void hub_solve(const HubParams& p, int h, const HubDesc hd, const Ctx& cx,
                                       HubRed& r) {
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const GlobalView<BF16> gv{p.dst, p.ca2, p.ca};
  // the unit statistics, in unit order
  float rmax = -CUDART_INF_F, mb = -CUDART_INF_F;
  double s0 = 0.0;
  const int nu = hd.nch * kHubWarps;
  const HubUnitStat* st = p.stat + (int64_t)hd.c0 * kHubWarps;
  for (int q = tid; q < nu; q += kHubThreads) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(st + q));
    const long long bits = __double_as_longlong(v.y);
    rmax = fmaxf(rmax, __int_as_float((int)(bits & 0xffffffffll)));
    mb = fmaxf(mb, __int_as_float((int)(bits >> 32)));
    s0 += v.x;
  }
  rmax = warp_max(rmax);
  mb = warp_max(mb);
  s0 = warp_dsum(s0);
  if (lane == 0) {
    r.f[0][w] = rmax;
    r.f[1][w] = mb;
    r.d[w] = s0;
  }
  __syncthreads();
  rmax = r.f[0][0];
  mb = r.f[1][0];
  s0 = r.d[0];
  for (int k = 1; k < kHubWarps; ++k) {
    rmax = fmaxf(rmax, r.f[0][k]);
    mb = fmaxf(mb, r.f[1][k]);
    s0 += r.d[k];
  }
  __syncthreads();
  const unsigned N = __ldcg(p.cnt + 2 * h);
  const float4* L = p.cand + hd.cand0;
  const int mode = rmax <= 0.f ? 0 : (s0 <= 1.0 ? 1 : 2);
  // Shifted scores d = (hi - r_max) + lo, as in the block class: FP32 for
  // unweighted sources, FP64 with primal scaling (widely spread weights make
  // x = alpha (d - t) cancel in FP32; see the multi-pass path).
  auto shifted = [&](const float4& v) -> double {
    return W ? ((double)v.x - (double)rmax) + (double)v.y
             : (double)__fadd_rn(__fsub_rn(v.x, rmax), v.y);
  };
  double t = 0.0;
  if (mode == 2) {
    // a lower bound of the threshold lowered by the FP32 rounding of the scores
    const float slack = __fmul_rn(fabsf(rmax), 0x1p-20f);
    const double lb = W ? (double)__fsub_rn(fminf(__fsub_rn(mb, rmax), 0.f), slack)
                        : (double)__fsub_rn(-cx.gamma, slack);
    // magnitudes of the summed terms, for the fixed-point scales
    double m1 = 0.0, m2 = 0.0;
    for (unsigned q = tid; q < N; q += kHubThreads) {
      const float4 v = __ldcg(L + q);
      const double dk = shifted(v);
      if (dk > lb) {
        m1 = fmax(m1, fabs(W ? (double)v.z * dk : dk));
        m2 = fmax(m2, (double)v.z);
      }
    }
    m1 = warp_dmax(m1);
    m2 = warp_dmax(m2);
    if (lane == 0) {
      r.d[w] = m1;
      r.e[w] = m2;
    }
    __syncthreads();
    m1 = r.d[0];
    m2 = r.e[0];
    for (int k = 1; k < kHubWarps; ++k) {
      m1 = fmax(m1, r.d[k]);
      m2 = fmax(m2, r.e[k]);
    }
    __syncthreads();
    const int s1 = hub_fixed_exp(N, m1), s2 = hub_fixed_exp(N, m2);
    double theta = lb;
    long long nprev = -1;
    t = lb;
    for (unsigned it = 0; it <= N; ++it) {
      long long sa = 0, sb = 0, nn = 0;
      for (unsigned q = tid; q < N; q += kHubThreads) {
        const float4 v = __ldcg(L + q);
        const double dk = shifted(v);
        if (dk > theta) {
          sa += __double2ll_rn(ldexp(W ? (double)v.z * dk : dk, s1));
          if (W) sb += __double2ll_rn(ldexp((double)v.z, s2));
          ++nn;
        }
      }
      sa = warp_isum64(sa);
      sb = warp_isum64(sb);
      nn = warp_isum64(nn);
      if (lane == 0) {
        r.q[0][w] = sa;
        r.q[1][w] = sb;
        r.q[2][w] = nn;
      }
      __syncthreads();
      sa = sb = nn = 0;
      for (int k = 0; k < kHubWarps; ++k) {
        sa += r.q[0][k];
        sb += r.q[1][k];
        nn += r.q[2][k];
      }
      __syncthreads();
      if (nn == nprev || nn == 0) break;
      const double A = ldexp((double)sa, -s1);
      const double tt = W ? (A - 1.0) / ldexp((double)sb, -s2)
                          : (A - (double)cx.gamma) / (double)nn;
      // unweighted: the threshold in FP32, as the other classes take it
      t = W ? tt : (double)(float)tt;
      nprev = nn;
      theta = theta > t ? theta : t;
    }
  }
  // x of the candidates (every other edge of the source has x = 0)
  Sums acc;
  for (unsigned q = tid; q < N; q += kHubThreads) {
    const float4 v = __ldcg(L + q);
    const int64_t e = hd.e0 + __float_as_int(v.w);
    float x = 0.f;
    if (mode == 1) {
      const float rf = __fadd_rn(v.x, v.y);
      x = rf > 0.f ? __fmul_rn(v.z, rf) : 0.f;
    } else if (mode == 2) {
      const double dk = shifted(v);
      if (dk > t)
        x = W ? (float)((double)v.z * (dk - t))
              : __fmul_rn(v.z, __fsub_rn((float)dk, (float)t));
    }
    if (x > 0.f) {
      int j;
      float c, a;
      gv.edge(e, j, c, a);
      acc.account(cx, j, c, a, edge_w<W>(a), x);
    }
    if (WX) p.x_out[e] = x;
  }
  const long long cs = warp_isum64(acc.cx), ws = warp_isum64(acc.wxx);
  if (lane == 0) {
    r.q[0][w] = cs;
    r.q[1][w] = ws;
  }
  __syncthreads();
  if (tid == 0) {
    longlong2 tot = make_longlong2(0, 0);
    for (int k = 0; k < kHubWarps; ++k) {
      tot.x += r.q[0][k];
      tot.y += r.q[1][k];
    }
    p.part[h] = tot;
    // rewind the source's counters for the next evaluation
    p.cnt[2 * h] = 0u;
    p.cnt[2 * h + 1] = 0u;
  }
  __syncthreads();
}

template <bool BF16, bool W, bool WX>
__global__ void __launch_bounds__(kHubThreads, kHubCtasPerSm) hub_kernel(HubParams p) {
  __shared__ HubRed r;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  Ctx cx;
  cx.mu_a = 0u;
  cx.mu_g = p.mu_r;
  cx.h_mu = 0;  // no shared caches: mu and A x go through L2
  cx.y_a = 0u;
  cx.h_y = 0;
  cx.y = p.y;
  cx.sy = ldexpf(1.f, p.ey);
  cx.sc = ldexpf(1.f, p.ec);
  cx.sw = ldexpf(1.f, p.ew);
  cx.one_w = p.ew >= 0 && p.ew <= 62 ? (1ll << p.ew) : 0ll;
  cx.x_out = WX ? p.x_out : nullptr;
  cx.dst_g = p.dst;
  cx.ca2_g = p.ca2;
  cx.ca_g = p.ca;
  const GlobalView<BF16> gv{p.dst, p.ca2, p.ca};
  const int64_t c_begin = (int64_t)blockIdx.x * p.nchunks / gridDim.x;
  const int64_t c_end = (int64_t)(blockIdx.x + 1) * p.nchunks / gridDim.x;
  pdl_wait();  // mu of this evaluation; A x rewound by the last epilogue
  pdl_trigger();
  cx.gamma = p.gamma_dev ? *p.gamma_dev : p.gamma;
  cx.inv_gamma = __frcp_rn(cx.gamma);
  unsigned run = 0u;  // chunks of the current source since the last ticket
  int h = c_begin < c_end ? __ldg(p.chunk_hub + c_begin) : 0;
  HubDesc hd = p.hubs[h];
  for (int64_t c = c_begin; c < c_end; ++c) {
    const int k0 = (int)(c - hd.c0) * kHubChunk + w * kHubUnit;  // this warp's unit
    const int n = hd.deg - k0 < 0 ? 0 : (hd.deg - k0 < kHubUnit ? hd.deg - k0 : kHubUnit);
    const int64_t eb = hd.e0 + k0;
    // r = -(c + a mu) rounded once (one FMA): the high word of the exact pair
    // that the candidates carry
    float rr[kHubU], mv[kHubU];
    float rmax = -CUDART_INF_F, mb = -CUDART_INF_F, s0 = 0.f;
    {
      int j[kHubU];
      float cv[kHubU], av[kHubU];
#pragma unroll
      for (int u = 0; u < kHubU; ++u) {  // the loads first
        const int k = u * 32 + lane;
        j[u] = 0;
        cv[u] = av[u] = 0.f;
        if (k < n) gv.edge(eb + k, j[u], cv[u], av[u]);
      }
#pragma unroll
      for (int u = 0; u < kHubU; ++u) mv[u] = __ldg(p.mu_r + j[u]);  // every gather in flight
#pragma unroll
      for (int u = 0; u < kHubU; ++u) {
        const float rv = -__fmaf_rn(av[u], mv[u], cv[u]);
        const bool in = u * 32 + lane < n;
        rr[u] = in ? rv : -CUDART_INF_F;
        if (in) {
          rmax = fmaxf(rmax, rv);
          if (W) {
            // the saturation sum only sorts units into slack and saturated
            // (the projection is continuous where the two meet), so alpha r
            // may be rounded loosely here
            const float gw = __fmul_rn(cx.gamma, edge_w<W>(av[u]));
            if (rv > 0.f) s0 += __fdividef(rv, gw);
            mb = fmaxf(mb, __fsub_rn(rv, gw));
          } else {
            s0 += fmaxf(rv, 0.f);
          }
        }
      }
    }
    rmax = warp_max(rmax);
    mb = W ? warp_max(mb) : __fsub_rn(rmax, cx.gamma);
    s0 = warp_sum(s0);
    if (!W) s0 = __fmul_rn(s0, cx.inv_gamma);
    // candidate threshold: m_u less a margin that covers the rounding of the
    // FP32 scores and of m_u itself (both below 2^-21 (|r_max| + |m_u|));
    // every r > 0 joins where the unit alone leaves the constraint slack
    float thr = __fsub_rn(mb, __fmul_rn(__fadd_rn(fabsf(rmax), fabsf(mb)), 0x1p-19f));
    if (!(s0 > 1.f)) thr = fminf(thr, 0.f);
    unsigned total = 0u;
    unsigned bal[kHubU];
#pragma unroll
    for (int u = 0; u < kHubU; ++u) {
      bal[u] = __ballot_sync(0xffffffffu, rr[u] > thr);
      total += __popc(bal[u]);
    }
    unsigned base = 0u;
    if (lane == 0 && total) base = atomicAdd(p.cnt + 2 * h, total);
    base = __shfl_sync(0xffffffffu, base, 0);
    const bool fits = (uint64_t)base + total <= (uint64_t)hd.deg;
    if (lane == 0 && !fits) atomicOr(&p.status->err, kErrBounds);
    // candidate u of this lane goes after every candidate of u' < u, then the
    // lanes below it; it carries the exact score pair and alpha
    unsigned pos = base;
#pragma unroll
    for (int u = 0; u < kHubU; ++u) {
      const int k = u * 32 + lane;
      if ((bal[u] >> lane) & 1u) {
        const unsigned q = pos + __popc(bal[u] & ((1u << lane) - 1u));
        int j;
        float cv, av, hi, lo;
        gv.edge(eb + k, j, cv, av);
        score(cv, av, mv[u], hi, lo);
        const float al = edge_alpha<W>(cx, edge_w<W>(av));
        if (fits) p.cand[hd.cand0 + q] = make_float4(hi, lo, al, __int_as_float(k0 + k));
      } else if (WX && k < n) {
        p.x_out[eb + k] = 0.f;
      }
      pos += __popc(bal[u]);
    }
    if (lane == 0) {
      HubUnitStat su;
      su.s0 = (double)s0;
      su.rmax = rmax;
      su.mb = mb;
      p.stat[c * kHubWarps + w] = su;
    }
    ++run;
    // the end of this CTA's run of the source: a ticket for its chunks; the
    // ticket that completes the source projects it
    const int hn = c + 1 < c_end ? __ldg(p.chunk_hub + c + 1) : -1;
    if (hn != h) {
      __syncthreads();  // every warp's candidates and statistics of the run are written
      if (tid == 0) {
        __threadfence();
        r.last = atomicAdd(p.cnt + 2 * h + 1, run) + run == (unsigned)hd.nch;
      }
      __syncthreads();
      if (r.last) {
        __threadfence();
        hub_solve<BF16, W, WX>(p, h, hd, cx, r);
      }
      run = 0u;
      h = hn;
      if (hn >= 0) hd = p.hubs[hn];
    }
  }
}

// ----------------------------------------------------------- the pass ----
// MU_SMEM: every destination's mu is cached in shared memory (J <= the cache).
// WRITE_X: the primal x is written for every edge (dualip_get_primal); every
// source then takes the general path.
// BATCH: the tiles come from a joint list over several problems (slots).  At
// a tile of another slot the consumer warps meet at a shared barrier, flush
// the previous slot's shared bins and objective partials, load the new slot's
// mu cache, and meet again; the producer never waits for them there.
// BIG: the problem has sources larger than a stage, which the block class
// projects (its call lives only in these instances and in the WRITE_X ones,
// so the other instances keep the hot loop's registers to themselves).
template <bool BF16, bool W, bool MU_SMEM, bool WRITE_X, bool BATCH, bool BOX = false,
          bool TINY = false, bool BIG = false>
__global__ void __launch_bounds__(kThreads, 1) dualgrad_pass_kernel(PassParams p) {
  using L = Layout<BF16>;
  extern __shared__ __align__(128) unsigned char smem[];
  float* mu_s = reinterpret_cast<float*>(smem + L::kMu);
  unsigned long long* y_s = reinterpret_cast<unsigned long long*>(smem + L::kY);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::kBars);
  uint64_t* empty = full + kStages;
  uint64_t* cbar = empty + kStages;  // consumer-only barriers (slot switch)
  StageInfo* info = reinterpret_cast<StageInfo*>(smem + L::kInfo);
  volatile int* abort = reinterpret_cast<volatile int*>(smem + L::kMisc);
  // [kMisc+16, kMisc+320): per-warp reduction slots (float4)
  float* dred = reinterpret_cast<float*>(smem + L::kMisc + 16);
  // per-stage batch claim counters (reset by the producer when it refills)
  unsigned* claim = reinterpret_cast<unsigned*>(smem + L::kMisc + 320);

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int64_t t_begin = (int64_t)blockIdx.x * p.ntiles / gridDim.x;
  const int64_t t_end = (int64_t)(blockIdx.x + 1) * p.ntiles / gridDim.x;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
      claim[s] = 0u;
    }
    if (BATCH) {
      mbar_init(&cbar[0], kConsumerWarps);
      mbar_init(&cbar[1], kConsumerWarps);
    }
    *abort = 0;
    fence_mbar_init();
  }
  for (int s = 0; s < kStages; ++s) {
    uint32_t* d = reinterpret_cast<uint32_t*>(smem + (size_t)s * L::kStageBytes + L::kOffBytes);
    for (int k = tid; k < (int)(L::kDstArr / 4); k += blockDim.x) d[k] = 0u;
  }
  __syncthreads();

  Ctx cx;
  Sums acc;
  cx.mu_a = smem_u32(mu_s);
  cx.y_a = smem_u32(y_s);
  cx.x_out = WRITE_X ? p.x_out : nullptr;
  if (!BATCH) {
    cx.mu_g = p.mu_r;
    cx.h_mu = p.h_mu;
    cx.h_y = p.h_y;
    cx.y = p.y;
    cx.sy = ldexpf(1.f, p.ey);
    cx.sc = ldexpf(1.f, p.ec);
    cx.sw = ldexpf(1.f, p.ew);
    cx.one_w = p.ew >= 0 && p.ew <= 62 ? (1ll << p.ew) : 0ll;
    cx.gamma = p.gamma_dev ? *p.gamma_dev : p.gamma;
    cx.inv_gamma = __frcp_rn(cx.gamma);
    cx.dst_g = p.dst;
    cx.ca2_g = p.ca2;
    cx.ca_g = p.ca;
  } else {  // set at the first tile (slot switch)
    cx.mu_g = nullptr;
    cx.h_mu = 0;
    cx.h_y = 0;
    cx.y = nullptr;
    cx.sy = 1.f;
    cx.sc = 1.f;
    cx.sw = 1.f;
    cx.one_w = 0ll;
    cx.gamma = 1.f;
    cx.inv_gamma = 1.f;
    cx.dst_g = nullptr;
    cx.ca2_g = nullptr;
    cx.ca_g = nullptr;
  }
  int cur = -1;  // batched pass: the slot of the consumers' current tile

  if (warp == 0) {
    // ------------------------------------------------------ producer ----
    // The warp fetches tile descriptors a group at a time; lane 0 waits and
    // issues the copies.
    int64_t it = 0;
    bool stop = false;
    int pslot = -1;  // batched pass: slot of the edge pointers below
    const uint32_t* offp = p.off;
    const int32_t* dstp = p.dst;
    const float2* ca2p = p.ca2;
    const uint32_t* cap = p.ca;
    // Lane 0 stages one tile (or, with done, the end marker) into the next
    // ring slot once every consumer has left the slot's previous tile, and
    // counts it in `it` (so the drain below waits only for armed stages).
    auto stage = [&](int64_t s0, int64_t s1, int64_t e0, int64_t e1, int slot, bool done) {
      if (lane != 0) return;
      if (BATCH && slot != pslot) {
        const SlotDesc* d = p.slots + slot;
        offp = d->off;
        dstp = d->dst;
        ca2p = d->ca2;
        cap = d->ca;
        pslot = slot;
      }
      const int s = (int)(it % kStages);
      const uint32_t round = (uint32_t)(it / kStages);
      if (round > 0 && !wait_phase(&empty[s], (round - 1) & 1u, abort, p.status, 1)) {
        stop = true;
        return;
      }
      claim[s] = 0u;  // every consumer has left this stage's last tile
      StageInfo si;
      si.s0 = s0;
      si.s1 = s1;
      si.e0 = e0;
      si.e1 = e1;
      const bool bad = !done && (s1 - s0 > kTileSources || s1 < s0 || e1 < e0 ||
                                 (e1 - e0 > L::kTile && s1 - s0 != 1));
      if (bad) {
        atomicOr(&p.status->err, kErrBounds);
        si.s1 = s0;  // skip the tile; results are flagged invalid
      }
      // a hub source: the multi-block class has projected it before the pass
      const bool hub = !done && !bad && e1 - e0 >= p.mb_min;
      if (hub) si.s1 = s0;
      si.big = done ? 2 : ((!bad && !hub && e1 - e0 > L::kTile) ? 1 : 0);
      si.slot = slot;
      si.a0 = e0 & ~int64_t(3);
      si.o0 = s0 & ~int64_t(3);
      info[s] = si;
      ++it;
      if (bad || hub || si.big) {
        mbar_arrive(&full[s]);
        return;
      }
      const int64_t a1 = (e1 + 3) & ~int64_t(3);
      const int64_t o1 = (s1 + 4) & ~int64_t(3);
      const uint32_t ne = (uint32_t)(a1 - si.a0), no = (uint32_t)(o1 - si.o0);
      const uint32_t bytes = no * 4u + ne * (BF16 ? 8u : 12u);
      mbar_arrive_expect_tx(&full[s], bytes);
      unsigned char* base = smem + (size_t)s * L::kStageBytes;
      bulk_g2s(base, offp + si.o0, no * 4u, &full[s]);
      if (ne) {
        bulk_g2s(base + L::kOffBytes, dstp + si.a0, ne * 4u, &full[s]);
        if (BF16) {
          bulk_g2s(base + L::kOffBytes + L::kDstArr, cap + si.a0, ne * 4u, &full[s]);
        } else {
          bulk_g2s(base + L::kOffBytes + L::kDstArr, ca2p + si.a0, ne * 8u, &full[s]);
        }
      }
    };
    // A host-set abort request (fault injection) stops the staging; it is
    // read once per group of descriptors, next to them.
    auto injected_abort = [&](int flag) {
      if (!__any_sync(0xffffffffu, flag != 0)) return false;
      if (lane == 0) {
        *abort = 1;
        atomicOr(&p.status->err, kErrTimeout);
        atomicCAS(&p.status->where, 0, 6);
      }
      stop = true;
      return true;
    };
    if (BATCH) {
      // a contiguous range of the joint list (slot switches stay rare)
      for (int64_t t0 = t_begin; t0 < t_end && !stop; t0 += 32) {
        const JointTile jt = p.jt[t0 + lane < t_end ? t0 + lane : t_end - 1];
        const int ab = lane == 31 ? *reinterpret_cast<volatile int*>(&p.status->abort_req) : 0;
        if (injected_abort(ab)) break;
        const int cnt = (int)(t_end - t0 < 32 ? t_end - t0 : 32);
        for (int k = 0; k < cnt; ++k) {
          const int64_t s0 = __shfl_sync(0xffffffffu, jt.s0, k);
          const int64_t e0 = __shfl_sync(0xffffffffu, jt.e0, k);
          const int64_t s1 = __shfl_sync(0xffffffffu, jt.s1, k);
          const int64_t e1 = __shfl_sync(0xffffffffu, jt.e1, k);
          const int slot = __shfl_sync(0xffffffffu, jt.slot, k);
          stage(s0, s1, e0, e1, slot, false);
          stop = __shfl_sync(0xffffffffu, stop ? 1 : 0, 0) != 0;
          if (stop) break;
        }
      }
    } else {
      // Dynamic tile grabs of kGrab tiles from a counter shared by all CTAs
      // (balanced ends); the next grab is requested while this one is
      // staged.  The end marker stops the consumers.
      const int kGrab = p.grab;
      unsigned long long* next = &p.status->tile_next;
      long long nxt = 0;
      if (lane == 0) nxt = (long long)atomicAdd(next, (unsigned long long)kGrab);
      nxt = __shfl_sync(0xffffffffu, nxt, 0);
      while (!stop && nxt < p.ntiles) {
        const int64_t t0 = nxt;
        const int64_t te = t0 + kGrab < p.ntiles ? t0 + kGrab : p.ntiles;
        long long fut = 0;
        if (lane == 0) fut = (long long)atomicAdd(next, (unsigned long long)kGrab);
        const int64_t tl = t0 + lane < te ? t0 + lane : te;
        const int64_t my_s = p.tiles[tl], my_e = p.tile_e[tl];
        // issued after the descriptor loads, so both are in flight together
        const int ab = lane == 31 ? *reinterpret_cast<volatile int*>(&p.status->abort_req) : 0;
        if (injected_abort(ab)) break;
        const int cnt = (int)(te - t0);
        for (int k = 0; k < cnt; ++k) {
          const int64_t s0 = __shfl_sync(0xffffffffu, my_s, k);
          const int64_t e0 = __shfl_sync(0xffffffffu, my_e, k);
          const int64_t s1 = __shfl_sync(0xffffffffu, my_s, k + 1);
          const int64_t e1 = __shfl_sync(0xffffffffu, my_e, k + 1);
          stage(s0, s1, e0, e1, 0, false);
          stop = __shfl_sync(0xffffffffu, stop ? 1 : 0, 0) != 0;
          if (stop) break;
        }
        nxt = __shfl_sync(0xffffffffu, fut, 0);
      }
      if (!stop) {
        const int ab = lane == 31 ? *reinterpret_cast<volatile int*>(&p.status->abort_req) : 0;
        if (!injected_abort(ab)) stage(0, 0, 0, 0, 0, true);
      }
    }
    // drain: every armed stage must have landed before the CTA may exit
    if (lane == 0) {
      const int64_t issued = it;
      for (int64_t k = issued > kStages ? issued - kStages : 0; k < issued; ++k) {
        const int s = (int)(k % kStages);
        // bounded, and independent of the abort flag: bulk copies always complete
        const uint64_t w0 = globaltimer();
        while (!mbar_try_wait(&full[s], (uint32_t)(k / kStages) & 1u)) {
          if (globaltimer() - w0 > kWaitLimitNs) {
            atomicOr(&p.status->err, kErrTimeout);
            atomicCAS(&p.status->where, 0, 3);
            break;
          }
        }
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------ consumers ----
    // The mu cache and the shared bins, while the producer already streams;
    // the consumer warps then meet (the producer does not take part).
    pdl_wait();  // mu (and every per-evaluation input) comes from the prologue
    pdl_trigger();
    if (!BATCH) {
      for (int j = tid - 32; j < p.h_mu; j += kConsumerWarps * 32) mu_s[j] = p.mu_r[j];
      for (int j = tid - 32; j < p.h_y; j += kConsumerWarps * 32) y_s[j] = 0ull;
    }
    asm volatile("bar.sync 1, %0;" ::"r"(kConsumerWarps * 32) : "memory");
    // Every consumer warp visits every tile and claims work from it through
    // the stage's counter (one batch of eight sources per claim), so a warp
    // that is done early takes the next batch, of this tile or the next.  A
    // warp leaves a tile (arrives on its empty barrier) once the counter runs
    // past the tile's batches; the producer resets the counter only after
    // every warp has left, so no claim can reach a refilled stage.
    int64_t it = 0;
    uint32_t nsw = 0;  // slot switches so far (phase of the consumer barriers)
    // (a batched pass takes a fixed range of tiles; otherwise the producer's
    // end marker closes the stream)
    for (int64_t t = t_begin; !BATCH || t < t_end; ++t, ++it) {
      const int s = (int)(it % kStages);
      const uint32_t round = (uint32_t)(it / kStages);
      const bool ok = wait_phase(&full[s], round & 1u, abort, p.status, 2);
      if (!__all_sync(0xffffffffu, ok)) break;
      const StageInfo si = info[s];
      if (si.big == 2) break;
      if (BATCH && si.slot != cur) {
        // Every consumer warp visits every tile, so all of them switch here.
        // Meet once the previous slot's tiles are done, move the shared
        // bins and the mu cache to the new slot, meet again.
        if (cur >= 0) flush_sums(acc, p.slot_part + 2 * cur, lane);
        acc = Sums{};
        __syncwarp();
        if (lane == 0) mbar_arrive(&cbar[0]);
        if (!__all_sync(0xffffffffu, wait_phase(&cbar[0], nsw & 1u, abort, p.status, 4))) break;
        const SlotDesc* d = p.slots + si.slot;
        const int h_mu = d->h_mu, h_y = d->h_y;
        const float* mu_r = d->mu_r;
        const int hy_old = cur >= 0 ? cx.h_y : 0;
        const int hmax = hy_old > h_y ? hy_old : h_y;
        for (int j = tid - 32; j < hmax; j += kConsumerWarps * 32) {
          if (j < hy_old) {
            const unsigned long long v = y_s[j];
            if (v != 0ull) atomicAdd(cx.y + j, v);
          }
          y_s[j] = 0ull;
        }
        for (int j = tid - 32; j < h_mu; j += kConsumerWarps * 32) mu_s[j] = mu_r[j];
        __syncwarp();
        if (lane == 0) mbar_arrive(&cbar[1]);
        if (!__all_sync(0xffffffffu, wait_phase(&cbar[1], nsw & 1u, abort, p.status, 5))) break;
        ++nsw;
        cur = si.slot;
        cx.mu_g = mu_r;
        cx.h_mu = h_mu;
        cx.h_y = h_y;
        cx.y = d->y;
        cx.sy = d->sy;
        cx.sc = ldexpf(1.f, d->ec);
        cx.sw = ldexpf(1.f, d->ew);
        cx.one_w = d->ew >= 0 && d->ew <= 62 ? (1ll << d->ew) : 0ll;
        cx.gamma = p.gamma_of[cur];
        cx.inv_gamma = __frcp_rn(cx.gamma);
        cx.dst_g = d->dst;
        cx.ca2_g = d->ca2;
        cx.ca_g = d->ca;
      }
      const uint32_t claim_a = smem_u32(claim + s);
      if (BOX) {
        // unit-box projection: every edge on its own; a warp takes the edges
        // of a claimed batch of eight sources (or of an oversized source)
        if (si.big) {  // every consumer thread takes a share of the edges
          GlobalView<BF16> gv{cx.dst_g, cx.ca2_g, cx.ca_g};
          project_box<BF16, W, WRITE_X>(gv, si.e0, si.e1, si.e0, tid - 32, kConsumerWarps * 32,
                                        cx, acc);
        } else {
          const StageView<BF16> sv = stage_view<BF16>(smem, s);
          const int nsrc = (int)(si.s1 - si.s0);
          const int li0 = (int)(si.s0 - si.o0);
          const unsigned nb = (unsigned)((nsrc + 7) >> 3);
          for (;;) {
            unsigned bi = 0u;
            if (lane == 0) bi = atoms_add_u32(claim_a, 1u);
            bi = __shfl_sync(0xffffffffu, bi, 0);
            if (bi >= nb) break;
            const int li = li0 + 8 * (int)bi;
            const int n8 = nsrc - 8 * (int)bi < 8 ? nsrc - 8 * (int)bi : 8;
            const uint32_t a0 = (uint32_t)si.a0;
            const int e_lo = (int)(sv.off(li) - a0), e_hi = (int)(sv.off(li + n8) - a0);
            project_box<BF16, W, WRITE_X>(sv, e_lo, e_hi, si.a0 + e_lo, lane, 32, cx, acc);
          }
        }
      } else if (si.big) {
        // a source larger than a stage: every consumer warp projects it
        // together from global memory (block class), or (kBlockClass off)
        // the warp that claims it does
        GlobalView<BF16> gv{cx.dst_g, cx.ca2_g, cx.ca_g};
        if (kBlockClass && (BIG || WRITE_X)) {
          const longlong2 ps = project_block<BF16, W>(gv, si.e0, si.e1 - si.e0, si.e0, tid - 32,
                                                      warp - 1, lane, cx, dred);
          acc.cx += ps.x;
          acc.wxx += ps.y;
        } else {
          unsigned b = 0u;
          if (lane == 0) b = atoms_add_u32(claim_a, 1u);
          b = __shfl_sync(0xffffffffu, b, 0);
          if (b == 0u) project_multipass<BF16, W>(gv, si.e0, si.e1 - si.e0, si.e0, lane, cx, acc);
        }
      } else {
        const StageView<BF16> sv = stage_view<BF16>(smem, s);
        const int nsrc = (int)(si.s1 - si.s0);
        const int li0 = (int)(si.s0 - si.o0);
        // Sources are taken in batches of eight (32 in the small-degree
        // variant TINY).  The span of a source (stage slot of its first edge
        // mod 4, plus its degree) picks the group width: 1 lane (TINY only,
        // span <= 16, 32 sources per warp), 4 lanes (span <= 64, eight
        // sources per warp), 8 (<= 128), 16 (<= 256), 32 (<= 512), else the
        // multi-pass path.  Whatever the lean path leaves (unsaturated
        // sources, near-ties, the primal output) goes through the candidate
        // or multi-pass path.
        constexpr int NB = TINY ? 32 : 8;
        const unsigned nb = (unsigned)((nsrc + NB - 1) / NB);
        for (;;) {
          unsigned bi = 0u;
          if (lane == 0) bi = atoms_add_u32(claim_a, 1u);
          bi = __shfl_sync(0xffffffffu, bi, 0);
          if (bi >= nb) break;
          const int li = li0 + NB * (int)bi;
          const int n8 = nsrc - NB * (int)bi < NB ? nsrc - NB * (int)bi : NB;
          const uint32_t oq = sv.off(li + (lane <= n8 ? lane : n8));
          uint32_t on = __shfl_down_sync(0xffffffffu, oq, 1);
          if (TINY && lane == 31) on = sv.off(li + n8);  // the batch's end offset
          const int dq = lane < n8 ? (int)(on - oq) : 0;
          const int bq = (int)(oq - (uint32_t)si.a0);
          const int spq = dq > 0 ? (bq & 3) + dq : 0;
          unsigned needm, needm_tiny = 0u;
          if (WRITE_X) {
            needm = __ballot_sync(0xffffffffu, dq > 0);
          } else {
            // 4-lane groups take spans up to 64 (window 64 slots), or with
            // lean80 up to 80 in one pass (a window of 64 or 80 slots, by the
            // batch's largest span) unless the batch needs an 8-lane pass
            // anyway: then spans over 64 join that pass
            const bool in1 = TINY && dq > 0 && spq <= 16;
            const bool over80 = !p.lean80 || __any_sync(0xffffffffu, spq > 80 && spq <= 128);
            const int span4 = over80 ? 64 : 80;
            const bool in4 = dq > 0 && spq <= span4 && !in1;
            if (TINY) {
              const unsigned m1 = __ballot_sync(0xffffffffu, in1);
              if (m1) needm_tiny = lean_over<1, 4, BF16, W, MU_SMEM, BATCH>(sv, m1, bq, dq, lane,
                                                                            cx, acc);
            }
            const unsigned m4 = __ballot_sync(0xffffffffu, in4);
            const unsigned m128 = __ballot_sync(0xffffffffu, spq > span4 && spq <= 128);
            const unsigned m256 = __ballot_sync(0xffffffffu, spq > 128 && spq <= 256);
            const unsigned m512 = __ballot_sync(0xffffffffu, spq > 256 && spq <= 512);
            needm = __ballot_sync(0xffffffffu, spq > 512);
            if (m4) {
              // batched problems are stored in degree order, so a batch's
              // spans are alike: their 4-lane window is sized to the batch's
              // largest span (32, 48, 64 or 80 slots)
              const int mx4 = BATCH ? __reduce_max_sync(0xffffffffu, in4 ? spq : 0) : 64;
              if (p.lean80 && __any_sync(0xffffffffu, in4 && spq > 64))
                needm |= lean_over<4, 5, BF16, W, MU_SMEM, BATCH>(sv, m4, bq, dq, lane, cx, acc);
              else if (BATCH && mx4 <= 32)
                needm |= lean_over<4, 2, BF16, W, MU_SMEM, BATCH>(sv, m4, bq, dq, lane, cx, acc);
              else if (BATCH && mx4 <= 48)
                needm |= lean_over<4, 3, BF16, W, MU_SMEM, BATCH>(sv, m4, bq, dq, lane, cx, acc);
              else
                needm |= lean_over<4, 4, BF16, W, MU_SMEM, BATCH>(sv, m4, bq, dq, lane, cx, acc);
            }
            if (m128) needm |= lean_over<8, 4, BF16, W, MU_SMEM, BATCH>(sv, m128, bq, dq, lane, cx, acc);
            if (m256) needm |= lean_over<16, 4, BF16, W, MU_SMEM, BATCH>(sv, m256, bq, dq, lane, cx, acc);
            if (m512) needm |= lean_over<32, 4, BF16, W, MU_SMEM, BATCH>(sv, m512, bq, dq, lane, cx, acc);
            needm |= needm_tiny;
          }
          while (needm) {
            const int q = __ffs(needm) - 1;
            needm &= needm - 1u;
            const int b = __shfl_sync(0xffffffffu, bq, q);
            const int dd = __shfl_sync(0xffffffffu, dq, q);
            // (the result is the same for every lane: it follows warp sums)
            const bool done = !W && !WRITE_X && kWarpCand && dd <= 512 &&
                              (dd <= 32    ? project_warp_cand<BF16, MU_SMEM, 1>(sv, b, dd, lane, cx, acc)
                               : dd <= 64  ? project_warp_cand<BF16, MU_SMEM, 2>(sv, b, dd, lane, cx, acc)
                               : dd <= 128 ? project_warp_cand<BF16, MU_SMEM, 4>(sv, b, dd, lane, cx, acc)
                                           : project_warp_cand<BF16, MU_SMEM, 16>(sv, b, dd, lane, cx, acc));
            if (!done)
              project_multipass<BF16, W>(sv, (int64_t)b, (int64_t)dd, si.a0 + b, lane, cx, acc);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
    if (BATCH && cur >= 0) flush_sums(acc, p.slot_part + 2 * cur, lane);
  }
  __syncthreads();

  if (BATCH) {
    // the last slot's shared bins (consumer threads hold its pointers)
    if (warp > 0 && cur >= 0) {
      for (int j = tid - 32; j < cx.h_y; j += kConsumerWarps * 32) {
        const unsigned long long v = y_s[j];
        if (v != 0ull) atomicAdd(cx.y + j, v);
      }
    }
  } else {
    // flush the shared-memory accumulators of the hot destinations
    for (int j = tid; j < p.h_y; j += blockDim.x) {
      const unsigned long long v = y_s[j];
      if (v != 0ull) atomicAdd(p.y + j, v);
    }
    // per-CTA objective partials: exact integer sums through the shuffle and
    // warp trees
    const long long csum = warp_isum64(acc.cx), wsum = warp_isum64(acc.wxx);
    longlong2* wred = reinterpret_cast<longlong2*>(dred);  // one per warp
    if (lane == 0) wred[warp] = make_longlong2(csum, wsum);
    __syncthreads();
    if (tid == 0) {
      longlong2 t = wred[0];
      for (int w = 1; w < kThreads / 32; ++w) {
        t.x += wred[w].x;
        t.y += wred[w].y;
      }
      p.part[blockIdx.x] = t;
      // the last CTA to finish rewinds the tile counter for the next launch
      __threadfence();
      if (atomicAdd(&p.status->done, 1u) == gridDim.x - 1) {
        p.status->tile_next = 0ull;
        p.status->done = 0u;
      }
    }
  }
}

// ---------------------------------------------------- J-length kernels ----
__global__ void prep_mu_kernel(int32_t J, const float* __restrict__ lambda,
                               const float* __restrict__ D, const int32_t* __restrict__ orig_of,
                               float* __restrict__ mu_r) {
  pdl_wait();
  pdl_trigger();
  for (int64_t jr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; jr < J;
       jr += (int64_t)gridDim.x * blockDim.x) {
    const int jo = orig_of ? orig_of[jr] : (int)jr;
    const float l = lambda[jo];
    mu_r[jr] = D ? __fmul_rn(D[jo], l) : l;
  }
}

__global__ void epilogue_kernel(EpiParams q) {
  __shared__ float4 red[32];
  __shared__ long long finq[2][32];
  __shared__ double find[2][32];
  __shared__ bool last;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  pdl_wait();  // A x and the partials of the pass
  pdl_trigger();
  EpiAcc r;
  epi_rows(q, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x, r);
  warp_pair_sum(r.mh, r.ml);
  warp_pair_sum(r.nh, r.nl);
  if (lane == 0) red[w] = make_float4(r.mh, r.ml, r.nh, r.nl);
  __syncthreads();
  if (threadIdx.x == 0) {
    float4 t = red[0];
    for (int k = 1; k < nw; ++k) {
      pair_addp(t.x, t.y, red[k].x, red[k].y);
      pair_addp(t.z, t.w, red[k].z, red[k].w);
    }
    q.epi_part[blockIdx.x] = t;
    __threadfence();
    const unsigned prev = atomicAdd(&q.status->ticket, 1u);
    last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // fixed-order combination of every partial (strided per thread, then a
  // fixed shuffle tree and a fixed warp order): the pass's fixed-point sums
  // exactly in 64-bit integers, the row partials in FP64
  long long cq = 0, wq = 0;
  double mg = 0.0, nn = 0.0;
  for (int k = threadIdx.x; k < q.npart; k += blockDim.x) {
    const longlong2 u = __ldcg(q.part + k);
    cq += u.x;
    wq += u.y;
  }
  for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
    const float4 u = __ldcg(q.epi_part + k);
    mg += pair_value(u.x, u.y);
    nn += pair_value(u.z, u.w);
  }
  cq = warp_isum64(cq);
  wq = warp_isum64(wq);
  mg = warp_dsum(mg);
  nn = warp_dsum(nn);
  if (lane == 0) {
    finq[0][w] = cq;
    finq[1][w] = wq;
    find[0][w] = mg;
    find[1][w] = nn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long tc = 0, tw = 0;
    double tm = 0.0, tn = 0.0;
    for (int k = 0; k < nw; ++k) {
      tc += finq[0][k];
      tw += finq[1][k];
      tm += find[0][k];
      tn += find[1][k];
    }
    epi_write(q, ldexp((double)tc, -q.ec), ldexp((double)tw, -q.ew), tm, tn);
    q.status->ticket = 0u;
  }
}

__global__ void histogram_kernel(const int32_t* __restrict__ dst, int64_t E, int32_t J,
                                 unsigned* __restrict__ counts, DeviceStatus* st) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t j = dst[e];
    if (j < 0 || j >= J) {
      atomicOr(&st->err, kErrBounds);
      continue;
    }
    atomicAdd(counts + j, 1u);
  }
}

__global__ void renumber_kernel(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                const int32_t* __restrict__ new_of, int64_t E, int32_t J,
                                DeviceStatus* st) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t j = in[e];
    if (j < 0 || j >= J) {
      atomicOr(&st->err, kErrBounds);
      out[e] = 0;
      continue;
    }
    out[e] = new_of[j];
  }
}

__global__ void pack_f32_kernel(const float* __restrict__ c, const float* __restrict__ a,
                                float2* __restrict__ ca2, int64_t E) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x)
    ca2[e] = make_float2(c[e], a[e]);
}

__global__ void pack_bf16_kernel(const float* __restrict__ c, const float* __restrict__ a,
                                 uint32_t* __restrict__ ca, int64_t E) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t cb = __bfloat16_as_ushort(__float2bfloat16_rn(c[e]));
    const uint32_t ab = __bfloat16_as_ushort(__float2bfloat16_rn(a[e]));
    ca[e] = cb | (ab << 16);
  }
}

__global__ void check_finite_kernel(const float* __restrict__ v, int64_t n, DeviceStatus* st) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (!isfinite(v[e])) atomicOr(&st->err, kErrBounds);
  }
}

__global__ void absmax_kernel(const float* __restrict__ v, int64_t n, unsigned* out) {
  unsigned m = 0u;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    m = max(m, __float_as_uint(fabsf(v[e])));
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

int grid_for(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace

size_t pass_smem_bytes(int storage) {
  return storage == DUALIP_EDGE_BF16 ? Layout<true>::kTotal : Layout<false>::kTotal;
}

template <bool BF16, bool W, bool MU, bool WX, bool B = false, bool BOX = false,
          bool TINY = false, bool BIG = false>
static cudaError_t set_smem() {
  return cudaFuncSetAttribute(dualgrad_pass_kernel<BF16, W, MU, WX, B, BOX, TINY, BIG>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Layout<BF16>::kTotal);
}

cudaError_t configure_pass_kernels() {
  const cudaError_t es[] = {
      set_smem<false, false, false, false>(), set_smem<false, false, true, false>(),
      set_smem<false, true, false, false>(),  set_smem<false, true, true, false>(),
      set_smem<true, false, false, false>(),  set_smem<true, false, true, false>(),
      set_smem<true, true, false, false>(),   set_smem<true, true, true, false>(),
      set_smem<false, false, false, true>(),  set_smem<false, true, false, true>(),
      set_smem<true, false, false, true>(),   set_smem<true, true, false, true>(),
      set_smem<false, false, false, false, true>(), set_smem<false, true, false, false, true>(),
      set_smem<true, false, false, false, true>(),  set_smem<true, true, false, false, true>(),
      set_smem<false, false, false, false, false, true>(),
      set_smem<false, true, false, false, false, true>(),
      set_smem<true, false, false, false, false, true>(),
      set_smem<true, true, false, false, false, true>(),
      set_smem<false, false, false, true, false, true>(),
      set_smem<false, true, false, true, false, true>(),
      set_smem<true, false, false, true, false, true>(),
      set_smem<true, true, false, true, false, true>(),
      set_smem<false, false, false, false, false, false, true>(),
      set_smem<false, false, true, false, false, false, true>(),
      set_smem<false, true, false, false, false, false, true>(),
      set_smem<false, true, true, false, false, false, true>(),
      set_smem<true, false, false, false, false, false, true>(),
      set_smem<true, false, true, false, false, false, true>(),
      set_smem<true, true, false, false, false, false, true>(),
      set_smem<true, true, true, false, false, false, true>(),
      set_smem<false, false, false, false, false, false, false, true>(),
      set_smem<false, false, true, false, false, false, false, true>(),
      set_smem<false, true, false, false, false, false, false, true>(),
      set_smem<false, true, true, false, false, false, false, true>(),
      set_smem<true, false, false, false, false, false, false, true>(),
      set_smem<true, false, true, false, false, false, false, true>(),
      set_smem<true, true, false, false, false, false, false, true>(),
      set_smem<true, true, true, false, false, false, false, true>(),
      set_smem<false, false, false, false, true, false, false, true>(),
      set_smem<false, true, false, false, true, false, false, true>(),
      set_smem<true, false, false, false, true, false, false, true>(),
      set_smem<true, true, false, false, true, false, false, true>()};
  for (cudaError_t e : es)
    if (e != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t launch_prep(const Problem& P, const float* lambda, const float* D, cudaStream_t s) {
  prep_mu_kernel<<<grid_for(P.J, 256, 4 * P.num_sms), 256, 0, s>>>(P.J, lambda, D, P.orig_of,
                                                                     P.mu_r);
  return cudaGetLastError();
}

static PassParams pass_params(const Problem& P, const float* gamma_dev, float gamma,
                              float* x_out) {
  PassParams p;
  p.off = P.off32;
  p.dst = P.dst;
  p.ca2 = P.ca2;
  p.ca = P.ca;
  p.tiles = P.tiles;
  p.tile_e = P.tile_e;
  p.ntiles = P.ntiles;
  p.I = P.I;
  p.J = P.J;
  p.h_mu = P.h_mu;
  p.h_y = P.h_y;
  p.mu_r = P.mu_r;
  p.gamma_dev = gamma_dev;
  p.gamma = gamma;
  p.y = P.y;
  p.ey = P.exp_y;
  p.ec = P.exp_c;
  p.ew = P.exp_w;
  p.part = P.part;
  p.x_out = x_out;
  p.status = P.status;
  p.jt = nullptr;
  p.slots = nullptr;
  p.gamma_of = nullptr;
  p.slot_part = nullptr;
  p.lean80 = 1;
  // a tile holding a source larger than a stage takes a whole CTA for a
  // while: one tile per grab keeps two of them off the same CTA
  p.grab = P.has_big ? 1 : DUALIP_GRAB;
  p.mb_min = P.nhub > 0 ? P.mb_min : INT64_MAX;
  return p;
}

static cudaError_t dispatch_pass(const Problem& P, const PassParams& p, bool x_out,
                                 cudaStream_t s);

// The multi-block class: every hub source, over the whole grid.
static cudaError_t launch_hubs(const Problem& P, const float* gamma_dev, float gamma,
                               float* x_out, cudaStream_t s) {
  HubParams h;
  h.dst = P.dst;
  h.ca2 = P.ca2;
  h.ca = P.ca;
  h.mu_r = P.mu_r;
  h.gamma_dev = gamma_dev;
  h.gamma = gamma;
  h.y = P.y;
  h.ey = P.exp_y;
  h.ec = P.exp_c;
  h.ew = P.exp_w;
  h.x_out = x_out;
  h.hubs = P.hubs;
  h.chunk_hub = P.chunk_hub;
  h.nchunks = P.nchunks;
  h.stat = P.hub_stat;
  h.cand = P.hub_cand;
  h.cnt = P.hub_cnt;
  h.part = P.part + P.grid;
  h.status = P.status;
  const int64_t slots = (int64_t)kHubCtasPerSm * P.num_sms;  // one wave of resident CTAs
  const int64_t g64 = P.nchunks < slots ? P.nchunks : slots;
  const dim3 grid((unsigned)(g64 > 0 ? g64 : 1)), block(kHubThreads);
  const bool bf16 = P.storage == DUALIP_EDGE_BF16;
#define DUALIP_HUB(B, W) \
  (x_out ? launch_pdl(hub_kernel<B, W, true>, grid, block, 0, s, h) \
         : launch_pdl(hub_kernel<B, W, false>, grid, block, 0, s, h))
  if (bf16) return P.weighted ? DUALIP_HUB(true, true) : DUALIP_HUB(true, false);
  return P.weighted ? DUALIP_HUB(false, true) : DUALIP_HUB(false, false);
#undef DUALIP_HUB
}

cudaError_t launch_pass(const Problem& P, const float* gamma_dev, float gamma, float* x_out,
                        cudaStream_t s) {
  if (P.m > 1) return launch_pass_multi(P, gamma_dev, gamma, x_out, s);
  if (P.nhub > 0) {
    const cudaError_t e = launch_hubs(P, gamma_dev, gamma, x_out, s);
    if (e != cudaSuccess) return e;
  }
  return dispatch_pass(P, pass_params(P, gamma_dev, gamma, x_out), x_out != nullptr, s);
}

static cudaError_t dispatch_pass(const Problem& P, const PassParams& p, bool x_out,
                                 cudaStream_t s) {
  const bool bf16 = P.storage == DUALIP_EDGE_BF16;
  const bool mu_all = P.J <= P.h_mu;
  const size_t smem = pass_smem_bytes(P.storage);
  const dim3 grid(P.grid), block(kThreads);
  cudaError_t e = cudaSuccess;
#define DUALIP_LAUNCH(B, W, M, X)                                                            \
  e = (!(X) && P.has_big)                                                                    \
          ? launch_pdl(dualgrad_pass_kernel<B, W, M, false, false, false, false, true>, grid,   \
                       block, smem, s, p)                                                    \
      : (!(X) && P.tiny)                                                                     \
          ? launch_pdl(dualgrad_pass_kernel<B, W, M, false, false, false, true>, grid, block,   \
                       smem, s, p)                                                           \
          : launch_pdl(dualgrad_pass_kernel<B, W, M, X, false>, grid, block, smem, s, p)
#define DUALIP_LAUNCH_BOX(B, W, X) \
  e = launch_pdl(dualgrad_pass_kernel<B, W, false, X, false, true>, grid, block, smem, s, p)
  if (P.box) {
    if (x_out) {
      if (bf16) {
        if (P.weighted) DUALIP_LAUNCH_BOX(true, true, true);
        else DUALIP_LAUNCH_BOX(true, false, true);
      } else {
        if (P.weighted) DUALIP_LAUNCH_BOX(false, true, true);
        else DUALIP_LAUNCH_BOX(false, false, true);
      }
    } else if (bf16) {
      if (P.weighted) DUALIP_LAUNCH_BOX(true, true, false);
      else DUALIP_LAUNCH_BOX(true, false, false);
    } else {
      if (P.weighted) DUALIP_LAUNCH_BOX(false, true, false);
      else DUALIP_LAUNCH_BOX(false, false, false);
    }
  } else if (x_out) {
    if (bf16) {
      if (P.weighted) DUALIP_LAUNCH(true, true, false, true);
      else DUALIP_LAUNCH(true, false, false, true);
    } else {
      if (P.weighted) DUALIP_LAUNCH(false, true, false, true);
      else DUALIP_LAUNCH(false, false, false, true);
    }
  } else if (bf16) {
    if (P.weighted) {
      if (mu_all) DUALIP_LAUNCH(true, true, true, false);
      else DUALIP_LAUNCH(true, true, false, false);
    } else {
      if (mu_all) DUALIP_LAUNCH(true, false, true, false);
      else DUALIP_LAUNCH(true, false, false, false);
    }
  } else {
    if (P.weighted) {
      if (mu_all) DUALIP_LAUNCH(false, true, true, false);
      else DUALIP_LAUNCH(false, true, false, false);
    } else {
      if (mu_all) DUALIP_LAUNCH(false, false, true, false);
      else DUALIP_LAUNCH(false, false, false, false);
    }
  }
#undef DUALIP_LAUNCH
#undef DUALIP_LAUNCH_BOX
  return e;
}

cudaError_t launch_pass_batch(int storage, int weighted, const JointTile* jt, int64_t ntiles,
                              const SlotDesc* slots, const float* gamma_of, long long* slot_part,
                              DeviceStatus* status, int grid, int lean80, bool big,
                              cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  PassParams p{};
  p.grab = DUALIP_GRAB;  // (the batched pass takes contiguous ranges)
  p.lean80 = lean80;
  p.ntiles = ntiles;
  p.jt = jt;
  p.slots = slots;
  p.gamma_of = gamma_of;
  p.slot_part = slot_part;
  p.status = status;
  p.mb_min = INT64_MAX;  // hub sources of a batch stay in the pass
  const bool bf16 = storage == DUALIP_EDGE_BF16;
  const size_t smem = pass_smem_bytes(storage);
  const int g = (int)(ntiles < grid ? ntiles : grid);
  const dim3 gd(g), bd(kThreads);
  // a batch holding a source larger than a tile takes the instance with the
  // block class (all consumer warps on that source)
#define DUALIP_LAUNCH_B(B_, W_)                                                                 \
  (big ? launch_pdl(dualgrad_pass_kernel<B_, W_, false, false, true, false, false, true>, gd, bd, \
                    smem, s, p)                                                                 \
       : launch_pdl(dualgrad_pass_kernel<B_, W_, false, false, true>, gd, bd, smem, s, p))
  if (bf16) return weighted ? DUALIP_LAUNCH_B(true, true) : DUALIP_LAUNCH_B(true, false);
  return weighted ? DUALIP_LAUNCH_B(false, true) : DUALIP_LAUNCH_B(false, false);
#undef DUALIP_LAUNCH_B
}

cudaError_t launch_epilogue(const Problem& P, const float* D, float* grad, const float* gamma_dev,
                            double gamma, double* eval_out, cudaStream_t s, bool identity) {
  EpiParams q;
  q.J = P.J;
  q.orig_of = identity ? nullptr : P.orig_of;
  q.b_r = P.b_r;
  q.mu_r = P.mu_r;
  q.D = D;
  q.y = P.y;
  q.sy = ldexpf(1.0f, -P.exp_y);
  q.grad = grad;
  q.part = P.part;
  q.ec = P.exp_c;
  q.ew = P.exp_w;
  q.npart = P.grid + P.nhub;
  q.epi_part = P.epi_part;
  q.gamma_dev = gamma_dev;
  q.gamma = gamma;
  q.eval_out = eval_out;
  q.status = P.status;
  return launch_pdl(epilogue_kernel, dim3(P.epi_blocks), dim3(256), 0, s, q);
}

cudaError_t launch_histogram(const int32_t* dst, int64_t E, int32_t J, unsigned* counts,
                             DeviceStatus* st, cudaStream_t s) {
  histogram_kernel<<<grid_for(E, 256, 8192), 256, 0, s>>>(dst, E, J, counts, st);
  return cudaGetLastError();
}

cudaError_t launch_renumber(const int32_t* dst_in, int32_t* dst_out, const int32_t* new_of,
                            int64_t E, int32_t J, DeviceStatus* st, cudaStream_t s) {
  renumber_kernel<<<grid_for(E, 256, 8192), 256, 0, s>>>(dst_in, dst_out, new_of, E, J, st);
  return cudaGetLastError();
}

cudaError_t launch_pack_f32(const float* c, const float* a, float2* ca2, int64_t E,
                            cudaStream_t s) {
  pack_f32_kernel<<<grid_for(E, 256, 8192), 256, 0, s>>>(c, a, ca2, E);
  return cudaGetLastError();
}

cudaError_t launch_pack_bf16(const float* c, const float* a, uint32_t* ca, int64_t E,
                             cudaStream_t s) {
  pack_bf16_kernel<<<grid_for(E, 256, 8192), 256, 0, s>>>(c, a, ca, E);
  return cudaGetLastError();
}

cudaError_t launch_absmax(const float* v, int64_t n, unsigned* out, cudaStream_t s) {
  absmax_kernel<<<grid_for(n, 256, 4096), 256, 0, s>>>(v, n, out);
  return cudaGetLastError();
}

cudaError_t launch_check_finite(const float* v, int64_t n, DeviceStatus* st, cudaStream_t s) {
  check_finite_kernel<<<grid_for(n, 256, 8192), 256, 0, s>>>(v, n, st);
  return cudaGetLastError();
}

}  // namespace dualip
