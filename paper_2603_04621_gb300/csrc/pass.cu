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
//  * one persistent CTA per SM walks a contiguous range of "tiles" (runs of
//    whole sources holding <= kTileEdges edges); warp 0 streams each tile's
//    offsets and edge arrays into a kStages-deep shared-memory ring with
//    cp.async.bulk + mbarrier transaction counts, 16 consumer warps project;
//  * a consumer warp owns one source at a time; degrees <= 128 live in
//    registers (up to 4 edges per lane), larger ones are re-read from the
//    staged tile, and a source too large for a tile is projected by one warp
//    straight from global memory;
//  * scores are formed as an unevaluated FP32 pair (hi + lo = -(c + a mu) to
//    about 2^-48 relative) and, when the sum constraint binds, shifted by the
//    block maximum (exact by Sterbenz's lemma near the top), so the threshold
//    and x keep FP32 accuracy even when gamma is small and r/gamma is large;
//  * the threshold follows Michelot's finite iteration started from the set
//    {d_e > max_e(d_e - gamma w_e)}, which contains the active set;
//  * y = A x uses FP32 atomics with an exact TwoSum error term accumulated in a
//    second array; hot destinations (ids renumbered by in-degree) accumulate
//    in shared memory first; objective partials use per-lane FP32 TwoSum
//    accumulators and FP64 only for the final per-CTA reduction.
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
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
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
// Bounded wait on an mbarrier phase.  Gives up after kWaitLimitNs or when
// another thread has raised `abort`, recording the site in the status word.
__device__ bool wait_phase(uint64_t* bar, uint32_t parity, volatile int* abort,
                           DeviceStatus* st, int site) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 0) {
      if (*abort) return false;
      if (globaltimer() - t0 > kWaitLimitNs) {
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
// and is rounded once to an integer; integer adds are exact and independent
// of their order, so A x and the objective partials are reproducible bit for
// bit.  The scales are chosen at create so that no sum can exceed 2^61.
__device__ __forceinline__ long long to_fixed(float v, float scale) {
  return __float2ll_rn(__fmul_rn(v, scale));
}

// --------------------------------------------------------- smem layout ----
struct StageInfo {
  int64_t s0, s1;  // sources [s0, s1)
  int64_t e0, e1;  // edges [e0, e1)
  int64_t a0;      // first staged edge (multiple of 4)
  int64_t o0;      // first staged offset (even)
  int32_t big;     // single source larger than a stage: read from global
  int32_t pad;
};

template <bool BF16>
struct Layout {
  static constexpr size_t kOffBytes = sizeof(int64_t) * kStageOffSlots;
  static constexpr size_t kEdgeArr = sizeof(uint32_t) * kStageEdgeSlots;
  static constexpr size_t kStageBytes = kOffBytes + kEdgeArr * (BF16 ? 2 : 3);
  static constexpr size_t kMu = kStages * kStageBytes;
  static constexpr size_t kY = kMu + sizeof(float) * kMaxCachedDests;
  static constexpr size_t kBars = kY + sizeof(unsigned long long) * kMaxPrivDests;
  static constexpr size_t kInfo = kBars + sizeof(uint64_t) * 2 * kStages;
  static constexpr size_t kMisc = kInfo + sizeof(StageInfo) * kStages;
  static constexpr size_t kTotal = kMisc + 512;
  static_assert(kOffBytes % 16 == 0 && kEdgeArr % 16 == 0, "16-byte staging");
  static_assert(kTotal <= 227 * 1024, "shared memory budget");
};

template <bool BF16>
struct StageView {
  const int64_t* off;
  const int32_t* dst;
  const float* c;
  const float* a;
  const uint32_t* ca;
  __device__ __forceinline__ void edge(int k, int& j, float& cv, float& av) const {
    j = dst[k];
    if (BF16) {
      const uint32_t u = ca[k];
      cv = __uint_as_float(u << 16);
      av = __uint_as_float(u & 0xffff0000u);
    } else {
      cv = c[k];
      av = a[k];
    }
  }
};

template <bool BF16>
__device__ __forceinline__ StageView<BF16> stage_view(unsigned char* smem, int s) {
  using L = Layout<BF16>;
  unsigned char* base = smem + (size_t)s * L::kStageBytes;
  StageView<BF16> v;
  v.off = reinterpret_cast<const int64_t*>(base);
  v.dst = reinterpret_cast<const int32_t*>(base + L::kOffBytes);
  v.c = reinterpret_cast<const float*>(base + L::kOffBytes + L::kEdgeArr);
  v.a = BF16 ? nullptr : reinterpret_cast<const float*>(base + L::kOffBytes + 2 * L::kEdgeArr);
  v.ca = reinterpret_cast<const uint32_t*>(base + L::kOffBytes + L::kEdgeArr);
  return v;
}

// global edge reader (sources too large for a stage)
template <bool BF16>
struct GlobalView {
  const int32_t* dst;
  const float* c;
  const float* a;
  const uint32_t* ca;
  __device__ __forceinline__ void edge(int64_t k, int& j, float& cv, float& av) const {
    j = __ldg(dst + k);
    if (BF16) {
      const uint32_t u = __ldg(ca + k);
      cv = __uint_as_float(u << 16);
      av = __uint_as_float(u & 0xffff0000u);
    } else {
      cv = __ldg(c + k);
      av = __ldg(a + k);
    }
  }
};

// ------------------------------------------------------ per-thread state ----
// Read-only context of a pass (passed by value to out-of-line paths).
struct Ctx {
  const float* mu_s;
  const float* mu_g;
  int h_mu;
  unsigned long long* y_s;
  int h_y;
  unsigned long long* y;
  float gamma, inv_gamma;
  float sy, sc, sw;
  float* x_out;

  __device__ __forceinline__ float mu(int j) const { return j < h_mu ? mu_s[j] : __ldg(mu_g + j); }
  __device__ __forceinline__ void scatter(int j, float v) const {
    const unsigned long long q = (unsigned long long)to_fixed(v, sy);
    if (q == 0ull) return;
    if (j < h_y) atomicAdd(y_s + j, q);
    else atomicAdd(y + j, q);
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

// Per-lane objective partials sum c x and sum w x^2, in fixed point.
struct Sums {
  long long cx = 0, wxx = 0;
  __device__ __forceinline__ void account(const Ctx& c, int j, float cv, float a, float w,
                                          float x) {
    c.scatter(j, __fmul_rn(a, x));
    cx += to_fixed(__fmul_rn(cv, x), c.sc);
    wxx += to_fixed(__fmul_rn(w, __fmul_rn(x, x)), c.sw);
  }
  __device__ __forceinline__ void merge(const Sums& o) {
    cx += o.cx;
    wxx += o.wxx;
  }
};

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

// The hot path: 32/G sources per warp, G lanes per source, K edges per lane
// (degree <= G K).  Plain FP32 scores (FMA), one fused group reduction (max,
// saturation sum, weighted bound), a per-lane count of the candidates near
// the top, and x = 1 for a saturated source with a single candidate.
// Returns (warp-uniform) bit q set for every source li + q of the batch that
// is unsaturated or has near-ties at the top; those take the general path.
template <int G, int K, bool BF16, bool W, bool MU_SMEM>
__device__ __forceinline__ unsigned project_lean(const StageView<BF16>& sv, int li, int nsrc,
                                                 int64_t a0, int lane, const Ctx& cx,
                                                 Sums& acc) {
  const int g = lane / G, l = lane % G;
  const bool gvalid = g < nsrc;
  const int lis = gvalid ? li + g : li;
  const int64_t eb = sv.off[lis];
  const int d = gvalid ? (int)(sv.off[lis + 1] - eb) : 0;
  const int base = (int)(eb - a0);
  float rf[K];
  float rmax = -CUDART_INF_F, s0 = 0.f, m2 = -CUDART_INF_F;
  // branch-free: out-of-range slots re-read the group's last edge (or the
  // first staged slot of an empty group, still inside the stage) and are
  // masked with -inf
  const int dl = d > 0 ? d - 1 : 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int idx = l + G * k;
    const bool v = idx < d;
    float c, a;
    int j;
    sv.edge(base + (v ? idx : dl), j, c, a);
    const float m = MU_SMEM ? cx.mu_s[j] : cx.mu(j);
    rf[k] = v ? -__fmaf_rn(a, m, c) : -CUDART_INF_F;
    rmax = fmaxf(rmax, rf[k]);
    if (W) {
      const float w = edge_w<W>(a);
      s0 += rf[k] > 0.f ? __fmul_rn(edge_alpha<W>(cx, w), rf[k]) : 0.f;
      m2 = fmaxf(m2, __fsub_rn(rf[k], __fmul_rn(cx.gamma, w)));
    } else {
      s0 += fmaxf(rf[k], 0.f);
    }
  }
#pragma unroll
  for (int o = G / 2; o; o >>= 1) {
    rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    if (W) m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, o));
  }
  if (!W) s0 = __fmul_rn(s0, cx.inv_gamma);
  const int mode = rmax <= 0.f ? 0 : (s0 <= 1.f ? 1 : 2);
  const float lb = (W ? fminf(__fsub_rn(m2, rmax), 0.f) : -cx.gamma) - ldexpf(fabsf(rmax), -20);
  int lc = 0, kc = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (__fsub_rn(rf[k], rmax) > lb) {
      ++lc;
      kc = k;
    }
  }
  if (mode != 2) lc = 0;
  const int cnt = group_isum<G>(lc);
  if (mode == 2 && cnt == 1 && lc == 1) {
    // the only candidate is the only active edge: x = 1 exactly
    float c, a;
    int j;
    sv.edge(base + l + G * kc, j, c, a);
    acc.account(cx, j, c, a, edge_w<W>(a), 1.f);
  }
  const unsigned lead =
      __ballot_sync(0xffffffffu, l == 0 && gvalid && (mode == 1 || (mode == 2 && cnt > 1)));
  unsigned need = 0u;
#pragma unroll
  for (int q = 0; q < 32 / G; ++q) need |= ((lead >> (G * q)) & 1u) << q;
  return need;
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
  float rmax = -CUDART_INF_F, s0 = 0.f;
  for (int64_t k = g.rank(); k < d; k += g.size()) {
    int j;
    float c, a, hi, lo;
    load(k, j, c, a, hi, lo);
    const float rf = __fadd_rn(hi, lo);
    rmax = fmaxf(rmax, rf);
    if (rf > 0.f) s0 += __fmul_rn(edge_alpha<W>(cx, edge_w<W>(a)), rf);
  }
  rmax = g.max(rmax);
  s0 = g.sum(s0);
  int mode = rmax <= 0.f ? 0 : (s0 <= 1.f ? 1 : 2);
  float t = 0.f;
  if (mode == 2) {
    float lb = -CUDART_INF_F;
    for (int64_t k = g.rank(); k < d; k += g.size()) {
      int j;
      float c, a, hi, lo;
      load(k, j, c, a, hi, lo);
      const float dk = __fadd_rn(__fsub_rn(hi, rmax), lo);
      lb = fmaxf(lb, __fsub_rn(dk, W ? __fmul_rn(cx.gamma, edge_w<W>(a)) : cx.gamma));
    }
    lb = g.max(lb);
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
    } else if (mode == 2) {
      const float dk = __fadd_rn(__fsub_rn(hi, rmax), lo);
      x = dk > t ? __fmul_rn(al, __fsub_rn(dk, t)) : 0.f;
    }
    if (x > 0.f) acc.account(cx, j, c, a, w, x);
    if (cx.x_out != nullptr) cx.x_out[e_glob + k] = x;
  }
}

// ----------------------------------------------------------- the pass ----
// MU_SMEM: every destination's mu is cached in shared memory (J <= the cache).
// WRITE_X: the primal x is written for every edge (dualip_get_primal); every
// source then takes the general path.
template <bool BF16, bool W, bool MU_SMEM, bool WRITE_X>
__global__ void __launch_bounds__(kThreads, 1) dualgrad_pass_kernel(PassParams p) {
  using L = Layout<BF16>;
  extern __shared__ __align__(128) unsigned char smem[];
  float* mu_s = reinterpret_cast<float*>(smem + L::kMu);
  unsigned long long* y_s = reinterpret_cast<unsigned long long*>(smem + L::kY);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::kBars);
  uint64_t* empty = full + kStages;
  StageInfo* info = reinterpret_cast<StageInfo*>(smem + L::kInfo);
  volatile int* abort = reinterpret_cast<volatile int*>(smem + L::kMisc);
  long long* dred = reinterpret_cast<long long*>(smem + L::kMisc + 16);  // 2 per warp

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int64_t t_begin = (int64_t)blockIdx.x * p.ntiles / gridDim.x;
  const int64_t t_end = (int64_t)(blockIdx.x + 1) * p.ntiles / gridDim.x;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    *abort = 0;
    fence_mbar_init();
  }
  for (int j = tid; j < p.h_mu; j += blockDim.x) mu_s[j] = p.mu_r[j];
  for (int j = tid; j < p.h_y; j += blockDim.x) y_s[j] = 0ull;
  __syncthreads();

  Ctx cx;
  Sums acc;
  cx.mu_s = mu_s;
  cx.mu_g = p.mu_r;
  cx.h_mu = p.h_mu;
  cx.y_s = y_s;
  cx.h_y = p.h_y;
  cx.y = p.y;
  cx.sy = p.sy;
  cx.sc = p.sc;
  cx.sw = p.sw;
  cx.gamma = p.gamma_dev ? *p.gamma_dev : p.gamma;
  cx.inv_gamma = __frcp_rn(cx.gamma);
  cx.x_out = WRITE_X ? p.x_out : nullptr;

  if (warp == 0) {
    // ------------------------------------------------------ producer ----
    // The warp fetches 32 tile descriptors per load; lane 0 waits and issues.
    int64_t it = 0;
    bool stop = false;
    for (int64_t t0 = t_begin; t0 < t_end && !stop; t0 += 32) {
      const int64_t tl = t0 + lane < t_end ? t0 + lane : t_end;
      const int64_t my_s = p.tiles[tl], my_e = p.tile_e[tl];
      const int64_t ext = t0 + 32 < t_end ? t0 + 32 : t_end;
      const int64_t ext_s = p.tiles[ext], ext_e = p.tile_e[ext];
      const int cnt = (int)(t_end - t0 < 32 ? t_end - t0 : 32);
      for (int k = 0; k < cnt; ++k, ++it) {
        const int64_t s0 = __shfl_sync(0xffffffffu, my_s, k);
        const int64_t e0 = __shfl_sync(0xffffffffu, my_e, k);
        const int64_t s1n = __shfl_sync(0xffffffffu, my_s, (k + 1) & 31);
        const int64_t e1n = __shfl_sync(0xffffffffu, my_e, (k + 1) & 31);
        const int64_t s1 = k < 31 ? s1n : ext_s;
        const int64_t e1 = k < 31 ? e1n : ext_e;
        if (lane == 0) {
          const int s = (int)(it % kStages);
          const uint32_t round = (uint32_t)(it / kStages);
          if (round > 0 && !wait_phase(&empty[s], (round - 1) & 1u, abort, p.status, 1)) {
            stop = true;
          } else {
            StageInfo si;
            si.s0 = s0;
            si.s1 = s1;
            si.e0 = e0;
            si.e1 = e1;
            const bool bad = s1 - s0 > kTileSources || s1 < s0 || e1 < e0 ||
                             (e1 - e0 > kTileEdges && s1 - s0 != 1);
            if (bad) {
              atomicOr(&p.status->err, kErrBounds);
              si.s1 = s0;  // skip the tile; results are flagged invalid
            }
            si.big = (!bad && e1 - e0 > kTileEdges) ? 1 : 0;
            si.a0 = e0 & ~int64_t(3);
            si.o0 = s0 & ~int64_t(1);
            info[s] = si;
            if (bad || si.big) {
              mbar_arrive(&full[s]);
            } else {
              const int64_t a1 = (e1 + 3) & ~int64_t(3);
              const int64_t o1 = (s1 + 2) & ~int64_t(1);
              const uint32_t ne = (uint32_t)(a1 - si.a0), no = (uint32_t)(o1 - si.o0);
              const uint32_t bytes = no * 8u + ne * (BF16 ? 8u : 12u);
              mbar_arrive_expect_tx(&full[s], bytes);
              unsigned char* base = smem + (size_t)s * L::kStageBytes;
              bulk_g2s(base, p.off + si.o0, no * 8u, &full[s]);
              if (ne) {
                bulk_g2s(base + L::kOffBytes, p.dst + si.a0, ne * 4u, &full[s]);
                if (BF16) {
                  bulk_g2s(base + L::kOffBytes + L::kEdgeArr, p.ca + si.a0, ne * 4u, &full[s]);
                } else {
                  bulk_g2s(base + L::kOffBytes + L::kEdgeArr, p.c + si.a0, ne * 4u, &full[s]);
                  bulk_g2s(base + L::kOffBytes + 2 * L::kEdgeArr, p.a + si.a0, ne * 4u,
                           &full[s]);
                }
              }
            }
          }
        }
        stop = __shfl_sync(0xffffffffu, stop ? 1 : 0, 0) != 0;
        if (stop) break;
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
    const int cw = warp - 1;
    int rot = 0;  // batches seen in earlier tiles, mod kConsumerWarps
    int64_t it = 0;
    for (int64_t t = t_begin; t < t_end; ++t, ++it) {
      const int s = (int)(it % kStages);
      const uint32_t round = (uint32_t)(it / kStages);
      const bool ok = wait_phase(&full[s], round & 1u, abort, p.status, 2);
      if (!__all_sync(0xffffffffu, ok)) break;
      const StageInfo si = info[s];
      if (si.big) {
        // one warp (chosen by tile index) projects a source larger than a
        // stage straight from global memory; no cross-warp barrier is used
        if (cw == (int)(t % kConsumerWarps)) {
          GlobalView<BF16> gv{p.dst, p.c, p.a, p.ca};
          project_multipass<BF16, W>(gv, si.e0, si.e1 - si.e0, si.e0, lane, cx, acc);
        }
      } else {
        const StageView<BF16> sv = stage_view<BF16>(smem, s);
        const int nsrc = (int)(si.s1 - si.s0);
        const int li0 = (int)(si.s0 - si.o0);
        // sources are taken in batches of four: four 8-lane groups when every
        // degree is <= 64, else pairs of 16-lane groups (<= 128), else one
        // warp per source (<= 256); what the lean path leaves (unsaturated
        // sources, near-ties, larger degrees, the primal output) goes through
        // the multi-pass path.  Batches are dealt round robin across tiles
        // (rot), so a tile whose batch count is not a multiple of the warp
        // count loads different warps.
        const int nb = (nsrc + 3) >> 2;
        const int first = (cw - rot + kConsumerWarps) % kConsumerWarps;
        rot = (rot + nb) % kConsumerWarps;
        for (int bi = first; bi < nb; bi += kConsumerWarps) {
          const int li = li0 + 4 * bi;
          const int n4 = nsrc - 4 * bi < 4 ? nsrc - 4 * bi : 4;
          int dg[4];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            dg[q] = q < n4 ? (int)(sv.off[li + q + 1] - sv.off[li + q]) : 0;
          const int dm = max(max(dg[0], dg[1]), max(dg[2], dg[3]));
          if (dm <= 0) continue;
          unsigned need = 0u;
          if (WRITE_X) {
            need = (1u << n4) - 1u;
          } else if (dm <= 64) {
            need = project_lean<8, 8, BF16, W, MU_SMEM>(sv, li, n4, si.a0, lane, cx, acc);
          } else {
            for (int h = 0; h < n4; h += 2) {
              const int np = n4 - h < 2 ? n4 - h : 2;
              const int d2 = np == 2 ? max(dg[h], dg[h + 1]) : dg[h];
              if (d2 <= 0) continue;
              if (d2 <= 128) {
                need |= project_lean<16, 8, BF16, W, MU_SMEM>(sv, li + h, np, si.a0, lane, cx,
                                                              acc) << h;
                continue;
              }
              for (int q = h; q < h + np; ++q) {
                if (dg[q] <= 0) continue;
                if (dg[q] <= 256)
                  need |= project_lean<32, 8, BF16, W, MU_SMEM>(sv, li + q, 1, si.a0, lane, cx,
                                                                acc) << q;
                else need |= 1u << q;
              }
            }
          }
          while (need) {
            const int q = __ffs(need) - 1;
            need &= need - 1u;
            const int64_t eb = sv.off[li + q];
            project_multipass<BF16, W>(sv, eb - si.a0, (int64_t)dg[q], eb, lane, cx, acc);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
  }
  __syncthreads();

  // flush the shared-memory accumulators of the hot destinations
  for (int j = tid; j < p.h_y; j += blockDim.x) {
    const unsigned long long v = y_s[j];
    if (v != 0ull) atomicAdd(p.y + j, v);
  }
  // per-CTA objective partials: exact integer sums, converted once
  long long v0 = acc.cx, v1 = acc.wxx;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    v0 += __shfl_xor_sync(0xffffffffu, v0, o);
    v1 += __shfl_xor_sync(0xffffffffu, v1, o);
  }
  if (lane == 0) {
    dred[2 * warp] = v0;
    dred[2 * warp + 1] = v1;
  }
  __syncthreads();
  if (tid == 0) {
    long long s0 = 0, s1 = 0;
    for (int w = 0; w < kThreads / 32; ++w) {
      s0 += dred[2 * w];
      s1 += dred[2 * w + 1];
    }
    p.part[2 * blockIdx.x] = (double)s0 * p.inv_sc;
    p.part[2 * blockIdx.x + 1] = (double)s1 * p.inv_sw;
  }
}

// ---------------------------------------------------- J-length kernels ----
__global__ void prep_mu_kernel(int32_t J, const float* __restrict__ lambda,
                               const float* __restrict__ D, const int32_t* __restrict__ orig_of,
                               float* __restrict__ mu_r) {
  for (int64_t jr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; jr < J;
       jr += (int64_t)gridDim.x * blockDim.x) {
    const int jo = orig_of ? orig_of[jr] : (int)jr;
    const float l = lambda[jo];
    mu_r[jr] = D ? __fmul_rn(D[jo], l) : l;
  }
}

__global__ void epilogue_kernel(EpiParams q) {
  __shared__ double red[3][32];
  double s_mug = 0.0, s_inf = 0.0;
  for (int64_t jr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; jr < q.J;
       jr += (int64_t)gridDim.x * blockDim.x) {
    const double ax = (double)(long long)q.y[jr] * q.inv_sy;
    q.y[jr] = 0ull;
    const double gj = ax - (double)q.b_r[jr];
    const int jo = q.orig_of ? q.orig_of[jr] : (int)jr;
    s_mug += (double)q.mu_r[jr] * gj;
    if (gj > 0.0) s_inf += gj * gj;
    q.grad[jo] = (float)(q.D ? (double)q.D[jo] * gj : gj);
  }
  for (int o = 16; o; o >>= 1) {
    s_mug += __shfl_xor_sync(0xffffffffu, s_mug, o);
    s_inf += __shfl_xor_sync(0xffffffffu, s_inf, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) {
    red[0][w] = s_mug;
    red[1][w] = s_inf;
  }
  __syncthreads();
  __shared__ bool last;
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < nw; ++k) {
      a += red[0][k];
      b += red[1][k];
    }
    q.epi_part[2 * blockIdx.x] = a;
    q.epi_part[2 * blockIdx.x + 1] = b;
    __threadfence();
    const unsigned prev = atomicAdd(&q.status->ticket, 1u);
    last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // fixed-order FP64 combination of every partial (strided per thread, then a
  // fixed shuffle tree and a fixed warp order)
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = threadIdx.x; k < q.npart; k += blockDim.x) {
    v[0] += q.part[2 * k];
    v[1] += q.part[2 * k + 1];
  }
  for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) {
    v[2] += q.epi_part[2 * k];
    v[3] += q.epi_part[2 * k + 1];
  }
  for (int o = 16; o; o >>= 1)
    for (int i = 0; i < 4; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  __shared__ double fin[4][32];
  if (lane == 0)
    for (int i = 0; i < 4; ++i) fin[i][w] = v[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    double cxs = 0.0, wxx = 0.0, mug = 0.0, inf = 0.0;
    for (int k = 0; k < nw; ++k) {
      cxs += fin[0][k];
      wxx += fin[1][k];
      mug += fin[2][k];
      inf += fin[3][k];
    }
    const double gamma = q.gamma_dev ? (double)*q.gamma_dev : q.gamma;
    const double reg = 0.5 * gamma * wxx;
    q.eval_out[0] = cxs + reg + mug;
    q.eval_out[1] = cxs;
    q.eval_out[2] = reg;
    q.eval_out[3] = sqrt(inf);
    q.eval_out[4] = mug;
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

template <bool BF16, bool W, bool MU, bool WX>
static cudaError_t set_smem() {
  return cudaFuncSetAttribute(dualgrad_pass_kernel<BF16, W, MU, WX>,
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
      set_smem<true, false, false, true>(),   set_smem<true, true, false, true>()};
  for (cudaError_t e : es)
    if (e != cudaSuccess) return e;
  return cudaSuccess;
}

cudaError_t launch_prep(const Problem& P, const float* lambda, const float* D, cudaStream_t s) {
  prep_mu_kernel<<<grid_for(P.J, 256, 4 * P.num_sms), 256, 0, s>>>(P.J, lambda, D, P.orig_of,
                                                                     P.mu_r);
  return cudaGetLastError();
}

cudaError_t launch_pass(const Problem& P, const float* gamma_dev, float gamma, float* x_out,
                        cudaStream_t s) {
  PassParams p;
  p.off = P.off;
  p.dst = P.dst;
  p.c = P.c;
  p.a = P.a;
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
  p.sy = ldexpf(1.f, P.exp_y);
  p.sc = ldexpf(1.f, P.exp_c);
  p.sw = ldexpf(1.f, P.exp_w);
  p.inv_sc = ldexp(1.0, -P.exp_c);
  p.inv_sw = ldexp(1.0, -P.exp_w);
  p.part = P.part;
  p.x_out = x_out;
  p.status = P.status;
  const bool bf16 = P.storage == DUALIP_EDGE_BF16;
  const bool mu_all = P.J <= P.h_mu;
  const size_t smem = pass_smem_bytes(P.storage);
  const dim3 grid(P.grid), block(kThreads);
#define DUALIP_LAUNCH(B, W, M, X) dualgrad_pass_kernel<B, W, M, X><<<grid, block, smem, s>>>(p)
  if (x_out) {
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
  return cudaGetLastError();
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
  q.inv_sy = ldexp(1.0, -P.exp_y);
  q.grad = grad;
  q.part = P.part;
  q.npart = P.grid;
  q.epi_part = P.epi_part;
  q.gamma_dev = gamma_dev;
  q.gamma = gamma;
  q.eval_out = eval_out;
  q.status = P.status;
  epilogue_kernel<<<P.epi_blocks, 256, 0, s>>>(q);
  return cudaGetLastError();
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
