// dualip_dual_grad_noalloc: one dual evaluation that performs no device
// allocation of any kind.
//
// Who needs it: a caller whose device memory is owned by someone else (a
// framework's caching allocator or a pre-planned arena that forbids raw
// cudaMalloc), or a latency-critical request path that cannot afford the
// implicit device synchronisation of cudaMalloc / cudaFree, or a process
// running with the device nearly full.  Such a caller cannot build a problem
// handle (dualip_create allocates the staged copy of the edges), so this entry
// point reads the caller's own device arrays directly and keeps its scratch
// (the A x accumulator, per-block partials and a completion counter) in one
// file-scope __device__ array of fixed size, held by every GPU that loads the
// library until the process exits.
//
// Limits and behaviour:
//  * at most kNaMaxDests destinations (J); larger J is rejected with
//    DUALIP_EINVAL before any device work;
//  * the first call on a device looks up the scratch array's device address
//    (cudaGetSymbolAddress, with that device current) and caches it; make that
//    first call before any stream capture;
//  * every call shares the one scratch array and clears it at its start, so
//    calls whose work overlaps on the GPU (two streams, two threads) race and
//    give wrong results: serialise them;
//  * results are the same quantities as dualip_dual_grad (Section 3.1, Eq. 2
//    and Danskin's gradient), computed by a simpler kernel (one warp per
//    source reading global memory, FP64 atomics for A x), so they agree with
//    the handle-based path within rounding, not bit for bit.  The FP64
//    atomics add in whatever order the warps reach them, so two calls on the
//    same inputs may differ in the last bits;
//  * the cached scratch address belongs to the CUDA context it was looked up
//    in: after a device reset (cudaDeviceReset, or a reset of the primary
//    context by another component of the process) this entry point must not
//    be called again in the same process.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "internal.h"

namespace dualip {
namespace {

constexpr int kNaMaxDests = 1 << 20;   // J limit: 8 MiB of FP64 accumulator
constexpr int kNaMaxBlocks = 1024;     // pass blocks (per-block partial slots)
constexpr int kNaMaxEpiBlocks = 1024;  // epilogue blocks
constexpr int kNaThreads = 256;
constexpr int kNaDevices = 64;
// layout (in 8-byte words): y[kNaMaxDests] | part[2*kNaMaxBlocks] |
// epi[2*kNaMaxEpiBlocks] | ticket
constexpr size_t kNaWords = (size_t)kNaMaxDests + 2 * kNaMaxBlocks + 2 * kNaMaxEpiBlocks + 32;

static __device__ __align__(256) unsigned long long na_scratch[kNaWords];

struct NaParams {
  int64_t I;
  int32_t J;
  const int64_t* off;
  const int32_t* dst;
  const float* c;
  const float* a;
  const float* b;
  const float* lambda;
  float gamma, inv_gamma;
  double gamma_d;
  int weighted;
  double* y;         // scratch [J]
  double* part;      // scratch [2 * pass blocks]
  double* epi;       // scratch [2 * epilogue blocks]
  unsigned* ticket;  // scratch
  unsigned* bad;     // scratch: set when a destination is outside [0, J)
  float* grad;
  double* out;       // [5] dualip_eval order
};

__device__ __forceinline__ float na_two_sum_err(float u, float v, float s) {
  const float bp = __fsub_rn(s, u);
  return __fadd_rn(__fsub_rn(u, __fsub_rn(s, bp)), __fsub_rn(v, bp));
}
// r = -(c + a m) as a normalised pair hi + lo
__device__ __forceinline__ void na_score(float c, float a, float m, float& hi, float& lo) {
  const float p = __fmul_rn(a, m);
  const float pe = __fmaf_rn(a, m, -p);
  const float s = __fadd_rn(c, p);
  const float se = na_two_sum_err(c, p, s);
  const float h0 = -s, l0 = -__fadd_rn(se, pe);
  hi = __fadd_rn(h0, l0);
  lo = na_two_sum_err(h0, l0, hi);
}
__device__ __forceinline__ float na_wsum(float v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float na_wmax(float v) {
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double na_dsum(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double na_dmax(double v) {
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__global__ void na_clear_kernel(NaParams p) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < p.J;
       j += (int64_t)gridDim.x * blockDim.x)
    p.y[j] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *p.ticket = 0u;
    *p.bad = 0u;
  }
}

// One warp per source, exact threshold in shifted coordinates (as the main
// pass): scores r = hi + lo, d = (hi - r_max) + lo, Michelot rounds from
// {d > max(d - gamma w)}, x = alpha (d - t)_+ (or alpha r_+ when the sum
// constraint is slack).
__global__ void __launch_bounds__(kNaThreads) na_pass_kernel(NaParams p) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double acc_cx = 0.0, acc_wxx = 0.0;
  for (int64_t src = wid; src < p.I; src += nw) {
    const int64_t e0 = p.off[src];
    const int64_t d = p.off[src + 1] - e0;
    auto wgt = [&](float av) { return p.weighted ? (av != 0.f ? av * av : 1.f) : 1.f; };
    auto alpha = [&](float w) { return p.weighted ? __frcp_rn(__fmul_rn(p.gamma, w)) : p.inv_gamma; };
    // an edge whose destination is outside [0, J) is skipped (score -inf)
    // and flagged; the call's scalars then come out as NaN
    auto load = [&](int64_t k, int& j, float& c, float& a, float& hi, float& lo) {
      j = __ldg(p.dst + e0 + k);
      c = __ldg(p.c + e0 + k);
      a = __ldg(p.a + e0 + k);
      if ((unsigned)j >= (unsigned)p.J) {
        atomicOr(p.bad, 1u);
        j = 0;
        hi = -CUDART_INF_F;
        lo = 0.f;
        return;
      }
      na_score(c, a, __ldg(p.lambda + j), hi, lo);
    };
    float rmax = -CUDART_INF_F, s0 = 0.f;
    for (int64_t k = lane; k < d; k += 32) {
      int j;
      float c, a, hi, lo;
      load(k, j, c, a, hi, lo);
      rmax = fmaxf(rmax, hi);
      if (hi > 0.f) s0 += __fmul_rn(alpha(wgt(a)), hi);
    }
    rmax = na_wmax(rmax);
    s0 = na_wsum(s0);
    const int mode = rmax <= 0.f ? 0 : (s0 <= 1.f ? 1 : 2);
    if (mode == 0) continue;
    // shifted scores d, the sums, t and x in FP64: with primal scaling the
    // weights of one source may spread widely, and x = alpha (d - t) then
    // cancels in FP32
    auto shifted = [&](float hi, float lo) { return ((double)hi - (double)rmax) + (double)lo; };
    double t = 0.0;
    if (mode == 2) {
      double lb = -CUDART_INF;
      for (int64_t k = lane; k < d; k += 32) {
        int j;
        float c, a, hi, lo;
        load(k, j, c, a, hi, lo);
        lb = fmax(lb, shifted(hi, lo) - (double)__fmul_rn(p.gamma, wgt(a)));
      }
      lb = na_dmax(lb);
      double theta = lb;
      float nprev = -1.f;
      t = lb;
      for (int64_t it = 0; it <= d; ++it) {
        double sr = 0.0, sa = 0.0;
        float n = 0.f;
        for (int64_t k = lane; k < d; k += 32) {
          int j;
          float c, a, hi, lo;
          load(k, j, c, a, hi, lo);
          const double dk = shifted(hi, lo);
          if (dk > theta) {
            const double al = (double)alpha(wgt(a));
            sr += al * dk;
            sa += al;
            n += 1.f;
          }
        }
        sr = na_dsum(sr);
        sa = na_dsum(sa);
        n = na_wsum(n);
        if (n == nprev) break;
        t = (sr - 1.0) / sa;
        nprev = n;
        theta = theta > t ? theta : t;
      }
    }
    for (int64_t k = lane; k < d; k += 32) {
      int j;
      float c, a, hi, lo;
      load(k, j, c, a, hi, lo);
      const float w = wgt(a), al = alpha(w);
      float x = 0.f;
      if (mode == 1) {
        x = hi > 0.f ? __fmul_rn(al, __fadd_rn(hi, lo)) : 0.f;
      } else {
        const double dk = shifted(hi, lo);
        x = dk > t ? (float)((double)al * (dk - t)) : 0.f;
      }
      if (x > 0.f) {
        atomicAdd(p.y + j, (double)a * (double)x);
        acc_cx += (double)c * (double)x;
        acc_wxx += (double)w * (double)x * (double)x;
      }
    }
  }
  for (int o = 16; o; o >>= 1) {
    acc_cx += __shfl_xor_sync(0xffffffffu, acc_cx, o);
    acc_wxx += __shfl_xor_sync(0xffffffffu, acc_wxx, o);
  }
  __shared__ double red[2][kNaThreads / 32];
  if (lane == 0) {
    red[0][threadIdx.x >> 5] = acc_cx;
    red[1][threadIdx.x >> 5] = acc_wxx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0, v = 0.0;
    for (int w = 0; w < kNaThreads / 32; ++w) {
      u += red[0][w];
      v += red[1][w];
    }
    p.part[2 * blockIdx.x] = u;
    p.part[2 * blockIdx.x + 1] = v;
  }
}

// grad = A x - b and the FP64 scalars; the last block combines every partial
// in a fixed order and writes out[0..4].
__global__ void __launch_bounds__(kNaThreads) na_epilogue_kernel(NaParams p, int npart) {
  double s_mug = 0.0, s_inf = 0.0;
  // an edge with a destination outside [0, J) was skipped by the pass: every
  // output is then marked invalid, the gradient as well as the scalars
  const bool bad = *reinterpret_cast<volatile unsigned*>(p.bad) != 0u;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < p.J;
       j += (int64_t)gridDim.x * blockDim.x) {
    const double gj = p.y[j] - (double)p.b[j];
    p.grad[j] = bad ? CUDART_NAN_F : (float)gj;
    s_mug += (double)p.lambda[j] * gj;
    if (gj > 0.0) s_inf += gj * gj;
  }
  for (int o = 16; o; o >>= 1) {
    s_mug += __shfl_xor_sync(0xffffffffu, s_mug, o);
    s_inf += __shfl_xor_sync(0xffffffffu, s_inf, o);
  }
  __shared__ double red[2][kNaThreads / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][w] = s_mug;
    red[1][w] = s_inf;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0, v = 0.0;
    for (int k = 0; k < kNaThreads / 32; ++k) {
      u += red[0][k];
      v += red[1][k];
    }
    p.epi[2 * blockIdx.x] = u;
    p.epi[2 * blockIdx.x + 1] = v;
    __threadfence();
    last = atomicAdd(p.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double cx = 0.0, wxx = 0.0, mug = 0.0, inf = 0.0;
  for (int k = 0; k < npart; ++k) {
    cx += p.part[2 * k];
    wxx += p.part[2 * k + 1];
  }
  for (unsigned k = 0; k < gridDim.x; ++k) {
    mug += p.epi[2 * k];
    inf += p.epi[2 * k + 1];
  }
  const double reg = 0.5 * p.gamma_d * wxx;
  p.out[0] = cx + reg + mug;
  p.out[1] = cx;
  p.out[2] = reg;
  p.out[3] = sqrt(inf);
  p.out[4] = mug;
  if (*p.bad)
    for (int k = 0; k < 5; ++k) p.out[k] = CUDART_NAN;
  *p.ticket = 0u;
}

struct NaDevice {
  unsigned long long* scratch = nullptr;  // device address of na_scratch
  int num_sms = 0;
};
std::mutex g_na_mu;
NaDevice g_na_dev[kNaDevices];

// Once per device, with that device current: the device address of the
// scratch array (host code never names the array itself as an address).
dualip_status na_setup(int dev, NaDevice** out) {
  if (dev < 0 || dev >= kNaDevices) return fail(DUALIP_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_na_mu);
  NaDevice& D = g_na_dev[dev];
  if (!D.scratch) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, na_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "looking up the no-allocation scratch array");
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "querying the SM count");
    D.num_sms = sms;
    D.scratch = static_cast<unsigned long long*>(ptr);
  }
  *out = &D;
  return DUALIP_OK;
}

}  // namespace
}  // namespace dualip

using namespace dualip;

extern "C" dualip_status dualip_dual_grad_noalloc(
    int64_t num_sources, int32_t num_dests, const int64_t* src_offsets, const int32_t* dst,
    const float* c, const float* a, const float* b, int32_t primal_scaling,
    const float* lambda, double gamma, float* grad, double* out_dev, void* stream) {
  if (num_sources < 0 || num_dests < 1)
    return fail(DUALIP_EINVAL, "need num_sources >= 0 and num_dests >= 1");
  if (num_dests > kNaMaxDests)
    return fail(DUALIP_EINVAL, "num_dests exceeds the no-allocation limit of 1048576");
  if (!src_offsets || !b || !lambda || !grad || !out_dev ||
      (num_sources > 0 && (!dst || !c || !a)))
    return fail(DUALIP_EINVAL, "device pointers must be non-NULL");
  if (primal_scaling != 0 && primal_scaling != 1)
    return fail(DUALIP_EINVAL, "primal_scaling must be 0 or 1");
  if (!std::isfinite(gamma) || !(gamma >= 1e-30) || !(gamma <= 1e30))
    return fail(DUALIP_EINVAL, "gamma must be finite and in [1e-30, 1e30]");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  NaDevice* D = nullptr;
  dualip_status st = na_setup(dev, &D);
  if (st) return st;
  NaParams p;
  p.I = num_sources;
  p.J = num_dests;
  p.off = src_offsets;
  p.dst = dst;
  p.c = c;
  p.a = a;
  p.b = b;
  p.lambda = lambda;
  p.gamma = (float)gamma;
  p.inv_gamma = 1.0f / p.gamma;
  p.gamma_d = gamma;
  p.weighted = primal_scaling;
  p.y = reinterpret_cast<double*>(D->scratch);
  p.part = p.y + kNaMaxDests;
  p.epi = p.part + 2 * kNaMaxBlocks;
  p.ticket = reinterpret_cast<unsigned*>(p.epi + 2 * kNaMaxEpiBlocks);
  p.bad = p.ticket + 1;
  p.grad = grad;
  p.out = out_dev;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int jblocks = (int)std::min<int64_t>((num_dests + kNaThreads - 1) / kNaThreads,
                                             std::min(2 * D->num_sms, kNaMaxEpiBlocks));
  int64_t want = (num_sources * 32 + kNaThreads - 1) / kNaThreads;
  const int pblocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, std::min(4 * D->num_sms,
                                                                                 kNaMaxBlocks)));
  na_clear_kernel<<<jblocks, kNaThreads, 0, s>>>(p);
  if ((e = cudaGetLastError())) return cuda_fail(e, "launching the scratch clear");
  na_pass_kernel<<<pblocks, kNaThreads, 0, s>>>(p);
  if ((e = cudaGetLastError())) return cuda_fail(e, "launching the no-allocation pass");
  na_epilogue_kernel<<<jblocks, kNaThreads, 0, s>>>(p, pblocks);
  if ((e = cudaGetLastError())) return cuda_fail(e, "launching the no-allocation epilogue");
  return DUALIP_OK;
}
