// The dual evaluation with several constraint families (Section 3.2,
// Definition 1): every source block of A stacks m diagonal blocks, so an edge
// e = (i, j) carries m coefficients a_{k,e} and enters rows k Jd + j.  The
// projection of a source sees the scores
//     r_e = -(c_e + sum_k a_{k,e} mu_{k Jd + j})
// and the pass scatters a_{k,e} x_e into each of the m rows.  Everything else
// (the J-length prologue and epilogue, the solver) runs on the handle's m Jd
// rows unchanged.
//
// One warp per source, eight per block, reading global memory: the edges of
// a source are contiguous, so a warp's loads coalesce, and the Michelot
// passes over a source re-read lines its first pass brought into L1.  Scores
// are unevaluated FP32 pairs (TwoProduct by FMA for each family, TwoSum
// accumulation) shifted by the source maximum as in the single-family pass,
// so x keeps FP32 accuracy relative to gamma; A x and the objective partials
// are 64-bit fixed-point sums with the handle's scales.
#include <algorithm>

#include "internal.h"

namespace dualip {
namespace {

constexpr int kMultiThreads = 256;
constexpr int kMultiRegs = 4;  // edges per lane held in registers (sources of up to 128 edges)

struct MultiParams {
  const int64_t* off;
  const int32_t* dst;
  const float* c;
  const float* a;  // [m E], family-major
  int64_t I, E;
  int32_t Jd, m;
  const float* mu;  // [m Jd] rows
  const float* gamma_dev;
  float gamma;
  unsigned long long* y;  // [m Jd] fixed point, scale 2^ey
  int ey, ec, ew;
  int weighted, box;
  longlong2* part;  // [gridDim.x]
  float* x_out;     // [E] or null
};

__device__ __forceinline__ float m_two_sum_err(float u, float v, float s) {
  const float bp = __fsub_rn(s, u);
  return __fadd_rn(__fsub_rn(u, __fsub_rn(s, bp)), __fsub_rn(v, bp));
}
__device__ __forceinline__ float m_wsum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float m_wmax(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double m_dsum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ long long m_isum(long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// r = -(c + sum_k a_k mu_k) of edge e as a normalised pair, and its weight
// w = sum_k a_k^2 (1 for a zero column) with primal scaling, else 1.
__device__ __forceinline__ void m_score(const MultiParams& p, int64_t e, int j, float& hi,
                                        float& lo, float& w) {
  float s = p.c[e], err = 0.f, ww = 0.f;
  for (int k = 0; k < p.m; ++k) {
    const float a = __ldg(p.a + (int64_t)k * p.E + e);
    const float mu = __ldg(p.mu + (int64_t)k * p.Jd + j);
    const float q = __fmul_rn(a, mu);
    const float qe = __fmaf_rn(a, mu, -q);
    const float t = __fadd_rn(s, q);
    err = __fadd_rn(err, __fadd_rn(m_two_sum_err(s, q, t), qe));
    s = t;
    ww = __fmaf_rn(a, a, ww);
  }
  const float h0 = -s, l0 = -err;
  hi = __fadd_rn(h0, l0);
  lo = m_two_sum_err(h0, l0, hi);
  w = p.weighted ? (ww != 0.f ? ww : 1.f) : 1.f;
}

// WGT: primal scaling (p.weighted); its instance carries the FP64 rounds.
template <bool WGT>
__global__ void __launch_bounds__(kMultiThreads, WGT ? 3 : 4) multi_pass_kernel(MultiParams p) {
  pdl_wait();  // mu (and the reset accumulator) of the kernels before
  pdl_trigger();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float gamma = p.gamma_dev ? *p.gamma_dev : p.gamma;
  const float sy = ldexpf(1.f, p.ey), sc = ldexpf(1.f, p.ec), sw = ldexpf(1.f, p.ew);
  long long acx = 0, awxx = 0;
  const int64_t nw = (int64_t)gridDim.x * (kMultiThreads / 32);
  auto alpha = [&](float w) { return __frcp_rn(__fmul_rn(gamma, w)); };
  // x of one edge, its scatter into every family's row and its objective terms
  auto emit = [&](int64_t e, int j, float w, float x) {
    if (x > 0.f) {
      for (int f = 0; f < p.m; ++f) {
        const float a = __ldg(p.a + (int64_t)f * p.E + e);
        const long long q = __float2ll_rn(__fmul_rn(__fmul_rn(a, x), sy));
        if (q) atomicAdd(p.y + (int64_t)f * p.Jd + j, (unsigned long long)q);
      }
      acx += __float2ll_rn(__fmul_rn(__fmul_rn(__ldg(p.c + e), x), sc));
      awxx += __float2ll_rn(__fmul_rn(__fmul_rn(w, __fmul_rn(x, x)), sw));
    }
    if (p.x_out) p.x_out[e] = x;
  };
  // one source by the whole warp
  auto warp_source = [&](int64_t e0, int64_t d) {
    if (d <= 32 * kMultiRegs) {
      // the source's scores stay in registers (kMultiRegs per lane): one read
      // of its edges, every gather in flight at once, Michelot's rounds and x
      // from the registers
      int jj[kMultiRegs];
      float hi[kMultiRegs], lo[kMultiRegs], wv[kMultiRegs];
#pragma unroll
      for (int u = 0; u < kMultiRegs; ++u) {
        const int64_t k = lane + 32 * u;
        jj[u] = k < d ? __ldg(p.dst + e0 + k) : 0;
      }
      float rmax = -INFINITY, s0 = 0.f, mb = -INFINITY;
#pragma unroll
      for (int u = 0; u < kMultiRegs; ++u) {
        const int64_t k = lane + 32 * u;
        hi[u] = -INFINITY;
        lo[u] = 0.f;
        wv[u] = 1.f;
        if (k < d) {
          m_score(p, e0 + k, jj[u], hi[u], lo[u], wv[u]);
          const float rf = __fadd_rn(hi[u], lo[u]);
          rmax = fmaxf(rmax, rf);
          if (rf > 0.f) s0 += __fmul_rn(alpha(wv[u]), rf);
          mb = fmaxf(mb, __fsub_rn(rf, __fmul_rn(gamma, wv[u])));
        }
      }
      rmax = m_wmax(rmax);
      s0 = m_wsum(s0);
      mb = m_wmax(mb);
      const int mode = p.box ? 3 : (rmax <= 0.f ? 0 : (s0 <= 1.f ? 1 : 2));
      float t = 0.f;
      double td = 0.0;
      if (mode == 2 && WGT) {
        // FP64 d, sums, t and x: widely spread weights cancel in FP32
        const float slack = __fmul_rn(fabsf(rmax), 0x1p-20f);
        double theta = (double)__fsub_rn(fminf(__fsub_rn(mb, rmax), 0.f), slack);
        float nprev = -1.f;
        td = theta;
        for (int64_t it = 0; it <= d; ++it) {
          double sr = 0.0, sa = 0.0;
          float n = 0.f;
#pragma unroll
          for (int u = 0; u < kMultiRegs; ++u) {
            const double dd = ((double)hi[u] - (double)rmax) + (double)lo[u];
            if (lane + 32 * u < d && dd > theta) {
              const double al = (double)alpha(wv[u]);
              sr += al * dd;
              sa += al;
              n += 1.f;
            }
          }
          sr = m_dsum(sr);
          sa = m_dsum(sa);
          n = m_wsum(n);
          if (n == nprev) break;
          td = (sr - 1.0) / sa;
          nprev = n;
          theta = theta > td ? theta : td;
        }
      } else if (mode == 2) {
        const float slack = __fmul_rn(fabsf(rmax), 0x1p-20f);
        float theta = __fsub_rn(fminf(__fsub_rn(mb, rmax), 0.f), slack), nprev = -1.f;
        t = theta;
        for (int64_t it = 0; it <= d; ++it) {
          float sr = 0.f, sa = 0.f, n = 0.f;
#pragma unroll
          for (int u = 0; u < kMultiRegs; ++u) {
            const float dk = __fadd_rn(__fsub_rn(hi[u], rmax), lo[u]);
            if (lane + 32 * u < d && dk > theta) {
              const float al = alpha(wv[u]);
              sr += __fmul_rn(al, dk);
              sa += al;
              n += 1.f;
            }
          }
          sr = m_wsum(sr);
          sa = m_wsum(sa);
          n = m_wsum(n);
          if (n == nprev) break;
          t = __fdiv_rn(sr - 1.f, sa);
          nprev = n;
          theta = fmaxf(theta, t);
        }
      }
#pragma unroll
      for (int u = 0; u < kMultiRegs; ++u) {
        const int64_t k = lane + 32 * u;
        if (k >= d) continue;
        const float al = alpha(wv[u]);
        float x = 0.f;
        if (mode == 1) {
          const float rf = __fadd_rn(hi[u], lo[u]);
          x = rf > 0.f ? __fmul_rn(al, rf) : 0.f;
        } else if (mode == 2 && WGT) {
          const double dd = ((double)hi[u] - (double)rmax) + (double)lo[u];
          x = dd > td ? (float)((double)al * (dd - td)) : 0.f;
        } else if (mode == 2) {
          const float dk = __fadd_rn(__fsub_rn(hi[u], rmax), lo[u]);
          x = dk > t ? __fmul_rn(al, __fsub_rn(dk, t)) : 0.f;
        } else if (mode == 3) {
          x = fminf(fmaxf(__fmul_rn(al, __fadd_rn(hi[u], lo[u])), 0.f), 1.f);
        }
        emit(e0 + k, jj[u], wv[u], x);
      }
      return;
    }
    // pass 1: maximum score, saturation sum, and the bound max(r - gamma w)
    float rmax = -INFINITY, s0 = 0.f, mb = -INFINITY;
    for (int64_t k = lane; k < d; k += 32) {
      const int64_t e = e0 + k;
      float hi, lo, w;
      m_score(p, e, __ldg(p.dst + e), hi, lo, w);
      const float rf = __fadd_rn(hi, lo);
      rmax = fmaxf(rmax, rf);
      if (rf > 0.f) s0 += __fmul_rn(alpha(w), rf);
      mb = fmaxf(mb, __fsub_rn(rf, __fmul_rn(gamma, w)));
    }
    rmax = m_wmax(rmax);
    s0 = m_wsum(s0);
    mb = m_wmax(mb);
    const int mode = p.box ? 3 : (rmax <= 0.f ? 0 : (s0 <= 1.f ? 1 : 2));
    float t = 0.f;
    double td = 0.0;
    if (mode == 2 && WGT) {  // FP64, as in the register path
      const float slack = __fmul_rn(fabsf(rmax), 0x1p-20f);
      double theta = (double)__fsub_rn(fminf(__fsub_rn(mb, rmax), 0.f), slack);
      float nprev = -1.f;
      td = theta;
      for (int64_t it = 0; it <= d; ++it) {
        double sr = 0.0, sa = 0.0;
        float n = 0.f;
        for (int64_t k = lane; k < d; k += 32) {
          const int64_t e = e0 + k;
          float hi, lo, w;
          m_score(p, e, __ldg(p.dst + e), hi, lo, w);
          const double dd = ((double)hi - (double)rmax) + (double)lo;
          if (dd > theta) {
            const double al = (double)alpha(w);
            sr += al * dd;
            sa += al;
            n += 1.f;
          }
        }
        sr = m_dsum(sr);
        sa = m_dsum(sa);
        n = m_wsum(n);
        if (n == nprev) break;
        td = (sr - 1.0) / sa;
        nprev = n;
        theta = theta > td ? theta : td;
      }
    } else if (mode == 2) {  // Michelot's iteration from a set that holds the active set
      const float slack = __fmul_rn(fabsf(rmax), 0x1p-20f);
      float theta = __fsub_rn(fminf(__fsub_rn(mb, rmax), 0.f), slack), nprev = -1.f;
      t = theta;
      for (int64_t it = 0; it <= d; ++it) {
        float sr = 0.f, sa = 0.f, n = 0.f;
        for (int64_t k = lane; k < d; k += 32) {
          const int64_t e = e0 + k;
          float hi, lo, w;
          m_score(p, e, __ldg(p.dst + e), hi, lo, w);
          const float dk = __fadd_rn(__fsub_rn(hi, rmax), lo);
          if (dk > theta) {
            const float al = alpha(w);
            sr += __fmul_rn(al, dk);
            sa += al;
            n += 1.f;
          }
        }
        sr = m_wsum(sr);
        sa = m_wsum(sa);
        n = m_wsum(n);
        if (n == nprev) break;
        t = __fdiv_rn(sr - 1.f, sa);
        nprev = n;
        theta = fmaxf(theta, t);
      }
    }
    // x, the scatter into every family's row, the objective partials
    for (int64_t k = lane; k < d; k += 32) {
      const int64_t e = e0 + k;
      const int j = __ldg(p.dst + e);
      float hi, lo, w;
      m_score(p, e, j, hi, lo, w);
      const float al = alpha(w);
      float x = 0.f;
      if (mode == 1) {
        const float rf = __fadd_rn(hi, lo);
        x = rf > 0.f ? __fmul_rn(al, rf) : 0.f;
      } else if (mode == 2 && WGT) {
        const double dd = ((double)hi - (double)rmax) + (double)lo;
        x = dd > td ? (float)((double)al * (dd - td)) : 0.f;
      } else if (mode == 2) {
        const float dk = __fadd_rn(__fsub_rn(hi, rmax), lo);
        x = dk > t ? __fmul_rn(al, __fsub_rn(dk, t)) : 0.f;
      } else if (mode == 3) {  // unit box
        x = fminf(fmaxf(__fmul_rn(al, __fadd_rn(hi, lo)), 0.f), 1.f);
      }
      emit(e, j, w, x);
    }
  };
  for (int64_t src = (int64_t)blockIdx.x * (kMultiThreads / 32) + warp; src < p.I; src += nw)
    warp_source(__ldg(p.off + src), __ldg(p.off + src + 1) - __ldg(p.off + src));
  // per-block partials: exact integer sums
  __shared__ longlong2 red[kMultiThreads / 32];
  acx = m_isum(acx);
  awxx = m_isum(awxx);
  if (lane == 0) red[warp] = make_longlong2(acx, awxx);
  __syncthreads();
  if (threadIdx.x == 0) {
    longlong2 tot = red[0];
    for (int w = 1; w < kMultiThreads / 32; ++w) {
      tot.x += red[w].x;
      tot.y += red[w].y;
    }
    p.part[blockIdx.x] = tot;
  }
}

__global__ void row_norm_multi_kernel(const int32_t* __restrict__ dst,
                                      const float* __restrict__ a, int64_t E, int32_t Jd, int m,
                                      int weighted, double* __restrict__ acc) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    double w = 0.0;
    for (int k = 0; k < m; ++k) {
      const double v = (double)a[(int64_t)k * E + e];
      w += v * v;
    }
    if (!weighted) w = 1.0;
    else if (w == 0.0) w = 1.0;
    const int j = dst[e];
    for (int k = 0; k < m; ++k) {
      const double v = (double)a[(int64_t)k * E + e];
      if (v != 0.0) atomicAdd(acc + (int64_t)k * Jd + j, v * v / w);
    }
  }
}

}  // namespace

cudaError_t launch_pass_multi(const Problem& P, const float* gamma_dev, float gamma, float* x_out,
                              cudaStream_t s) {
  MultiParams p;
  p.off = P.off;
  p.dst = P.dst;
  p.c = P.cm;
  p.a = P.am;
  p.I = P.I;
  p.E = P.E;
  p.Jd = P.Jd;
  p.m = P.m;
  p.mu = P.mu_r;
  p.gamma_dev = gamma_dev;
  p.gamma = gamma;
  p.y = P.y;
  p.ey = P.exp_y;
  p.ec = P.exp_c;
  p.ew = P.exp_w;
  p.weighted = P.weighted;
  p.box = P.box;
  p.part = P.part;
  p.x_out = x_out;
  return P.weighted ? launch_pdl(multi_pass_kernel<true>, dim3(P.grid), dim3(kMultiThreads), 0, s, p)
                    : launch_pdl(multi_pass_kernel<false>, dim3(P.grid), dim3(kMultiThreads), 0, s, p);
}

cudaError_t launch_row_norm_multi(const Problem& P, double* acc, cudaStream_t s) {
  if (P.E == 0) return cudaSuccess;
  const int64_t g = std::min<int64_t>((P.E + 255) / 256, 8192);
  row_norm_multi_kernel<<<(int)g, 256, 0, s>>>(P.dst, P.am, P.E, P.Jd, P.m, P.weighted, acc);
  return cudaGetLastError();
}

}  // namespace dualip
