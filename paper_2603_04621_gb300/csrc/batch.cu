// Batched form: several matching LPs evaluated, and solved, together.
//
// Each problem keeps the arrays dualip_create made for it (packed edges,
// renumbering, fixed-point scale) and occupies a slot of a device table.  One
// launch of the pass walks a joint list of tiles of all active slots; the
// J-length work walks a joint list of row chunks.  The ascent (Section 5 and
// Appendix B of the paper, as in the single-problem solver) runs per slot:
// every slot has its own gamma schedule, step, momentum and stopping test, and
// a slot that has converged leaves the lists, so its edges are no longer
// streamed.  Every per-problem result equals the problem's own evaluation:
// A x and the objective partials (sum c x, sum w x^2) are exact fixed-point
// sums, so the gradient, c^T x and the ridge term do not depend on the other
// problems; lambda^T (A x - b) and ||(A x - b)_+|| differ from a lone
// evaluation only in the order of their partial sums (chunk order here), and
// are the same in any mix of problems.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "batch.h"

namespace dualip {
namespace {

// ------------------------------------------------ double-float helpers ----
__device__ __forceinline__ float b_two_sum_err(float u, float v, float s) {
  const float vv = __fsub_rn(s, u);
  return __fadd_rn(__fsub_rn(u, __fsub_rn(s, vv)), __fsub_rn(v, vv));
}
__device__ __forceinline__ void b_pair_add(float& h, float& l, float v) {
  const float t = __fadd_rn(h, v);
  l = __fadd_rn(l, b_two_sum_err(h, v, t));
  h = t;
}
__device__ __forceinline__ void b_pair_addp(float& h, float& l, float h2, float l2) {
  const float t = __fadd_rn(h, h2);
  l = __fadd_rn(__fadd_rn(l, l2), b_two_sum_err(h, h2, t));
  h = t;
}
__device__ __forceinline__ void b_warp_pair_sum(float& h, float& l) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, h, o);
    const float l2 = __shfl_xor_sync(0xffffffffu, l, o);
    b_pair_addp(h, l, h2, l2);
  }
}
// Block sum of two pairs (blockDim.x = 256), result in thread 0.
__device__ __forceinline__ float4 block_pair_sum2(float4 v) {
  __shared__ float4 red[8];
  b_warp_pair_sum(v.x, v.y);
  b_warp_pair_sum(v.z, v.w);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      b_pair_addp(t.x, t.y, red[k].x, red[k].y);
      b_pair_addp(t.z, t.w, red[k].z, red[k].w);
    }
  return t;
}

__host__ __device__ inline double slot_gamma(const SlotSolve& s, int32_t k) {
  double g = s.gamma0;
  if (s.halve_every > 0) g = ldexp(s.gamma0, -(k / s.halve_every));
  return g > s.gamma_final ? g : s.gamma_final;
}
__device__ inline bool slot_restart(const SlotSolve& s, int32_t k) {
  return s.restart && k > 0 && slot_gamma(s, k) != slot_gamma(s, k - 1);
}

// ------------------------------------------------- J-length kernels ----
// Rows of chunk c are rows [r0, r1) of the chunk's slot in renumbered order.
// API mode: mu_r[jr] = lambda[joff + orig_of[jr]].  Solver mode (before a
// slot's first iteration; later ones get theirs from bstep and bnorms): the
// ascent's point y (renumbered) times the row scale, with the momentum restart
// at a gamma change; the first chunk of a slot publishes the slot's gamma.
__global__ void bprep_kernel(const RowChunk* __restrict__ rc, const SlotDesc* __restrict__ sd,
                             const float* __restrict__ lam, int solver, SlotSolve* ss,
                             float* gamma_f, double* gamma_d) {
  pdl_trigger();  // the pass may launch (this kernel itself is a plain launch)
  const RowChunk ch = rc[blockIdx.x];
  const SlotDesc& d = sd[ch.slot];
  if (!solver) {
    for (int jr = ch.r0 + threadIdx.x; jr < ch.r1; jr += blockDim.x)
      d.mu_r[jr] = lam[d.joff + d.orig_of[jr]];
    return;
  }
  const SlotSolve& st = ss[ch.slot];
  const bool rs = slot_restart(st, st.k);
  for (int jr = ch.r0 + threadIdx.x; jr < ch.r1; jr += blockDim.x) {
    float yj = d.yv[jr];
    if (rs) {
      yj = d.lam[jr];
      d.yv[jr] = yj;
    }
    d.mu_r[jr] = __fmul_rn(d.D[jr], yj);
  }
  if (ch.r0 == 0 && threadIdx.x == 0) {
    const double g = slot_gamma(st, st.k);
    gamma_f[ch.slot] = (float)g;
    gamma_d[ch.slot] = (double)(float)g;  // the pass projects with the FP32 value
  }
}

// grad = D (A x - b) (solver: renumbered G; API: caller's order at joff),
// the fixed-point accumulator reset, and per-chunk FP32-pair partials
// (mu^T g, ||g_+||^2).  The last block combines, per active slot and in chunk
// order, the chunk partials with the pass's per-slot sums into the five
// scalars of dualip_eval.
__global__ void bepi_kernel(const RowChunk* __restrict__ rc, int nchunks,
                            const SlotDesc* __restrict__ sd, float* __restrict__ grad, int solver,
                            float4* __restrict__ cpart, const int32_t* __restrict__ act, int nact,
                            const int2* __restrict__ crange, long long* slot_part,
                            const double* __restrict__ gamma_d, double* eval, unsigned* ticket) {
  pdl_wait();  // A x and the partials of the pass
  pdl_trigger();
  const RowChunk ch = rc[blockIdx.x];
  const SlotDesc& d = sd[ch.slot];
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int jr = ch.r0 + threadIdx.x; jr < ch.r1; jr += blockDim.x) {
    const long long yq = (long long)__ldcg(d.y + jr);
    d.y[jr] = 0ull;
    const float fh = __ll2float_rn(yq);
    const float fl = __ll2float_rn(yq - __float2ll_rn(fh));
    const float ah = __fmul_rn(fh, d.inv_sy), al = __fmul_rn(fl, d.inv_sy);
    const float b = d.b_r[jr];
    const float t = __fsub_rn(ah, b);
    const float e = __fadd_rn(b_two_sum_err(ah, -b, t), al);
    const float g = __fadd_rn(t, e);
    const float gl = b_two_sum_err(t, e, g);
    const float m = d.mu_r[jr];
    const float pm = __fmul_rn(m, g);
    b_pair_add(v.x, v.y, pm);
    v.y = __fadd_rn(v.y, __fmaf_rn(m, gl, __fmaf_rn(m, g, -pm)));
    if (g > 0.f) {
      const float sq = __fmul_rn(g, g);
      b_pair_add(v.z, v.w, sq);
      v.w = __fadd_rn(v.w, __fmaf_rn(2.f * g, gl, __fmaf_rn(g, g, -sq)));
    }
    if (solver) {
      const float dj = d.D[jr];
      d.G[jr] = __fmaf_rn(dj, g, __fmul_rn(dj, gl));
    } else {
      grad[d.joff + d.orig_of[jr]] = __fadd_rn(g, gl);
    }
  }
  const float4 t = block_pair_sum2(v);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    cpart[blockIdx.x] = t;
    __threadfence();
    last = atomicAdd(ticket, 1u) == (unsigned)nchunks - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int a = threadIdx.x; a < nact; a += blockDim.x) {
    const int s = act[a];
    const int2 cr = crange[s];
    double mug = 0.0, inf = 0.0;  // chunk pairs combined in FP64, in chunk order
    for (int c = cr.x; c < cr.y; ++c) {
      const float4 u = __ldcg(cpart + c);
      mug += (double)u.x + (double)u.y;
      inf += (double)u.z + (double)u.w;
    }
    // the pass's exact fixed-point sums, in the slot's scales
    const SlotDesc& ds = sd[s];
    const double cx = ldexp((double)__ldcg(slot_part + 2 * s), -ds.ec);
    const double wxx = ldexp((double)__ldcg(slot_part + 2 * s + 1), -ds.ew);
    slot_part[2 * s] = 0;
    slot_part[2 * s + 1] = 0;
    const double reg = 0.5 * gamma_d[s] * wxx;
    double* o = eval + 5 * (size_t)s;
    o[0] = cx + reg + mug;
    o[1] = cx;
    o[2] = reg;
    o[3] = sqrt(inf);
    o[4] = mug;
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

// ||y_k - y_{k-1}||^2 and ||G_k - G_{k-1}||^2 per chunk; the last block turns
// them, per active slot, into the step (secant estimate capped by
// max_step gamma / gamma0), the momentum weight and the stopping quantities,
// and advances the slot's iteration counter.
__global__ void bnorms_kernel(const RowChunk* __restrict__ rc, int nchunks,
                              const SlotDesc* __restrict__ sd, SlotSolve* ss,
                              float4* __restrict__ cpart, const int32_t* __restrict__ act,
                              int nact, const int2* __restrict__ crange,
                              const double* __restrict__ eval, unsigned* ticket,
                              float* gamma_f, double* gamma_d) {
  pdl_wait();  // G and the scalars of the epilogue
  pdl_trigger();
  const RowChunk ch = rc[blockIdx.x];
  const SlotDesc& d = sd[ch.slot];
  const SlotSolve& st = ss[ch.slot];
  const bool have_prev = st.k > 0 && !slot_restart(st, st.k);
  // FP64 per row and through the trees (the step and the restart test read them)
  double dy = 0.0, dg = 0.0;
  if (have_prev) {
    for (int j = ch.r0 + threadIdx.x; j < ch.r1; j += blockDim.x) {
      const double u = (double)d.yv[j] - (double)d.yp[j];
      const double w = (double)d.G[j] - (double)d.Gp[j];
      dy += u * u;
      dg += w * w;
    }
  }
  __shared__ double2 red[8];
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    dy += __shfl_xor_sync(0xffffffffu, dy, o);
    dg += __shfl_xor_sync(0xffffffffu, dg, o);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_double2(dy, dg);
  __syncthreads();
  __shared__ bool last;
  double2* cpd = reinterpret_cast<double2*>(cpart);  // same 16 bytes per chunk
  if (threadIdx.x == 0) {
    double2 t = red[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
      t.x += red[k].x;
      t.y += red[k].y;
    }
    cpd[blockIdx.x] = t;
    __threadfence();
    last = atomicAdd(ticket, 1u) == (unsigned)nchunks - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int a = threadIdx.x; a < nact; a += blockDim.x) {
    const int s = act[a];
    const int2 cr = crange[s];
    double sdy = 0.0, sdg = 0.0;
    for (int c = cr.x; c < cr.y; ++c) {
      const double2 u = __ldcg(cpd + c);
      sdy += u.x;
      sdg += u.y;
    }
    SlotSolve& S = ss[s];
    const int32_t k = S.k;
    const bool hp = k > 0 && !slot_restart(S, k);
    const double gk = slot_gamma(S, k);
    const double eta_max = S.max_step * gk / S.gamma0;
    double eta;
    if (hp) eta = sdg > 0.0 ? fmin(eta_max, sqrt(sdy) / sqrt(sdg)) : eta_max;
    else eta = fmin(S.init_step, eta_max);
    const double* o = eval + 5 * (size_t)s;
    const double g = o[0], p = o[1] + o[2];
    // momentum restarts at a gamma change, and (restart_dec) when the dual
    // objective fell since the previous evaluation at the same gamma
    const bool dec = S.restart_dec && hp && g < S.g_prev;
    const double tk = (slot_restart(S, k) || dec) ? 1.0 : S.t;
    const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tk * tk));
    S.eta = eta;
    S.beta = (tk - 1.0) / tn;
    S.t = tn;
    S.sdy = sdy;
    S.sdg = sdg;
    S.g_prev = g;
    S.gap_rel = fabs(o[4]) / fmax(1.0, fmax(fabs(p), fabs(g)));
    S.infeas_rel = o[3] / fmax(1.0, S.bnorm);
    S.last_gamma = gk;
    S.k = k + 1;
    const double gn = slot_gamma(S, k + 1);  // for the next iteration's pass and scalars
    gamma_f[s] = (float)gn;
    gamma_d[s] = (double)(float)gn;
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

// lambda_{k+1} = max(0, y_k + eta G_k), y_{k+1} = max(0, lambda_{k+1} +
// beta (lambda_{k+1} - lambda_k)), per slot with its own eta and beta.  Runs
// after bnorms, which has already advanced k; eta and beta are those of the
// evaluated point.
__global__ void bstep_kernel(const RowChunk* __restrict__ rc, const SlotDesc* __restrict__ sd,
                             const SlotSolve* __restrict__ ss) {
  pdl_wait();  // eta and beta of bnorms
  pdl_trigger();
  const RowChunk ch = rc[blockIdx.x];
  const SlotDesc& d = sd[ch.slot];
  const SlotSolve& st = ss[ch.slot];
  const float eta = (float)st.eta, beta = (float)st.beta;
  // the next iteration's point (bnorms has advanced k): a restart at a gamma
  // change puts y at lambda; then its mu
  const bool rs = slot_restart(st, st.k);
  for (int j = ch.r0 + threadIdx.x; j < ch.r1; j += blockDim.x) {
    const float yk = d.yv[j], g = d.G[j], lk = d.lam[j];
    float ln = __fmaf_rn(eta, g, yk);
    ln = ln > 0.f ? ln : 0.f;
    float yn = __fmaf_rn(beta, __fsub_rn(ln, lk), ln);
    yn = yn > 0.f ? yn : 0.f;
    if (rs) yn = ln;
    d.yp[j] = yk;
    d.Gp[j] = g;
    d.lam[j] = ln;
    d.yv[j] = yn;
    d.mu_r[j] = __fmul_rn(d.D[j], yn);
  }
}

// lambda' = max(0, lambda_caller / D) in renumbered order (0 without an
// input), y = y_prev = lambda'.
__global__ void binit_kernel(const RowChunk* __restrict__ rc, const SlotDesc* __restrict__ sd,
                             const float* __restrict__ lam_in) {
  const RowChunk ch = rc[blockIdx.x];
  const SlotDesc& d = sd[ch.slot];
  for (int j = ch.r0 + threadIdx.x; j < ch.r1; j += blockDim.x) {
    const float l = lam_in ? lam_in[d.joff + d.orig_of[j]] / d.D[j] : 0.f;
    const float c = l > 0.f ? l : 0.f;
    d.lam[j] = c;
    d.yv[j] = c;
    d.yp[j] = c;
    d.G[j] = 0.f;
    d.Gp[j] = 0.f;
  }
}

// lambda_caller = D y_prev (the point of the last evaluation), caller's order.
__global__ void bfinal_kernel(const RowChunk* __restrict__ rc, const SlotDesc* __restrict__ sd,
                              float* __restrict__ lam_out) {
  const RowChunk ch = rc[blockIdx.x];
  const SlotDesc& d = sd[ch.slot];
  for (int j = ch.r0 + threadIdx.x; j < ch.r1; j += blockDim.x)
    lam_out[d.joff + d.orig_of[j]] = __fmul_rn(d.D[j], d.yp[j]);
}

}  // namespace

// ------------------------------------------------------------ host side ----

void free_prof(Batch& B) {
  for (cudaEvent_t ev : B.prof_ev)
    if (ev) cudaEventDestroy(ev);
  B.prof_ev.clear();
  B.prof_used = B.prof_max = 0;
}


void batch_free(Batch& B) {
  if (B.stream) cudaStreamSynchronize(B.stream);
  if (B.graph) cudaGraphExecDestroy(B.graph);
  void* bufs[] = {B.d_slots, B.d_gamma_f, B.d_gamma_d, B.d_slot_part, B.d_eval, B.d_ss, B.d_act,
                  B.d_crange, B.d_tickets, B.d_status, B.d_jt, B.d_rc, B.d_cpart, B.d_rc2};
  for (void* p : bufs)
    if (p) cudaFree(p);
  for (float* p : B.vecs)
    if (p) cudaFree(p);
  if (B.h_gamma) cudaFreeHost(B.h_gamma);
  if (B.h_eval) cudaFreeHost(B.h_eval);
  if (B.h_ss) cudaFreeHost(B.h_ss);
  if (B.ev) cudaEventDestroy(B.ev);
  if (B.ev_stage) cudaEventDestroy(B.ev_stage);
  if (B.ev_use) cudaEventDestroy(B.ev_use);
  free_prof(B);
  if (B.stream) cudaStreamDestroy(B.stream);
}

void slot_tiles(const Problem& P, int slot, int64_t max_e, int64_t max_s,
                std::vector<JointTile>& out) {
  std::vector<int64_t> t, te;
  build_tiles(P.off_host, t, te, max_e, max_s);
  out.clear();
  out.reserve(t.size());
  for (size_t k = 0; k + 1 < t.size(); ++k)
    out.push_back(JointTile{t[k], t[k + 1], te[k], te[k + 1], slot, 0});
}

cudaError_t build_slot_tiles(Batch& B) {
  B.tiles.assign(B.n, {});
  for (int s = 0; s < B.n; ++s)
    if (B.prob[s]) slot_tiles(*B.prob[s], s, B.tile_edges, B.tile_sources, B.tiles[s]);
  B.lists_ok = false;
  return cudaSuccess;
}

// Joint tile and row-chunk lists of the active slots, uploaded on B.stream.
cudaError_t rebuild_lists(Batch& B) {
  if (B.lists_ok) return cudaSuccess;
  B.jt_host.clear();
  B.rc_host.clear();
  B.act_host.clear();
  B.crange_host.assign(B.n, int2{0, 0});
  B.has_big = false;
  for (int s = 0; s < B.n; ++s) {
    if (!B.active[s]) continue;
    B.act_host.push_back(s);
    B.jt_host.insert(B.jt_host.end(), B.tiles[s].begin(), B.tiles[s].end());
    for (const JointTile& t : B.tiles[s])  // a source larger than a stage is read from memory
      B.has_big = B.has_big || t.e1 - t.e0 > tile_edges_for(B.storage);
    const int c0 = (int)B.rc_host.size();
    for (int32_t r = 0; r < B.prob[s]->J; r += kChunkRows)
      B.rc_host.push_back(RowChunk{s, r, std::min<int32_t>(B.prob[s]->J, r + kChunkRows), 0});
    B.crange_host[s] = int2{c0, (int)B.rc_host.size()};
  }
  B.ntiles = (int64_t)B.jt_host.size();
  B.nchunks = (int)B.rc_host.size();
  if (B.lean_auto) {
    // 80-edge lean windows pay off when few sources need an 8-lane pass
    int64_t over = 0, all = 0;
    for (int s = 0; s < B.n; ++s)
      if (B.active[s]) {
        over += B.over76[s];
        all += B.prob[s]->I;
      }
    B.lean80 = over * 50 < all ? 1 : 0;
  }
  cudaError_t e;
  // the lists may still be read by queued work, here or on a caller's stream
  cudaStreamSynchronize(B.stream);
  cudaEventSynchronize(B.ev_use);
  if ((e = grow(&B.d_jt, B.jt_cap, B.jt_host.size()))) return e;
  size_t rc_cap = B.rc_cap;
  if ((e = grow(&B.d_rc, B.rc_cap, B.rc_host.size()))) return e;
  if (B.rc_cap != rc_cap || !B.d_cpart) {
    if (B.d_cpart) cudaFree(B.d_cpart);
    if ((e = cudaMalloc(&B.d_cpart, sizeof(float4) * B.rc_cap))) return e;
  }
  if ((!B.jt_host.empty() &&
       (e = cudaMemcpyAsync(B.d_jt, B.jt_host.data(), sizeof(JointTile) * B.jt_host.size(),
                            cudaMemcpyHostToDevice, B.stream))) ||
      (!B.rc_host.empty() &&
       (e = cudaMemcpyAsync(B.d_rc, B.rc_host.data(), sizeof(RowChunk) * B.rc_host.size(),
                            cudaMemcpyHostToDevice, B.stream))) ||
      (!B.act_host.empty() &&
       (e = cudaMemcpyAsync(B.d_act, B.act_host.data(), sizeof(int32_t) * B.act_host.size(),
                            cudaMemcpyHostToDevice, B.stream))) ||
      (e = cudaMemcpyAsync(B.d_crange, B.crange_host.data(), sizeof(int2) * B.n,
                           cudaMemcpyHostToDevice, B.stream)) ||
      (e = cudaStreamSynchronize(B.stream)))
    return e;
  B.grid = (int)std::max<int64_t>(1, std::min<int64_t>(B.num_sms, B.ntiles));
  if (B.graph) cudaGraphExecDestroy(B.graph);
  B.graph = nullptr;
  B.lists_ok = true;
  return cudaSuccess;
}

cudaError_t upload_slots(Batch& B) {
  return cudaMemcpyAsync(B.d_slots, B.desc.data(), sizeof(SlotDesc) * B.n, cudaMemcpyHostToDevice,
                         B.stream);
}

// One evaluation of every active slot on stream s.  solver: the ascent's
// point and vectors; otherwise lam / grad are joint caller vectors.
cudaError_t enqueue_batch_eval(Batch& B, const float* lam, float* grad, int solver,
                               cudaStream_t s) {
  if (B.nchunks == 0) return cudaSuccess;
  cudaError_t e;
  cudaEvent_t* ev = nullptr;
  if (!solver && B.prof_used < B.prof_max) ev = &B.prof_ev[4 * (size_t)B.prof_used++];
  if (ev && (e = cudaEventRecord(ev[0], s))) return e;
  if (!solver) {  // the solver's mu and gamma come from the previous iteration
    bprep_kernel<<<B.nchunks, 256, 0, s>>>(B.d_rc, B.d_slots, lam, solver, B.d_ss, B.d_gamma_f,
                                           B.d_gamma_d);
    if ((e = cudaGetLastError())) return e;
  }
  if (ev && (e = cudaEventRecord(ev[1], s))) return e;
  if ((e = launch_pass_batch(B.storage, B.weighted, B.d_jt, B.ntiles, B.d_slots, B.d_gamma_f,
                             B.d_slot_part, B.d_status, B.grid, B.lean80, B.has_big, s)))
    return e;
  if (ev && (e = cudaEventRecord(ev[2], s))) return e;
  if ((e = launch_pdl(bepi_kernel, dim3(B.nchunks), dim3(256), 0, s, (const RowChunk*)B.d_rc,
                      B.nchunks, (const SlotDesc*)B.d_slots, grad, solver, B.d_cpart,
                      (const int32_t*)B.d_act, (int)B.act_host.size(), (const int2*)B.d_crange,
                      B.d_slot_part, (const double*)B.d_gamma_d, B.d_eval, B.d_tickets)))
    return e;
  if (ev && (e = cudaEventRecord(ev[3], s))) return e;
  return cudaSuccess;
}

cudaError_t enqueue_batch_iteration(Batch& B, cudaStream_t s) {
  cudaError_t e;
  if ((e = enqueue_batch_eval(B, nullptr, nullptr, 1, s))) return e;
  if (B.nchunks == 0) return cudaSuccess;
  if ((e = launch_pdl(bnorms_kernel, dim3(B.nchunks), dim3(256), 0, s, (const RowChunk*)B.d_rc,
                      B.nchunks, (const SlotDesc*)B.d_slots, B.d_ss, B.d_cpart,
                      (const int32_t*)B.d_act, (int)B.act_host.size(), (const int2*)B.d_crange,
                      (const double*)B.d_eval, B.d_tickets + 1, B.d_gamma_f, B.d_gamma_d)))
    return e;
  return launch_pdl(bstep_kernel, dim3(B.nchunks), dim3(256), 0, s, (const RowChunk*)B.d_rc,
                    (const SlotDesc*)B.d_slots, (const SlotSolve*)B.d_ss);
}

cudaError_t run_batch_chunk(Batch& B, int n, bool use_graph) {
  cudaError_t e;
  if (!use_graph) {
    for (int i = 0; i < n; ++i)
      if ((e = enqueue_batch_iteration(B, B.stream))) return e;
    return cudaSuccess;
  }
  if (!B.graph || B.graph_len != n) {
    if (B.graph) cudaGraphExecDestroy(B.graph);
    B.graph = nullptr;
    cudaGraph_t g = nullptr;
    if ((e = cudaStreamBeginCapture(B.stream, cudaStreamCaptureModeThreadLocal))) return e;
    for (int i = 0; i < n && !e; ++i) e = enqueue_batch_iteration(B, B.stream);
    const cudaError_t e2 = cudaStreamEndCapture(B.stream, &g);
    if (e || e2) {
      if (g) cudaGraphDestroy(g);
      return e ? e : e2;
    }
    e = cudaGraphInstantiate(&B.graph, g, 0);
    cudaGraphDestroy(g);
    if (e) return e;
    B.graph_len = n;
  }
  return cudaGraphLaunch(B.graph, B.stream);
}

dualip_status batch_status(Batch& B) {
  DeviceStatus h{};
  cudaError_t e = cudaMemcpyAsync(&h, B.d_status, sizeof(h), cudaMemcpyDeviceToHost, B.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B.stream);
  if (e != cudaSuccess) return cuda_fail(e, "reading the batch status");
  if (h.err & kErrTimeout) return fail(DUALIP_ETIMEOUT, "a device wait timed out in a batched pass");
  if (h.err) return fail(DUALIP_EINVAL, "a batched pass met an invalid tile");
  return DUALIP_OK;
}

static cudaError_t batch_alloc_parts(Batch& B, int capacity, int storage, int weighted,
                                     int num_sms) {
  const int n = capacity;
  B.tile_edges = tile_edges_for(storage);
  B.n = n;
  B.storage = storage;
  B.weighted = weighted;
  B.num_sms = num_sms;
  B.prob.assign(n, nullptr);
  B.desc.assign(n, SlotDesc{});
  B.active.assign(n, 0);
  B.vecs.assign(n, nullptr);
  B.tiles.assign(n, {});
  B.over76.assign(n, 0);
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&B.stream, cudaStreamNonBlocking)) ||
      (e = cudaEventCreateWithFlags(&B.ev, cudaEventDisableTiming)) ||
      (e = cudaEventCreateWithFlags(&B.ev_stage, cudaEventDisableTiming)) ||
      (e = cudaEventCreateWithFlags(&B.ev_use, cudaEventDisableTiming)) ||
      (e = cudaMalloc(&B.d_slots, sizeof(SlotDesc) * n)) ||
      (e = cudaMalloc(&B.d_gamma_f, sizeof(float) * n)) ||
      (e = cudaMalloc(&B.d_gamma_d, sizeof(double) * n)) ||
      (e = cudaMalloc(&B.d_slot_part, sizeof(long long) * 2 * n)) ||
      (e = cudaMalloc(&B.d_eval, sizeof(double) * 5 * n)) ||
      (e = cudaMalloc(&B.d_ss, sizeof(SlotSolve) * n)) ||
      (e = cudaMalloc(&B.d_act, sizeof(int32_t) * n)) ||
      (e = cudaMalloc(&B.d_crange, sizeof(int2) * n)) ||
      (e = cudaMalloc(&B.d_tickets, sizeof(unsigned) * 2)) ||
      (e = cudaMalloc(&B.d_status, sizeof(DeviceStatus))) ||
      (e = cudaMallocHost(&B.h_gamma, sizeof(double) * 2 * n)) ||
      (e = cudaMallocHost(&B.h_eval, sizeof(double) * 5 * n)) ||
      (e = cudaMallocHost(&B.h_ss, sizeof(SlotSolve) * n)))
    return e;
  if ((e = cudaMemsetAsync(B.d_slot_part, 0, sizeof(long long) * 2 * n, B.stream)) ||
      (e = cudaMemsetAsync(B.d_tickets, 0, sizeof(unsigned) * 2, B.stream)) ||
      (e = cudaMemsetAsync(B.d_status, 0, sizeof(DeviceStatus), B.stream)) ||
      (e = cudaMemsetAsync(B.d_eval, 0, sizeof(double) * 5 * n, B.stream)) ||
      (e = cudaMemsetAsync(B.d_ss, 0, sizeof(SlotSolve) * n, B.stream)) ||
      (e = cudaMemsetAsync(B.d_slots, 0, sizeof(SlotDesc) * n, B.stream)) ||
      (e = cudaEventRecord(B.ev_stage, B.stream)) || (e = cudaEventRecord(B.ev_use, B.stream)) ||
      (e = cudaStreamSynchronize(B.stream)))
    return e;
  return cudaSuccess;
}

// On failure, everything allocated so far is released and B is left empty.
cudaError_t batch_alloc(Batch& B, int capacity, int storage, int weighted, int num_sms) {
  const cudaError_t e = batch_alloc_parts(B, capacity, storage, weighted, num_sms);
  if (e) {
    batch_free(B);
    B = Batch{};
  }
  return e;
}

SlotDesc slot_desc(Problem& P, int64_t joff) {
  SlotDesc d{};
  d.off = P.off32;
  d.dst = P.dst;
  d.ca2 = P.ca2;
  d.ca = P.ca;
  d.mu_r = P.mu_r;
  d.y = P.y;
  d.orig_of = P.orig_of;
  d.b_r = P.b_r;
  d.J = P.J;
  d.h_mu = P.h_mu;
  d.h_y = P.h_y;
  d.sy = ldexpf(1.0f, P.exp_y);
  d.inv_sy = ldexpf(1.0f, -P.exp_y);
  d.ec = P.exp_c;
  d.ew = P.exp_w;
  d.joff = joff;
  return d;
}

static cudaError_t slot_chunks(Batch& B, int slot) {
  std::vector<RowChunk> rc;
  for (int32_t r = 0; r < B.prob[slot]->J; r += kChunkRows)
    rc.push_back(RowChunk{slot, r, std::min<int32_t>(B.prob[slot]->J, r + kChunkRows), 0});
  cudaError_t e;
  if ((e = grow(&B.d_rc2, B.rc2_cap, rc.size()))) return e;
  B.nrc2 = (int)rc.size();
  return rc.empty() ? cudaSuccess
                    : cudaMemcpyAsync(B.d_rc2, rc.data(), sizeof(RowChunk) * rc.size(),
                                      cudaMemcpyHostToDevice, B.stream);
}

SlotSolve slot_solve_init(const dualip_solve_opts& o, double bnorm) {
  SlotSolve S;
  std::memset(&S, 0, sizeof(S));
  S.gamma0 = o.gamma0;
  S.gamma_final = o.gamma_final;
  S.max_step = o.max_step;
  S.init_step = o.init_step;
  S.bnorm = bnorm;
  S.halve_every = o.halve_every;
  S.restart = o.restart_on_gamma_change ? 1 : 0;
  S.restart_dec = o.restart_on_decrease ? 1 : 0;
  S.t = 1.0;
  return S;
}

int batch_attach(Batch& B, Problem* P, const dualip_solve_opts& o, cudaError_t* err) {
  *err = cudaSuccess;
  int s = -1;
  for (int k = 0; k < B.n && s < 0; ++k)
    if (!B.prob[k]) s = k;
  if (s < 0) return -1;
  cudaError_t e;
  float* v = nullptr;
  const int32_t J = P->J;
  // stream-ordered: no device-wide synchronisation while other work runs
  if ((e = cudaMallocAsync(&v, sizeof(float) * 6 * std::max<int32_t>(J, 1), B.stream))) {
    *err = e;
    return -1;
  }
  B.prob[s] = P;
  B.vecs[s] = v;
  SlotDesc d = slot_desc(*P, 0);
  d.lam = v;
  d.yv = v + J;
  d.yp = v + 2 * (size_t)J;
  d.G = v + 3 * (size_t)J;
  d.Gp = v + 4 * (size_t)J;
  d.D = v + 5 * (size_t)J;
  B.desc[s] = d;
  slot_tiles(*P, s, B.tile_edges, B.tile_sources, B.tiles[s]);
  int64_t over = 0;
  for (size_t i = 0; i + 1 < P->off_host.size(); ++i)
    over += P->off_host[i + 1] - P->off_host[i] > 76 ? 1 : 0;
  B.over76[s] = over;
  B.h_ss[s] = slot_solve_init(o, P->bnorm);
  if ((e = compute_row_scale(*P, o.row_normalize ? 1 : 0, d.D, B.stream)) ||
      (e = upload_slots(B)) ||
      (e = cudaMemcpyAsync(B.d_ss + s, B.h_ss + s, sizeof(SlotSolve), cudaMemcpyHostToDevice,
                           B.stream)) ||
      (e = cudaMemsetAsync(B.d_slot_part + 2 * s, 0, 2 * sizeof(long long), B.stream)) ||
      (e = slot_chunks(B, s))) {
    *err = e;
    batch_detach(B, s);
    return -1;
  }
  if (B.nrc2) {
    binit_kernel<<<B.nrc2, 256, 0, B.stream>>>(B.d_rc2, B.d_slots, nullptr);
    bprep_kernel<<<B.nrc2, 256, 0, B.stream>>>(B.d_rc2, B.d_slots, nullptr, 1, B.d_ss,
                                               B.d_gamma_f, B.d_gamma_d);
    if ((e = cudaGetLastError()) || (e = cudaStreamSynchronize(B.stream))) {
      *err = e;
      batch_detach(B, s);
      return -1;
    }
  }
  B.active[s] = 1;
  B.lists_ok = false;
  return s;
}

cudaError_t batch_write_lambda(Batch& B, int slot, float* lam_out) {
  cudaError_t e = slot_chunks(B, slot);
  if (e) return e;
  if (B.nrc2) {
    bfinal_kernel<<<B.nrc2, 256, 0, B.stream>>>(B.d_rc2, B.d_slots, lam_out);
    if ((e = cudaGetLastError())) return e;
  }
  return cudaStreamSynchronize(B.stream);
}

void batch_detach(Batch& B, int slot) {
  if (B.vecs[slot]) cudaFreeAsync(B.vecs[slot], B.stream);
  cudaStreamSynchronize(B.stream);
  B.vecs[slot] = nullptr;
  B.prob[slot] = nullptr;
  B.desc[slot] = SlotDesc{};
  B.tiles[slot].clear();
  B.active[slot] = 0;
  B.lists_ok = false;
}

cudaError_t batch_read_state(Batch& B) {
  cudaError_t e;
  if ((e = cudaMemcpyAsync(B.h_ss, B.d_ss, sizeof(SlotSolve) * B.n, cudaMemcpyDeviceToHost,
                           B.stream)) ||
      (e = cudaMemcpyAsync(B.h_eval, B.d_eval, sizeof(double) * 5 * B.n, cudaMemcpyDeviceToHost,
                           B.stream)))
    return e;
  return cudaStreamSynchronize(B.stream);
}

}  // namespace dualip

struct dualip_batch {
  dualip::Batch b;
};

using namespace dualip;

namespace {

bool gamma_ok(double g) { return std::isfinite(g) && g >= 1e-30 && g <= 1e30; }

// joint lists of every slot (API calls evaluate all problems)
dualip_status ensure_all_active(Batch& B) {
  bool all = true;
  for (int s = 0; s < B.n; ++s) all = all && B.active[s];
  if (all && B.lists_ok) return DUALIP_OK;
  std::fill(B.active.begin(), B.active.end(), 1);
  B.lists_ok = false;
  cudaError_t e = rebuild_lists(B);
  return e ? cuda_fail(e, "building the batch lists") : DUALIP_OK;
}

// order stream b after stream a
cudaError_t order(Batch& B, cudaStream_t a, cudaStream_t b) {
  cudaError_t e = cudaEventRecord(B.ev, a);
  if (!e) e = cudaStreamWaitEvent(b, B.ev, 0);
  return e;
}

dualip_status stage_gammas(Batch& B, const double* gammas, cudaStream_t s) {
  for (int k = 0; k < B.n; ++k)
    if (!gamma_ok(gammas[k])) return fail(DUALIP_EINVAL, "every gamma must be in [1e-30, 1e30]");
  // the staging buffer may still be read by an earlier call's copy
  cudaError_t e = cudaEventSynchronize(B.ev_stage);
  if (e) return cuda_fail(e, "waiting for the gamma staging buffer");
  float* gf = reinterpret_cast<float*>(B.h_gamma + B.n);
  for (int k = 0; k < B.n; ++k) {
    B.h_gamma[k] = gammas[k];
    gf[k] = (float)gammas[k];
  }
  if ((e = cudaMemcpyAsync(B.d_gamma_d, B.h_gamma, sizeof(double) * B.n, cudaMemcpyHostToDevice,
                           s)) ||
      (e = cudaMemcpyAsync(B.d_gamma_f, gf, sizeof(float) * B.n, cudaMemcpyHostToDevice, s)) ||
      (e = cudaEventRecord(B.ev_stage, s)))
    return cuda_fail(e, "uploading gammas");
  return DUALIP_OK;
}

}  // namespace

extern "C" {

dualip_status dualip_batch_create(int32_t n, dualip_problem* const* problems, dualip_batch** out) {
  if (!out) return fail(DUALIP_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || !problems) return fail(DUALIP_EINVAL, "need n >= 1 problems");
  for (int k = 0; k < n; ++k) {
    if (!problems[k]) return fail(DUALIP_EINVAL, "a problem handle is NULL");
    const Problem& P = problems[k]->p;
    const Problem& P0 = problems[0]->p;
    if (P.storage != P0.storage || P.weighted != P0.weighted || P.device != P0.device)
      return fail(DUALIP_EINVAL, "problems of a batch share storage, primal_scaling and device");
    if (P.box || P.m > 1)
      return fail(DUALIP_EINVAL,
                  "the batched form takes simplex problems with one constraint family only");
    for (int m = 0; m < k; ++m)
      if (problems[m] == problems[k]) return fail(DUALIP_EINVAL, "a problem appears twice");
  }
  dualip_batch* h = new dualip_batch();
  Batch& B = h->b;
  auto bail = [&](dualip_status st) {
    batch_free(B);
    delete h;
    return st;
  };
  cudaError_t e = batch_alloc(B, n, problems[0]->p.storage, problems[0]->p.weighted,
                              problems[0]->p.num_sms);
  if (e) return bail(cuda_fail(e, "allocating the batch"));
  int64_t joff = 0;
  for (int k = 0; k < n; ++k) {
    Problem& P = problems[k]->p;
    B.prob[k] = &P;
    B.desc[k] = slot_desc(P, joff);
    B.active[k] = 1;
    joff += P.J;
  }
  if ((e = upload_slots(B)) || (e = build_slot_tiles(B)) || (e = rebuild_lists(B)) ||
      (e = cudaStreamSynchronize(B.stream)))
    return bail(cuda_fail(e, "initialising the batch"));
  *out = h;
  return DUALIP_OK;
}

void dualip_batch_destroy(dualip_batch* b) {
  if (!b) return;
  batch_free(b->b);
  delete b;
}

dualip_status dualip_batch_dual_grad_async(dualip_batch* b, const float* lambda,
                                           const double* gammas, float* grad, double* out_dev,
                                           void* stream) {
  NvtxRange nvtx_("dualip_batch_dual_grad");
  if (!b || !lambda || !gammas || !grad) return fail(DUALIP_EINVAL, "NULL argument");
  Batch& B = b->b;
  cudaStream_t s = as_stream(stream);
  dualip_status st = ensure_all_active(B);
  if (st) return st;
  if ((st = stage_gammas(B, gammas, s))) return st;
  cudaError_t e = enqueue_batch_eval(B, lambda, grad, 0, s);
  if (!e) e = cudaEventRecord(B.ev_use, s);
  if (!e && out_dev)
    e = cudaMemcpyAsync(out_dev, B.d_eval, sizeof(double) * 5 * B.n, cudaMemcpyDeviceToDevice, s);
  return e ? cuda_fail(e, "launching the batched evaluation") : DUALIP_OK;
}

dualip_status dualip_batch_dual_grad(dualip_batch* b, const float* lambda, const double* gammas,
                                     float* grad, dualip_eval* out, void* stream) {
  dualip_status st = dualip_batch_dual_grad_async(b, lambda, gammas, grad, nullptr, stream);
  if (st) return st;
  Batch& B = b->b;
  cudaStream_t s = as_stream(stream);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(B.h_eval, B.d_eval, sizeof(double) * 5 * B.n, cudaMemcpyDeviceToHost,
                           s)) ||
      (e = cudaStreamSynchronize(s)))
    return cuda_fail(e, "reading the batched scalars");
  if ((e = order(B, s, B.stream))) return cuda_fail(e, "ordering streams");
  if ((st = batch_status(B))) return st;
  if (out)
    for (int k = 0; k < B.n; ++k) {
      const double* o = B.h_eval + 5 * k;
      out[k].dual_obj = o[0];
      out[k].primal_obj = o[1];
      out[k].reg = o[2];
      out[k].infeas_l2 = o[3];
      out[k].lambda_dot_grad = o[4];
    }
  return DUALIP_OK;
}

dualip_status dualip_batch_set_tile_shape(dualip_batch* b, int32_t edges, int32_t sources) {
  if (!b) return fail(DUALIP_EINVAL, "batch is NULL");
  if (edges < 1 || edges > tile_edges_for(b->b.storage) || sources < 1 || sources > kTileSources)
    return fail(DUALIP_EINVAL, "tile shape out of range");
  Batch& B = b->b;
  B.tile_edges = edges;
  B.tile_sources = sources;
  cudaError_t e = build_slot_tiles(B);
  if (!e) e = rebuild_lists(B);
  return e ? cuda_fail(e, "retiling the batch") : DUALIP_OK;
}

dualip_status dualip_batch_get_info(const dualip_batch* b, int32_t* n, int64_t* total_J,
                                    int64_t* total_E, int64_t* ntiles, int32_t* tile_edges,
                                    int32_t* tile_sources) {
  if (!b) return fail(DUALIP_EINVAL, "batch is NULL");
  const Batch& B = b->b;
  int64_t J = 0, E = 0, T = 0;
  for (int s = 0; s < B.n; ++s) {
    J += B.prob[s]->J;
    E += B.prob[s]->E;
    T += (int64_t)B.tiles[s].size();
  }
  if (n) *n = B.n;
  if (total_J) *total_J = J;
  if (total_E) *total_E = E;
  if (ntiles) *ntiles = T;
  if (tile_edges) *tile_edges = (int32_t)B.tile_edges;
  if (tile_sources) *tile_sources = (int32_t)B.tile_sources;
  return DUALIP_OK;
}

dualip_status dualip_batch_solve(dualip_batch* b, const dualip_solve_opts* opts, int32_t n_opts,
                                 float* lambda_inout, dualip_solve_result* results,
                                 void* stream) {
  NvtxRange nvtx_("dualip_batch_solve");
  if (!b || !opts || !lambda_inout) return fail(DUALIP_EINVAL, "NULL argument");
  Batch& B = b->b;
  if (n_opts != 1 && n_opts != B.n) return fail(DUALIP_EINVAL, "n_opts must be 1 or n");
  for (int k = 0; k < n_opts; ++k) {
    const dualip_solve_opts& o = opts[k];
    if (!(o.gamma0 > 0) || !(o.gamma_final > 0) || !std::isfinite(o.gamma0) ||
        o.gamma_final > o.gamma0 || o.gamma_final < 1e-30)
      return fail(DUALIP_EINVAL, "need 1e-30 <= gamma_final <= gamma0 < inf");
    if (o.max_iters < 1 || o.check_every < 1 || !(o.max_step > 0) || !(o.init_step > 0))
      return fail(DUALIP_EINVAL, "need max_iters >= 1, check_every >= 1, positive steps");
  }
  auto O = [&](int k) -> const dualip_solve_opts& { return opts[n_opts == 1 ? 0 : k]; };
  const int check_every = opts[0].check_every;
  const bool use_graph = opts[0].use_graph != 0;
  cudaStream_t us = as_stream(stream);
  cudaError_t e;
  // solver vectors (renumbered): lam, y, y_prev, G, G_prev, D per slot
  for (int k = 0; k < B.n; ++k) {
    if (B.vecs[k]) continue;
    if ((e = cudaMalloc(&B.vecs[k], sizeof(float) * 6 * std::max<int32_t>(B.prob[k]->J, 1))))
      return cuda_fail(e, "allocating solver vectors");
    const int32_t J = B.prob[k]->J;
    float* v = B.vecs[k];
    SlotDesc& d = B.desc[k];
    d.lam = v;
    d.yv = v + J;
    d.yp = v + 2 * (size_t)J;
    d.G = v + 3 * (size_t)J;
    d.Gp = v + 4 * (size_t)J;
    d.D = v + 5 * (size_t)J;
    B.row_normalize = -1;
  }
  if ((e = order(B, us, B.stream))) return cuda_fail(e, "ordering streams");
  const int rn = opts[0].row_normalize ? 1 : 0;
  if (B.row_normalize != rn) {
    for (int k = 0; k < B.n; ++k)
      if ((e = compute_row_scale(*B.prob[k], rn, B.desc[k].D, B.stream)))
        return cuda_fail(e, "computing row scales");
    B.row_normalize = rn;
  }
  for (int k = 0; k < B.n; ++k) B.h_ss[k] = slot_solve_init(O(k), B.prob[k]->bnorm);
  std::fill(B.active.begin(), B.active.end(), 1);
  B.lists_ok = false;
  if ((e = upload_slots(B)) ||
      (e = cudaMemcpyAsync(B.d_ss, B.h_ss, sizeof(SlotSolve) * B.n, cudaMemcpyHostToDevice,
                           B.stream)) ||
      (e = rebuild_lists(B)))
    return cuda_fail(e, "initialising the batched solver");
  if (B.nchunks) {
    binit_kernel<<<B.nchunks, 256, 0, B.stream>>>(B.d_rc, B.d_slots, lambda_inout);
    if ((e = cudaGetLastError())) return cuda_fail(e, "initialising lambda");
    bprep_kernel<<<B.nchunks, 256, 0, B.stream>>>(B.d_rc, B.d_slots, nullptr, 1, B.d_ss,
                                                  B.d_gamma_f, B.d_gamma_d);
    if ((e = cudaGetLastError())) return cuda_fail(e, "preparing the first iteration");
  }
  std::vector<int32_t> iters(B.n, 0);
  std::vector<char> conv(B.n, 0);
  std::vector<double> evals(5 * (size_t)B.n, 0.0);
  std::vector<SlotSolve> last(B.n);
  int n_active = B.n;
  while (n_active > 0) {
    int n_it = check_every;
    for (int k = 0; k < B.n; ++k)
      if (B.active[k]) n_it = std::min(n_it, O(k).max_iters - iters[k]);
    if ((e = run_batch_chunk(B, n_it, use_graph && n_it == check_every)))
      return cuda_fail(e, "running batched iterations");
    if ((e = cudaMemcpyAsync(B.h_ss, B.d_ss, sizeof(SlotSolve) * B.n, cudaMemcpyDeviceToHost,
                             B.stream)) ||
        (e = cudaMemcpyAsync(B.h_eval, B.d_eval, sizeof(double) * 5 * B.n,
                             cudaMemcpyDeviceToHost, B.stream)) ||
        (e = cudaStreamSynchronize(B.stream)))
      return cuda_fail(e, "reading the solver state");
    dualip_status st = batch_status(B);
    if (st) return st;
    std::vector<RowChunk> fin;
    for (int k = 0; k < B.n; ++k) {
      if (!B.active[k]) continue;
      iters[k] += n_it;
      const SlotSolve& S = B.h_ss[k];
      const bool ok = O(k).stop_on_tol && iters[k] % check_every == 0 &&
                      S.last_gamma == O(k).gamma_final && S.gap_rel <= O(k).tol_gap &&
                      S.infeas_rel <= O(k).tol_infeas;
      if (ok || iters[k] >= O(k).max_iters) {
        conv[k] = ok ? 1 : 0;
        last[k] = S;
        std::copy(B.h_eval + 5 * k, B.h_eval + 5 * k + 5, evals.begin() + 5 * k);
        B.active[k] = 0;
        --n_active;
        for (int32_t r = 0; r < B.prob[k]->J; r += kChunkRows)
          fin.push_back(RowChunk{k, r, std::min<int32_t>(B.prob[k]->J, r + kChunkRows), 0});
      }
    }
    if (!fin.empty()) {
      // lambda of the finished problems; the joint lists are rebuilt after
      if ((e = cudaMemcpyAsync(B.d_rc, fin.data(), sizeof(RowChunk) * fin.size(),
                               cudaMemcpyHostToDevice, B.stream)))
        return cuda_fail(e, "uploading chunks");
      bfinal_kernel<<<(int)fin.size(), 256, 0, B.stream>>>(B.d_rc, B.d_slots, lambda_inout);
      if ((e = cudaGetLastError()) || (e = cudaStreamSynchronize(B.stream)))
        return cuda_fail(e, "writing lambda");
      B.lists_ok = false;
      if ((e = rebuild_lists(B))) return cuda_fail(e, "rebuilding the batch lists");
    }
  }
  if ((e = order(B, B.stream, us))) return cuda_fail(e, "ordering streams");
  bool all = true;
  for (int k = 0; k < B.n; ++k) {
    all = all && conv[k];
    if (!results) continue;
    dualip_solve_result& r = results[k];
    r.iters = iters[k];
    r.converged = conv[k];
    r.last.dual_obj = evals[5 * k];
    r.last.primal_obj = evals[5 * k + 1];
    r.last.reg = evals[5 * k + 2];
    r.last.infeas_l2 = evals[5 * k + 3];
    r.last.lambda_dot_grad = evals[5 * k + 4];
    r.gap_rel = last[k].gap_rel;
    r.infeas_rel = last[k].infeas_rel;
    r.gamma = last[k].last_gamma;
  }
  // the lists of every slot again, for later evaluations
  std::fill(B.active.begin(), B.active.end(), 1);
  B.lists_ok = false;
  if (!all && opts[0].stop_on_tol)
    return fail(DUALIP_ENOTCONVERGED, "some problem reached max_iters before its tolerances");
  return DUALIP_OK;
}

dualip_status dualip_batch_autotune(dualip_batch* b, dualip_autotune_result* result,
                                    void* stream) {
  NvtxRange nvtx_("dualip_batch_autotune");
  if (!b) return fail(DUALIP_EINVAL, "batch is NULL");
  Batch& B = b->b;
  cudaStream_t s = as_stream(stream);
  dualip_autotune_result r;
  std::memset(&r, 0, sizeof(r));
  // segment-length histogram: sources by degree, log2 buckets
  int64_t nsrc = 0, nedge = 0;
  for (int k = 0; k < B.n; ++k) {
    const std::vector<int64_t>& off = B.prob[k]->off_host;
    for (size_t i = 0; i + 1 < off.size(); ++i) ++r.degree_hist[degree_bucket(off[i + 1] - off[i])];
    nsrc += (int64_t)off.size() - 1;
    nedge += off.empty() ? 0 : off.back();
  }
  // candidate shapes, pruned by the degree histogram (plan.h)
  const int32_t emax = tile_edges_for(B.storage);
  const int32_t cand[][2] = {{emax, 256}, {emax, 128}, {2048, 256}, {2048, 128},
                             {1536, 128}, {1024, 128}, {1024, 64},   {512, 64}};
  const std::vector<int> keep = prune_shapes(r.degree_hist, nsrc, nedge, cand, 8);
  dualip_status st = DUALIP_OK;
  std::vector<float*> bufs(2, nullptr);
  int64_t Jt = 0;
  for (int k = 0; k < B.n; ++k) Jt += B.prob[k]->J;
  cudaError_t e;
  if ((e = cudaMalloc(&bufs[0], sizeof(float) * std::max<int64_t>(Jt, 1))) ||
      (e = cudaMalloc(&bufs[1], sizeof(float) * std::max<int64_t>(Jt, 1))) ||
      (e = cudaMemsetAsync(bufs[0], 0, sizeof(float) * std::max<int64_t>(Jt, 1), s)))
    st = cuda_fail(e, "allocating autotune buffers");
  std::vector<double> gam(B.n, 1e-2);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!st && ((e = cudaEventCreate(&e0)) || (e = cudaEventCreate(&e1))))
    st = cuda_fail(e, "creating events");
  // mean time of 3 evaluations (after one more) with the current shape and policy
  auto time_evals = [&](double* out_ms) -> dualip_status {
    dualip_status t = ensure_all_active(B);
    const int reps = 3;
    for (int w = 0; w < 1 + reps && !t; ++w) {
      if (w == 1 && (e = cudaEventRecord(e0, s))) t = cuda_fail(e, "timing");
      if (!t) t = dualip_batch_dual_grad_async(b, bufs[0], gam.data(), bufs[1], nullptr, s);
    }
    float ms = 0.f;
    if (!t && ((e = cudaEventRecord(e1, s)) || (e = cudaEventSynchronize(e1)) ||
               (e = cudaEventElapsedTime(&ms, e0, e1))))
      t = cuda_fail(e, "timing");
    *out_ms = ms / reps;
    return t;
  };
  double best = 1e300;
  int best_c = keep.empty() ? 0 : keep[0];
  B.lean80 = 0;
  for (size_t q = 0; q < keep.size() && !st; ++q) {
    const int c = keep[q];
    if ((st = dualip_batch_set_tile_shape(b, cand[c][0], cand[c][1]))) break;
    double ms = 0.0;
    if ((st = time_evals(&ms))) break;
    const int slot = (int)q;
    r.tile_edges[slot] = cand[c][0];
    r.tile_sources[slot] = cand[c][1];
    r.ms[slot] = ms;
    r.n_candidates = slot + 1;
    if (ms < best) {
      best = ms;
      best_c = c;
      r.chosen = slot;
    }
  }
  // the lean-window policy, on the chosen shape: 4-lane windows of up to 80
  // slots pay off when few batches need an 8-lane pass anyway
  if (!st && !keep.empty() && !(st = dualip_batch_set_tile_shape(b, cand[best_c][0], cand[best_c][1]))) {
    B.lean80 = 1;
    st = time_evals(&r.ms_lean80);
    r.lean80 = r.ms_lean80 < best ? 1 : 0;
    B.lean80 = r.lean80;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  for (float* p : bufs)
    if (p) cudaFree(p);
  if (st) return st;
  if ((st = dualip_batch_set_tile_shape(b, cand[best_c][0], cand[best_c][1]))) return st;
  if ((st = batch_status(B))) return st;
  if (result) *result = r;
  return DUALIP_OK;
}

dualip_status dualip_batch_profile_enable(dualip_batch* b, int32_t max_evals) {
  if (!b || max_evals < 1) return fail(DUALIP_EINVAL, "need a batch and max_evals >= 1");
  Batch& B = b->b;
  free_prof(B);
  B.prof_ev.resize(4 * (size_t)max_evals, nullptr);
  for (auto& ev : B.prof_ev) {
    const cudaError_t e = cudaEventCreate(&ev);
    if (e) {
      ev = nullptr;
      free_prof(B);
      return cuda_fail(e, "creating timing events");
    }
  }
  B.prof_max = max_evals;
  return DUALIP_OK;
}

dualip_status dualip_batch_profile_collect(dualip_batch* b, double* ms_prologue, double* ms_pass,
                                           double* ms_epilogue, int32_t* count) {
  if (!b) return fail(DUALIP_EINVAL, "batch is NULL");
  Batch& B = b->b;
  double t[3] = {0, 0, 0};
  for (int i = 0; i < B.prof_used; ++i) {
    cudaEvent_t* ev = &B.prof_ev[4 * (size_t)i];
    cudaError_t e = cudaEventSynchronize(ev[3]);
    for (int k = 0; k < 3 && !e; ++k) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
      t[k] += ms;
    }
    if (e) {
      free_prof(B);
      return cuda_fail(e, "reading timing events");
    }
  }
  if (ms_prologue) *ms_prologue = t[0];
  if (ms_pass) *ms_pass = t[1];
  if (ms_epilogue) *ms_epilogue = t[2];
  if (count) *count = B.prof_used;
  free_prof(B);
  return DUALIP_OK;
}

}  // extern "C"
