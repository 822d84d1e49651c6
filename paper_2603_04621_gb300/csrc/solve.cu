// Dual ascent on the GPU (Section 5 and Appendix B of the DuaLip-GPU report).
//
// The iteration lives entirely on the device so that check_every iterations
// can be replayed as one CUDA graph with no host synchronisation:
//   pass        projection + A x (pass.cu), gamma read from the state
//   epi    (J)  G = D (A x - b) and the FP64 scalars (pass.cu)
//   norms  (J)  ||y - y_prev||, ||G - G_prev|| in FP64; the last block picks
//               the step (secant estimate capped by max_step * gamma / gamma0),
//               the momentum weight (reset when gamma changes, or when the
//               dual objective fell: an adaptive restart), the stopping
//               scalars and the trace row, advances k and publishes gamma_{k+1}
//   step   (J)  lam+ = max(0, y + eta G); y+ = max(0, lam+ + beta (lam+ - lam)),
//               or y+ = lam+ when gamma changes at k+1 (momentum restart);
//               mu = D y+ for the next pass
// A prep kernel forms mu and gamma of the first iteration.  Every kernel but
// the first of the chain is launched with programmatic stream serialisation
// and waits for its predecessor before it reads.
// Vectors are kept in the renumbered destination order and in the
// normalised coordinates lam' of Section 5.1 (mu = D lam').
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace dualip {
namespace {

struct SolveState {
  // options (read-only during the run)
  double gamma0, gamma_final, max_step, init_step, bnorm;
  int32_t halve_every, restart;
  int32_t restart_dec;  // adaptive restart when the dual objective falls
  int32_t pad0;
  double* trace;
  // iteration state
  int32_t k;
  int32_t last_k;
  int32_t k0;       // k at the start of this dualip_solve call (trace row 0)
  int32_t pad_k;
  float gamma_f;  // gamma of the current iteration, read by the pass
  float pad;
  double t, eta, beta;
  double gap_rel, infeas_rel, last_gamma;
  double g_prev;   // dual objective of the previous evaluation
  int32_t restarts;  // adaptive restarts taken so far
  int32_t pad1;
  double eval[5];  // written by the epilogue
  unsigned ticket;
  int32_t pad2;
};

__host__ __device__ inline double gamma_at(const SolveState& s, int32_t k) {
  double g = s.gamma0;
  if (s.halve_every > 0) g = ldexp(s.gamma0, -(k / s.halve_every));
  return g > s.gamma_final ? g : s.gamma_final;
}
__device__ inline bool restart_at(const SolveState& s, int32_t k) {
  return s.restart && k > 0 && gamma_at(s, k) != gamma_at(s, k - 1);
}

struct Vecs {
  float *lam, *y, *yp, *G, *Gp, *D;
};

__global__ void solve_init_kernel(int32_t J, const float* __restrict__ lam_in,
                                  const int32_t* __restrict__ orig_of, Vecs v) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < J;
       j += (int64_t)gridDim.x * blockDim.x) {
    const float l = lam_in[orig_of[j]] / v.D[j];
    const float c = l > 0.f ? l : 0.f;
    v.lam[j] = c;
    v.y[j] = c;
    v.yp[j] = c;
    v.G[j] = 0.f;
    v.Gp[j] = 0.f;
  }
}

// mu and gamma of the first iteration (later iterations get them from the
// step and norms kernels of the iteration before)
__global__ void solve_prep_kernel(int32_t J, SolveState* st, Vecs v, float* __restrict__ mu_r) {
  const int32_t k = st->k;
  const bool rs = restart_at(*st, k);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < J;
       j += (int64_t)gridDim.x * blockDim.x) {
    float yj = v.y[j];
    if (rs) {
      yj = v.lam[j];
      v.y[j] = yj;
    }
    mu_r[j] = __fmul_rn(v.D[j], yj);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) st->gamma_f = (float)gamma_at(*st, k);
}

__global__ void solve_norms_kernel(int32_t J, SolveState* st, Vecs v, double* part) {
  pdl_wait();  // G and the scalars of the epilogue
  pdl_trigger();
  const int32_t k = st->k;
  const bool have_prev = k > 0 && !restart_at(*st, k);
  double dy = 0.0, dg = 0.0;
  if (have_prev) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < J;
         j += (int64_t)gridDim.x * blockDim.x) {
      const double u = (double)v.y[j] - (double)v.yp[j];
      const double w = (double)v.G[j] - (double)v.Gp[j];
      dy += u * u;
      dg += w * w;
    }
  }
  for (int o = 16; o; o >>= 1) {
    dy += __shfl_xor_sync(0xffffffffu, dy, o);
    dg += __shfl_xor_sync(0xffffffffu, dg, o);
  }
  __shared__ double red[2][32];
  __shared__ bool last;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red[0][w] = dy;
    red[1][w] = dg;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      a += red[0][i];
      b += red[1][i];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
    __threadfence();
    last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double sdy = 0.0, sdg = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    sdy += part[2 * i];
    sdg += part[2 * i + 1];
  }
  for (int o = 16; o; o >>= 1) {
    sdy += __shfl_xor_sync(0xffffffffu, sdy, o);
    sdg += __shfl_xor_sync(0xffffffffu, sdg, o);
  }
  __syncthreads();
  if (lane == 0) {
    red[0][w] = sdy;
    red[1][w] = sdg;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  sdy = 0.0;
  sdg = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
    sdy += red[0][i];
    sdg += red[1][i];
  }
  const double gk = gamma_at(*st, k);
  const double eta_max = st->max_step * gk / st->gamma0;
  double eta;
  if (have_prev) eta = sdg > 0.0 ? fmin(eta_max, sqrt(sdy) / sqrt(sdg)) : eta_max;
  else eta = fmin(st->init_step, eta_max);
  const double g = st->eval[0], p = st->eval[1] + st->eval[2];
  // momentum restarts at a gamma change and, adaptively, when the dual
  // objective fell since the previous evaluation at the same gamma
  const bool dec = st->restart_dec && have_prev && g < st->g_prev;
  st->restarts += dec ? 1 : 0;
  const double t = (restart_at(*st, k) || dec) ? 1.0 : st->t;
  const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
  st->eta = eta;
  st->beta = (t - 1.0) / tn;
  st->t = tn;
  st->g_prev = g;
  const double den = fmax(1.0, fmax(fabs(p), fabs(g)));
  st->gap_rel = fabs(st->eval[4]) / den;
  st->infeas_rel = st->eval[3] / fmax(1.0, st->bnorm);
  st->last_k = k;
  st->last_gamma = gk;
  if (st->trace) {
    double* tr = st->trace + 8 * (size_t)(k - st->k0);
    tr[0] = gk;
    tr[1] = g;
    tr[2] = p;
    tr[3] = st->eval[3];
    tr[4] = st->gap_rel;
    tr[5] = st->infeas_rel;
    tr[6] = eta;
    tr[7] = st->eval[4];
  }
  st->k = k + 1;
  st->gamma_f = (float)gamma_at(*st, k + 1);  // read by the next iteration's pass
  st->ticket = 0u;
}

// The step, then the next iteration's point: y restarts at lambda when gamma
// changes there (the norms kernel has already advanced k), and its mu.
__global__ void solve_step_kernel(int32_t J, const SolveState* st, Vecs v,
                                  float* __restrict__ mu_r) {
  pdl_wait();  // eta and beta of the norms kernel
  pdl_trigger();
  const float eta = (float)st->eta, beta = (float)st->beta;
  const bool rs = restart_at(*st, st->k);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < J;
       j += (int64_t)gridDim.x * blockDim.x) {
    const float yk = v.y[j], g = v.G[j], lk = v.lam[j];
    float ln = __fmaf_rn(eta, g, yk);
    ln = ln > 0.f ? ln : 0.f;
    float yn = __fmaf_rn(beta, __fsub_rn(ln, lk), ln);
    yn = yn > 0.f ? yn : 0.f;
    if (rs) yn = ln;
    v.yp[j] = yk;
    v.Gp[j] = g;
    v.lam[j] = ln;
    v.y[j] = yn;
    mu_r[j] = __fmul_rn(v.D[j], yn);
  }
}

__global__ void solve_final_kernel(int32_t J, Vecs v, const int32_t* __restrict__ orig_of,
                                   float* __restrict__ lam_out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < J;
       j += (int64_t)gridDim.x * blockDim.x)
    lam_out[orig_of[j]] = __fmul_rn(v.D[j], v.yp[j]);
}

// The six ascent vectors (lam', y, y_prev, G, G_prev, D) between the solver's
// renumbered order and a [6][J] array in the caller's numbering.
__global__ void state_gather_kernel(int32_t J, Vecs v, const int32_t* __restrict__ orig_of,
                                    float* __restrict__ out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < J;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = orig_of[j];
    out[o] = v.lam[j];
    out[J + o] = v.y[j];
    out[2 * (int64_t)J + o] = v.yp[j];
    out[3 * (int64_t)J + o] = v.G[j];
    out[4 * (int64_t)J + o] = v.Gp[j];
    out[5 * (int64_t)J + o] = v.D[j];
  }
}
__global__ void state_scatter_kernel(int32_t J, Vecs v, const int32_t* __restrict__ orig_of,
                                     const float* __restrict__ in) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < J;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = orig_of[j];
    v.lam[j] = in[o];
    v.y[j] = in[J + o];
    v.yp[j] = in[2 * (int64_t)J + o];
    v.G[j] = in[3 * (int64_t)J + o];
    v.Gp[j] = in[4 * (int64_t)J + o];
    v.D[j] = in[5 * (int64_t)J + o];
  }
}

// D_j = (sum_{e -> j} a_e^2 / w_e)^(-1/2), 1 for a zero row (Section 5.1)
__global__ void row_norm_kernel(const int32_t* __restrict__ dst, const float2* __restrict__ ca2,
                                const uint32_t* __restrict__ ca, int64_t E, int weighted,
                                double* __restrict__ acc) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float av = ca2 ? ca2[e].y : __uint_as_float(ca[e] & 0xffff0000u);
    double v = (double)av * (double)av;
    if (weighted) v = av != 0.f ? 1.0 : 0.0;
    if (v != 0.0) atomicAdd(acc + dst[e], v);
  }
}
__global__ void row_scale_kernel(int32_t J, const double* __restrict__ acc, float* __restrict__ D) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < J;
       j += (int64_t)gridDim.x * blockDim.x)
    D[j] = acc[j] > 0.0 ? (float)(1.0 / sqrt(acc[j])) : 1.0f;
}
__global__ void fill_kernel(int32_t J, float* __restrict__ D, float v) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < J;
       j += (int64_t)gridDim.x * blockDim.x)
    D[j] = v;
}

}  // namespace

struct SolveCtx {
  int row_normalize = -1;  // row scale currently held in D (-1: none yet)
  bool has_state = false;  // the vectors and SolveState hold an ascent (solve or import)
  float *lam = nullptr, *y = nullptr, *yp = nullptr, *G = nullptr, *Gp = nullptr, *D = nullptr;
  double* part = nullptr;
  SolveState* st = nullptr;
  SolveState* st_host = nullptr;  // pinned
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_len = 0;
  int blocks = 0;
};

void solve_ctx_free(Problem& P) {
  SolveCtx* C = static_cast<SolveCtx*>(P.solve_ctx);
  if (!C) return;
  if (C->stream) cudaStreamSynchronize(C->stream);
  if (C->graph) cudaGraphExecDestroy(C->graph);
  void* bufs[] = {C->lam, C->y, C->yp, C->G, C->Gp, C->D, C->part, C->st};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (C->st_host) cudaFreeHost(C->st_host);
  if (C->ev) cudaEventDestroy(C->ev);
  if (C->stream) cudaStreamDestroy(C->stream);
  delete C;
  P.solve_ctx = nullptr;
}

static cudaError_t solve_ctx_get(Problem& P, SolveCtx** out) {
  if (P.solve_ctx) {
    *out = static_cast<SolveCtx*>(P.solve_ctx);
    return cudaSuccess;
  }
  SolveCtx* C = new SolveCtx();
  P.solve_ctx = C;
  const size_t n = (size_t)P.J * sizeof(float);
  C->blocks = (int)std::max<int64_t>(1, std::min<int64_t>((P.J + 255) / 256, 2 * P.num_sms));
  cudaError_t e;
  if ((e = cudaMalloc(&C->lam, n)) || (e = cudaMalloc(&C->y, n)) || (e = cudaMalloc(&C->yp, n)) ||
      (e = cudaMalloc(&C->G, n)) || (e = cudaMalloc(&C->Gp, n)) || (e = cudaMalloc(&C->D, n)) ||
      (e = cudaMalloc(&C->part, sizeof(double) * 2 * C->blocks)) ||
      (e = cudaMalloc(&C->st, sizeof(SolveState))) ||
      (e = cudaMallocHost(&C->st_host, sizeof(SolveState))) ||
      (e = cudaStreamCreateWithFlags(&C->stream, cudaStreamNonBlocking)) ||
      (e = cudaEventCreateWithFlags(&C->ev, cudaEventDisableTiming))) {
    solve_ctx_free(P);  // a later call starts again from nothing
    return e;
  }
  *out = C;
  return cudaSuccess;
}

cudaError_t compute_row_scale(const Problem& P, int row_normalize, float* D, cudaStream_t s) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((P.J + 255) / 256, 2 * P.num_sms));
  cudaError_t e;
  if (!row_normalize) {
    fill_kernel<<<blocks, 256, 0, s>>>(P.J, D, 1.0f);
    return cudaGetLastError();
  }
  double* acc = nullptr;
  if ((e = cudaMalloc(&acc, sizeof(double) * std::max<int32_t>(P.J, 1)))) return e;
  e = cudaMemsetAsync(acc, 0, sizeof(double) * P.J, s);
  if (!e && P.E > 0 && P.m > 1) {
    e = launch_row_norm_multi(P, acc, s);
  } else if (!e && P.E > 0) {
    const int64_t g = std::min<int64_t>((P.E + 255) / 256, 8192);
    row_norm_kernel<<<(int)g, 256, 0, s>>>(P.dst, P.ca2, P.ca, P.E, P.weighted, acc);
    e = cudaGetLastError();
  }
  if (!e) {
    row_scale_kernel<<<blocks, 256, 0, s>>>(P.J, acc, D);
    e = cudaGetLastError();
  }
  cudaStreamSynchronize(s);
  cudaFree(acc);
  return e;
}

static cudaError_t ensure_row_scale(Problem& P, SolveCtx& C, int row_normalize, cudaStream_t s) {
  if (C.row_normalize == row_normalize) return cudaSuccess;
  cudaError_t e = compute_row_scale(P, row_normalize, C.D, s);
  if (e) return e;
  C.row_normalize = row_normalize;
  return cudaSuccess;
}

// prof: record the handle's timing events (dualip_profile_enable) around the
// pass and the epilogue; only outside graph capture.
static cudaError_t enqueue_iteration(Problem& P, SolveCtx& C, cudaStream_t s, bool prof) {
  Vecs v{C.lam, C.y, C.yp, C.G, C.Gp, C.D};
  cudaError_t e;
  cudaEvent_t* ev = nullptr;
  if (prof && P.prof_used < P.prof_max) ev = &P.prof_ev[4 * (size_t)P.prof_used++];
  // mu and gamma of this iteration come from the previous one (or the prep
  // before the first); every kernel waits for its predecessor's writes
  if (ev && ((e = cudaEventRecord(ev[0], s)) || (e = cudaEventRecord(ev[1], s)))) return e;
  if ((e = launch_pass(P, &C.st->gamma_f, 0.f, nullptr, s))) return e;
  if (ev && (e = cudaEventRecord(ev[2], s))) return e;
  if ((e = launch_epilogue(P, C.D, C.G, &C.st->gamma_f, 0.0, C.st->eval, s, true))) return e;
  if (ev && (e = cudaEventRecord(ev[3], s))) return e;
  if ((e = launch_pdl(solve_norms_kernel, dim3(C.blocks), dim3(256), 0, s, P.J, C.st, v,
                      C.part)))
    return e;
  return launch_pdl(solve_step_kernel, dim3(C.blocks), dim3(256), 0, s, P.J,
                    (const SolveState*)C.st, v, P.mu_r);
}

static cudaError_t run_chunk(Problem& P, SolveCtx& C, int n, bool use_graph) {
  cudaError_t e;
  if (use_graph) {
    if (!C.graph || C.graph_len != n) {
      if (C.graph) cudaGraphExecDestroy(C.graph);
      C.graph = nullptr;
      cudaGraph_t g = nullptr;
      if ((e = cudaStreamBeginCapture(C.stream, cudaStreamCaptureModeThreadLocal))) return e;
      for (int i = 0; i < n; ++i) {
        e = enqueue_iteration(P, C, C.stream, false);
        if (e) break;
      }
      cudaError_t e2 = cudaStreamEndCapture(C.stream, &g);
      if (e) {
        if (g) cudaGraphDestroy(g);
        return e;
      }
      if (e2) return e2;
      e = cudaGraphInstantiate(&C.graph, g, 0);
      cudaGraphDestroy(g);
      if (e) return e;
      C.graph_len = n;
    }
    return cudaGraphLaunch(C.graph, C.stream);
  }
  for (int i = 0; i < n; ++i)
    if ((e = enqueue_iteration(P, C, C.stream, true))) return e;
  return cudaSuccess;
}

}  // namespace dualip

using namespace dualip;

extern "C" {

void dualip_solve_opts_default(dualip_solve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->gamma0 = 0.1;
  o->gamma_final = 1e-3;
  o->halve_every = 25;
  o->max_step = 10.0;
  o->init_step = 1e-5;
  o->max_iters = 5000;
  o->tol_gap = 1e-4;
  o->tol_infeas = 1e-4;
  o->check_every = 10;
  o->row_normalize = 1;
  o->restart_on_gamma_change = 1;
  o->stop_on_tol = 1;
  o->use_graph = 1;
  o->restart_on_decrease = 1;
}

dualip_status dualip_solve(dualip_problem* h, const dualip_solve_opts* o, float* lambda_io,
                           dualip_solve_result* res, double* trace, void* stream) {
  NvtxRange nvtx_("dualip_solve");
  if (!h || !o || !lambda_io) return fail(DUALIP_EINVAL, "handle, opts and lambda must be non-NULL");
  if (!(o->gamma0 > 0) || !(o->gamma_final > 0) || !std::isfinite(o->gamma0) ||
      o->gamma_final > o->gamma0 || o->gamma_final < 1e-30)
    return fail(DUALIP_EINVAL, "need 1e-30 <= gamma_final <= gamma0 < inf");
  if (o->max_iters < 1 || o->check_every < 1 || !(o->max_step > 0) || !(o->init_step > 0))
    return fail(DUALIP_EINVAL, "need max_iters >= 1, check_every >= 1, positive steps");
  Problem& P = h->p;
  cudaStream_t us = static_cast<cudaStream_t>(stream);
  P.last_stream = us;
  SolveCtx* Cp = nullptr;
  cudaError_t e = solve_ctx_get(P, &Cp);
  if (e) return cuda_fail(e, "allocating solver state");
  SolveCtx& C = *Cp;
  // order the private stream after the caller's stream
  if ((e = cudaEventRecord(C.ev, us)) || (e = cudaStreamWaitEvent(C.stream, C.ev, 0)))
    return cuda_fail(e, "ordering streams");
  const bool resume = o->resume != 0;
  if (resume && !C.has_state)
    return fail(DUALIP_EINVAL, "resume needs a solver state (a previous solve or an import)");
  if (resume && C.row_normalize != (o->row_normalize ? 1 : 0))
    return fail(DUALIP_EINVAL, "resume needs the row normalisation of the saved state");
  if ((e = ensure_row_scale(P, C, o->row_normalize ? 1 : 0, C.stream)))
    return cuda_fail(e, "computing the row scale");
  SolveState& H = *C.st_host;
  if (resume) {  // the iteration state as it stands; the options from opts
    if ((e = cudaMemcpyAsync(&H, C.st, sizeof(H), cudaMemcpyDeviceToHost, C.stream)) ||
        (e = cudaStreamSynchronize(C.stream)))
      return cuda_fail(e, "reading solver state");
  } else {
    std::memset(&H, 0, sizeof(H));
    H.t = 1.0;
  }
  H.gamma0 = o->gamma0;
  H.gamma_final = o->gamma_final;
  H.max_step = o->max_step;
  H.init_step = o->init_step;
  H.bnorm = P.bnorm;
  H.halve_every = o->halve_every;
  H.restart = o->restart_on_gamma_change ? 1 : 0;
  H.restart_dec = o->restart_on_decrease ? 1 : 0;
  H.trace = trace;
  H.k0 = H.k;
  H.ticket = 0u;
  if ((e = cudaMemcpyAsync(C.st, &H, sizeof(H), cudaMemcpyHostToDevice, C.stream)))
    return cuda_fail(e, "uploading solver state");
  C.has_state = true;
  {
    Vecs v{C.lam, C.y, C.yp, C.G, C.Gp, C.D};
    if (!resume) {
      solve_init_kernel<<<C.blocks, 256, 0, C.stream>>>(P.J, lambda_io, P.orig_of, v);
      if ((e = cudaGetLastError())) return cuda_fail(e, "initialising the solver");
    }
    // mu and gamma of the next iteration (a resumed ascent continues at k)
    solve_prep_kernel<<<C.blocks, 256, 0, C.stream>>>(P.J, C.st, v, P.mu_r);
    if ((e = cudaGetLastError())) return cuda_fail(e, "initialising the solver");
  }
  int done = 0;
  bool converged = false;
  dualip_status st = DUALIP_OK;
  while (done < o->max_iters) {
    const int n = std::min(o->check_every, o->max_iters - done);
    if ((e = run_chunk(P, C, n, o->use_graph && n == o->check_every)))
      return cuda_fail(e, "running solver iterations");
    done += n;
    if ((e = cudaMemcpyAsync(C.st_host, C.st, sizeof(SolveState), cudaMemcpyDeviceToHost,
                             C.stream)) ||
        (e = cudaStreamSynchronize(C.stream)))
      return cuda_fail(e, "reading solver state");
    if ((st = dualip_check_device_status(h, C.stream))) return st;
    if (o->stop_on_tol && done % o->check_every == 0 && H.last_gamma == o->gamma_final &&
        H.gap_rel <= o->tol_gap && H.infeas_rel <= o->tol_infeas) {
      converged = true;
      break;
    }
  }
  {
    Vecs v{C.lam, C.y, C.yp, C.G, C.Gp, C.D};
    solve_final_kernel<<<C.blocks, 256, 0, C.stream>>>(P.J, v, P.orig_of, lambda_io);
    if ((e = cudaGetLastError())) return cuda_fail(e, "writing lambda");
  }
  if ((e = cudaEventRecord(C.ev, C.stream)) || (e = cudaStreamWaitEvent(us, C.ev, 0)) ||
      (e = cudaStreamSynchronize(C.stream)))
    return cuda_fail(e, "finishing the solve");
  if (res) {
    res->iters = done;
    res->converged = converged ? 1 : 0;
    std::memcpy(&res->last, H.eval, sizeof(res->last));
    res->gap_rel = H.gap_rel;
    res->infeas_rel = H.infeas_rel;
    res->gamma = H.last_gamma;
  }
  if (!converged && o->stop_on_tol)
    return fail(DUALIP_ENOTCONVERGED, "max_iters reached before the tolerances held");
  return DUALIP_OK;
}

}  // extern "C"

namespace dualip {
namespace {
// Saved ascent: this header, then lam', y, y_prev, G, G_prev and the row
// scale D, J floats each, in the caller's destination numbering.
struct StateHeader {
  char magic[8];           // "DUALIPS1"
  int32_t J, row_normalize;
  int32_t k, last_k, restarts, pad;
  double t, eta, beta, g_prev, gap_rel, infeas_rel, last_gamma;
  double eval[5];
};
constexpr char kStateMagic[8] = {'D', 'U', 'A', 'L', 'I', 'P', 'S', '1'};
int64_t state_bytes(int32_t J) { return (int64_t)sizeof(StateHeader) + 24 * (int64_t)J; }
}  // namespace
}  // namespace dualip

extern "C" {

dualip_status dualip_solve_state_size(const dualip_problem* h, int64_t* bytes) {
  if (!h || !bytes) return fail(DUALIP_EINVAL, "handle and bytes must be non-NULL");
  *bytes = state_bytes(h->p.J);
  return DUALIP_OK;
}

dualip_status dualip_solve_state_export(dualip_problem* h, void* buf, int64_t bytes,
                                        void* stream) {
  NvtxRange nvtx_("dualip_solve_state_export");
  if (!h || !buf) return fail(DUALIP_EINVAL, "handle and buffer must be non-NULL");
  Problem& P = h->p;
  if (bytes < state_bytes(P.J)) return fail(DUALIP_EINVAL, "buffer smaller than the state");
  SolveCtx* C = static_cast<SolveCtx*>(P.solve_ctx);
  if (!C || !C->has_state) return fail(DUALIP_EINVAL, "the handle holds no solver state");
  cudaStream_t us = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  float* tmp = nullptr;
  if ((e = cudaEventRecord(C->ev, us)) || (e = cudaStreamWaitEvent(C->stream, C->ev, 0)) ||
      (e = cudaMemcpyAsync(C->st_host, C->st, sizeof(SolveState), cudaMemcpyDeviceToHost,
                           C->stream)) ||
      (e = cudaMallocAsync(&tmp, sizeof(float) * 6 * std::max<int32_t>(P.J, 1), C->stream)))
    return cuda_fail(e, "reading solver state");
  Vecs v{C->lam, C->y, C->yp, C->G, C->Gp, C->D};
  state_gather_kernel<<<C->blocks, 256, 0, C->stream>>>(P.J, v, P.orig_of, tmp);
  unsigned char* out = static_cast<unsigned char*>(buf);
  if (!(e = cudaGetLastError()))
    e = cudaMemcpyAsync(out + sizeof(StateHeader), tmp, sizeof(float) * 6 * (size_t)P.J,
                        cudaMemcpyDeviceToHost, C->stream);
  cudaFreeAsync(tmp, C->stream);
  if (!e) e = cudaStreamSynchronize(C->stream);
  if (e) return cuda_fail(e, "exporting solver state");
  const SolveState& S = *C->st_host;
  StateHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, kStateMagic, 8);
  hd.J = P.J;
  hd.row_normalize = C->row_normalize;
  hd.k = S.k;
  hd.last_k = S.last_k;
  hd.restarts = S.restarts;
  hd.t = S.t;
  hd.eta = S.eta;
  hd.beta = S.beta;
  hd.g_prev = S.g_prev;
  hd.gap_rel = S.gap_rel;
  hd.infeas_rel = S.infeas_rel;
  hd.last_gamma = S.last_gamma;
  std::memcpy(hd.eval, S.eval, sizeof(hd.eval));
  std::memcpy(out, &hd, sizeof(hd));
  return DUALIP_OK;
}

dualip_status dualip_solve_state_import(dualip_problem* h, const void* buf, int64_t bytes,
                                        void* stream) {
  NvtxRange nvtx_("dualip_solve_state_import");
  if (!h || !buf) return fail(DUALIP_EINVAL, "handle and buffer must be non-NULL");
  Problem& P = h->p;
  StateHeader hd;
  if (bytes < (int64_t)sizeof(hd)) return fail(DUALIP_EINVAL, "buffer smaller than a state");
  std::memcpy(&hd, buf, sizeof(hd));
  if (std::memcmp(hd.magic, kStateMagic, 8) != 0)
    return fail(DUALIP_EINVAL, "not a saved solver state");
  if (hd.J != P.J || bytes < state_bytes(P.J))
    return fail(DUALIP_EINVAL, "the saved state belongs to a problem of another size");
  if ((hd.row_normalize != 0 && hd.row_normalize != 1) || hd.k < 0)
    return fail(DUALIP_EINVAL, "corrupt solver state");
  SolveCtx* Cp = nullptr;
  cudaError_t e = solve_ctx_get(P, &Cp);
  if (e) return cuda_fail(e, "allocating solver state");
  SolveCtx& C = *Cp;
  cudaStream_t us = static_cast<cudaStream_t>(stream);
  SolveState& S = *C.st_host;
  std::memset(&S, 0, sizeof(S));
  S.bnorm = P.bnorm;
  S.k = hd.k;
  S.last_k = hd.last_k;
  S.restarts = hd.restarts;
  S.t = hd.t;
  S.eta = hd.eta;
  S.beta = hd.beta;
  S.g_prev = hd.g_prev;
  S.gap_rel = hd.gap_rel;
  S.infeas_rel = hd.infeas_rel;
  S.last_gamma = hd.last_gamma;
  std::memcpy(S.eval, hd.eval, sizeof(S.eval));
  float* tmp = nullptr;
  if ((e = cudaEventRecord(C.ev, us)) || (e = cudaStreamWaitEvent(C.stream, C.ev, 0)) ||
      (e = cudaMemcpyAsync(C.st, &S, sizeof(S), cudaMemcpyHostToDevice, C.stream)) ||
      (e = cudaMallocAsync(&tmp, sizeof(float) * 6 * std::max<int32_t>(P.J, 1), C.stream)) ||
      (e = cudaMemcpyAsync(tmp, static_cast<const unsigned char*>(buf) + sizeof(hd),
                           sizeof(float) * 6 * (size_t)P.J, cudaMemcpyHostToDevice, C.stream))) {
    if (tmp) cudaFreeAsync(tmp, C.stream);
    C.has_state = false;  // the device state may be half written
    return cuda_fail(e, "importing solver state");
  }
  Vecs v{C.lam, C.y, C.yp, C.G, C.Gp, C.D};
  state_scatter_kernel<<<C.blocks, 256, 0, C.stream>>>(P.J, v, P.orig_of, tmp);
  e = cudaGetLastError();
  cudaFreeAsync(tmp, C.stream);
  if (!e) e = cudaStreamSynchronize(C.stream);
  if (e) {
    C.has_state = false;
    return cuda_fail(e, "importing solver state");
  }
  C.row_normalize = hd.row_normalize;
  C.has_state = true;
  return DUALIP_OK;
}

}  // extern "C"
