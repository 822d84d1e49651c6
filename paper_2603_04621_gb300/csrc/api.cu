// C ABI of the dual-gradient engine: validation, problem construction and
// the single-evaluation entry points.  Every device step runs in this
// library's kernels (pass.cu, solve.cu); nothing falls back to the host.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "internal.h"

namespace dualip {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

dualip_status fail(dualip_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

dualip_status cuda_fail(cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  set_error(m);
  return e == cudaErrorMemoryAllocation ? DUALIP_ENOMEM : DUALIP_ECUDA;
}

namespace {

template <class T>
cudaError_t dev_alloc(Problem& P, T** ptr, size_t count) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  P.allocations.push_back(p);
  *ptr = static_cast<T*>(p);
  return cudaSuccess;
}

void free_events(Problem& P) {
  for (cudaEvent_t ev : P.prof_ev) cudaEventDestroy(ev);
  P.prof_ev.clear();
  P.prof_max = P.prof_used = 0;
}

void free_all(Problem& P) {
  solve_ctx_free(P);
  free_events(P);
  for (void* p : P.allocations) cudaFree(p);
  P.allocations.clear();
  if (P.eval_host) cudaFreeHost(P.eval_host);
  P.eval_host = nullptr;
}

// The pass kernels' shared-memory limits are set once per device (a function
// attribute is set on the current device), under a lock: problems may be
// created from several host threads at once.
cudaError_t configure_device_once(int device) {
  static std::mutex m;
  static std::vector<char> done;
  std::lock_guard<std::mutex> lk(m);
  if (device >= (int)done.size()) done.resize((size_t)device + 1, 0);
  if (done[device]) return cudaSuccess;
  const cudaError_t e = configure_pass_kernels();
  if (e == cudaSuccess) done[device] = 1;
  return e;
}

}  // namespace

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

namespace {

dualip_status read_status(Problem& P, cudaStream_t s) {
  DeviceStatus h{};
  cudaError_t e = cudaMemcpyAsync(&h, P.status, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "reading the device status");
  if (h.err == 0 && h.abort_req == 0) return DUALIP_OK;
  DeviceStatus z{};
  cudaMemcpyAsync(P.status, &z, sizeof(z), cudaMemcpyHostToDevice, s);
  cudaStreamSynchronize(s);
  if (h.err == 0) return DUALIP_OK;  // an abort request that no wait saw
  if (h.err & kErrTimeout)
    return fail(DUALIP_ETIMEOUT, "a bounded device wait gave up (site " + std::to_string(h.where) +
                                     "); results of the call are invalid");
  return fail(DUALIP_EDEVICE, "a device-side consistency check failed; results are invalid");
}

dualip_status check_eval_args(dualip_problem* h, const void* lambda, double gamma, const void* out) {
  if (!h) return fail(DUALIP_EINVAL, "problem handle is NULL");
  if (!lambda || !out) return fail(DUALIP_EINVAL, "lambda and output pointers must be non-NULL");
  if (!std::isfinite(gamma) || !(gamma >= 1e-30) || !(gamma <= 1e30))
    return fail(DUALIP_EINVAL, "gamma must be finite and in [1e-30, 1e30]");
  return DUALIP_OK;
}

}  // namespace

// One evaluation: prologue (renumbered mu), pass, epilogue.
static cudaError_t enqueue_eval(Problem& P, const float* lambda, double gamma, float* grad,
                                double* eval_out, float* x_out, cudaStream_t s) {
  cudaError_t e;
  cudaEvent_t* ev = nullptr;
  if (P.prof_used < P.prof_max) ev = &P.prof_ev[4 * (size_t)P.prof_used++];
  if (ev && (e = cudaEventRecord(ev[0], s))) return e;
  if ((e = launch_prep(P, lambda, nullptr, s))) return e;
  if (ev && (e = cudaEventRecord(ev[1], s))) return e;
  if ((e = launch_pass(P, nullptr, (float)gamma, x_out, s))) return e;
  if (ev && (e = cudaEventRecord(ev[2], s))) return e;
  if ((e = launch_epilogue(P, nullptr, grad, nullptr, gamma, eval_out, s))) return e;
  if (ev && (e = cudaEventRecord(ev[3], s))) return e;
  return cudaSuccess;
}

// A problem with m > 1 constraint families (Definition 1).  The edges keep
// the caller's order and destination ids (rows k Jd + j need no renumbering),
// c and the m coefficient arrays stay separate FP32 arrays, and every J-length
// array of the handle has m Jd rows in the caller's row order; the prologue,
// epilogue and solver kernels then work unchanged on those rows.
// Stores the edges of every hub source in order of destination: a stable
// counting sort of its renumbered ids on the host, then a gather of its
// (dst, c, a) on the device.  The source's simplex does not depend on the
// order of its edges; sorted ids let the lanes of a warp gather mu from
// shared sectors of L2 instead of one sector per edge.  The permutation stays
// in P.hub_perm for dualip_get_primal.
static cudaError_t sort_hub_edges(Problem& P, int64_t hub_edges, cudaStream_t s) {
  const size_t ce = P.storage == DUALIP_EDGE_BF16 ? 4 : 8;  // bytes of a stored (c, a)
  char* ca = P.storage == DUALIP_EDGE_BF16 ? reinterpret_cast<char*>(P.ca)
                                            : reinterpret_cast<char*>(P.ca2);
  std::vector<int32_t> dh((size_t)hub_edges);
  cudaError_t e;
  for (const HubDesc& hd : P.hub_host)
    if ((e = cudaMemcpyAsync(dh.data() + hd.cand0, P.dst + hd.e0, 4 * (size_t)hd.deg,
                             cudaMemcpyDeviceToHost, s)))
      return e;
  if ((e = cudaStreamSynchronize(s))) return e;
  std::vector<uint32_t> perm((size_t)hub_edges), start;
  for (const HubDesc& hd : P.hub_host)  // (the ids were range-checked at renumbering)
    destination_order(dh.data() + hd.cand0, hd.deg, P.J, start, perm.data() + hd.cand0);
  int32_t* tdst = nullptr;
  char* tca = nullptr;
  if ((e = dev_alloc(P, &P.hub_perm, (size_t)hub_edges)) ||
      (e = cudaMemcpyAsync(P.hub_perm, perm.data(), 4 * (size_t)hub_edges,
                           cudaMemcpyHostToDevice, s)) ||
      (e = cudaMallocAsync(&tdst, 4 * (size_t)hub_edges, s)) ||
      (e = cudaMallocAsync(&tca, ce * (size_t)hub_edges, s))) {
    if (tdst) cudaFreeAsync(tdst, s);
    cudaStreamSynchronize(s);
    return e;
  }
  for (const HubDesc& hd : P.hub_host) {
    if ((e = cudaMemcpyAsync(tdst + hd.cand0, P.dst + hd.e0, 4 * (size_t)hd.deg,
                             cudaMemcpyDeviceToDevice, s)) ||
        (e = cudaMemcpyAsync(tca + ce * hd.cand0, ca + ce * hd.e0, ce * (size_t)hd.deg,
                             cudaMemcpyDeviceToDevice, s)) ||
        (e = launch_gather_perm(tdst + hd.cand0, P.dst + hd.e0, P.hub_perm + hd.cand0, hd.deg,
                                4, s)) ||
        (e = launch_gather_perm(tca + ce * hd.cand0, ca + ce * hd.e0, P.hub_perm + hd.cand0,
                                hd.deg, (int)ce, s)))
      break;
  }
  cudaFreeAsync(tdst, s);
  cudaFreeAsync(tca, s);
  const cudaError_t e2 = cudaStreamSynchronize(s);
  return e ? e : e2;
}

dualip_status create_multi(const dualip_problem_desc* d, void* stream, dualip_problem** out) {
  const int64_t I = d->num_sources, E = d->num_edges;
  const int32_t Jd = d->num_dests, m = d->num_families;
  const int64_t R64 = (int64_t)m * Jd;
  if (R64 > INT32_MAX) return fail(DUALIP_EINVAL, "num_families * num_dests exceeds 2^31 - 1");
  const int32_t R = (int32_t)R64;
  if (d->storage != DUALIP_EDGE_F32)
    return fail(DUALIP_EINVAL, "several constraint families need FP32 edge storage");
  cudaStream_t s = as_stream(stream);
  const cudaMemcpyKind h2d = d->inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e;
  std::vector<int64_t> off((size_t)I + 1);
  if ((e = cudaMemcpyAsync(off.data(), d->src_offsets, sizeof(int64_t) * (I + 1),
                           d->inputs_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost,
                           s)) ||
      (e = cudaStreamSynchronize(s)))
    return cuda_fail(e, "reading src_offsets");
  if (off[0] != 0) return fail(DUALIP_EINVAL, "src_offsets[0] must be 0");
  for (int64_t i = 0; i < I; ++i)
    if (off[i + 1] < off[i]) return fail(DUALIP_EINVAL, "src_offsets must be nondecreasing");
  if (off[I] != E) return fail(DUALIP_EINVAL, "src_offsets[I] must equal num_edges");
  std::vector<float> b((size_t)R);
  if ((e = cudaMemcpyAsync(b.data(), d->b, sizeof(float) * R,
                           d->inputs_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost,
                           s)) ||
      (e = cudaStreamSynchronize(s)))
    return cuda_fail(e, "reading b");
  double bn = 0.0;
  for (int32_t r = 0; r < R; ++r) {
    if (!std::isfinite(b[r])) return fail(DUALIP_EINVAL, "b must be finite");
    bn += (double)b[r] * (double)b[r];
  }

  auto* h = new (std::nothrow) dualip_problem();
  if (!h) return fail(DUALIP_ENOMEM, "host allocation failed");
  Problem& P = h->p;
  P.I = I;
  P.E = E;
  P.J = R;
  P.Jd = Jd;
  P.m = m;
  P.storage = DUALIP_EDGE_F32;
  P.weighted = d->primal_scaling;
  P.box = d->projection == DUALIP_PROJ_BOX ? 1 : 0;
  P.bnorm = std::sqrt(bn);
  P.last_stream = s;
  auto bail = [&](dualip_status st) {
    cudaStreamSynchronize(s);
    free_all(P);
    delete h;
    return st;
  };
  if ((e = cudaGetDevice(&P.device))) return bail(cuda_fail(e, "cudaGetDevice"));
  if ((e = cudaDeviceGetAttribute(&P.num_sms, cudaDevAttrMultiProcessorCount, P.device)))
    return bail(cuda_fail(e, "querying the SM count"));
  // one warp per source, eight warps per block, a few blocks per SM
  P.grid = (int)std::max<int64_t>(1, std::min<int64_t>(8 * (int64_t)P.num_sms, (I + 7) / 8));
  P.epi_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((R + 255) / 256, 2 * P.num_sms));
  std::vector<int32_t> ident((size_t)R);
  std::iota(ident.begin(), ident.end(), 0);
  if ((e = dev_alloc(P, &P.off, (size_t)I + 1)) || (e = dev_alloc(P, &P.dst, (size_t)E)) ||
      (e = dev_alloc(P, &P.cm, (size_t)E)) || (e = dev_alloc(P, &P.am, (size_t)m * E)) ||
      (e = dev_alloc(P, &P.b_r, R)) || (e = dev_alloc(P, &P.orig_of, R)) ||
      (e = dev_alloc(P, &P.new_of, R)) || (e = dev_alloc(P, &P.mu_r, R)) ||
      (e = dev_alloc(P, &P.y, R)) || (e = dev_alloc(P, &P.part, (size_t)P.grid)) ||
      (e = dev_alloc(P, &P.epi_part, (size_t)P.epi_blocks)) || (e = dev_alloc(P, &P.eval_dev, 8)) ||
      (e = dev_alloc(P, &P.lam_stage, R)) || (e = dev_alloc(P, &P.grad_stage, R)) ||
      (e = dev_alloc(P, &P.status, 1)))
    return bail(cuda_fail(e, "allocating problem memory"));
  if ((e = cudaMallocHost(&P.eval_host, 16 * sizeof(double))))
    return bail(cuda_fail(e, "allocating pinned memory"));
  unsigned* counts = nullptr;
  if ((e = cudaMemsetAsync(P.y, 0, (size_t)R * 8, s)) ||
      (e = cudaMemsetAsync(P.status, 0, sizeof(DeviceStatus), s)) ||
      (e = cudaMemcpyAsync(P.off, off.data(), sizeof(int64_t) * (I + 1), cudaMemcpyHostToDevice,
                           s)) ||
      (E > 0 && (e = cudaMemcpyAsync(P.dst, d->dst, 4 * (size_t)E, h2d, s))) ||
      (E > 0 && (e = cudaMemcpyAsync(P.cm, d->c, 4 * (size_t)E, h2d, s))) ||
      (E > 0 && (e = cudaMemcpyAsync(P.am, d->a, 4 * (size_t)m * E, h2d, s))) ||
      (e = cudaMemcpyAsync(P.b_r, b.data(), 4 * (size_t)R, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(P.orig_of, ident.data(), 4 * (size_t)R, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(P.new_of, ident.data(), 4 * (size_t)R, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMallocAsync(&counts, sizeof(unsigned) * (Jd + 2), s)) ||
      (e = cudaMemsetAsync(counts, 0, sizeof(unsigned) * (Jd + 2), s)) ||
      (E > 0 && (e = launch_histogram(P.dst, E, Jd, counts, P.status, s))) ||
      (E > 0 && (e = launch_check_finite(P.cm, E, P.status, s))) ||
      (E > 0 && (e = launch_check_finite(P.am, (int64_t)m * E, P.status, s))) ||
      (E > 0 && (e = launch_absmax(P.cm, E, counts + Jd, s))) ||
      (E > 0 && (e = launch_absmax(P.am, (int64_t)m * E, counts + Jd + 1, s)))) {
    if (counts) cudaFreeAsync(counts, s);
    return bail(cuda_fail(e, "building the problem"));
  }
  std::vector<unsigned> cnt((size_t)Jd + 2);
  e = cudaMemcpyAsync(cnt.data(), counts, sizeof(unsigned) * (Jd + 2), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(counts, s);
  DeviceStatus st{};
  if (e || (e = cudaMemcpyAsync(&st, P.status, sizeof(st), cudaMemcpyDeviceToHost, s)) ||
      (e = cudaStreamSynchronize(s)))
    return bail(cuda_fail(e, "building the problem"));
  if (st.err) return bail(fail(DUALIP_EINVAL, "dst out of [0, J) or non-finite c / a"));
  // fixed-point scales: |(A x)_r| <= max in-degree max|a|; |sum c x| <= U max|c|
  // and sum w x^2 <= U max w with w = sum_k a_k^2 (primal scaling) or 1, where
  // U = I on the simplex (sum_e x_e <= 1 per source) and E on the unit box
  float mc, ma;
  std::memcpy(&mc, &cnt[Jd], 4);
  std::memcpy(&ma, &cnt[Jd + 1], 4);
  const unsigned maxcnt = Jd > 0 ? *std::max_element(cnt.begin(), cnt.begin() + Jd) : 0u;
  const double mw = P.weighted ? std::max(1.0, (double)m * (double)ma * (double)ma) : 1.0;
  const double units = (double)(P.box ? E : I);
  int ex = 0;
  std::frexp(std::max((double)maxcnt * ma, 1e-30), &ex);
  P.exp_y = std::max(-100, std::min(100, 61 - ex));
  std::frexp(std::max(units * mc, 1e-30), &ex);
  P.exp_c = std::max(-100, std::min(100, 61 - ex));
  std::frexp(std::max(units * mw, 1e-30), &ex);
  P.exp_w = std::max(-100, std::min(100, 61 - ex));
  P.off_host = std::move(off);
  *out = h;
  return DUALIP_OK;
}

}  // namespace dualip

using namespace dualip;

extern "C" {

const char* dualip_last_error(void) { return g_last_error.c_str(); }

dualip_status dualip_create(const dualip_problem_desc* d, void* stream, dualip_problem** out) {
  NvtxRange nvtx_("dualip_create");
  if (!out) return fail(DUALIP_EINVAL, "out is NULL");
  *out = nullptr;
  if (!d) return fail(DUALIP_EINVAL, "desc is NULL");
  const int64_t I = d->num_sources, E = d->num_edges;
  const int32_t J = d->num_dests;
  if (I < 0 || E < 0 || J < 1) return fail(DUALIP_EINVAL, "need I >= 0, E >= 0, J >= 1");
  if (!d->src_offsets || !d->b || (E > 0 && (!d->dst || !d->c || !d->a)))
    return fail(DUALIP_EINVAL, "input arrays must be non-NULL");
  if (d->storage != DUALIP_EDGE_F32 && d->storage != DUALIP_EDGE_BF16)
    return fail(DUALIP_EINVAL, "unknown edge storage");
  if (d->primal_scaling != 0 && d->primal_scaling != 1)
    return fail(DUALIP_EINVAL, "primal_scaling must be 0 or 1");
  if (d->projection != DUALIP_PROJ_SIMPLEX && d->projection != DUALIP_PROJ_BOX)
    return fail(DUALIP_EINVAL, "unknown projection");
  if (d->inputs_on_device != 0 && d->inputs_on_device != 1)
    return fail(DUALIP_EINVAL, "inputs_on_device must be 0 or 1");
  if (d->num_families < 0) return fail(DUALIP_EINVAL, "num_families must be >= 0");
  if (d->num_families > 1) return create_multi(d, stream, out);
  cudaStream_t s = as_stream(stream);
  const cudaMemcpyKind h2d = d->inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e;

  // offsets on the host: validation and tiling
  std::vector<int64_t> off((size_t)I + 1);
  if (d->inputs_on_device) {
    e = cudaMemcpyAsync(off.data(), d->src_offsets, sizeof(int64_t) * (I + 1),
                        cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "reading src_offsets");
  } else {
    std::memcpy(off.data(), d->src_offsets, sizeof(int64_t) * (I + 1));
  }
  if (off[0] != 0) return fail(DUALIP_EINVAL, "src_offsets[0] must be 0");
  for (int64_t i = 0; i < I; ++i)
    if (off[i + 1] < off[i]) return fail(DUALIP_EINVAL, "src_offsets must be nondecreasing");
  if (off[I] != E) return fail(DUALIP_EINVAL, "src_offsets[I] must equal num_edges");

  // Degree order: when the pass's cost model says so, sources are stored by
  // increasing degree (ties in the caller's order), so that the pass's
  // batches of eight consecutive sources have similar spans and one window
  // width serves all eight.  Sources are independent blocks of the problem:
  // the gradient and the objective partials are exact sums in any order, and
  // dualip_get_primal maps x back to the caller's order.
  std::vector<int64_t> src_of, off_st;
  choose_degree_order(off, tile_edges_for(d->storage), kTileSources, src_of, off_st);
  const bool seg = !src_of.empty();
  const std::vector<int64_t>& off_s = seg ? off_st : off;  // offsets as stored

  auto* h = new (std::nothrow) dualip_problem();
  if (!h) return fail(DUALIP_ENOMEM, "host allocation failed");
  Problem& P = h->p;
  P.I = I;
  P.E = E;
  P.J = J;
  P.storage = d->storage;
  P.weighted = d->primal_scaling;
  P.box = d->projection == DUALIP_PROJ_BOX ? 1 : 0;
  // small mean degree (at most 16 edges per source): the pass takes sources
  // 32 at a time and gives a span of up to 16 slots one lane
  P.tiny = (kTinyBatches && I > 0 && E <= 16 * I) ? 1 : 0;
  P.last_stream = s;
  auto bail = [&](dualip_status st) {
    cudaStreamSynchronize(s);
    free_all(P);
    delete h;
    return st;
  };
  if ((e = cudaGetDevice(&P.device))) return bail(cuda_fail(e, "cudaGetDevice"));
  if ((e = cudaDeviceGetAttribute(&P.num_sms, cudaDevAttrMultiProcessorCount, P.device)))
    return bail(cuda_fail(e, "querying the SM count"));
  if ((e = configure_device_once(P.device)))
    return bail(cuda_fail(e, "configuring the pass kernel"));

  std::vector<int64_t> tiles, tile_e;
  build_tiles(off_s, tiles, tile_e, tile_edges_for(P.storage), kTileSources);
  P.ntiles = (int64_t)tiles.size() - 1;
  // Segment classes of the sources larger than a stage: the block class up
  // to kMultiBlockStages stages, the multi-block class (hub sources) from
  // there (not for the unit box, whose edges are independent, and not for a
  // source past the hub kernel's 32-bit edge indices).
  const int64_t stage_e = tile_edges_for(P.storage);
  std::vector<HubPlan> hub_plan;
  std::vector<int32_t> chunk_hub;
  bool big = false;
  plan_hubs(tile_e, stage_e, kMultiBlockStages, P.box != 0, kHubChunk, P.mb_min, hub_plan,
            chunk_hub, big);
  P.has_big = big ? 1 : 0;
  std::vector<HubDesc> hubs(hub_plan.size());
  int64_t hub_edges = 0;
  for (size_t h = 0; h < hub_plan.size(); ++h) {
    hubs[h] = HubDesc{};
    hubs[h].e0 = hub_plan[h].e0;
    hubs[h].cand0 = hub_plan[h].cand0;
    hubs[h].deg = hub_plan[h].deg;
    hubs[h].c0 = hub_plan[h].c0;
    hubs[h].nch = hub_plan[h].nch;
    hub_edges += hub_plan[h].deg;
  }
  P.nhub = (int)hubs.size();
  P.nchunks = (int64_t)chunk_hub.size();
  P.grid = (int)std::max<int64_t>(1, std::min<int64_t>(P.num_sms, P.ntiles));
  P.h_mu = std::min(J, kMaxCachedDests);
  P.h_y = std::min(J, kMaxPrivDests);
  P.epi_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((J + 255) / 256, 2 * P.num_sms));

  const size_t e_pad = (size_t)((E + 3) & ~int64_t(3)) + 4;
  const size_t i_pad = (size_t)I + 4;
  std::vector<int64_t> off_pad(i_pad, E);
  std::copy(off_s.begin(), off_s.end(), off_pad.begin());

  std::vector<uint32_t> off32_pad(i_pad);
  for (size_t i = 0; i < i_pad; ++i) off32_pad[i] = (uint32_t)off_pad[i];
  if ((e = dev_alloc(P, &P.off, i_pad)) || (e = dev_alloc(P, &P.off32, i_pad)) ||
      (e = dev_alloc(P, &P.dst, e_pad)) ||
      (e = dev_alloc(P, &P.tiles, tiles.size())) || (e = dev_alloc(P, &P.tile_e, tiles.size())) ||
      (e = dev_alloc(P, &P.b_r, J)) || (e = dev_alloc(P, &P.orig_of, J)) ||
      (e = dev_alloc(P, &P.new_of, J)) || (e = dev_alloc(P, &P.mu_r, J)) ||
      (e = dev_alloc(P, &P.y, J)) ||
      (e = dev_alloc(P, &P.part, (size_t)P.grid + P.nhub)) ||
      (e = dev_alloc(P, &P.epi_part, (size_t)P.epi_blocks)) ||
      (e = dev_alloc(P, &P.eval_dev, 8)) || (e = dev_alloc(P, &P.lam_stage, J)) ||
      (e = dev_alloc(P, &P.grad_stage, J)) || (e = dev_alloc(P, &P.status, 1)))
    return bail(cuda_fail(e, "allocating problem memory"));
  if (P.nhub > 0) {
    if ((e = dev_alloc(P, &P.hubs, hubs.size())) ||
        (e = dev_alloc(P, &P.chunk_hub, chunk_hub.size())) ||
        (e = dev_alloc(P, &P.hub_stat, chunk_hub.size() * (kHubThreads / 32))) ||
        (e = dev_alloc(P, &P.hub_cand, (size_t)hub_edges)) ||
        (e = dev_alloc(P, &P.hub_cnt, 2 * hubs.size())))
      return bail(cuda_fail(e, "allocating hub-source memory"));
    if ((e = cudaMemcpyAsync(P.hubs, hubs.data(), hubs.size() * sizeof(HubDesc),
                             cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(P.chunk_hub, chunk_hub.data(), chunk_hub.size() * sizeof(int32_t),
                             cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemsetAsync(P.hub_cnt, 0, 2 * hubs.size() * sizeof(unsigned), s)))
      return bail(cuda_fail(e, "uploading hub sources"));
  }
  if (P.storage == DUALIP_EDGE_F32) {
    if ((e = dev_alloc(P, &P.ca2, e_pad))) return bail(cuda_fail(e, "allocating edge memory"));
  } else {
    if ((e = dev_alloc(P, &P.ca, e_pad))) return bail(cuda_fail(e, "allocating edge memory"));
  }
  if ((e = cudaMallocHost(&P.eval_host, 16 * sizeof(double))))
    return bail(cuda_fail(e, "allocating pinned memory"));

  // zero everything that must start at zero (padding included)
  if ((e = cudaMemsetAsync(P.dst, 0, e_pad * 4, s)) || (e = cudaMemsetAsync(P.y, 0, J * 8, s)) ||
      (e = cudaMemsetAsync(P.status, 0, sizeof(DeviceStatus), s)))
    return bail(cuda_fail(e, "clearing problem memory"));
  if (P.ca2 && (e = cudaMemsetAsync(P.ca2, 0, e_pad * 8, s)))
    return bail(cuda_fail(e, "clearing edge memory"));
  if (P.ca && (e = cudaMemsetAsync(P.ca, 0, e_pad * 4, s)))
    return bail(cuda_fail(e, "clearing edge memory"));
  if ((e = cudaMemcpyAsync(P.off, off_pad.data(), i_pad * 8, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(P.off32, off32_pad.data(), i_pad * 4, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(P.tiles, tiles.data(), tiles.size() * 8, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(P.tile_e, tile_e.data(), tile_e.size() * 8, cudaMemcpyHostToDevice, s)))
    return bail(cuda_fail(e, "uploading offsets"));

  // raw destinations -> in-degree histogram (validates the range)
  const int32_t* dst_raw = d->dst;
  int32_t* dst_tmp = nullptr;
  unsigned* counts = nullptr;
  int64_t *seg_src = nullptr, *seg_orig = nullptr;  // degree order: device copies of the map
  // temporaries are stream-ordered (cudaMallocAsync / cudaFreeAsync on s): no
  // device-wide synchronisation, so a build overlaps other streams' kernels
  auto free_seg = [&]() {
    if (seg_src) cudaFreeAsync(seg_src, s);
    if (seg_orig) cudaFreeAsync(seg_orig, s);
    seg_src = seg_orig = nullptr;
  };
  if (seg && ((e = cudaMallocAsync(&seg_src, sizeof(int64_t) * I, s)) ||
              (e = cudaMallocAsync(&seg_orig, sizeof(int64_t) * (I + 1), s)) ||
              (e = cudaMemcpyAsync(seg_src, src_of.data(), sizeof(int64_t) * I,
                                   cudaMemcpyHostToDevice, s)) ||
              (e = cudaMemcpyAsync(seg_orig, off.data(), sizeof(int64_t) * (I + 1),
                                   cudaMemcpyHostToDevice, s)))) {
    free_seg();
    return bail(cuda_fail(e, "uploading the source order"));
  }
  const SegMap segmap{P.off, seg_src, seg_orig, I};
  if ((e = cudaMallocAsync(&counts, sizeof(unsigned) * J, s))) {
    free_seg();
    return bail(cuda_fail(e, "allocating"));
  }
  auto free_tmp = [&]() {
    if (dst_tmp) cudaFreeAsync(dst_tmp, s);
    if (counts) cudaFreeAsync(counts, s);
    dst_tmp = nullptr;
    counts = nullptr;
    free_seg();
  };
  if (!d->inputs_on_device && E > 0) {
    if ((e = cudaMallocAsync(&dst_tmp, sizeof(int32_t) * E, s)) ||
        (e = cudaMemcpyAsync(dst_tmp, d->dst, sizeof(int32_t) * E, cudaMemcpyHostToDevice, s))) {
      free_tmp();
      return bail(cuda_fail(e, "uploading dst"));
    }
    dst_raw = dst_tmp;
  }
  std::vector<unsigned> cnt(J);
  if ((e = cudaMemsetAsync(counts, 0, sizeof(unsigned) * J, s)) ||
      (E > 0 && (e = launch_histogram(dst_raw, E, J, counts, P.status, s))) ||
      (e = cudaMemcpyAsync(cnt.data(), counts, sizeof(unsigned) * J, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaStreamSynchronize(s))) {
    free_tmp();
    return bail(cuda_fail(e, "counting in-degrees"));
  }
  // renumber destinations by decreasing in-degree (ties by id): the hot ones
  // get the smallest ids, which the pass caches in shared memory
  std::vector<int32_t> orig_of(J), new_of(J);
  std::iota(orig_of.begin(), orig_of.end(), 0);
  std::stable_sort(orig_of.begin(), orig_of.end(),
                   [&](int32_t x, int32_t y) { return cnt[x] > cnt[y]; });
  for (int32_t r = 0; r < J; ++r) new_of[orig_of[r]] = r;
  std::vector<float> b_host(J), b_r(J);
  if ((e = cudaMemcpyAsync(b_host.data(), d->b, sizeof(float) * J,
                           d->inputs_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost,
                           s)) ||
      (e = cudaStreamSynchronize(s))) {
    free_tmp();
    return bail(cuda_fail(e, "reading b"));
  }
  double bn = 0.0;
  for (int32_t j = 0; j < J; ++j) bn += (double)b_host[j] * (double)b_host[j];
  P.bnorm = std::sqrt(bn);
  for (int32_t r = 0; r < J; ++r) {
    b_r[r] = b_host[orig_of[r]];
    if (!std::isfinite(b_r[r])) {
      free_tmp();
      return bail(fail(DUALIP_EINVAL, "b must be finite"));
    }
  }
  if ((e = cudaMemcpyAsync(P.orig_of, orig_of.data(), 4 * (size_t)J, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(P.new_of, new_of.data(), 4 * (size_t)J, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(P.b_r, b_r.data(), 4 * (size_t)J, cudaMemcpyHostToDevice, s)) ||
      (E > 0 && !seg && (e = launch_renumber(dst_raw, P.dst, P.new_of, E, J, P.status, s))) ||
      (E > 0 && seg &&
       (e = launch_renumber_seg(dst_raw, P.dst, P.new_of, segmap, J, P.status, s)))) {
    free_tmp();
    return bail(cuda_fail(e, "renumbering destinations"));
  }
  if (dst_tmp) cudaFreeAsync(dst_tmp, s);
  if (counts) cudaFreeAsync(counts, s);
  dst_tmp = nullptr;
  counts = nullptr;

  // edge values
  unsigned absmax[2] = {0u, 0u};  // bit patterns of max |c|, max |a|
  unsigned* counts_max = nullptr;
  if ((e = cudaMallocAsync(&counts_max, 2 * sizeof(unsigned), s))) {
    free_seg();
    return bail(cuda_fail(e, "allocating"));
  }
  if (E > 0) {
    float *c_tmp = nullptr, *a_tmp = nullptr;
    const float *c_src = d->c, *a_src = d->a;
    if (!d->inputs_on_device) {
      if ((e = cudaMallocAsync(&c_tmp, 4 * (size_t)E, s)) ||
          (e = cudaMallocAsync(&a_tmp, 4 * (size_t)E, s)) ||
          (e = cudaMemcpyAsync(c_tmp, d->c, 4 * (size_t)E, h2d, s)) ||
          (e = cudaMemcpyAsync(a_tmp, d->a, 4 * (size_t)E, h2d, s))) {
        if (c_tmp) cudaFreeAsync(c_tmp, s);
        if (a_tmp) cudaFreeAsync(a_tmp, s);
        cudaFreeAsync(counts_max, s);
        free_seg();
        return bail(cuda_fail(e, "uploading c and a"));
      }
      c_src = c_tmp;
      a_src = a_tmp;
    }
    if ((e = launch_check_finite(c_src, E, P.status, s)) ||
        (e = launch_check_finite(a_src, E, P.status, s)) ||
        (e = cudaMemsetAsync(counts_max, 0, 2 * sizeof(unsigned), s)) ||
        (e = launch_absmax(c_src, E, counts_max, s)) ||
        (e = launch_absmax(a_src, E, counts_max + 1, s)) ||
        (e = cudaMemcpyAsync(absmax, counts_max, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost,
                             s)) ||
        (!seg && P.storage == DUALIP_EDGE_BF16 &&
         (e = launch_pack_bf16(c_src, a_src, P.ca, E, s))) ||
        (!seg && P.storage == DUALIP_EDGE_F32 &&
         (e = launch_pack_f32(c_src, a_src, P.ca2, E, s))) ||
        (seg && (e = launch_pack_seg(c_src, a_src, P.storage,
                                     P.storage == DUALIP_EDGE_BF16 ? (void*)P.ca : (void*)P.ca2,
                                     segmap, s)))) {
      if (c_tmp) cudaFreeAsync(c_tmp, s);
      if (a_tmp) cudaFreeAsync(a_tmp, s);
      cudaFreeAsync(counts_max, s);
      free_seg();
      return bail(cuda_fail(e, "checking edge values"));
    }
    if (c_tmp) cudaFreeAsync(c_tmp, s);
    if (a_tmp) cudaFreeAsync(a_tmp, s);
  }
  cudaFreeAsync(counts_max, s);
  free_seg();
  e = cudaStreamSynchronize(s);
  if (e) return bail(cuda_fail(e, "building the problem"));
  // Fixed-point scale 2^exp_y of A x: |(A x)_j| <= max in-degree * max |a|
  // (x <= 1), kept below 2^61 so no sum can overflow.
  {
    float ma;
    std::memcpy(&ma, &absmax[1], 4);
    const unsigned maxcnt = cnt.empty() ? 0u : *std::max_element(cnt.begin(), cnt.end());
    int ex = 0;
    std::frexp(std::max((double)maxcnt * ma, 1e-30), &ex);  // bound < 2^ex
    P.exp_y = std::max(-100, std::min(100, 61 - ex));
    // Objective partials: on the simplex every source has sum_e x_e <= 1 and
    // x_e <= 1, so |sum c x| <= I max|c| and sum w x^2 <= I max w (w = a^2, or
    // 1 where a = 0, with primal scaling; w = 1 without); on the unit box only
    // x_e <= 1 holds, and E takes the place of I.  The BF16 rounding of c and
    // a stays far inside the two bits of headroom below 2^63.
    float mc;
    std::memcpy(&mc, &absmax[0], 4);
    const double mw = P.weighted ? std::max(1.0, (double)ma * (double)ma) : 1.0;
    const double units = (double)(P.box ? E : I);
    std::frexp(std::max(units * mc, 1e-30), &ex);
    P.exp_c = std::max(-100, std::min(100, 61 - ex));
    std::frexp(std::max(units * mw, 1e-30), &ex);
    P.exp_w = std::max(-100, std::min(100, 61 - ex));
  }
  DeviceStatus st{};
  if ((e = cudaMemcpyAsync(&st, P.status, sizeof(st), cudaMemcpyDeviceToHost, s)) ||
      (e = cudaStreamSynchronize(s)))
    return bail(cuda_fail(e, "reading the device status"));
  if (st.err) return bail(fail(DUALIP_EINVAL, "dst out of [0, J) or non-finite c / a"));
  if (P.nhub > 0) {
    P.hub_host = hubs;
    P.hub_caller0.resize(hubs.size());
    for (size_t k = 0; k < hubs.size(); ++k)
      P.hub_caller0[k] = caller_segment_start(off_s, off, src_of, hubs[k].e0);
    if ((e = sort_hub_edges(P, hub_edges, s)))
      return bail(cuda_fail(e, "storing the hub sources in destination order"));
  }
  if (seg) {
    P.off_host = std::move(off_st);
    P.orig_off_host = std::move(off);
    P.src_of_host = std::move(src_of);
  } else {
    P.off_host = std::move(off);
  }
  *out = h;
  return DUALIP_OK;
}

void dualip_destroy(dualip_problem* h) {
  if (!h) return;
  cudaStreamSynchronize(h->p.last_stream);
  free_all(h->p);
  delete h;
}

dualip_status dualip_get_info(const dualip_problem* h, int64_t* I, int32_t* J, int64_t* E,
                              int64_t* ntiles) {
  if (!h) return fail(DUALIP_EINVAL, "problem handle is NULL");
  if (I) *I = h->p.I;
  if (J) *J = h->p.J;
  if (E) *E = h->p.E;
  if (ntiles) *ntiles = h->p.ntiles;
  return DUALIP_OK;
}

dualip_status dualip_dual_grad_async(dualip_problem* h, const float* lambda, double gamma,
                                     float* grad, double* out_dev, void* stream) {
  NvtxRange nvtx_("dualip_dual_grad_async");
  dualip_status st = check_eval_args(h, lambda, gamma, grad);
  if (st) return st;
  if (!out_dev) return fail(DUALIP_EINVAL, "out_dev is NULL");
  cudaStream_t s = as_stream(stream);
  h->p.last_stream = s;
  cudaError_t e = enqueue_eval(h->p, lambda, gamma, grad, out_dev, nullptr, s);
  return e ? cuda_fail(e, "launching the dual evaluation") : DUALIP_OK;
}

dualip_status dualip_dual_grad(dualip_problem* h, const float* lambda, double gamma, float* grad,
                               dualip_eval* out, void* stream) {
  NvtxRange nvtx_("dualip_dual_grad");
  dualip_status st = check_eval_args(h, lambda, gamma, grad);
  if (st) return st;
  Problem& P = h->p;
  cudaStream_t s = as_stream(stream);
  P.last_stream = s;
  cudaError_t e = enqueue_eval(P, lambda, gamma, grad, P.eval_dev, nullptr, s);
  if (e) return cuda_fail(e, "launching the dual evaluation");
  if (!out) return DUALIP_OK;
  if ((e = cudaMemcpyAsync(P.eval_host, P.eval_dev, 5 * sizeof(double), cudaMemcpyDeviceToHost, s)))
    return cuda_fail(e, "reading the scalars");
  if ((st = read_status(P, s))) return st;
  std::memcpy(out, P.eval_host, sizeof(dualip_eval));
  return DUALIP_OK;
}

dualip_status dualip_dual_grad_host(dualip_problem* h, const float* lambda_host, double gamma,
                                    float* grad_host, dualip_eval* out, void* stream) {
  dualip_status st = check_eval_args(h, lambda_host, gamma, grad_host);
  if (st) return st;
  Problem& P = h->p;
  cudaStream_t s = as_stream(stream);
  P.last_stream = s;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(P.lam_stage, lambda_host, 4 * (size_t)P.J, cudaMemcpyHostToDevice, s)))
    return cuda_fail(e, "copying lambda in");
  if ((e = enqueue_eval(P, P.lam_stage, gamma, P.grad_stage, P.eval_dev, nullptr, s)))
    return cuda_fail(e, "launching the dual evaluation");
  if ((e = cudaMemcpyAsync(grad_host, P.grad_stage, 4 * (size_t)P.J, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(P.eval_host, P.eval_dev, 5 * sizeof(double), cudaMemcpyDeviceToHost, s)))
    return cuda_fail(e, "copying results out");
  if ((st = read_status(P, s))) return st;
  if (out) std::memcpy(out, P.eval_host, sizeof(dualip_eval));
  return DUALIP_OK;
}

dualip_status dualip_get_primal(dualip_problem* h, const float* lambda, double gamma, float* x,
                                void* stream) {
  NvtxRange nvtx_("dualip_get_primal");
  dualip_status st = check_eval_args(h, lambda, gamma, x);
  if (st) return st;
  Problem& P = h->p;
  cudaStream_t s = as_stream(stream);
  P.last_stream = s;
  cudaError_t e;
  const bool seg = !P.src_of_host.empty();
  if (!seg && P.nhub == 0) {
    e = enqueue_eval(P, lambda, gamma, P.grad_stage, P.eval_dev, x, s);
    return e ? cuda_fail(e, "launching the primal evaluation") : DUALIP_OK;
  }
  // degree order: x in stored order, then each source's segment back to the
  // caller's place; hub sources: their edges back from destination order
  // (stream-ordered temporaries)
  float* xs = nullptr;
  int64_t *src = nullptr, *orig = nullptr;
  const int64_t I = P.I;
  if (!(e = cudaMallocAsync(&xs, sizeof(float) * std::max<int64_t>(P.E, 1), s)) &&
      !(e = enqueue_eval(P, lambda, gamma, P.grad_stage, P.eval_dev, xs, s))) {
    if (seg) {
      if (!(e = cudaMallocAsync(&src, sizeof(int64_t) * I, s)) &&
          !(e = cudaMallocAsync(&orig, sizeof(int64_t) * (I + 1), s)) &&
          !(e = cudaMemcpyAsync(src, P.src_of_host.data(), sizeof(int64_t) * I,
                                cudaMemcpyHostToDevice, s)) &&
          !(e = cudaMemcpyAsync(orig, P.orig_off_host.data(), sizeof(int64_t) * (I + 1),
                                cudaMemcpyHostToDevice, s)))
        e = launch_unpermute_seg(xs, x, SegMap{P.off, src, orig, I}, s);
    } else if (P.E > 0) {
      e = cudaMemcpyAsync(x, xs, sizeof(float) * P.E, cudaMemcpyDeviceToDevice, s);
    }
    for (size_t k = 0; !e && k < P.hub_host.size(); ++k) {
      const HubDesc& hd = P.hub_host[k];
      e = launch_scatter_perm(xs + hd.e0, x + P.hub_caller0[k], P.hub_perm + hd.cand0, hd.deg,
                              s);
    }
  }
  if (xs) cudaFreeAsync(xs, s);
  if (src) cudaFreeAsync(src, s);
  if (orig) cudaFreeAsync(orig, s);
  return e ? cuda_fail(e, "launching the primal evaluation") : DUALIP_OK;
}

dualip_status dualip_profile_enable(dualip_problem* h, int32_t max_evals) {
  if (!h || max_evals < 1) return fail(DUALIP_EINVAL, "need a handle and max_evals >= 1");
  Problem& P = h->p;
  free_events(P);
  P.prof_ev.resize(4 * (size_t)max_evals, nullptr);
  for (auto& ev : P.prof_ev) {
    cudaError_t e = cudaEventCreate(&ev);
    if (e) {
      ev = nullptr;
      free_events(P);
      return cuda_fail(e, "creating timing events");
    }
  }
  P.prof_max = max_evals;
  P.prof_used = 0;
  return DUALIP_OK;
}

dualip_status dualip_profile_collect(dualip_problem* h, double* ms_prep, double* ms_pass,
                                     double* ms_epi, int32_t* count) {
  if (!h) return fail(DUALIP_EINVAL, "problem handle is NULL");
  Problem& P = h->p;
  double t[3] = {0, 0, 0};
  for (int i = 0; i < P.prof_used; ++i) {
    cudaEvent_t* ev = &P.prof_ev[4 * (size_t)i];
    cudaError_t e = cudaEventSynchronize(ev[3]);
    for (int k = 0; k < 3 && !e; ++k) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
      t[k] += ms;
    }
    if (e) {
      free_events(P);
      return cuda_fail(e, "reading timing events");
    }
  }
  if (ms_prep) *ms_prep = t[0];
  if (ms_pass) *ms_pass = t[1];
  if (ms_epi) *ms_epi = t[2];
  if (count) *count = P.prof_used;
  free_events(P);
  return DUALIP_OK;
}

dualip_status dualip_debug_abort_waits(dualip_problem* h, void* stream) {
  if (!h) return fail(DUALIP_EINVAL, "problem handle is NULL");
  static const int one = 1;
  const cudaError_t e =
      cudaMemcpyAsync(&h->p.status->abort_req, &one, sizeof(int), cudaMemcpyHostToDevice,
                      as_stream(stream));
  if (e == cudaSuccess) cudaStreamSynchronize(as_stream(stream));
  return e ? cuda_fail(e, "setting the abort request") : DUALIP_OK;
}

dualip_status dualip_check_device_status(dualip_problem* h, void* stream) {
  if (!h) return fail(DUALIP_EINVAL, "problem handle is NULL");
  return read_status(h->p, as_stream(stream));
}

}  // extern "C"
