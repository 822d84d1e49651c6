// Serving form: a request loop with continuous batching over the batched
// ascent (batch.cu).
//
// Two host threads share the device.  The admission thread takes queued
// requests in arrival order while a slot is free and the request's estimated
// footprint fits the HBM budget, and builds each on the device with
// dualip_create on its own stream (so the upload overlaps the iterations of
// the resident requests).  A request stays QUEUED while it is built, since the
// build reads the caller's arrays; it turns RUNNING once they are copied.  The scheduler thread attaches built requests to
// the batch of their storage kind at a chunk boundary, runs every non-empty
// batch for check_every iterations (one CUDA graph per batch membership),
// reads the per-request stopping quantities, and retires requests that have
// met their tolerances or max_iters: lambda to host memory, slot and device
// memory released.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "batch.h"

namespace dualip {
namespace {

constexpr int kKinds = 4;  // (storage, primal scaling)

struct Request {
  dualip_problem_desc desc{};
  dualip_solve_opts opts{};
  int state = DUALIP_REQ_QUEUED;
  dualip_status status = DUALIP_OK;
  std::string error;
  double t_submit = -1, t_admit = -1, t_done = -1;
  int64_t footprint = 0, transient = 0;
  dualip_problem* h = nullptr;  // built, waiting for a slot, or resident
  int kind = 0, slot = -1;
  int32_t iters = 0;
  bool building = false;  // admitted; dualip_create is reading the caller's arrays
  bool cancel = false;    // leaves when its build ends or at the next chunk boundary
  dualip_solve_result result{};
  std::vector<float> lam;
};

int64_t resident_bytes(const dualip_problem_desc& d) {
  return request_resident_bytes(d.num_sources, d.num_edges, d.num_dests,
                                d.storage == DUALIP_EDGE_BF16);
}
int64_t transient_bytes(const dualip_problem_desc& d) {
  return request_transient_bytes(d.num_edges, d.inputs_on_device != 0);
}

}  // namespace

struct Server {
  dualip_server_opts o{};
  int device = 0, num_sms = 0;
  std::mutex mu;
  std::condition_variable cv;       // submissions, built problems, completions
  std::deque<int64_t> queue;        // QUEUED, in arrival order
  std::deque<int64_t> built;        // RUNNING, built, not yet attached
  std::map<int64_t, Request> reqs;
  int64_t next_ticket = 1;
  int64_t resident = 0, peak = 0;
  int slots_used[kKinds] = {0, 0, 0, 0};  // admitted (built or attached) per kind
  bool stop = false;
  Batch batch[kKinds];
  bool batch_ok[kKinds] = {false, false, false, false};
  std::vector<int64_t> slot_ticket[kKinds];
  std::thread admitter, scheduler;
  std::chrono::steady_clock::time_point t0;
  int64_t chunks = 0, slot_iters = 0, n_done = 0, n_failed = 0;
  double busy = 0.0;
  cudaStream_t admit_stream = nullptr;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  void finish_locked(Request& r, int state) {
    r.state = state;
    r.t_done = now();
    resident -= r.footprint;
    slots_used[r.kind] -= 1;
    if (state == DUALIP_REQ_DONE) ++n_done;
    else ++n_failed;
    cv.notify_all();
  }
  void admit_loop();
  void schedule_loop();
  void run_chunks();
};

void Server::admit_loop() {
  cudaSetDevice(device);
  for (;;) {
    int64_t t = 0;
    dualip_problem_desc d{};
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        if (stop) return;
        if (!queue.empty()) {
          Request& r = reqs[queue.front()];
          const Admission a = admission(resident, r.footprint, r.transient, o.hbm_budget_bytes,
                                        slots_used[r.kind] < o.max_slots);
          if (a == Admission::kAdmit) break;
          if (a == Admission::kReject) {  // can never fit
            r.status = DUALIP_ENOMEM;
            r.error = "the request's footprint exceeds the HBM budget";
            r.state = DUALIP_REQ_FAILED;
            r.t_done = now();
            ++n_failed;
            queue.pop_front();
            cv.notify_all();
            continue;
          }
        }
        cv.wait_for(lk, std::chrono::milliseconds(20));
      }
      t = queue.front();
      queue.pop_front();
      Request& r = reqs[t];
      r.building = true;
      r.t_admit = now();
      resident += r.footprint;
      peak = std::max(peak, resident + r.transient);
      slots_used[r.kind] += 1;
      d = r.desc;
    }
    dualip_problem* h = nullptr;
    const dualip_status st = dualip_create(&d, admit_stream, &h);
    std::string msg = st ? dualip_last_error() : "";
    std::lock_guard<std::mutex> lk(mu);
    Request& r = reqs[t];
    r.building = false;
    if (st) {
      r.status = st;
      r.error = msg;
      finish_locked(r, DUALIP_REQ_FAILED);
    } else {
      r.h = h;
      r.state = DUALIP_REQ_RUNNING;  // a cancel taken during the build is honoured at attach
      built.push_back(t);
      cv.notify_all();
    }
  }
}

// One chunk of every non-empty batch, then the stopping tests.
void Server::run_chunks() {
  NvtxRange nvtx_("serve_chunk");
  for (int k = 0; k < kKinds; ++k) {
    Batch& B = batch[k];
    if (!batch_ok[k]) continue;
    bool any = false;
    // a chunk runs check_every iterations, or fewer when a request has fewer
    // left before its max_iters (so that no request runs past it)
    int n_it = o.check_every;
    {
      std::lock_guard<std::mutex> lk(mu);
      for (int s = 0; s < B.n; ++s) {
        if (!B.active[s]) continue;
        any = true;
        const Request& r = reqs[slot_ticket[k][s]];
        n_it = std::min(n_it, std::max(1, r.opts.max_iters - r.iters));
      }
    }
    if (!any) continue;
    const double c0 = now();
    cudaError_t e = rebuild_lists(B);
    if (!e) e = run_batch_chunk(B, n_it, n_it == o.check_every);
    if (!e) e = batch_read_state(B);
    dualip_status st = e ? cuda_fail(e, "running a serving chunk") : batch_status(B);
    {
      std::lock_guard<std::mutex> lk(mu);
      busy += now() - c0;
      ++chunks;
    }
    for (int s = 0; s < B.n; ++s) {
      if (!B.active[s]) continue;
      const int64_t t = slot_ticket[k][s];
      Request* rp;
      int32_t iters;
      bool cancelled;
      {
        std::lock_guard<std::mutex> lk(mu);
        rp = &reqs[t];
        rp->iters += n_it;
        iters = rp->iters;
        cancelled = rp->cancel;
        slot_iters += n_it;
      }
      Request& r = *rp;  // the fields below are written by this thread only
      const SlotSolve& S = B.h_ss[s];
      const bool conv = !st && r.opts.stop_on_tol && S.last_gamma == r.opts.gamma_final &&
                        S.gap_rel <= r.opts.tol_gap && S.infeas_rel <= r.opts.tol_infeas;
      if (!st && !cancelled && !conv && iters < r.opts.max_iters) continue;
      // retire: lambda to host, slot and memory back
      std::vector<float> lam;
      dualip_status rst = st ? st : (cancelled ? DUALIP_ECANCELED : DUALIP_OK);
      if (!rst) {
        float* lam_dev = nullptr;  // stream-ordered, like the copy below
        e = cudaMallocAsync(&lam_dev, sizeof(float) * std::max<int32_t>(r.desc.num_dests, 1),
                            B.stream);
        if (!e) e = batch_write_lambda(B, s, lam_dev);
        lam.resize(r.desc.num_dests);
        if (!e)
          e = cudaMemcpyAsync(lam.data(), lam_dev, sizeof(float) * r.desc.num_dests,
                              cudaMemcpyDeviceToHost, B.stream);
        if (lam_dev) cudaFreeAsync(lam_dev, B.stream);
        if (!e) e = cudaStreamSynchronize(B.stream);
        if (e) rst = cuda_fail(e, "reading a finished request's lambda");
      }
      dualip_solve_result res{};
      const double* ev = B.h_eval + 5 * s;
      res.iters = iters;
      res.converged = conv ? 1 : 0;
      res.last.dual_obj = ev[0];
      res.last.primal_obj = ev[1];
      res.last.reg = ev[2];
      res.last.infeas_l2 = ev[3];
      res.last.lambda_dot_grad = ev[4];
      res.gap_rel = S.gap_rel;
      res.infeas_rel = S.infeas_rel;
      res.gamma = S.last_gamma;
      batch_detach(B, s);
      dualip_destroy(r.h);
      const std::string msg =
          rst == DUALIP_ECANCELED ? std::string("cancelled") : (rst ? dualip_last_error() : "");
      std::lock_guard<std::mutex> lk(mu);
      r.h = nullptr;
      r.slot = -1;
      r.result = res;
      r.lam.swap(lam);
      if (rst) {
        r.status = rst;
        r.error = msg;
      }
      finish_locked(r, rst ? DUALIP_REQ_FAILED : DUALIP_REQ_DONE);
    }
  }
}

void Server::schedule_loop() {
  cudaSetDevice(device);
  for (;;) {
    std::vector<int64_t> ready;
    bool running = false;
    {
      std::unique_lock<std::mutex> lk(mu);
      for (int k = 0; k < kKinds; ++k)
        for (int s = 0; s < (int)slot_ticket[k].size(); ++s) running = running || slot_ticket[k][s];
      if (stop) return;
      if (built.empty() && !running) {
        cv.wait_for(lk, std::chrono::milliseconds(20));
        continue;
      }
      ready.assign(built.begin(), built.end());
      built.clear();
    }
    // joins at the chunk boundary
    for (int64_t t : ready) {
      Request* rp;
      {
        std::lock_guard<std::mutex> lk(mu);
        rp = &reqs[t];
      }
      Request& r = *rp;
      const int k = r.kind;
      bool cancelled;
      {
        std::lock_guard<std::mutex> lk(mu);
        cancelled = r.cancel;
      }
      if (cancelled) {
        dualip_destroy(r.h);
        std::lock_guard<std::mutex> lk(mu);
        r.h = nullptr;
        r.status = DUALIP_ECANCELED;
        r.error = "cancelled";
        finish_locked(r, DUALIP_REQ_FAILED);
        continue;
      }
      cudaError_t e = cudaSuccess;
      if (!batch_ok[k]) {
        e = batch_alloc(batch[k], o.max_slots, r.desc.storage, r.desc.primal_scaling, num_sms);
        batch[k].lean_auto = true;
        batch_ok[k] = e == cudaSuccess;
        slot_ticket[k].assign(o.max_slots, 0);
      }
      int s = -1;
      if (!e) s = batch_attach(batch[k], &r.h->p, r.opts, &e);
      std::lock_guard<std::mutex> lk(mu);
      if (s < 0) {
        r.status = e ? DUALIP_ECUDA : DUALIP_EBUSY;
        r.error = e ? cudaGetErrorString(e) : "no free slot";
        dualip_destroy(r.h);
        r.h = nullptr;
        finish_locked(r, DUALIP_REQ_FAILED);
        continue;
      }
      r.slot = s;
      slot_ticket[k][s] = t;
    }
    run_chunks();
    std::lock_guard<std::mutex> lk(mu);
    for (int k = 0; k < kKinds; ++k)
      for (int s = 0; s < (int)slot_ticket[k].size(); ++s)
        if (slot_ticket[k][s] && reqs[slot_ticket[k][s]].slot != s) slot_ticket[k][s] = 0;
  }
}

}  // namespace dualip

struct dualip_server {
  dualip::Server s;
};

using namespace dualip;

namespace {

void fill_info(const Request& r, dualip_request_info* info) {
  std::memset(info, 0, sizeof(*info));
  info->state = r.state;
  info->status = r.status;
  info->result = r.result;
  info->t_submit = r.t_submit;
  info->t_admit = r.t_admit;
  info->t_done = r.t_done;
  info->footprint_bytes = r.footprint;
  info->num_dests = r.desc.num_dests;
}

}  // namespace

extern "C" {

dualip_status dualip_server_create(const dualip_server_opts* opts, dualip_server** out) {
  if (!out || !opts) return fail(DUALIP_EINVAL, "NULL argument");
  *out = nullptr;
  if (opts->hbm_budget_bytes <= 0 || opts->max_slots < 1 || opts->max_slots > 1024 ||
      opts->check_every < 1)
    return fail(DUALIP_EINVAL, "need a positive budget, 1..1024 slots and check_every >= 1");
  dualip_server* h = new dualip_server();
  Server& S = h->s;
  S.o = *opts;
  cudaError_t e;
  if ((e = cudaGetDevice(&S.device)) ||
      (e = cudaDeviceGetAttribute(&S.num_sms, cudaDevAttrMultiProcessorCount, S.device)) ||
      (e = cudaStreamCreateWithFlags(&S.admit_stream, cudaStreamNonBlocking))) {
    delete h;
    return cuda_fail(e, "starting the server");
  }
  S.t0 = std::chrono::steady_clock::now();
  S.admitter = std::thread([&S] { S.admit_loop(); });
  S.scheduler = std::thread([&S] { S.schedule_loop(); });
  *out = h;
  return DUALIP_OK;
}

dualip_status dualip_server_submit(dualip_server* h, const dualip_problem_desc* desc,
                                   const dualip_solve_opts* opts, int64_t* ticket) {
  if (!h || !desc || !ticket) return fail(DUALIP_EINVAL, "NULL argument");
  if (desc->storage != DUALIP_EDGE_F32 && desc->storage != DUALIP_EDGE_BF16)
    return fail(DUALIP_EINVAL, "unknown storage");
  if (desc->num_sources < 0 || desc->num_edges < 0 || desc->num_dests < 1)
    return fail(DUALIP_EINVAL, "need I >= 0, E >= 0, J >= 1");
  dualip_solve_opts o;
  if (opts) {
    o = *opts;
  } else {
    dualip_solve_opts_default(&o);
  }
  if (!(o.gamma0 > 0) || !(o.gamma_final > 0) || !std::isfinite(o.gamma0) ||
      o.gamma_final > o.gamma0 || o.gamma_final < 1e-30 || o.max_iters < 1 ||
      !(o.max_step > 0) || !(o.init_step > 0))
    return fail(DUALIP_EINVAL, "invalid solve options");
  if (desc->projection != DUALIP_PROJ_SIMPLEX || desc->num_families > 1)
    return fail(DUALIP_EINVAL,
                "the serving form takes simplex problems with one constraint family only");
  Server& S = h->s;
  std::lock_guard<std::mutex> lk(S.mu);
  const int64_t t = S.next_ticket++;
  Request& r = S.reqs[t];
  r.desc = *desc;
  r.opts = o;
  r.kind = (desc->storage == DUALIP_EDGE_BF16 ? 2 : 0) + (desc->primal_scaling ? 1 : 0);
  r.footprint = resident_bytes(*desc);
  r.transient = transient_bytes(*desc);
  r.t_submit = S.now();
  S.queue.push_back(t);
  S.cv.notify_all();
  *ticket = t;
  return DUALIP_OK;
}

dualip_status dualip_server_poll(dualip_server* h, int64_t ticket, dualip_request_info* info,
                                 float* lambda_out) {
  if (!h || !info) return fail(DUALIP_EINVAL, "NULL argument");
  Server& S = h->s;
  std::lock_guard<std::mutex> lk(S.mu);
  auto it = S.reqs.find(ticket);
  if (it == S.reqs.end()) return fail(DUALIP_EINVAL, "unknown ticket");
  const Request& r = it->second;
  fill_info(r, info);
  if (r.state == DUALIP_REQ_DONE && lambda_out && !r.lam.empty())
    std::memcpy(lambda_out, r.lam.data(), sizeof(float) * r.lam.size());
  if (r.state == DUALIP_REQ_FAILED) set_error(r.error);
  return DUALIP_OK;
}

dualip_status dualip_server_wait(dualip_server* h, int64_t ticket, double timeout_s,
                                 dualip_request_info* info, float* lambda_out) {
  if (!h || !info) return fail(DUALIP_EINVAL, "NULL argument");
  Server& S = h->s;
  {
    std::unique_lock<std::mutex> lk(S.mu);
    auto it = S.reqs.find(ticket);
    if (it == S.reqs.end()) return fail(DUALIP_EINVAL, "unknown ticket");
    const auto until =
        std::chrono::steady_clock::now() + std::chrono::duration<double>(std::max(0.0, timeout_s));
    const Request& r = it->second;
    while (r.state != DUALIP_REQ_DONE && r.state != DUALIP_REQ_FAILED) {
      if (S.cv.wait_until(lk, until) == std::cv_status::timeout &&
          r.state != DUALIP_REQ_DONE && r.state != DUALIP_REQ_FAILED)
        break;
    }
  }
  const dualip_status st = dualip_server_poll(h, ticket, info, lambda_out);
  if (st) return st;
  if (info->state != DUALIP_REQ_DONE && info->state != DUALIP_REQ_FAILED)
    return fail(DUALIP_ETIMEOUT, "the request did not finish in time");
  return DUALIP_OK;
}

dualip_status dualip_server_get_stats(dualip_server* h, dualip_server_stats* st) {
  if (!h || !st) return fail(DUALIP_EINVAL, "NULL argument");
  Server& S = h->s;
  std::lock_guard<std::mutex> lk(S.mu);
  std::memset(st, 0, sizeof(*st));
  for (const auto& kv : S.reqs) {
    ++st->submitted;
    if (kv.second.state == DUALIP_REQ_QUEUED) ++st->queued;
    if (kv.second.state == DUALIP_REQ_RUNNING) ++st->running;
  }
  st->done = S.n_done;
  st->failed = S.n_failed;
  st->resident_bytes = S.resident;
  st->peak_resident_bytes = S.peak;
  st->chunks = S.chunks;
  st->slot_iterations = S.slot_iters;
  st->busy_seconds = S.busy;
  return DUALIP_OK;
}

dualip_status dualip_server_cancel(dualip_server* h, int64_t ticket) {
  if (!h) return fail(DUALIP_EINVAL, "server is NULL");
  Server& S = h->s;
  std::lock_guard<std::mutex> lk(S.mu);
  auto it = S.reqs.find(ticket);
  if (it == S.reqs.end()) return fail(DUALIP_EINVAL, "unknown ticket");
  Request& r = it->second;
  if (r.state == DUALIP_REQ_QUEUED && !r.building) {
    for (auto q = S.queue.begin(); q != S.queue.end(); ++q)
      if (*q == ticket) {
        S.queue.erase(q);
        break;
      }
    r.state = DUALIP_REQ_FAILED;
    r.status = DUALIP_ECANCELED;
    r.error = "cancelled";
    r.t_done = S.now();
    ++S.n_failed;
    S.cv.notify_all();
  } else if (r.state == DUALIP_REQ_QUEUED || r.state == DUALIP_REQ_RUNNING) {
    r.cancel = true;  // being built or resident: leaves at the next chunk boundary
  }
  return DUALIP_OK;
}

void dualip_server_destroy(dualip_server* h) {
  if (!h) return;
  Server& S = h->s;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    S.stop = true;
    S.cv.notify_all();
  }
  if (S.admitter.joinable()) S.admitter.join();
  if (S.scheduler.joinable()) S.scheduler.join();
  for (int k = 0; k < kKinds; ++k)
    if (S.batch_ok[k]) {
      for (int s = 0; s < S.batch[k].n; ++s)
        if (S.batch[k].prob[s]) batch_detach(S.batch[k], s);
      batch_free(S.batch[k]);
    }
  for (auto& kv : S.reqs)
    if (kv.second.h) dualip_destroy(kv.second.h);
  if (S.admit_stream) cudaStreamDestroy(S.admit_stream);
  delete h;
}

}  // extern "C"
