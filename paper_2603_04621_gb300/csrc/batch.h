// Host-side batch of problems: the slot table, the joint tile and row-chunk
// lists of the active slots, and the batched solver's state.  Used by the
// batch entry points and by the server.
#pragma once

#include <algorithm>
#include <vector>

#include "internal.h"

namespace dualip {

constexpr int kChunkRows = 2048;  // rows of a J-length chunk

struct Batch {
  int n = 0;
  int storage = DUALIP_EDGE_F32, weighted = 0;
  int num_sms = 0;
  std::vector<Problem*> prob;     // per slot
  std::vector<SlotDesc> desc;     // host copy of the slot table
  std::vector<char> active;       // slots in the joint lists
  int64_t tile_edges = kTileEdges, tile_sources = kTileSources;
  int lean80 = 0;  // lean-window policy of the pass (the autotuner may change it)
  bool has_big = false;  // an active tile holds a source larger than a stage (block class)
  bool lean_auto = false;  // pick lean80 from the degrees of the active slots
  std::vector<int64_t> over76;  // per slot: sources with more than 76 edges
  // per-slot tile lists for the current tile shape (host), and their joint
  // concatenation for the active slots (device)
  std::vector<std::vector<JointTile>> tiles;
  std::vector<JointTile> jt_host;
  std::vector<RowChunk> rc_host;
  std::vector<int32_t> act_host;
  std::vector<int2> crange_host;
  int64_t ntiles = 0;
  int nchunks = 0;
  bool lists_ok = false;
  // device
  SlotDesc* d_slots = nullptr;
  float* d_gamma_f = nullptr;
  double* d_gamma_d = nullptr;
  long long* d_slot_part = nullptr;  // [2 n] fixed-point (sum c x, sum w x^2) per slot
  double* d_eval = nullptr;
  SlotSolve* d_ss = nullptr;
  int32_t* d_act = nullptr;
  int2* d_crange = nullptr;
  unsigned* d_tickets = nullptr;
  DeviceStatus* d_status = nullptr;
  JointTile* d_jt = nullptr;
  size_t jt_cap = 0;
  RowChunk* d_rc = nullptr;
  float4* d_cpart = nullptr;
  size_t rc_cap = 0;
  RowChunk* d_rc2 = nullptr;  // chunks of one slot (attach, lambda output)
  size_t rc2_cap = 0;
  int nrc2 = 0;
  // pinned staging
  double* h_gamma = nullptr;  // n doubles then n floats
  double* h_eval = nullptr;   // 5 n
  SlotSolve* h_ss = nullptr;  // n
  // solver vectors (6 per slot, renumbered order), allocated by the solver
  std::vector<float*> vecs;
  int row_normalize = -1;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;        // stream ordering
  cudaEvent_t ev_stage = nullptr;  // the gamma staging copies have been read
  cudaEvent_t ev_use = nullptr;    // the last queued use of the joint lists
  cudaGraphExec_t graph = nullptr;
  int graph_len = 0;
  int grid = 0;
  // kernel timing of API evaluations (4 events each)
  std::vector<cudaEvent_t> prof_ev;
  int prof_used = 0, prof_max = 0;
};


template <class T>
cudaError_t grow(T** p, size_t& cap, size_t need) {
  if (need <= cap && *p) return cudaSuccess;
  if (*p) cudaFree(*p);
  *p = nullptr;
  cap = 0;
  const size_t n = std::max<size_t>(need, 1) * 5 / 4 + 16;
  cudaError_t e = cudaMalloc(p, sizeof(T) * n);
  if (e == cudaSuccess) cap = n;
  return e;
}

void batch_free(Batch& B);
SlotDesc slot_desc(Problem& P, int64_t joff);
SlotSolve slot_solve_init(const dualip_solve_opts& o, double bnorm);
// per-slot tiles for the current tile shape (empty slots get none)
cudaError_t build_slot_tiles(Batch& B);
// joint lists of the active slots (waits for queued users of the old lists)
cudaError_t rebuild_lists(Batch& B);
cudaError_t upload_slots(Batch& B);
// one evaluation of every active slot: API (lam / grad joint caller vectors)
// or solver mode
cudaError_t enqueue_batch_eval(Batch& B, const float* lam, float* grad, int solver,
                               cudaStream_t s);
// n solver iterations of every active slot on B.stream (optionally a graph)
cudaError_t run_batch_chunk(Batch& B, int n, bool use_graph);
dualip_status batch_status(Batch& B);

// ---- dynamic slots (the server) ----
// device tables for `capacity` slots, no problem attached
cudaError_t batch_alloc(Batch& B, int capacity, int storage, int weighted, int num_sms);
// attach P to a free slot with the ascent's options; lambda starts at 0.
// Returns the slot, or -1 if none is free (err set on a CUDA failure).
int batch_attach(Batch& B, Problem* P, const dualip_solve_opts& o, cudaError_t* err);
// the slot's last evaluated dual point, caller's numbering, into lam_out [J]
cudaError_t batch_write_lambda(Batch& B, int slot, float* lam_out);
// frees the slot's solver vectors; the problem itself stays with the caller
void batch_detach(Batch& B, int slot);
// copies the solver states and scalars of every slot to B.h_ss / B.h_eval
cudaError_t batch_read_state(Batch& B);

}  // namespace dualip
