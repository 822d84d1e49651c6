// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/dualip.h"
#include "plan.h"
#include <nvtx3/nvToolsExt.h>

namespace dualip {

// ---- pass geometry --------------------------------------------------------
// A tile is a run of whole sources whose edges fit one shared-memory stage.
#ifndef DUALIP_TILE_EDGES
#define DUALIP_TILE_EDGES 3200
#endif
#ifndef DUALIP_STAGES
#define DUALIP_STAGES 4
#endif
#ifndef DUALIP_CONSUMER_WARPS
#define DUALIP_CONSUMER_WARPS 18
#endif
#ifndef DUALIP_PRIV_DESTS
#define DUALIP_PRIV_DESTS 1024
#endif
constexpr int kTileEdges = DUALIP_TILE_EDGES;       // edge capacity of a stage
#ifndef DUALIP_TILE_EDGES_BF16
#define DUALIP_TILE_EDGES_BF16 4800
#endif
// edge capacity of a stage with BF16 (c, a): 8 bytes per edge instead of 12
constexpr int kTileEdgesBF16 = DUALIP_TILE_EDGES_BF16;
constexpr int tile_edges_for(int storage) {
  return storage == DUALIP_EDGE_BF16 ? kTileEdgesBF16 : kTileEdges;
}
#ifndef DUALIP_TILE_SOURCES
#define DUALIP_TILE_SOURCES 256
#endif
constexpr int kTileSources = DUALIP_TILE_SOURCES;   // source capacity of a stage
constexpr int kStages = DUALIP_STAGES;               // depth of the staging ring
constexpr int kConsumerWarps = DUALIP_CONSUMER_WARPS;  // warps that project sources
// Tiles per grab of the single-problem pass's dynamic schedule (<= 31).
#ifndef DUALIP_GRAB
#define DUALIP_GRAB 4
#endif
// Programmatic dependent launch of the pass after the prologue and of the
// epilogue after the pass (1), or plain stream order (0).
#ifndef DUALIP_PDL
#define DUALIP_PDL 1
#endif
#ifndef DUALIP_SMEM_RED64
#define DUALIP_SMEM_RED64 0
#endif
constexpr bool kSmemRed64 = DUALIP_SMEM_RED64 != 0;  // shared bins: one 64-bit reduction
#ifndef DUALIP_WAIT_HINT_NS
#define DUALIP_WAIT_HINT_NS 0
#endif
constexpr unsigned kWaitHintNs = DUALIP_WAIT_HINT_NS;  // mbarrier suspend hint (0: none)
// Unweighted sources that the lane groups leave (unsaturated, near-ties) and
// whose span fits a warp's registers take the candidate path (1) instead of
// the multi-pass path (0).
#ifndef DUALIP_WARP_CAND
#define DUALIP_WARP_CAND 1
#endif
constexpr bool kWarpCand = DUALIP_WARP_CAND != 0;
constexpr int kCandRounds = 16;  // Michelot rounds before the multi-pass path takes over
// A source larger than a stage is projected by all consumer warps of the CTA
// (1) or by one warp (0).
#ifndef DUALIP_BLOCK_CLASS
#define DUALIP_BLOCK_CLASS 1
#endif
constexpr bool kBlockClass = DUALIP_BLOCK_CLASS != 0;
constexpr int kBlockUnroll = 4;  // edges in flight per consumer thread in the block class
constexpr int kBlockCand = 4;    // candidate edges a consumer thread keeps in registers
// Sources of at least DUALIP_MB_STAGES stages' edges are projected by the
// multi-block class (the hub kernel, over the whole grid, before the pass,
// which skips them); 0 leaves them to the block class.
#ifndef DUALIP_MB_STAGES
#define DUALIP_MB_STAGES 16
#endif
constexpr int kMultiBlockStages = DUALIP_MB_STAGES;
constexpr int kHubChunk = 4096;    // edges of a hub source per chunk (one CTA, one read)
constexpr int kHubThreads = 512;   // threads of a hub-kernel CTA
// Problems with at most 16 edges per source on average take the pass variant
// with 32-source batches and one-lane groups (1), or the standard one (0).
#ifndef DUALIP_TINY_BATCHES
#define DUALIP_TINY_BATCHES 1
#endif
constexpr bool kTinyBatches = DUALIP_TINY_BATCHES != 0;
constexpr int kThreads = 32 * (kConsumerWarps + 1);  // + one producer warp
constexpr int kMaxCachedDests = 10240; // hot destinations whose mu lives in smem
constexpr int kMaxPrivDests = DUALIP_PRIV_DESTS;  // hot destinations accumulated in smem
constexpr int kStageSlack = 8;                      // 16-byte alignment slack of a stage
constexpr int kDstPad = 512;                         // widest group window (32 lanes x 16)
constexpr int kStageOffSlots = kTileSources + 8;  // a tile's offsets, from a 16-byte boundary

// device error word bits
constexpr int kErrTimeout = 1;
constexpr int kErrBounds = 2;

struct alignas(128) DeviceStatus {
  int err;        // OR of kErr* bits
  int where;      // first wait site that timed out
  unsigned ticket;  // last-block counter of the epilogue (reset by the last block)
  unsigned done;    // CTAs of the pass that have finished (reset by the last one)
  int abort_req;    // set by the host: device waits give up at once (fault injection)
  int pad;
  // the dynamic schedule's counter takes every CTA's atomics: a line of its own
  alignas(128) unsigned long long tile_next;
};

// A source of the multi-block class: its stored edges [e0, e0 + deg), its
// chunks [c0, c0 + nch) of kHubChunk edges, its candidate list at cand0.
struct HubDesc {
  int64_t e0;
  int64_t cand0;
  int32_t deg, c0, nch, pad;
};
// Statistics of one warp's unit of a hub-source chunk: the saturation sum
// sum_{r > 0} alpha r, r_max and max (r - gamma w).
struct alignas(16) HubUnitStat {
  double s0;
  float rmax, mb;
};

// Kernel parameters of the J-length epilogue.
struct EpiParams {
  int32_t J;
  const int32_t* orig_of;  // renumbered -> caller's destination id
  const float* b_r;        // [J] budgets, renumbered
  const float* mu_r;       // [J] renumbered dual point of the pass
  const float* D;          // [J] optional row scale in caller numbering (solver)
  unsigned long long* y;   // [J] fixed-point A x, reset to 0 after reading
  float sy;                // 2^-exp_y (exact in FP32: |exp_y| <= 100)
  float* grad;             // [J] caller numbering: D (A x - b) (D = 1 if null)
  const longlong2* part;   // per-CTA fixed-point partials of the pass (see PassParams)
  int ec, ew;              // their exponents: sum c x = part.x 2^-ec, sum w x^2 = part.y 2^-ew
  int npart;
  float4* epi_part;        // [gridDim.x] per-block (lambda^T g, ||g_+||^2) as FP32 pairs
  const float* gamma_dev;
  double gamma;
  double* eval_out;        // [5] dualip_eval order
  DeviceStatus* status;
};

// ------------------------------------------------------------ batches ----
// Several problems evaluated by one launch of the pass.  Every problem keeps
// its own packed edges, renumbering, fixed-point scale and J-length arrays;
// it occupies a slot of a device table.  The pass walks a joint list of tiles
// (each tile belongs to one slot; tiles of a slot are contiguous), and the
// J-length kernels walk a joint list of row chunks.

// One tile of a batched pass: a run of whole sources of one slot's problem.
struct JointTile {
  int64_t s0, s1;  // sources [s0, s1) of the slot's problem
  int64_t e0, e1;  // edges [e0, e1)
  int32_t slot;
  int32_t pad;
};
// Rows [r0, r1) of one slot's problem, for the batched J-length kernels.
struct RowChunk {
  int32_t slot;
  int32_t r0, r1;
  int32_t pad;
};
// Per-slot arrays and scalars (device table).
struct SlotDesc {
  // the problem's own device arrays
  const uint32_t* off;        // low 32 bits of the stored source offsets
  const int32_t* dst;
  const float2* ca2;
  const uint32_t* ca;
  float* mu_r;                // [J] renumbered dual point of the pass
  unsigned long long* y;      // [J] fixed-point A x (reset by the epilogue)
  const int32_t* orig_of;     // [J] renumbered -> caller's id
  const float* b_r;           // [J] budgets, renumbered
  int32_t J, h_mu, h_y, pad;
  float sy, inv_sy;           // 2^exp_y, 2^-exp_y
  int32_t ec, ew;             // fixed-point exponents of the objective partials
  int64_t joff;               // offset of this problem in joint caller vectors
  // solver vectors in the caller's numbering (null outside the solver)
  float *lam, *yv, *yp, *G, *Gp, *D;
};
// Solver scalars of one slot (the ascent of the single-problem solver, per
// problem; every field is written on the device except the options).
struct SlotSolve {
  double gamma0, gamma_final, max_step, init_step, bnorm;
  double t, eta, beta;
  double gap_rel, infeas_rel, last_gamma;
  double sdy, sdg;            // ||y_k - y_{k-1}||^2, ||G_k - G_{k-1}||^2
  double g_prev;              // dual objective of the previous evaluation (same gamma)
  int32_t k, halve_every, restart, restart_dec;
};

// Kernel parameters of one pass (one dual evaluation).
struct PassParams {
  // edges
  // low 32 bits of the stored source offsets [I+1 (+ padding)]: a tile spans
  // fewer than 2^32 edges, so differences within it are exact modulo 2^32
  const uint32_t* off;
  const int32_t* dst;     // [E_pad] renumbered destinations
  const float2* ca2;      // [E_pad] (c, a) pairs (f32 storage)
  const uint32_t* ca;     // [E_pad] packed bf16 (c | a << 16) (bf16 storage)
  const int64_t* tiles;   // [ntiles+1] first source of each tile
  const int64_t* tile_e;  // [ntiles+1] first edge of each tile (= off[tiles[t]])
  int64_t ntiles;
  int64_t I;
  int32_t J;
  int32_t h_mu;           // destinations [0, h_mu) have their mu cached in smem
  int32_t h_y;            // destinations [0, h_y) accumulate in smem
  // dual point, renumbered: mu_r[jr]
  const float* mu_r;
  const float* gamma_dev;  // if non-null, gamma is read here (solver)
  float gamma;
  // outputs / scratch
  unsigned long long* y;  // [J] A x in fixed point (two's complement, scale 2^exp_y)
  int ey;                 // fixed-point exponent of A x (scale 2^ey)
  int ec, ew;             // fixed-point exponents of sum c x and sum w x^2
  longlong2* part;        // [gridDim.x] per-CTA (sum c x, sum w x^2) in fixed point
                          // (scales 2^ec, 2^ew): exact sums of once-rounded terms, so
                          // they do not depend on which CTA took which source
  float* x_out;           // [E] optional primal output (edge order)
  DeviceStatus* status;
  // batched pass: tiles from jt, per-slot arrays from slots, per-slot gamma,
  // per-slot FP64 partials (sum c x, sum w x^2) by atomics
  const JointTile* jt;
  const SlotDesc* slots;
  const float* gamma_of;
  long long* slot_part;   // per-slot fixed-point (sum c x, sum w x^2) (slot scales)
  int lean80;  // 4-lane lean groups may take spans up to 80 (else 64)
  int grab;    // tiles per grab of the single-problem schedule (1..31)
  int64_t mb_min;  // a tile of at least this many edges is a hub source (skipped)
};

struct Problem {
  int64_t I = 0, E = 0;
  int32_t J = 0;
  int storage = DUALIP_EDGE_F32;
  int weighted = 0;
  int box = 0;  // projection onto the unit box [0, 1]^E instead of per-source simplices
  int tiny = 0;  // small mean degree: the pass claims 32 sources at a time (1-lane groups)
  int has_big = 0;  // some source is larger than a stage: tiles are grabbed one at a time
  // multi-block class: sources of at least mb_min edges (INT64_MAX: none)
  int64_t mb_min = INT64_MAX;
  int nhub = 0;
  int64_t nchunks = 0;
  HubDesc* hubs = nullptr;           // [nhub]
  int32_t* chunk_hub = nullptr;      // [nchunks] hub of each chunk
  HubUnitStat* hub_stat = nullptr;   // [nchunks * units per chunk]
  float4* hub_cand = nullptr;        // [sum of hub degrees] candidate lists
  unsigned* hub_cnt = nullptr;       // [2 nhub] candidates so far, chunks done
  // A hub source's edges are stored in order of destination (renumbered id),
  // so that the mu gathers of a warp read neighbouring ids.  hub_perm[cand0 +
  // k] is the place, within the source's segment, that its stored edge k had
  // in the caller's order; hub_host and hub_caller0 (the segment's start in
  // the caller's edge order) serve dualip_get_primal.
  uint32_t* hub_perm = nullptr;      // [sum of hub degrees]
  std::vector<HubDesc> hub_host;
  std::vector<int64_t> hub_caller0;
  // constraint families (Definition 1): with m > 1, J counts rows (m Jd, row
  // k Jd + j), the edges keep the caller's order and destination ids, and c,
  // a (family-major, a[k E + e]) live in cm, am; the pass is multi.cu's
  int m = 1;
  int32_t Jd = 0;
  float* cm = nullptr;
  float* am = nullptr;
  int64_t ntiles = 0;
  int h_mu = 0, h_y = 0;
  int num_sms = 0, grid = 0;
  int device = 0;
  // device buffers (owned)
  int64_t* off = nullptr;     // stored source offsets (create, the primal's source map)
  uint32_t* off32 = nullptr;  // their low 32 bits, padded (the pass streams these)
  int32_t* dst = nullptr;
  float2* ca2 = nullptr;  // (c, a) pairs, FP32 storage
  uint32_t* ca = nullptr;
  int64_t* tiles = nullptr;
  int64_t* tile_e = nullptr;
  float* b_r = nullptr;
  int32_t* orig_of = nullptr;
  int32_t* new_of = nullptr;
  float* mu_r = nullptr;
  unsigned long long* y = nullptr;  // fixed-point accumulator of A x
  int exp_y = 0;                    // fixed-point scale of A x (power of two)
  // fixed-point exponents of the objective partials: sum_e c_e x_e and
  // sum_e w_e x_e^2 are bounded by I max|c| and I max w (sum_e x_e <= 1 per
  // source), kept below 2^61
  int exp_c = 0, exp_w = 0;
  longlong2* part = nullptr;  // [grid + nhub] fixed-point partials of the pass and hubs
  int epi_blocks = 0;
  float4* epi_part = nullptr;
  double* eval_dev = nullptr;
  float* lam_stage = nullptr;   // [J] staging for host-buffer calls
  float* grad_stage = nullptr;  // [J]
  DeviceStatus* status = nullptr;
  double* eval_host = nullptr;  // pinned [8]
  cudaStream_t last_stream = nullptr;
  double bnorm = 0.0;           // ||b||_2
  void* solve_ctx = nullptr;    // solver state, created by the first dualip_solve
  std::vector<cudaEvent_t> prof_ev;  // 4 per recorded evaluation
  std::vector<int64_t> off_host;     // source offsets as stored (tiling of batched passes)
  // degree order (empty: sources are stored in the caller's order): stored
  // source i is the caller's source src_of_host[i]; orig_off_host holds the
  // caller's offsets
  std::vector<int64_t> src_of_host, orig_off_host;
  int prof_max = 0, prof_used = 0;
  std::vector<void*> allocations;
};

// pass.cu
size_t pass_smem_bytes(int storage);
cudaError_t configure_pass_kernels();
cudaError_t launch_prep(const Problem& P, const float* lambda, const float* D, cudaStream_t s);
cudaError_t launch_pass(const Problem& P, const float* gamma_dev, float gamma, float* x_out,
                        cudaStream_t s);
// solve.cu: D_j = (sum_{e->j} a_e^2 / w_e)^(-1/2) (1 for an empty row), or 1
// everywhere without row normalisation, in renumbered order.  Synchronises s.
cudaError_t compute_row_scale(const Problem& P, int row_normalize, float* D, cudaStream_t s);
#ifdef __CUDACC__
// Programmatic dependent launch.  wait: the preceding kernel of the stream
// has finished and its writes are visible (immediate without the launch
// attribute).  trigger: the next kernel may start launching.  Every kernel of
// a chain triggers only after its own wait, so a kernel that starts early may
// rely on everything launched two kernels before it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
#endif

// Launch with programmatic stream serialisation: the kernel may start before
// the preceding kernel of the stream has finished and must call
// griddepcontrol.wait before it reads what that kernel writes.
template <typename... K, typename... A>
cudaError_t launch_pdl(void (*k)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = DUALIP_PDL;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<A&&>(args)...);
}

// Batched pass over the joint tile list (ntiles entries) with the given grid.
cudaError_t launch_pass_batch(int storage, int weighted, const JointTile* jt, int64_t ntiles,
                              const SlotDesc* slots, const float* gamma_of, long long* slot_part,
                              DeviceStatus* status, int grid, int lean80, bool big, cudaStream_t s);
cudaError_t launch_epilogue(const Problem& P, const float* D, float* grad, const float* gamma_dev,
                            double gamma, double* eval_out, cudaStream_t s, bool identity = false);
cudaError_t launch_renumber(const int32_t* dst_in, int32_t* dst_out, const int32_t* new_of,
                            int64_t E, int32_t J, DeviceStatus* st, cudaStream_t s);
cudaError_t launch_histogram(const int32_t* dst, int64_t E, int32_t J, unsigned* counts,
                             DeviceStatus* st, cudaStream_t s);
cudaError_t launch_pack_f32(const float* c, const float* a, float2* ca2, int64_t E,
                            cudaStream_t s);
cudaError_t launch_pack_bf16(const float* c, const float* a, uint32_t* ca, int64_t E,
                             cudaStream_t s);
cudaError_t launch_check_finite(const float* v, int64_t n, DeviceStatus* st, cudaStream_t s);
// Degree order: stored source i is the caller's source src_of[i]; its edges
// sit at off[i] .. off[i+1]-1 in storage and start at orig_off[src_of[i]] in
// the caller's arrays (all three are device arrays).
struct SegMap {
  const int64_t* off;
  const int64_t* src_of;
  const int64_t* orig_off;
  int64_t I;
};
cudaError_t launch_renumber_seg(const int32_t* dst_in, int32_t* dst_out, const int32_t* new_of,
                                const SegMap& m, int32_t J, DeviceStatus* st, cudaStream_t s);
cudaError_t launch_pack_seg(const float* c, const float* a, int storage, void* out,
                            const SegMap& m, cudaStream_t s);
cudaError_t launch_unpermute_seg(const float* in, float* out, const SegMap& m, cudaStream_t s);
// out[k] = in[perm[k]] (elements of 4 or 8 bytes) and out[perm[k]] = in[k],
// for k < n
cudaError_t launch_gather_perm(const void* in, void* out, const uint32_t* perm, int64_t n,
                               int elem_bytes, cudaStream_t s);
cudaError_t launch_scatter_perm(const float* in, float* out, const uint32_t* perm, int64_t n,
                                cudaStream_t s);
cudaError_t launch_absmax(const float* v, int64_t n, unsigned* out, cudaStream_t s);

// solve.cu
void solve_ctx_free(Problem& P);

// multi.cu: problems with several constraint families (m > 1)
dualip_status create_multi(const dualip_problem_desc* d, void* stream, dualip_problem** out);
cudaError_t launch_pass_multi(const Problem& P, const float* gamma_dev, float gamma, float* x_out,
                              cudaStream_t s);
// acc[r] += a_{k,e}^2 / w_e over the edges of row r = k Jd + j (row norms)
cudaError_t launch_row_norm_multi(const Problem& P, double* acc, cudaStream_t s);

// api.cu helpers (the tiling and the degree order are in plan.h)
cudaStream_t as_stream(void* s);
// NVTX range for the lifetime of a scope (shown by profilers; nothing
// happens without one attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

void set_error(const std::string& msg);
dualip_status fail(dualip_status st, const std::string& msg);
dualip_status cuda_fail(cudaError_t e, const char* what);

}  // namespace dualip

struct dualip_problem {
  dualip::Problem p;
};
