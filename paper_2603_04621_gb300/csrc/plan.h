// Host-side planning of a problem's stored layout (plain C++, no CUDA): the
// degree order of the sources and the tiling of the source-major edge list.
// dualip_create and the batched form use these; a CPU test compiles this
// header on its own and checks the invariants stated below.
#pragma once

#include <algorithm>
#include <cstdint>
#include <numeric>
#include <vector>

namespace dualip {

// Greedy tiling: consecutive whole sources while the edge count stays within
// max_edges and the source count within max_sources; a source larger than
// max_edges forms a tile of its own (projected from global memory).  On
// return tiles[t] .. tiles[t+1]-1 are the sources of tile t and tile_e[t] its
// first edge; tiles.back() = I and tile_e.back() = E.
inline void build_tiles(const std::vector<int64_t>& off, std::vector<int64_t>& tiles,
                        std::vector<int64_t>& tile_e, int64_t max_edges, int64_t max_sources) {
  const int64_t I = (int64_t)off.size() - 1;
  tiles.clear();
  tile_e.clear();
  int64_t s = 0;
  while (s < I) {
    tiles.push_back(s);
    tile_e.push_back(off[s]);
    int64_t e = 0, n = 0;
    if (off[s + 1] - off[s] > max_edges) {
      ++s;
      continue;
    }
    while (s < I && n < max_sources && e + (off[s + 1] - off[s]) <= max_edges) {
      e += off[s + 1] - off[s];
      ++n;
      ++s;
    }
  }
  tiles.push_back(I);
  tile_e.push_back(off[I]);
}

// Degree order: src_of[i] is the caller's source stored at position i, by
// increasing degree with ties in the caller's order; off_st are the stored
// offsets (off_st[i+1] - off_st[i] = the degree of src_of[i]).  A counting
// sort by degree (stable, O(I + max degree)) gives the order; when the
// largest degree exceeds 4 I + 1024 a comparison sort gives the same one.
inline void degree_order(const std::vector<int64_t>& off, std::vector<int64_t>& src_of,
                         std::vector<int64_t>& off_st) {
  const int64_t I = (int64_t)off.size() - 1;
  src_of.resize((size_t)I);
  int64_t dmax = 0;
  for (int64_t i = 0; i < I; ++i) dmax = std::max(dmax, off[i + 1] - off[i]);
  if (dmax <= 4 * I + 1024) {
    std::vector<int64_t> start((size_t)dmax + 2, 0);  // start[d + 1]: sources of degree d
    for (int64_t i = 0; i < I; ++i) ++start[(size_t)(off[i + 1] - off[i]) + 1];
    for (int64_t d = 0; d <= dmax; ++d) start[(size_t)d + 1] += start[(size_t)d];
    for (int64_t i = 0; i < I; ++i) src_of[(size_t)start[(size_t)(off[i + 1] - off[i])]++] = i;
  } else {
    std::iota(src_of.begin(), src_of.end(), int64_t(0));
    std::stable_sort(src_of.begin(), src_of.end(), [&](int64_t x, int64_t y) {
      return off[x + 1] - off[x] < off[y + 1] - off[y];
    });
  }
  off_st.resize((size_t)I + 1);
  off_st[0] = 0;
  for (int64_t i = 0; i < I; ++i)
    off_st[i + 1] = off_st[i] + (off[src_of[i] + 1] - off[src_of[i]]);
}

// Element slots the lane-group projection of the pass sweeps for a stored
// order (its offsets off), tiled greedily with max_edges / max_sources: each
// tile's sources go in batches of eight; a source's span is (first edge mod 4)
// + degree; per batch, one round per 32/G sources of each group width G, a
// round sweeping 32 lanes x 4 S slots: G = 4 for spans up to 64 (S = 4), or up
// to 80 (S = 5 when some span exceeds 64) when lean80 is set and no span of the
// batch lies in (80, 128]; G = 8, 16, 32 for spans up to 128, 256, 512 (S = 4).
// A source with a longer span is counted as four passes over it.  Used to pick
// the stored order: the kernel's cost per edge follows these slots.
inline double lean_slots(const std::vector<int64_t>& off, int64_t max_edges, int64_t max_sources,
                         bool lean80) {
  std::vector<int64_t> tiles, tile_e;
  build_tiles(off, tiles, tile_e, max_edges, max_sources);
  double slots = 0.0;
  for (size_t t = 0; t + 1 < tiles.size(); ++t) {
    for (int64_t b = tiles[t]; b < tiles[t + 1]; b += 8) {
      const int64_t be = std::min<int64_t>(b + 8, tiles[t + 1]);
      int64_t sp[8];
      bool mid = false, over64 = false;
      for (int64_t q = b; q < be; ++q) {
        const int64_t d = off[q + 1] - off[q];
        sp[q - b] = d > 0 ? (off[q] & 3) + d : 0;
        mid = mid || (sp[q - b] > 80 && sp[q - b] <= 128);
      }
      const int64_t span4 = (!lean80 || mid) ? 64 : 80;
      int64_t n4 = 0, n8 = 0, n16 = 0, n32 = 0;
      for (int64_t q = 0; q < be - b; ++q) {
        const int64_t s = sp[q];
        if (s == 0) continue;
        if (s <= span4) {
          ++n4;
          over64 = over64 || s > 64;
        } else if (s <= 128) {
          ++n8;
        } else if (s <= 256) {
          ++n16;
        } else if (s <= 512) {
          ++n32;
        } else {
          slots += 4.0 * (double)s;
        }
      }
      slots += (double)((n4 + 7) / 8) * 128.0 * (over64 ? 5 : 4);
      slots += (double)((n8 + 3) / 4 + (n16 + 1) / 2 + n32) * 512.0;
    }
  }
  return slots;
}

// The stored order of a problem: degree order (src_of, off_st filled) when the
// cost model above gives it at least 2% fewer element slots than the caller's
// order, for tiles of max_edges / max_sources; else the caller's order
// (src_of, off_st left empty).  DUALIP_DEGREE_ORDER = 0 or 1 forces never or
// always (for measurements).
#ifndef DUALIP_DEGREE_ORDER
#define DUALIP_DEGREE_ORDER -1
#endif
inline bool choose_degree_order(const std::vector<int64_t>& off, int64_t max_edges,
                                int64_t max_sources, std::vector<int64_t>& src_of,
                                std::vector<int64_t>& off_st) {
  src_of.clear();
  off_st.clear();
  const int64_t I = (int64_t)off.size() - 1;
  if (I < 2 || DUALIP_DEGREE_ORDER == 0) return false;
  degree_order(off, src_of, off_st);
  if (DUALIP_DEGREE_ORDER == 1) return true;
  if (lean_slots(off_st, max_edges, max_sources, true) <
      0.98 * lean_slots(off, max_edges, max_sources, true))
    return true;
  src_of.clear();
  off_st.clear();
  return false;
}

// Autotuner histogram bucket of a degree: 0 for degrees 0 and 1, else k for
// [2^k, 2^(k+1)), at most 31.
inline int degree_bucket(int64_t d) {
  int bk = 0;
  while (bk < 31 && (int64_t(2) << bk) <= d) ++bk;
  return bk;
}

// The degree below which 99% of the sources lie, as the upper bound of its
// histogram bucket (with no sources, bucket 0's bound: 2).
inline int64_t degree_p99(const int64_t hist[32], int64_t nsrc) {
  int64_t acc = 0;
  for (int bk = 0; bk < 32; ++bk) {
    acc += hist[bk];
    if (acc >= nsrc - nsrc / 100) return int64_t(2) << bk;
  }
  return 1;
}

// Tile shapes worth timing: candidate c = (edges, sources) is dropped when
// most of its tiles would hold a single source (p99 degree above half the
// edge budget), or when its source cap would stop tiles at under a quarter
// of the edge budget (sources x mean degree).  The first candidate is always
// kept.  Returns the indices kept, in order.
inline std::vector<int> prune_shapes(const int64_t hist[32], int64_t nsrc, int64_t nedge,
                                     const int32_t (*cand)[2], int ncand) {
  const int64_t p99 = degree_p99(hist, nsrc);
  const double mean = nsrc ? (double)nedge / (double)nsrc : 1.0;
  std::vector<int> keep;
  for (int c = 0; c < ncand; ++c) {
    const double e = cand[c][0], src = cand[c][1];
    if (p99 > e / 2 && c != 0) continue;
    if (src * mean < e / 4 && c != 0) continue;
    keep.push_back(c);
  }
  return keep;
}

// Segment classes of the sources larger than a stage (stage_e edges): the
// block class below mb_stages stages, the multi-block class (hub sources)
// from there.  A hub source is cut into chunks of `chunk` edges; hub h's
// candidate list starts at cand0 (the hub degrees before it).  The
// multi-block class is off (mb_min = INT64_MAX, no hubs) when mb_stages is 0,
// for the unit box, or when a tile reaches 2^31 - chunk edges (the hub
// kernel's edge indices are 32-bit).  big: some tile is larger than a stage
// and below mb_min (the block class's pass variant is needed).
struct HubPlan {
  int64_t e0, cand0;
  int32_t deg, c0, nch;
};
inline void plan_hubs(const std::vector<int64_t>& tile_e, int64_t stage_e, int mb_stages,
                      bool box, int64_t chunk, int64_t& mb_min, std::vector<HubPlan>& hubs,
                      std::vector<int32_t>& chunk_hub, bool& big) {
  const int64_t nt = (int64_t)tile_e.size() - 1;
  mb_min = mb_stages > 0 && !box ? (int64_t)mb_stages * stage_e : INT64_MAX;
  for (int64_t t = 0; t < nt; ++t)
    if (tile_e[t + 1] - tile_e[t] >= (int64_t)INT32_MAX - chunk) mb_min = INT64_MAX;
  hubs.clear();
  chunk_hub.clear();
  big = false;
  int64_t cand = 0;
  for (int64_t t = 0; t < nt; ++t) {
    const int64_t ne = tile_e[t + 1] - tile_e[t];
    if (ne >= mb_min) {
      HubPlan h;
      h.e0 = tile_e[t];
      h.cand0 = cand;
      h.deg = (int32_t)ne;
      h.c0 = (int32_t)chunk_hub.size();
      h.nch = (int32_t)((ne + chunk - 1) / chunk);
      chunk_hub.insert(chunk_hub.end(), (size_t)h.nch, (int32_t)hubs.size());
      hubs.push_back(h);
      cand += ne;
    } else if (ne > stage_e) {
      big = true;
    }
  }
}

// Where the segment of a non-empty stored source that starts at edge e0 starts
// in the caller's edge order.  With degree order (src_of not empty) stored
// source i is the caller's source src_of[i]; empty sources before it share
// its offset, so the source is the last one whose offset is at most e0.
inline int64_t caller_segment_start(const std::vector<int64_t>& off_stored,
                                    const std::vector<int64_t>& off_caller,
                                    const std::vector<int64_t>& src_of, int64_t e0) {
  if (src_of.empty()) return e0;
  const int64_t i =
      (int64_t)(std::upper_bound(off_stored.begin(), off_stored.end(), e0) - off_stored.begin()) -
      1;
  return off_caller[(size_t)src_of[(size_t)i]];
}

// Destination order of a hub source's edges: a stable counting sort of its
// renumbered ids d[0..n), each in [0, J).  perm[k] is the place in d of the
// k-th edge in destination order (equal ids keep their order); start is
// scratch, resized to J + 1.
inline void destination_order(const int32_t* d, int32_t n, int32_t J,
                              std::vector<uint32_t>& start, uint32_t* perm) {
  start.assign((size_t)J + 1, 0u);
  for (int32_t k = 0; k < n; ++k) ++start[(size_t)d[k] + 1];
  for (int32_t j = 0; j < J; ++j) start[(size_t)j + 1] += start[(size_t)j];
  for (int32_t k = 0; k < n; ++k) perm[start[(size_t)d[k]]++] = (uint32_t)k;
}

// Serving admission.  Resident footprint of a request (bytes): its edges
// (4 bytes of dst plus the stored c and a), offsets (8 bytes and their 4-byte
// low words), tiles and J-length arrays; the transient is the staging of host
// inputs during creation.
inline int64_t request_resident_bytes(int64_t I, int64_t E, int64_t J, bool bf16) {
  const int64_t eb = bf16 ? 8 : 12;
  return eb * (E + 8) + 12 * (I + 4) + 16 * (E / 1024 + I / 256 + 2) + 56 * J;
}
inline int64_t request_transient_bytes(int64_t E, bool inputs_on_device) {
  return inputs_on_device ? 0 : 12 * E;
}

// The head of the queue is admitted when a slot of its kind is free and its
// footprint and transient fit the budget beside what is resident; it is
// rejected when it cannot fit even with nothing resident; else it waits.
enum class Admission { kAdmit, kWait, kReject };
inline Admission admission(int64_t resident, int64_t footprint, int64_t transient, int64_t budget,
                           bool slot_free) {
  const bool fits = resident + footprint + transient <= budget;
  if (slot_free && fits) return Admission::kAdmit;
  if (!fits && resident == 0) return Admission::kReject;
  return Admission::kWait;
}

}  // namespace dualip
