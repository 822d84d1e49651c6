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

// Degrees spread widely when their standard deviation exceeds 0.3 of their
// mean.  Such problems are stored in degree order (dualip_create).
inline bool degrees_spread_widely(const std::vector<int64_t>& off) {
  const int64_t I = (int64_t)off.size() - 1;
  if (I < 2) return false;
  double s1 = 0.0, s2 = 0.0;
  for (int64_t i = 0; i < I; ++i) {
    const double d = (double)(off[i + 1] - off[i]);
    s1 += d;
    s2 += d * d;
  }
  const double mean = s1 / (double)I, var = s2 / (double)I - mean * mean;
  return mean > 0.0 && var > 0.09 * mean * mean;
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

// Serving admission.  Resident footprint of a request (bytes): its edges
// (4 bytes of dst plus the stored c and a), offsets, tiles and J-length
// arrays; the transient is the staging of host inputs during creation.
inline int64_t request_resident_bytes(int64_t I, int64_t E, int64_t J, bool bf16) {
  const int64_t eb = bf16 ? 8 : 12;
  return eb * (E + 8) + 8 * (I + 4) + 16 * (E / 1024 + I / 256 + 2) + 56 * J;
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
