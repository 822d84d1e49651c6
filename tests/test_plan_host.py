"""Host planning of the stored layout (paper_2603_04621_gb300/csrc/plan.h),
compiled on its own with g++ (no CUDA): the greedy tiling of the
source-major edge list, the lane-group slot model, the choice of the stored
order and the degree order.

* Tiles cover the sources in order.  Each tile is a single oversized source,
  or holds at most max_edges edges and max_sources sources.  It is greedy:
  the next source would break a limit.
* The slot model counts the element slots of the pass's lane-group rounds
  (checked by hand); degree order is stored when it saves at least 2%.
* The degree order is a stable permutation by degree, and its offsets move
  each source's edges as one segment.
* The autotuner's histogram buckets are [2^k, 2^(k+1)) (0 and 1 in bucket 0);
  its 99th-percentile degree is a bucket's upper bound; and it times only the
  shapes that neither make most tiles single-source nor cap tiles at under a
  quarter of their edge budget.
* Serving admission: the footprint estimate of the header, and the head of
  the queue admitted, kept waiting or rejected.
* Segment classes of large sources: hub sources (at least 16 stages) and
  their chunk table and candidate-list offsets; the block class's flag; the
  multi-block class off for the unit box.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2603_04621_gb300", "csrc")

SHIM = r"""
#include "plan.h"
extern "C" {
int64_t plan_tiles(const int64_t* off, int64_t I, int64_t max_e, int64_t max_s,
                   int64_t* tiles, int64_t* tile_e, int64_t cap) {
  std::vector<int64_t> o(off, off + I + 1), t, te;
  dualip::build_tiles(o, t, te, max_e, max_s);
  for (size_t k = 0; k < t.size() && (int64_t)k < cap; ++k) { tiles[k] = t[k]; tile_e[k] = te[k]; }
  return (int64_t)t.size();
}
double plan_lean_slots(const int64_t* off, int64_t I, int64_t max_e, int64_t max_s, int lean80) {
  return dualip::lean_slots(std::vector<int64_t>(off, off + I + 1), max_e, max_s, lean80 != 0);
}
int plan_choose(const int64_t* off, int64_t I, int64_t max_e, int64_t max_s) {
  std::vector<int64_t> s, os;
  return dualip::choose_degree_order(std::vector<int64_t>(off, off + I + 1), max_e, max_s, s,
                                     os) ? 1 : 0;
}
int plan_bucket(int64_t d) { return dualip::degree_bucket(d); }
int64_t plan_p99(const int64_t* hist, int64_t nsrc) { return dualip::degree_p99(hist, nsrc); }
int plan_prune(const int64_t* hist, int64_t nsrc, int64_t nedge, const int32_t* cand, int ncand,
               int* keep) {
  std::vector<int> k = dualip::prune_shapes(hist, nsrc, nedge,
                                            reinterpret_cast<const int32_t (*)[2]>(cand), ncand);
  for (size_t i = 0; i < k.size(); ++i) keep[i] = k[i];
  return (int)k.size();
}
int64_t plan_resident(int64_t I, int64_t E, int64_t J, int bf16) {
  return dualip::request_resident_bytes(I, E, J, bf16 != 0);
}
int64_t plan_transient(int64_t E, int on_device) {
  return dualip::request_transient_bytes(E, on_device != 0);
}
int plan_admission(int64_t resident, int64_t footprint, int64_t transient, int64_t budget,
                   int slot_free) {
  return (int)dualip::admission(resident, footprint, transient, budget, slot_free != 0);
}
int64_t plan_hubs_c(const int64_t* tile_e, int64_t nt, int64_t stage_e, int mb_stages, int box,
                    int64_t chunk, int64_t* mb_min, int64_t* hub_out, int64_t hub_cap,
                    int32_t* chunk_hub, int64_t chunk_cap, int64_t* nchunks, int* big) {
  std::vector<int64_t> te(tile_e, tile_e + nt + 1);
  std::vector<dualip::HubPlan> hubs;
  std::vector<int32_t> ch;
  bool b = false;
  dualip::plan_hubs(te, stage_e, mb_stages, box != 0, chunk, *mb_min, hubs, ch, b);
  for (size_t h = 0; h < hubs.size() && (int64_t)h < hub_cap; ++h) {
    hub_out[5 * h] = hubs[h].e0; hub_out[5 * h + 1] = hubs[h].cand0;
    hub_out[5 * h + 2] = hubs[h].deg; hub_out[5 * h + 3] = hubs[h].c0;
    hub_out[5 * h + 4] = hubs[h].nch;
  }
  for (size_t k = 0; k < ch.size() && (int64_t)k < chunk_cap; ++k) chunk_hub[k] = ch[k];
  *nchunks = (int64_t)ch.size();
  *big = b ? 1 : 0;
  return (int64_t)hubs.size();
}
int64_t plan_caller_start(const int64_t* off_st, const int64_t* off, const int64_t* src_of,
                          int64_t I, int64_t e0) {
  std::vector<int64_t> s(src_of, src_of + I);
  return dualip::caller_segment_start(std::vector<int64_t>(off_st, off_st + I + 1),
                                      std::vector<int64_t>(off, off + I + 1), s, e0);
}
void plan_destination_order(const int32_t* d, int32_t n, int32_t J, uint32_t* perm) {
  std::vector<uint32_t> start;
  dualip::destination_order(d, n, J, start, perm);
}
void plan_degree_order(const int64_t* off, int64_t I, int64_t* src_of, int64_t* off_st) {
  std::vector<int64_t> s, os;
  dualip::degree_order(std::vector<int64_t>(off, off + I + 1), s, os);
  for (int64_t i = 0; i < I; ++i) src_of[i] = s[i];
  for (int64_t i = 0; i <= I; ++i) off_st[i] = os[i];
}
}
"""


@pytest.fixture(scope="module")
def plan(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ is not available")
    d = tmp_path_factory.mktemp("plan")
    src = d / "shim.cpp"
    src.write_text(SHIM)
    lib = d / "libplan.so"
    subprocess.run([gxx, "-std=c++17", "-O2", "-shared", "-fPIC", "-I", CSRC, str(src), "-o",
                    str(lib)], check=True)
    L = ctypes.CDLL(str(lib))
    p64 = ctypes.POINTER(ctypes.c_int64)
    L.plan_tiles.argtypes = [p64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, p64, p64,
                             ctypes.c_int64]
    L.plan_tiles.restype = ctypes.c_int64
    i64 = ctypes.c_int64
    L.plan_lean_slots.argtypes = [p64, i64, i64, i64, ctypes.c_int]
    L.plan_lean_slots.restype = ctypes.c_double
    L.plan_choose.argtypes = [p64, i64, i64, i64]
    L.plan_choose.restype = ctypes.c_int
    L.plan_bucket.argtypes = [ctypes.c_int64]
    L.plan_bucket.restype = ctypes.c_int
    L.plan_p99.argtypes = [p64, ctypes.c_int64]
    L.plan_p99.restype = ctypes.c_int64
    L.plan_prune.argtypes = [p64, ctypes.c_int64, ctypes.c_int64,
                             ctypes.POINTER(ctypes.c_int32), ctypes.c_int,
                             ctypes.POINTER(ctypes.c_int)]
    L.plan_prune.restype = ctypes.c_int
    i64 = ctypes.c_int64
    L.plan_resident.argtypes = [i64, i64, i64, ctypes.c_int]
    L.plan_resident.restype = i64
    L.plan_transient.argtypes = [i64, ctypes.c_int]
    L.plan_transient.restype = i64
    L.plan_admission.argtypes = [i64, i64, i64, i64, ctypes.c_int]
    L.plan_admission.restype = ctypes.c_int
    L.plan_degree_order.argtypes = [p64, ctypes.c_int64, p64, p64]
    L.plan_destination_order.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_void_p]
    L.plan_destination_order.restype = None
    L.plan_caller_start.argtypes = [p64, p64, p64, ctypes.c_int64, ctypes.c_int64]
    L.plan_caller_start.restype = ctypes.c_int64
    vp = ctypes.c_void_p
    L.plan_hubs_c.argtypes = [vp, i64, i64, ctypes.c_int, ctypes.c_int, i64, vp, vp, i64, vp,
                              i64, vp, vp]
    L.plan_hubs_c.restype = i64
    L.plan_degree_order.restype = None
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def offsets(deg):
    return np.concatenate([[0], np.cumsum(deg)]).astype(np.int64)


def tiles_of(plan, off, max_e, max_s):
    I = len(off) - 1
    cap = I + 2
    t = np.zeros(cap, np.int64)
    te = np.zeros(cap, np.int64)
    n = plan.plan_tiles(_p(off), I, max_e, max_s, _p(t), _p(te), cap)
    assert n <= cap
    return t[:n], te[:n]


@pytest.mark.parametrize("law", ["poisson", "uniform", "with_giants", "zeros_and_ones"])
def test_tiles_cover_in_order_within_limits_and_greedily(plan, law):
    rng = np.random.default_rng({"poisson": 1, "uniform": 2, "with_giants": 3,
                                 "zeros_and_ones": 4}[law])
    if law == "poisson":
        deg = rng.poisson(50, 20_000)
    elif law == "uniform":
        deg = rng.integers(5, 101, 20_000)
    elif law == "with_giants":
        deg = rng.poisson(80, 5_000)
        deg[rng.choice(5_000, 40, replace=False)] = rng.integers(3_201, 20_000, 40)
    else:
        deg = rng.integers(0, 2, 30_000)
    off = offsets(deg)
    max_e, max_s = 3_200, 256
    t, te = tiles_of(plan, off, max_e, max_s)
    I = len(deg)
    assert t[0] == 0 and t[-1] == I and np.all(np.diff(t) >= 1)
    assert np.array_equal(te, off[t])
    for a, b in zip(t[:-1], t[1:]):
        e = off[b] - off[a]
        if b - a == 1 and deg[a] > max_e:
            continue  # an oversized source alone
        assert e <= max_e and b - a <= max_s
        assert np.all(deg[a:b] <= max_e)
        if b < I:  # greedy: the next source would break a limit, or is oversized
            assert b - a == max_s or e + deg[b] > max_e


def test_lean_slot_model_by_hand(plan):
    """Element slots of the lane-group projection, counted by hand."""
    def slots(deg, lean80=True, max_e=3200, max_s=256):
        off = offsets(np.asarray(deg))
        return plan.plan_lean_slots(_p(off), len(deg), max_e, max_s, int(lean80))

    # eight sources of 50 edges: spans 50 / 52 (first edge mod 4 is 0 or 2),
    # one 4-lane round of 64-slot windows = 32 lanes x 16 slots
    assert slots([50] * 8) == 512
    # spans of 70..73 take 80-slot windows under lean80 (one round, 640
    # slots), else two 8-lane rounds of 512
    assert slots([70] * 8) == 640
    assert slots([70] * 8, lean80=False) == 1024
    # a span in (80, 128] sends the spans over 64 to the 8-lane pass as well
    assert slots([70] * 7 + [100]) == 512 * 2
    # 16- and 32-lane rounds: two sources of 200 edges, one of 400
    assert slots([200, 200]) == 512 and slots([400]) == 512
    # a span over 512 is counted as four passes over it; empty sources cost nothing
    assert slots([600, 0, 0]) == 4 * 600
    # batches restart at every tile: 5-source tiles split 8 sources 5 + 3
    assert slots([10] * 8, max_s=5) == 2 * 512


def test_degree_order_is_chosen_by_the_slot_model(plan):
    rng = np.random.default_rng(5)

    def choose(deg, max_e=3200):
        off = offsets(np.asarray(deg))
        return plan.plan_choose(_p(off), len(deg), max_e, 256)

    # constant degrees: sorting changes nothing
    assert choose(np.full(1_000, 10)) == 0
    assert choose(np.array([7])) == 0 and choose(np.zeros(100, np.int64)) == 0
    # uniform 5..100 (the batched workload): batches of mixed spans
    assert choose(rng.integers(5, 101, 50_000)) == 1
    # Poisson(80) in [1, 2000] with 4800-edge BF16 tiles (the precision workload):
    # about half the spans exceed 80, so unsorted batches mix 4- and 8-lane rounds
    assert choose(np.clip(rng.poisson(80, 50_000), 1, 2000), max_e=4800) == 1
    # hub sources among the others (the two mixes of the GPU test of hub edges
    # in destination order): ascending degrees stay in the caller's order,
    # hubs among Uniform[5, 100] degrees are stored in degree order
    assert choose(np.array([3, 10, 40, 300, 70_000, 200_000])) == 0
    r47 = np.random.default_rng(47)
    assert choose(np.concatenate([[200_000], r47.integers(5, 101, 6_000), [70_000],
                                  r47.integers(5, 101, 6_000)])) == 1
    # whatever it picks, the model never prefers an order it scores higher
    for deg in (rng.poisson(50, 20_000), rng.poisson(40, 20_000), rng.integers(1, 300, 20_000)):
        off = offsets(deg)
        src, off_st = np.empty(len(deg), np.int64), np.empty(len(deg) + 1, np.int64)
        plan.plan_degree_order(_p(off), len(deg), _p(src), _p(off_st))
        a = plan.plan_lean_slots(_p(off), len(deg), 3200, 256, 1)
        b = plan.plan_lean_slots(_p(off_st), len(deg), 3200, 256, 1)
        assert choose(deg) == int(b < 0.98 * a)


@pytest.mark.parametrize("case", ["counting", "comparison"])
def test_degree_order_is_a_stable_permutation_with_consistent_offsets(plan, case):
    rng = np.random.default_rng(6)
    deg = rng.integers(0, 12, 5_000)
    if case == "comparison":  # a degree above 4 I + 1024 takes the comparison sort
        deg[17] = 4 * len(deg) + 5_000
        deg[4_000] = deg[17]  # a tie among the giants keeps the caller's order
    off = offsets(deg)
    I = len(deg)
    src = np.zeros(I, np.int64)
    off_st = np.zeros(I + 1, np.int64)
    plan.plan_degree_order(_p(off), I, _p(src), _p(off_st))
    assert np.array_equal(np.sort(src), np.arange(I))
    assert np.array_equal(src, np.argsort(deg, kind="stable"))  # ties keep the caller's order
    assert np.all(np.diff(deg[src]) >= 0)
    assert np.array_equal(np.diff(off_st), deg[src]) and off_st[-1] == off[-1]
    # moving each source's segment to its stored place is a bijection of the edges
    edge_of = np.concatenate([np.arange(off[s], off[s + 1]) for s in src])
    assert np.array_equal(np.sort(edge_of), np.arange(off[-1]))


def test_histogram_buckets_and_p99(plan):
    for d, bk in ((0, 0), (1, 0), (2, 1), (3, 1), (4, 2), (63, 5), (64, 6), (2**31, 31),
                  (2**40, 31)):
        assert plan.plan_bucket(d) == bk, d
    rng = np.random.default_rng(7)
    deg = rng.integers(5, 101, 100_000)
    hist = np.bincount([plan.plan_bucket(int(x)) for x in deg], minlength=32).astype(np.int64)
    p99 = plan.plan_p99(_p(hist), len(deg))
    q = np.quantile(deg, 0.99)
    assert p99 // 2 <= q < p99  # the bucket holding the 99th percentile, by its upper bound
    assert plan.plan_p99(_p(np.zeros(32, np.int64)), 0) == 2  # no sources: bucket 0's bound


CANDS = [(3200, 256), (3200, 128), (2048, 256), (2048, 128), (1536, 128), (1024, 128),
         (1024, 64), (512, 64)]


def kept(plan, deg):
    hist = np.bincount([plan.plan_bucket(int(x)) for x in deg], minlength=32).astype(np.int64)
    cand = np.array(CANDS, dtype=np.int32).ravel()
    keep = (ctypes.c_int * 8)()
    n = plan.plan_prune(_p(hist), len(deg), int(np.sum(deg)),
                        cand.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), 8, keep)
    return list(keep[:n]), plan.plan_p99(_p(hist), len(deg)), float(np.mean(deg))


@pytest.mark.parametrize("law", ["c4", "tiny", "huge"])
def test_shape_pruning_rule(plan, law):
    rng = np.random.default_rng(8)
    deg = {"c4": rng.integers(5, 101, 50_000), "tiny": rng.integers(1, 3, 50_000),
           "huge": rng.integers(2_000, 5_000, 5_000)}[law]
    keep, p99, mean = kept(plan, deg)
    expect = [c for c, (e, s) in enumerate(CANDS)
              if c == 0 or not (p99 > e / 2 or s * mean < e / 4)]
    assert keep == expect
    if law == "c4":  # moderate degrees: every shape is worth timing
        assert keep == list(range(8))
    if law == "huge":  # most tiles would hold one source: only the default shape
        assert keep == [0]
    if law == "tiny":  # small source caps would stop tiles early: they go
        assert 1 not in keep and 7 not in keep


def test_request_footprint_estimate(plan):
    I, E, J = 800_000, 32_000_000, 26_000
    tiles = E // 1024 + I // 256 + 2
    # E (4 + bytes of c and a) + 12 (I + 4) (offsets and their low words) + 16 tiles + 56 J,
    # with 8 edges of padding
    assert plan.plan_resident(I, E, J, 0) == 12 * (E + 8) + 12 * (I + 4) + 16 * tiles + 56 * J
    assert plan.plan_resident(I, E, J, 1) == 8 * (E + 8) + 12 * (I + 4) + 16 * tiles + 56 * J
    assert plan.plan_transient(E, 0) == 12 * E and plan.plan_transient(E, 1) == 0


ADMIT, WAIT, REJECT = 0, 1, 2


def test_admission_rule(plan):
    a = plan.plan_admission
    assert a(0, 60, 30, 100, 1) == ADMIT        # fits with its transient
    assert a(0, 60, 50, 100, 1) == REJECT       # never fits, even alone
    assert a(0, 60, 50, 100, 0) == REJECT       # no slot changes that
    assert a(20, 60, 30, 100, 1) == WAIT        # fits once something leaves
    assert a(10, 60, 30, 100, 0) == WAIT        # fits, but no slot of its kind is free
    assert a(10, 60, 30, 100, 1) == ADMIT       # exactly at the budget


def hub_plan(plan, tile_e, stage_e=3200, mb_stages=16, box=0, chunk=4096):
    te = np.ascontiguousarray(tile_e, dtype=np.int64)
    mb = np.zeros(1, np.int64)
    hubs = np.zeros(5 * 64, np.int64)
    ch = np.zeros(100_000, np.int32)
    nch = np.zeros(1, np.int64)
    big = ctypes.c_int(0)
    n = plan.plan_hubs_c(te.ctypes.data, len(te) - 1, stage_e, mb_stages, box, chunk,
                         mb.ctypes.data, hubs.ctypes.data, 64, ch.ctypes.data, len(ch),
                         nch.ctypes.data, ctypes.addressof(big))
    return int(mb[0]), hubs[: 5 * n].reshape(n, 5), ch[: int(nch[0])], bool(big.value)


def test_hub_sources_and_their_chunks(plan):
    """Sources of at least 16 stages are hub sources (the multi-block class),
    cut into 4096-edge chunks; those between a stage and 16 stages need the
    block class; the unit box and mb_stages = 0 turn the multi-block class off."""
    degs = [100, 3_201, 51_199, 51_200, 4_096 * 20 + 1, 7, 200_000]
    tile_e = np.concatenate([[0], np.cumsum(degs)])
    mb, hubs, ch, big = hub_plan(plan, tile_e)
    assert mb == 16 * 3200 and big  # 3,201 and 51,199 edges: block class
    assert hubs[:, 2].tolist() == [51_200, 81_921, 200_000]
    assert hubs[:, 0].tolist() == [tile_e[3], tile_e[4], tile_e[6]]
    assert hubs[:, 1].tolist() == [0, 51_200, 51_200 + 81_921]  # candidate lists back to back
    nch = [-(-d // 4096) for d in (51_200, 81_921, 200_000)]
    assert hubs[:, 4].tolist() == nch and hubs[:, 3].tolist() == [0, nch[0], nch[0] + nch[1]]
    assert ch.tolist() == [0] * nch[0] + [1] * nch[1] + [2] * nch[2]
    for kw in (dict(box=1), dict(mb_stages=0)):
        mb, hubs, ch, big = hub_plan(plan, tile_e, **kw)
        assert mb == 2**63 - 1 and len(hubs) == 0 and len(ch) == 0 and big
    mb, hubs, ch, big = hub_plan(plan, [0, 10, 3_000])
    assert len(hubs) == 0 and not big



@pytest.mark.parametrize("n,J", [(0, 5), (1, 1), (1000, 7), (50_000, 1_000_000), (20_000, 300)])
def test_destination_order_is_numpys_stable_argsort(plan, n, J):
    """The hub sources' edge order: a stable sort of the renumbered ids, checked
    against numpy's stable argsort, with repeated ids (small J) and sparse ones."""
    rng = np.random.default_rng(n + J)
    d = rng.integers(0, J, n).astype(np.int32)
    perm = np.full(n, 0xFFFFFFFF, np.uint32)
    plan.plan_destination_order(d.ctypes.data, n, J, perm.ctypes.data)
    assert np.array_equal(perm.astype(np.int64), np.argsort(d, kind="stable"))


def test_caller_segment_start_skips_empty_sources(plan):
    """A hub's segment in the caller's order, for sources stored in degree order:
    every non-empty stored source maps to its caller's offset, also where empty
    sources share its stored offset (they sort first)."""
    rng = np.random.default_rng(8)
    deg = rng.integers(0, 60, 3_000)
    deg[rng.integers(0, 3_000, 400)] = 0
    deg[[5, 700, 2_999]] = [90_000, 60_000, 75_000]
    off = offsets(deg)
    I = len(deg)
    src, off_st = np.empty(I, np.int64), np.empty(I + 1, np.int64)
    plan.plan_degree_order(_p(off), I, _p(src), _p(off_st))
    for i in range(I):
        if off_st[i + 1] > off_st[i]:
            assert plan.plan_caller_start(_p(off_st), _p(off), _p(src), I,
                                          int(off_st[i])) == off[src[i]]
