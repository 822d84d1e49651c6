"""Seeded synthetic matching-LP instances, shared by the oracle and the CUDA path.

This module only draws problem data (degrees, destinations, c, a, b); it holds
none of the dual-ascent arithmetic.  The heavy lifting is ``gen.c`` (compiled
to ``libsynth.so`` by :func:`build`), whose counter-based streams make every
instance independent of the thread count and of the machine.

Workloads (the paper's Appendix B generator is replaced by these recipes; the
paper uses no public dataset):

* ``c1`` -- 1,000 sources x 50 destinations, 10 distinct uniform destinations
  per source, c = -U(0,1), a ~ U(0.5,1.5), b_j = 0.3 * sum of a into j.
* ``c2`` -- 1M sources x 10k destinations, degree Poisson(50) clipped to
  [1, 500], Zipf(1.1) destinations, c = -LogNormal(0,1), a ~ U(0.5,1.5),
  b_j = 0.2 * sum of a into j.
* ``c3`` -- 25M sources x 1M destinations, degree Poisson(80) clipped to
  [1, 2000], otherwise as c2.
* ``c4`` -- 256 independent instances, sources log-uniform 1k..2M,
  destinations log-uniform 10..50k, degree uniform 5..100 (clipped to J).
* ``c5`` -- a Poisson request stream (20 requests/s), sources log-uniform
  10k..5M, destinations 100..200k, degree Poisson(40) clipped to [1, J],
  edge storage FP32 or BF16 with probability 1/2 each.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None

DEG_FIXED, DEG_POISSON, DEG_UNIFORM = 0, 1, 2
DST_UNIFORM, DST_ZIPF = 0, 1
C_NEG_UNIFORM, C_NEG_LOGNORMAL = 0, 1

CONFIG_SEEDS = {"c1": 1001, "c2": 1002, "c3": 1003, "c4": 1004, "c5": 1005, "appb": 1006}

# The unstated parameters of the paper's Appendix B generator (the paper gives
# the laws' families only; these values are this library's choices):
# lognormal scales of the resource breadth, the resource value scale v_j, the
# request responsiveness u_i, the edge noise eps_ij and the per-resource
# coefficient scale s_j; the value cap c_max; the budget slack eps.
APPB_DEFAULTS = dict(sig_breadth=1.0, sig_v=0.5, sig_u=0.5, sig_eps=0.25, c_max=10.0, mu_s=0.0,
                     sig_s=1.0, eps=0.01)


def build(force: bool = False) -> str:
    """Compile gen.c into libsynth.so next to it (gcc, OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, i32, u64, dbl, vp = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                  ctypes.c_double, ctypes.c_void_p)
        lib.synth_degrees.argtypes = [i64, u64, ctypes.c_int, dbl, dbl, i64, i64, vp]
        lib.synth_edges.argtypes = [i64, i32, vp, u64, ctypes.c_int, dbl, ctypes.c_int, dbl, dbl,
                                    vp, vp, vp]
        lib.synth_budgets.argtypes = [i64, i32, vp, vp, dbl, vp]
        lib.synth_budgets_greedy.argtypes = [i64, i32, vp, vp, vp, u64, dbl, dbl, dbl, vp]
        lib.synth_set_threads.argtypes = [ctypes.c_int]
        lib.synth_appb_degrees.argtypes = [i64, i32, dbl, u64, dbl, vp, vp]
        lib.synth_appb_fill.argtypes = [i64, i32, vp, u64, dbl, dbl, dbl, dbl, dbl, dbl, vp, vp,
                                        vp, vp]
        _lib = lib
    return _lib


def _ptr(x: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(x.ctypes.data)


@dataclass
class Instance:
    """One matching LP in source-major layout (see the module docstring)."""

    off: np.ndarray  # int64 [I+1]
    dst: np.ndarray  # int32 [E]
    c: np.ndarray  # float32 [E]
    a: np.ndarray  # float32 [E]
    b: np.ndarray  # float32 [J]
    J: int
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def I(self) -> int:  # noqa: E743 - the paper's notation
        return int(self.off.shape[0] - 1)

    @property
    def E(self) -> int:
        return int(self.dst.shape[0])

    def subset_sources(self, idx: np.ndarray) -> "Instance":
        """The sub-instance made of the given sources (same J and b)."""
        idx = np.asarray(idx, dtype=np.int64)
        deg = self.off[idx + 1] - self.off[idx]
        off = np.zeros(idx.shape[0] + 1, dtype=np.int64)
        np.cumsum(deg, out=off[1:])
        # edge ids of the chosen sources, in order: each source's first edge
        # repeated over its degree, plus the running position inside it
        E = int(off[-1])
        sel = np.repeat(self.off[idx] - off[:-1], deg) + np.arange(E, dtype=np.int64)
        return Instance(off, self.dst[sel], self.c[sel], self.a[sel], self.b.copy(), self.J,
                        name=self.name + "[subset]")


def greedy_budgets(inst: Instance, seed: int | None = None, rho=(0.5, 1.0),
                   eps: float = 0.01) -> Instance:
    """The same graph and values with the paper's Appendix B budgets
    b_j = rho_j (l_j + eps), l_j the greedy load (each source's largest-a edge),
    rho_j ~ U[0.5, 1].  Unlike the sum-fraction budgets these bind."""
    lib = _load()
    seed = inst.meta.get("seed", 0) if seed is None else seed
    b = np.empty(inst.J, dtype=np.float32)
    rc = lib.synth_budgets_greedy(inst.I, inst.J, _ptr(inst.off), _ptr(inst.dst), _ptr(inst.a),
                                  seed, rho[0], rho[1], eps, _ptr(b))
    if rc:
        raise ValueError(f"synth_budgets_greedy failed ({rc})")
    return Instance(inst.off, inst.dst, inst.c, inst.a, b, inst.J, name=inst.name + "g",
                    meta=dict(inst.meta, budgets="greedy"))


def degrees(I: int, seed: int, kind: int, p1: float, p2: float = 0.0, lo: int = 0,
            hi: int = 1 << 40) -> np.ndarray:
    lib = _load()
    deg = np.empty(I, dtype=np.int64)
    rc = lib.synth_degrees(I, seed, kind, p1, p2, lo, hi, _ptr(deg))
    if rc:
        raise ValueError(f"synth_degrees failed ({rc})")
    return deg


def from_degrees(deg: np.ndarray, J: int, seed: int, dst_law: int = DST_ZIPF, zipf_s: float = 1.1,
                 c_law: int = C_NEG_LOGNORMAL, a_lo: float = 0.5, a_hi: float = 1.5,
                 b_frac: float = 0.2, name: str = "") -> Instance:
    """Instance with the given per-source degrees (each <= J)."""
    lib = _load()
    deg = np.ascontiguousarray(deg, dtype=np.int64)
    I = deg.shape[0]
    off = np.zeros(I + 1, dtype=np.int64)
    np.cumsum(deg, out=off[1:])
    E = int(off[-1])
    dst = np.empty(E, dtype=np.int32)
    c = np.empty(E, dtype=np.float32)
    a = np.empty(E, dtype=np.float32)
    b = np.empty(J, dtype=np.float32)
    rc = lib.synth_edges(I, J, _ptr(off), seed, dst_law, zipf_s, c_law, a_lo, a_hi, _ptr(dst),
                         _ptr(c), _ptr(a))
    if rc:
        raise ValueError(f"synth_edges failed ({rc})")
    rc = lib.synth_budgets(E, J, _ptr(dst), _ptr(a), b_frac, _ptr(b))
    if rc:
        raise ValueError(f"synth_budgets failed ({rc})")
    return Instance(off, dst, c, a, b, J, name=name,
                    meta=dict(seed=seed, dst_law=dst_law, zipf_s=zipf_s, c_law=c_law,
                              a_lo=a_lo, a_hi=a_hi, b_frac=b_frac))


def matching(I: int, J: int, seed: int, degree=("poisson", 50, 1, 500), dst_law: str = "zipf",
             zipf_s: float = 1.1, c_law: str = "lognormal", a_range=(0.5, 1.5),
             b_frac: float = 0.2, name: str = "") -> Instance:
    """General recipe.  ``degree`` is ("fixed", d), ("poisson", mean, lo, hi) or
    ("uniform", lo, hi); degrees are clipped to J."""
    kind = degree[0]
    if kind == "fixed":
        deg = degrees(I, seed, DEG_FIXED, degree[1], 0, 0, J)
    elif kind == "poisson":
        deg = degrees(I, seed, DEG_POISSON, degree[1], 0, degree[2], min(degree[3], J))
    elif kind == "uniform":
        deg = degrees(I, seed, DEG_UNIFORM, degree[1], degree[2], 0, J)
    else:
        raise ValueError(kind)
    deg = np.minimum(deg, J)
    return from_degrees(deg, J, seed, DST_ZIPF if dst_law == "zipf" else DST_UNIFORM, zipf_s,
                        C_NEG_LOGNORMAL if c_law == "lognormal" else C_NEG_UNIFORM,
                        a_range[0], a_range[1], b_frac, name=name)


def config(name: str, scale: float = 1.0) -> Instance:
    """The named single-instance workloads c1, c2, c3.  ``scale`` < 1 shrinks the
    source count (J and every law unchanged) for quick runs."""
    seed = CONFIG_SEEDS[name]
    if name == "c1":
        return matching(max(1, int(1000 * scale)), 50, seed, ("fixed", 10), "uniform",
                        c_law="uniform", b_frac=0.3, name="c1")
    if name == "c2":
        return matching(max(1, int(1_000_000 * scale)), 10_000, seed, ("poisson", 50, 1, 500),
                        name="c2" if scale == 1.0 else f"c2x{scale:g}")
    if name == "c3":
        return matching(max(1, int(25_000_000 * scale)), 1_000_000, seed, ("poisson", 80, 1, 2000),
                        name="c3" if scale == 1.0 else f"c3x{scale:g}")
    raise ValueError(name)


def appb(I: int, J: int, nu: float = 10.0, seed: int = CONFIG_SEEDS["appb"], **params) -> Instance:
    """The paper's Appendix B instance: I requests (sources), J resources
    (destinations), nu edges per request on average, resource breadths
    lognormal, K_j ~ Poisson(p_j I nu) distinct requests per resource, values
    min(v_j u_i eps_ij, c_max) (c = -value), coefficients a = s_j value, and
    greedy-load budgets b_j = rho_j (l_j + eps), rho_j ~ U[0.5, 1].  Unstated
    parameters default to APPB_DEFAULTS."""
    lib = _load()
    p = dict(APPB_DEFAULTS, **params)
    K = np.empty(J, dtype=np.int64)
    E = ctypes.c_int64(0)
    rc = lib.synth_appb_degrees(I, J, float(nu), seed, p["sig_breadth"], _ptr(K), ctypes.byref(E))
    if rc:
        raise ValueError(f"synth_appb_degrees failed ({rc})")
    off = np.empty(I + 1, dtype=np.int64)
    dst = np.empty(E.value, dtype=np.int32)
    c = np.empty(E.value, dtype=np.float32)
    a = np.empty(E.value, dtype=np.float32)
    rc = lib.synth_appb_fill(I, J, _ptr(K), seed, p["sig_v"], p["sig_u"], p["sig_eps"],
                             p["c_max"], p["mu_s"], p["sig_s"], _ptr(off), _ptr(dst), _ptr(c),
                             _ptr(a))
    if rc:
        raise ValueError(f"synth_appb_fill failed ({rc})")
    inst = Instance(off, dst, c, a, np.zeros(J, dtype=np.float32), J, name=f"appb{I}x{J}",
                    meta=dict(seed=seed, nu=nu, **p))
    return greedy_budgets(inst, seed=seed, eps=p["eps"])


def add_families(inst: Instance, m: int, seed: int = 77, a_range=(0.5, 1.5),
                 rho=(0.5, 1.0), eps: float = 0.01) -> Instance:
    """The same graph and costs with m constraint families (Definition 1):
    family 0 keeps inst.a and inst.b; family k >= 1 draws its coefficients
    a_k ~ U(a_range) per edge and takes greedy-load budgets of its own (each
    source's largest a_k edge), b_k = rho (l_k + eps).  a becomes [m, E] and b
    [m J] (row k J + j)."""
    lib = _load()
    rng = np.random.Generator(np.random.PCG64(seed))
    a = np.empty((m, inst.E), dtype=np.float32)
    b = np.empty(m * inst.J, dtype=np.float32)
    a[0] = inst.a
    b[: inst.J] = inst.b
    for k in range(1, m):
        a[k] = rng.uniform(a_range[0], a_range[1], inst.E).astype(np.float32)
        bk = np.empty(inst.J, dtype=np.float32)
        ak = np.ascontiguousarray(a[k])
        rc = lib.synth_budgets_greedy(inst.I, inst.J, _ptr(inst.off), _ptr(inst.dst), _ptr(ak),
                                      seed * 1000 + k, rho[0], rho[1], eps, _ptr(bk))
        if rc:
            raise ValueError(f"synth_budgets_greedy failed ({rc})")
        b[k * inst.J:(k + 1) * inst.J] = bk
    return Instance(inst.off, inst.dst, inst.c, a, b, inst.J, name=f"{inst.name}x{m}families",
                    meta=dict(inst.meta, families=m))


def with_hubs(base: Instance, n_hubs: int = 100, deg_range=(100_000, 1_000_000),
              J: int = 1_000_000, seed: int = 1007) -> Instance:
    """The base instance plus n_hubs sources of log-uniform degree in deg_range,
    each linked to distinct destinations drawn uniformly from J >= base.J (the
    base keeps its destination ids), c and a by the base laws; greedy-load
    budgets on the whole."""
    rng = np.random.Generator(np.random.PCG64(seed))
    deg = np.round(np.exp(rng.uniform(np.log(deg_range[0]), np.log(deg_range[1]),
                                      n_hubs))).astype(np.int64)
    hubs = from_degrees(deg, J, seed, DST_UNIFORM)
    off = np.concatenate([base.off, base.off[-1] + hubs.off[1:]]).astype(np.int64)
    inst = Instance(off, np.concatenate([base.dst, hubs.dst]), np.concatenate([base.c, hubs.c]),
                    np.concatenate([base.a, hubs.a]), np.zeros(J, np.float32), J,
                    name=f"{base.name}+{n_hubs}hubs", meta=dict(base.meta, hubs=n_hubs))
    return greedy_budgets(inst, seed=seed)


def batch_shapes(n: int = 256, seed: int = CONFIG_SEEDS["c4"], i_range=(1_000, 2_000_000),
                 j_range=(10, 50_000)):
    """(I, J, seed) of each instance of the batched workload c4."""
    rng = np.random.Generator(np.random.PCG64(seed))
    li = rng.uniform(np.log(i_range[0]), np.log(i_range[1]), n)
    lj = rng.uniform(np.log(j_range[0]), np.log(j_range[1]), n)
    return [(int(round(np.exp(x))), int(round(np.exp(y))), seed * 1_000_000 + k)
            for k, (x, y) in enumerate(zip(li, lj))]


def batch_instance(I: int, J: int, seed: int) -> Instance:
    return matching(I, J, seed, ("uniform", 5, 100), name=f"c4:{seed}")


def request_trace(n: int = 400, rate: float = 20.0, seed: int = CONFIG_SEEDS["c5"],
                  i_range=(10_000, 5_000_000), j_range=(100, 200_000)):
    """Arrival time, (I, J, seed) and edge storage ("f32"/"bf16") of each request of c5."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, n)
    t = np.cumsum(gaps) - gaps[0]
    li = rng.uniform(np.log(i_range[0]), np.log(i_range[1]), n)
    lj = rng.uniform(np.log(j_range[0]), np.log(j_range[1]), n)
    st = rng.integers(0, 2, n)
    return [dict(t=float(t[k]), I=int(round(np.exp(li[k]))), J=int(round(np.exp(lj[k]))),
                 seed=seed * 1_000_000 + k, storage=("bf16" if st[k] else "f32"))
            for k in range(n)]


def request_instance(req: dict) -> Instance:
    return matching(req["I"], req["J"], req["seed"], ("poisson", 40, 1, req["J"]),
                    name=f"c5:{req['seed']}")
