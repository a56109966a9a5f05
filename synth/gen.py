"""Seeded generators for graphs and update batches (numpy, deterministic).

Every random number comes from splitmix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014) evaluated on a
counter, so a draw is a pure function of (seed, stream tag, index) and the
same on every machine.

Graphs are simple and undirected.  They are returned as a symmetric int32 CSR
``(row_ptr[n+1], col[2m])`` with every row sorted, or as a sorted array of
canonical uint64 keys ``min(u,v) << 32 | max(u,v)``.

The batch recipes follow the experiments of the paper (Sec. 5, batch creation
with p = 0.7) and the synthetic stand-ins for its SNAP datasets (Table 1):
Chung-Lu power-law graphs of the same sizes.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_LO32 = np.uint64(0xFFFFFFFF)


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """splitmix64 output for counters ``idx`` (uint64 array) under ``seed``."""
    with np.errstate(over="ignore"):
        x = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (idx.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (x ^ (x >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _substream(seed: int, tag: str) -> int:
    """Seed of an independent stream named ``tag`` derived from ``seed``."""
    h = 1469598103934665603
    for ch in tag.encode():
        h = ((h ^ ch) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return int(splitmix64(seed ^ h, np.array([0], dtype=np.uint64))[0])


def uniform01(seed: int, start: int, count: int) -> np.ndarray:
    """``count`` doubles in [0, 1) from counters ``start .. start+count-1``."""
    idx = np.arange(start, start + count, dtype=np.uint64)
    return (splitmix64(seed, idx) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _sorted_unique(a: np.ndarray) -> np.ndarray:
    """Sorted distinct values (sort + adjacent compare)."""
    a = np.sort(a)
    if a.size == 0:
        return a
    keep = np.empty(a.size, dtype=bool)
    keep[0] = True
    np.not_equal(a[1:], a[:-1], out=keep[1:])
    return a[keep]


def _canon(u: np.ndarray, v: np.ndarray) -> np.ndarray:
    a = np.minimum(u, v).astype(np.uint64)
    b = np.maximum(u, v).astype(np.uint64)
    return (a << np.uint64(32)) | b


def _collect(draw, target: int, sel_seed: int, exclude_sorted: np.ndarray | None = None) -> np.ndarray:
    """Exactly ``target`` distinct keys, sorted.

    ``draw(round, need)`` returns candidate keys.  Rounds continue until at
    least ``target`` distinct keys (not in ``exclude_sorted``) are known; the
    surplus is then trimmed by keeping the keys of smallest seeded hash, which
    is an unbiased choice and independent of the draw order.
    """
    keys = np.empty(0, dtype=np.uint64)
    rnd = 0
    while keys.size < target:
        cand = np.asarray(draw(rnd, target - keys.size), dtype=np.uint64)
        if exclude_sorted is not None and exclude_sorted.size and cand.size:
            pos = np.minimum(np.searchsorted(exclude_sorted, cand), exclude_sorted.size - 1)
            cand = cand[exclude_sorted[pos] != cand]
        keys = _sorted_unique(np.concatenate([keys, cand]))
        rnd += 1
        if rnd > 1000:
            raise RuntimeError("could not draw enough distinct pairs")
    if keys.size > target:
        h = splitmix64(sel_seed, keys)
        keys = np.sort(keys[np.argpartition(h, target - 1)[:target]])
    return keys


class _CdfSampler:
    """Inverse-CDF sampling: index i with cdf[i-1] <= r < cdf[i].

    Same result as ``searchsorted(cdf, r, side='right')`` clipped to the last
    index; a bucket table narrows each search first.
    """

    def __init__(self, cdf: np.ndarray):
        self.cdf = cdf
        self.nb = int(max(1024, min(1 << 22, 4 * cdf.size)))
        self.table = np.searchsorted(cdf, np.arange(self.nb, dtype=np.float64) / self.nb, side="right")

    def __call__(self, r: np.ndarray) -> np.ndarray:
        cdf, n = self.cdf, self.cdf.size
        idx = np.minimum(self.table[np.minimum((r * self.nb).astype(np.int64), self.nb - 1)], n - 1)
        act = np.nonzero(cdf[idx] <= r)[0]
        while act.size:
            idx[act] += 1
            np.minimum(idx, n - 1, out=idx)
            act = act[(cdf[idx[act]] <= r[act]) & (idx[act] < n - 1)]
        return idx


def csr_from_keys(n: int, keys: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Symmetric CSR (rows sorted) from canonical keys of an undirected graph."""
    keys = np.asarray(keys, dtype=np.uint64)
    u = (keys >> np.uint64(32)).astype(np.int64)
    v = (keys & _LO32).astype(np.int64)
    src = np.concatenate([u, v])
    directed = np.sort((src.astype(np.uint64) << np.uint64(32)) | np.concatenate([v, u]).astype(np.uint64))
    col = (directed & _LO32).astype(np.int32)
    counts = np.bincount(src, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("graph too large for an int32 CSR")
    return row_ptr.astype(np.int32), col


def keys_from_csr(row_ptr: np.ndarray, col: np.ndarray) -> np.ndarray:
    """Sorted canonical keys (u < v) of a symmetric CSR."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    n = row_ptr.size - 1
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    dst = np.asarray(col, dtype=np.int64)
    sel = src < dst
    return np.sort((src[sel].astype(np.uint64) << np.uint64(32)) | dst[sel].astype(np.uint64))


def _relabel(n: int, keys: np.ndarray, seed: int) -> np.ndarray:
    perm = np.argsort(uniform01(_substream(seed, "perm"), 0, n), kind="stable").astype(np.uint64)
    u = perm[(keys >> np.uint64(32)).astype(np.int64)]
    v = perm[(keys & _LO32).astype(np.int64)]
    return np.sort(_canon(u, v))


def er_graph(n: int, m: int, seed: int = 0) -> np.ndarray:
    """G(n, m): m distinct uniform non-loop pairs; sorted canonical keys."""
    if m > n * (n - 1) // 2:
        raise ValueError("m exceeds the number of vertex pairs")
    s = _substream(seed, "er")

    def draw(rnd, need):
        need = int(need * 1.3) + 64
        r = uniform01(s, rnd << 40, 2 * need)
        u = np.minimum((r[0::2] * n).astype(np.int64), n - 1)
        v = np.minimum((r[1::2] * n).astype(np.int64), n - 1)
        ok = u != v
        return _canon(u[ok], v[ok])

    return _collect(draw, m, _substream(seed, "er-sel"))


def chung_lu_weights(n: int, m: int, gamma: float, dmax: float) -> np.ndarray:
    """Expected degrees w_i proportional to i^(-1/(gamma-1)), capped at dmax, sum 2m."""
    alpha = 1.0 / (gamma - 1.0)
    base = np.arange(1, n + 1, dtype=np.float64) ** (-alpha)
    target = 2.0 * m
    if n * dmax < target:
        raise ValueError("dmax too small to reach 2m")
    lo, hi = 0.0, 1.0
    while np.minimum(hi * base, dmax).sum() < target:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.minimum(mid * base, dmax).sum() < target:
            lo = mid
        else:
            hi = mid
    return np.minimum(hi * base, dmax)


def chung_lu_graph(n: int, m: int, gamma: float, dmax: float, seed: int = 0) -> np.ndarray:
    """Chung-Lu graph with exactly m edges; sorted canonical keys.

    Endpoints are drawn i.i.d. proportional to the weights; pairs are
    canonicalised; self-loops and repeats are dropped; drawing continues until
    m distinct pairs exist.  Vertex ids are then randomly permuted so that hubs
    are not clustered at low ids.
    """
    w = chung_lu_weights(n, m, gamma, dmax)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    sample = _CdfSampler(cdf)
    s = _substream(seed, "cl")

    def draw(rnd, need):
        need = int(need * 1.25) + 1024
        e = sample(uniform01(s, rnd << 40, 2 * need))
        u, v = e[0::2], e[1::2]
        ok = u != v
        return _canon(u[ok], v[ok])

    return _relabel(n, _collect(draw, m, _substream(seed, "cl-sel")), seed)


def _degrees(n: int, keys: np.ndarray) -> np.ndarray:
    u = (keys >> np.uint64(32)).astype(np.int64)
    v = (keys & _LO32).astype(np.int64)
    return np.bincount(u, minlength=n) + np.bincount(v, minlength=n)


def random_batch(n: int, keys: np.ndarray, n_ins: int, n_del: int, seed: int,
                 ins_weighting: str = "degree", deg: np.ndarray | None = None):
    """One clean batch against the graph with sorted canonical ``keys``.

    Deletions are distinct existing edges chosen uniformly.  Insertions are
    distinct non-edges whose endpoints are drawn uniformly
    (``ins_weighting='uniform'``) or proportionally to degree + 1
    (``'degree'``).  Each pair's orientation is randomised.  Returns int32
    arrays ``ins[n_ins, 2]`` and ``dels[n_del, 2]``.
    """
    keys = np.asarray(keys, dtype=np.uint64)
    m = keys.size
    n_del = min(n_del, m)
    sd = _substream(seed, "del")
    # deletions: distinct existing edges, uniform
    def draw_del(rnd, need):
        idx = np.minimum((uniform01(sd, rnd << 40, need * 2 + 16) * m).astype(np.int64), m - 1)
        return keys[idx]

    dkeys = _collect(draw_del, n_del, _substream(seed, "del-sel")) if n_del else np.empty(0, np.uint64)
    # insertions: distinct non-edges
    si = _substream(seed, "ins")
    if ins_weighting == "degree":
        if deg is None:
            deg = _degrees(n, keys)
        cdf = np.cumsum(deg.astype(np.float64) + 1.0)
        cdf /= cdf[-1]
        sample = _CdfSampler(cdf)

    def draw_ins(rnd, need):
        r = uniform01(si, rnd << 40, 2 * (need * 2 + 64))
        if ins_weighting == "degree":
            e = sample(r)
        else:
            e = np.minimum((r * n).astype(np.int64), n - 1)
        u, v = e[0::2], e[1::2]
        ok = u != v
        return _canon(u[ok], v[ok])

    ikeys = (_collect(draw_ins, n_ins, _substream(seed, "ins-sel"), exclude_sorted=keys)
             if n_ins else np.empty(0, np.uint64))
    # present each batch in a seeded random order
    ikeys = ikeys[np.argsort(uniform01(_substream(seed, "ord-ins"), 0, ikeys.size), kind="stable")]
    dkeys = dkeys[np.argsort(uniform01(_substream(seed, "ord-del"), 0, dkeys.size), kind="stable")]

    def pairs(k, tag):
        a = (k >> np.uint64(32)).astype(np.int32)
        b = (k & _LO32).astype(np.int32)
        flip = uniform01(_substream(seed, tag), 0, k.size) < 0.5
        out = np.stack([np.where(flip, b, a), np.where(flip, a, b)], axis=1)
        return np.ascontiguousarray(out, dtype=np.int32)

    return pairs(ikeys, "flip-ins"), pairs(dkeys, "flip-del")


def apply_batch_keys(keys: np.ndarray, ins: np.ndarray, dels: np.ndarray) -> np.ndarray:
    """Sorted keys of the graph after a clean batch (test and bench plumbing)."""
    ik = _canon(ins[:, 0].astype(np.int64), ins[:, 1].astype(np.int64)) if len(ins) else np.empty(0, np.uint64)
    dk = _canon(dels[:, 0].astype(np.int64), dels[:, 1].astype(np.int64)) if len(dels) else np.empty(0, np.uint64)
    keys = np.asarray(keys, dtype=np.uint64)
    if dk.size:
        dk = np.sort(dk)
        pos = np.minimum(np.searchsorted(dk, keys), dk.size - 1)
        keys = keys[dk[pos] != keys]
    return _sorted_unique(np.concatenate([keys, ik]))


def batch_stream(n: int, keys: np.ndarray, sizes, ins_frac: float, seed: int,
                 sequential: bool = True, ins_weighting: str = "degree"):
    """A list of (ins, dels) batches.

    ``sequential``: each batch is drawn against the graph left by the previous
    ones.  Otherwise every batch is drawn against the same base graph.
    """
    out = []
    cur = np.asarray(keys, dtype=np.uint64)
    deg = _degrees(n, cur)
    for i, sz in enumerate(sizes):
        n_ins = int(round(sz * ins_frac))
        n_del = int(sz) - n_ins
        ins, dels = random_batch(n, cur, n_ins, n_del, _substream(seed, f"batch{i}"),
                                 ins_weighting=ins_weighting, deg=deg)
        out.append((ins, dels))
        if sequential:
            cur = apply_batch_keys(cur, ins, dels)
            deg = _degrees(n, cur)
    return out


def log_uniform_sizes(count: int, lo: int, hi: int, seed: int) -> list[int]:
    r = uniform01(_substream(seed, "sizes"), 0, count)
    return [int(round(math.exp(math.log(lo) + x * (math.log(hi) - math.log(lo))))) for x in r]


# The five workloads (stand-ins for the paper's SNAP graphs, Table 1; batch
# recipe of Sec. 5).  Graph seed 0; batch seed 1 + workload index.
WORKLOADS = {
    "c1": dict(kind="er", n=2000, m=20000, seed=0,
               desc="ER n=2,000 m=20,000; one batch of 200 deletions + 200 insertions"),
    "c2": dict(kind="cl", n=7000, m=100000, gamma=2.1, dmax=1000, seed=0,
               desc="Chung-Lu n=7,000 m=100,000 gamma=2.1 dmax=1,000; sequential 1k/10k batches"),
    "c3": dict(kind="cl", n=1600000, m=30000000, gamma=2.3, dmax=10000, seed=0,
               desc="Chung-Lu n=1.6M m=30M gamma=2.3 dmax=10,000; 100k batches 60% ins / 40% del"),
    "c4": dict(kind="cl", n=2400000, m=5000000, gamma=1.8, dmax=100000, seed=0,
               desc="Chung-Lu n=2.4M m=5M gamma=1.8 dmax=100,000; 64 independent batches of 10..50k"),
}


def c5_graph_params():
    """The eight resident graphs of the serving workload."""
    ns = np.exp(np.linspace(math.log(100_000), math.log(4_800_000), 8))
    ms = np.exp(np.linspace(math.log(1_000_000), math.log(69_000_000), 8))
    gs = np.linspace(2.0, 2.4, 8)
    return [dict(kind="cl", n=int(round(a)), m=int(round(b)), gamma=float(g),
                 dmax=float(math.sqrt(2 * b)), seed=0) for a, b, g in zip(ns, ms, gs)]


def workload_graph(name_or_params) -> tuple[int, np.ndarray]:
    """(n, sorted canonical keys) of a named workload's graph."""
    p = WORKLOADS[name_or_params] if isinstance(name_or_params, str) else name_or_params
    if p["kind"] == "er":
        return p["n"], er_graph(p["n"], p["m"], p["seed"])
    return p["n"], chung_lu_graph(p["n"], p["m"], p["gamma"], p["dmax"], p["seed"])
