"""ctypes front end of the plain C oracle (``gc_oracle.c``).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Functions here take
numpy CSR arrays (``row_ptr`` of n+1 offsets, ``col`` of int32 neighbours,
rows sorted) and return Python ints, so expected values never pass through
the CUDA library.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

GRAPHLETS = ("3-path", "3-star", "4-cycle", "tailed-triangle", "diamond", "4-clique")
SUMS = ("P", "S", "TT", "D", "K", "Q")


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (plain -O2, single-threaded)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            I64 = ctypes.c_int64
            lib.or_sums_literal.argtypes = [I64, i64p, i32p, ctypes.c_int, i64p]
            lib.or_sums_oriented.argtypes = [I64, i64p, i32p, i64p]
            lib.or_counts3.argtypes = [I64, i64p, i32p, i64p]
            lib.or_counts_from_sums.argtypes = [i64p, i64p]
            lib.or_counts_from_sums.restype = None
            lib.or_normalize.argtypes = [I64, i64p, i32p, i32p, I64, i32p, I64, u64p, i64p, u64p, i64p, i64p]
            lib.or_fdgc_step.argtypes = [I64, i64p, i32p, i32p, I64, i32p, I64, ctypes.c_int, ctypes.c_int,
                                         u64p, i64p, i64p, i64p, i64p, i64p, i64p, i32p, i32p]
            _lib = lib
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _csr(row_ptr, col):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    c = np.ascontiguousarray(col, dtype=np.int32)
    if c.size == 0:
        c = np.zeros(1, dtype=np.int32)
    return rp, c


def _pairs(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1, 2))
    buf = a if a.size else np.zeros((1, 2), dtype=np.int32)
    return buf, a.shape[0]


def sums_literal(row_ptr, col, with_ic4: bool = False) -> list[int]:
    """[P, S, TT, D, K, Q] (+ induced 4-cycles if ``with_ic4``) by plain definitions."""
    rp, c = _csr(row_ptr, col)
    out = np.zeros(7, dtype=np.int64)
    rc = _load().or_sums_literal(rp.size - 1, _p(rp, ctypes.c_int64), _p(c, ctypes.c_int32),
                                 1 if with_ic4 else 0, _p(out, ctypes.c_int64))
    if rc != 0:
        raise RuntimeError(f"or_sums_literal failed ({rc})")
    return [int(x) for x in (out if with_ic4 else out[:6])]


def sums_oriented(row_ptr, col) -> list[int]:
    """[P, S, TT, D, K, Q] by degree-oriented listing (large graphs)."""
    rp, c = _csr(row_ptr, col)
    out = np.zeros(6, dtype=np.int64)
    rc = _load().or_sums_oriented(rp.size - 1, _p(rp, ctypes.c_int64), _p(c, ctypes.c_int32), _p(out, ctypes.c_int64))
    if rc != 0:
        raise RuntimeError(f"or_sums_oriented failed ({rc})")
    return [int(x) for x in out]


def counts_from_sums(sums) -> list[int]:
    s = np.asarray(sums[:6], dtype=np.int64)
    out = np.zeros(6, dtype=np.int64)
    _load().or_counts_from_sums(_p(s, ctypes.c_int64), _p(out, ctypes.c_int64))
    return [int(x) for x in out]


def static_counts(row_ptr, col, variant: str = "oriented") -> list[int]:
    """Induced graphlet counts [g1..g6] of a whole graph."""
    s = sums_literal(row_ptr, col) if variant == "literal" else sums_oriented(row_ptr, col)
    return counts_from_sums(s)


def static_counts3(row_ptr, col) -> list[int]:
    """Induced 3-vertex counts [2-paths, triangles] of a whole graph (the
    by-product of the per-edge triangle counts and degrees, Sec. 3)."""
    rp, c = _csr(row_ptr, col)
    n = rp.size - 1
    out = np.zeros(2, np.int64)
    if _load().or_counts3(n, _p(rp, ctypes.c_int64), _p(c, ctypes.c_int32), _p(out, ctypes.c_int64)) != 0:
        raise RuntimeError("or_counts3 failed")
    return [int(x) for x in out]


ALL_TYPES = ("3-path", "3-star", "4-cycle", "tailed-triangle", "diamond", "4-clique",
             "triangle+isolated", "2-path+isolated", "two-disjoint-edges", "edge+2-isolated", "empty")


def counts_all(row_ptr, col) -> list[int]:
    """Induced counts of all eleven 4-vertex graphs: the six connected
    graphlets of Problem 1, then the five disconnected ones, as Python ints
    (they exceed 64 bits).  The disconnected counts follow from counting
    pairs (a sub-structure, a 4-set) two ways: every triangle with a fourth
    vertex, every 2-path with a fourth vertex, every pair of vertex-disjoint
    edges, and every edge with two more vertices lies in exactly one 4-set,
    and each induced type holds a fixed number of each; the empty sets are
    the rest of C(n, 4)."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    n = rp.size - 1
    m = int(rp[-1]) // 2
    deg = np.diff(rp)
    g1, g2, g3, g4, g5, g6 = static_counts(row_ptr, col)
    p2, tri = static_counts3(row_ptr, col)
    wedges = sum(int(d) * (int(d) - 1) // 2 for d in deg)   # non-induced 2-paths
    assert wedges == p2 + 3 * tri
    c = math.comb
    t_iso = tri * (n - 3) - g4 - 2 * g5 - 4 * g6
    w_iso = wedges * (n - 3) - (2 * g1 + 3 * g2 + 4 * g3 + 5 * g4 + 8 * g5 + 12 * g6 + 3 * t_iso)
    two = (c(m, 2) - wedges) - (g1 + 2 * g3 + g4 + 2 * g5 + 3 * g6)
    one = m * c(n - 2, 2) - (2 * (w_iso + two) + 3 * (t_iso + g1 + g2) + 4 * (g3 + g4) + 5 * g5 + 6 * g6)
    empty = c(n, 4) - (one + w_iso + two + t_iso + g1 + g2 + g3 + g4 + g5 + g6)
    return [g1, g2, g3, g4, g5, g6, t_iso, w_iso, two, one, empty]


def vertex_orbits(row_ptr, col) -> list[list[int]]:
    """Per vertex v, how many induced connected 4-vertex graphlets hold v in
    each orbit 4..14 (11 columns: 3-path end, middle; 3-star leaf, centre;
    4-cycle; tailed triangle tail end, other triangle corner, attachment;
    diamond degree-2, degree-3 corner; 4-clique).  Plain Python over
    adjacency sets, for graphs of a few thousand vertices.

    The containment identity behind the global counts holds per vertex and
    role: a 4-set S of induced type g holding v in orbit o contains a fixed
    number of copies of each subgraph H with v in each role r, so the
    non-induced role counts N_r(v) = sum_o M[r][o] I_o(v), and M is
    triangular.  The role counts (d degrees, t_e triangles per edge, tri(v)
    triangles at v, s(u) = sum_{w in N(u)} (d_w - 1)):
      3-path end: paths v-u-w-x; middle: sum_u ((d_v-1)(d_u-1) - t_vu)
      3-star leaf: sum_u C(d_u - 1, 2); centre: C(d_v, 3)
      4-cycle: pairs of common neighbours of v and an opposite corner w
      tailed triangle tail end: sum_z (tri(z) - t_vz); other corner:
        sum_y t_vy (d_y - 2); attachment: tri(v)(d_v - 2)
      diamond degree-2 corner: sum over triangles {v, a, b} of t_ab - 1;
        degree-3 corner: sum_u C(t_vu, 2)
      4-clique: cliques through v."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    c = np.asarray(col, dtype=np.int64)
    n = rp.size - 1
    N = [set(int(x) for x in c[rp[v]:rp[v + 1]]) for v in range(n)]
    d = [len(N[v]) for v in range(n)]
    t = {}
    for v in range(n):
        for u in N[v]:
            if u > v:
                t[(v, u)] = t[(u, v)] = len(N[v] & N[u])
    tri = [sum(t[(v, u)] for u in N[v]) // 2 for v in range(n)]
    out = []
    for v in range(n):
        p_end = 0
        for u in N[v]:
            for w in N[u]:
                if w != v:
                    p_end += len(N[w] - {u, v})   # x in N(w), x != u, x != v
        p_mid = sum((d[v] - 1) * (d[u] - 1) - t[(v, u)] for u in N[v])
        s_leaf = sum((d[u] - 1) * (d[u] - 2) // 2 for u in N[v])
        s_ctr = d[v] * (d[v] - 1) * (d[v] - 2) // 6
        cnt = {}
        for a in N[v]:
            for w in N[a]:
                if w != v:
                    cnt[w] = cnt.get(w, 0) + 1
        c4 = sum(x * (x - 1) // 2 for x in cnt.values())
        tt_tail = sum(tri[z] - t[(v, z)] for z in N[v])
        tt_oth = sum(t[(v, y)] * (d[y] - 2) for y in N[v])
        tt_att = tri[v] * (d[v] - 2)
        d3 = sum(t[(v, u)] * (t[(v, u)] - 1) // 2 for u in N[v])
        d2 = 0
        k4 = 0
        nb = sorted(N[v])
        for i, a in enumerate(nb):
            for b in nb[i + 1:]:
                if b in N[a]:
                    d2 += t[(a, b)] - 1
                    k4 += sum(1 for z in N[a] & N[b] & N[v] if z > b)
        # invert the role containment (triangular)
        o14 = k4
        o13 = d3 - 3 * o14
        o12 = d2 - 3 * o14
        o11 = tt_att - 2 * o13 - 3 * o14
        o10 = tt_oth - 2 * o12 - 2 * o13 - 6 * o14
        o9 = tt_tail - 2 * o12 - 3 * o14
        o8 = c4 - o12 - o13 - 3 * o14
        o7 = s_ctr - o11 - o13 - o14
        o6 = s_leaf - o9 - o10 - 2 * o12 - o13 - 3 * o14
        o5 = p_mid - 2 * o8 - o10 - 2 * o11 - 2 * o12 - 4 * o13 - 6 * o14
        o4 = p_end - 2 * o8 - 2 * o9 - o10 - 4 * o12 - 2 * o13 - 6 * o14
        out.append([o4, o5, o6, o7, o8, o9, o10, o11, o12, o13, o14])
    return out


def vertex_counts(row_ptr, col) -> list[list[int]]:
    """Per vertex v, the induced connected 4-vertex graphlets [g1..g6] that
    contain v: the sums of its orbits per graphlet."""
    return [[o[0] + o[1], o[2] + o[3], o[4], o[5] + o[6] + o[7], o[8] + o[9], o[10]]
            for o in vertex_orbits(row_ptr, col)]


EDGE_ORBITS = ("3-path end", "3-path middle", "3-star", "4-cycle", "tailed-triangle tail",
               "tailed-triangle opposite", "tailed-triangle attachment", "diamond outer", "diamond chord",
               "4-clique")


def edge_orbits(row_ptr, col, pairs=None):
    """Per edge {u, v}, how many induced connected 4-vertex graphlets hold it
    in each edge orbit (10 columns, EDGE_ORBITS: 3-path end, middle edge;
    3-star edge; 4-cycle edge; tailed triangle tail, triangle edge opposite
    the attachment, triangle edge at the attachment; diamond outer edge,
    chord; 4-clique edge).  Returns (edges, rows) over the sorted edges
    u < v, or over ``pairs`` (edges of the graph) when given; adjacency sets
    are built only for the rows touched, so a sample of edges of a large
    graph costs little.

    The containment identity behind the global counts (Sec. 3) holds per
    edge and role: an induced graphlet holding {u, v} in orbit o contains a
    fixed number of non-induced copies of each connected 4-vertex subgraph H
    that hold {u, v} in each edge role of H, so N_r(uv) = sum_o M[r][o]
    I_o(uv) with M triangular.  The non-induced copies are counted here
    directly by walking the neighbourhoods of u and v:
      3-path end: paths u-v-w-z and v-u-w-z; middle: paths x-u-v-y
      3-star: C(d_u - 1, 2) + C(d_v - 1, 2)
      4-cycle: cycles u-v-w-z-u
      tailed triangle tail: triangles at u without v, and at v without u;
        opposite: each common neighbour w with a further neighbour of w;
        attachment: each common neighbour w with a further neighbour of u
        or of v
      diamond outer: each common neighbour w with a vertex adjacent to u
        and w (chord uw) or to v and w (chord vw); chord: pairs of common
        neighbours
      4-clique: adjacent pairs of common neighbours."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    c = np.asarray(col, dtype=np.int64)
    cache = {}

    def N(x):
        s = cache.get(x)
        if s is None:
            s = cache[x] = set(int(y) for y in c[rp[x]:rp[x + 1]])
        return s

    if pairs is None:
        n = rp.size - 1
        pairs = [(u, v) for u in range(n) for v in sorted(N(u)) if v > u]
    keys = []
    rows = []
    for a, b in pairs:
        u, v = (int(a), int(b)) if a < b else (int(b), int(a))
        Nu, Nv = N(u), N(v)
        if v not in Nu:
            raise ValueError(f"({u}, {v}) is not an edge")
        T = Nu & Nv
        Nu_v, Nv_u = Nu - {v}, Nv - {u}   # (no set of a hub is copied per neighbour below)
        p_end = sum(len(N(w) - {u, v}) for w in Nv_u) + sum(len(N(w) - {u, v}) for w in Nu_v)
        p_mid = sum(len(Nv_u) - (x in Nv_u) for x in Nu_v)            # y in N(v) - {u, x}
        star = math.comb(len(Nu) - 1, 2) + math.comb(len(Nv) - 1, 2)
        cyc = sum(len((N(w) & Nu) - {v}) for w in Nv_u)
        tail = sum(len(N(x) & Nu_v) for x in Nu_v) // 2 + sum(len(N(x) & Nv_u) for x in Nv_u) // 2
        opp = sum(len(N(w) - {u, v}) for w in T)
        att = sum((len(Nu_v) - (w in Nu_v)) + (len(Nv_u) - (w in Nv_u)) for w in T)   # N(u) - {v, w} and N(v) - {u, w}
        outer = sum(len((Nu & N(w)) - {v}) + len((Nv & N(w)) - {u}) for w in T)
        chord = math.comb(len(T), 2)
        k4 = sum(len(N(w) & T) for w in T) // 2
        # invert the edge-role containment (triangular)
        i9 = k4
        i8 = chord - i9
        i7 = outer - 4 * i9
        i6 = att - 4 * i8 - i7 - 4 * i9
        i5 = opp - i7 - 2 * i9
        i4 = tail - i7 - 2 * i9
        i3 = cyc - i7 - 2 * i9
        i2 = star - i6 - i4 - 2 * i8 - i7 - 2 * i9
        i1 = p_mid - i3 - i6 - 2 * i8 - i7 - 2 * i9
        i0 = p_end - 2 * i3 - 2 * i5 - 2 * i4 - 3 * i7 - 4 * i9
        keys.append((u, v))
        rows.append([i0, i1, i2, i3, i4, i5, i6, i7, i8, i9])
    return keys, rows


def normalize(row_ptr, col, ins, dels):
    """Normalised batch: (A keys, D keys, stats) or raises ValueError."""
    rp, c = _csr(row_ptr, col)
    ib, ni = _pairs(ins)
    db, nd = _pairs(dels)
    A = np.zeros(max(ni, 1), dtype=np.uint64)
    D = np.zeros(max(nd, 1), dtype=np.uint64)
    na = ctypes.c_int64(0)
    ndd = ctypes.c_int64(0)
    st = np.zeros(8, dtype=np.int64)
    rc = _load().or_normalize(rp.size - 1, _p(rp, ctypes.c_int64), _p(c, ctypes.c_int32),
                              _p(ib, ctypes.c_int32), ni, _p(db, ctypes.c_int32), nd,
                              _p(A, ctypes.c_uint64), ctypes.byref(na), _p(D, ctypes.c_uint64), ctypes.byref(ndd),
                              _p(st, ctypes.c_int64))
    if rc == -1:
        raise ValueError("invalid batch (self-loop or vertex out of range)")
    if rc != 0:
        raise RuntimeError(f"or_normalize failed ({rc})")
    return A[: na.value].copy(), D[: ndd.value].copy(), [int(x) for x in st]


def fdgc_step(row_ptr, col, ins, dels, F, hops: int = 3, variant: str = "oriented", want_region: bool = False):
    """One step of Algorithm 2.  Returns a dict with the new F, C_a, C_b, the
    sums of G_a and G_b, info and the committed CSR."""
    rp, c = _csr(row_ptr, col)
    n = rp.size - 1
    ib, ni = _pairs(ins)
    db, nd = _pairs(dels)
    Fa = np.asarray([int(x) & 0xFFFFFFFFFFFFFFFF for x in F], dtype=np.uint64)
    Ca = np.zeros(6, dtype=np.int64)
    Cb = np.zeros(6, dtype=np.int64)
    sa = np.zeros(6, dtype=np.int64)
    sb = np.zeros(6, dtype=np.int64)
    info = np.zeros(8, dtype=np.int64)
    new_rp = np.zeros(n + 1, dtype=np.int64)
    new_col = np.zeros(int(rp[-1]) + 2 * ni + 1, dtype=np.int32)
    region = np.zeros(max(n, 1), dtype=np.int32)
    rc = _load().or_fdgc_step(n, _p(rp, ctypes.c_int64), _p(c, ctypes.c_int32),
                              _p(ib, ctypes.c_int32), ni, _p(db, ctypes.c_int32), nd,
                              int(hops), 0 if variant == "literal" else 1,
                              _p(Fa, ctypes.c_uint64), _p(Ca, ctypes.c_int64), _p(Cb, ctypes.c_int64),
                              _p(sa, ctypes.c_int64), _p(sb, ctypes.c_int64), _p(info, ctypes.c_int64),
                              _p(new_rp, ctypes.c_int64), _p(new_col, ctypes.c_int32),
                              _p(region, ctypes.c_int32) if want_region else None)
    if rc == -1:
        raise ValueError("invalid batch (self-loop or vertex out of range)")
    if rc != 0:
        raise RuntimeError(f"or_fdgc_step failed ({rc})")
    out = dict(F=[int(x) for x in Fa], Ca=[int(x) for x in Ca], Cb=[int(x) for x in Cb],
               sums_a=[int(x) for x in sa], sums_b=[int(x) for x in sb],
               n_ins=int(info[0]), n_del=int(info[1]), region_vertices=int(info[2]),
               edges_a=int(info[3]), edges_b=int(info[4]), cancelled=int(info[5]),
               noops=int(info[6]), repeats=int(info[7]),
               row_ptr=new_rp, col=new_col[: int(new_rp[-1])].copy())
    if want_region:
        out["region"] = region[: int(info[2])].copy()
    return out


class OracleGraph:
    """A graph under a stream of batches, maintained by the oracle alone."""

    def __init__(self, row_ptr, col, variant: str = "oriented", hops: int = 3):
        self.row_ptr = np.asarray(row_ptr, dtype=np.int64).copy()
        self.col = np.asarray(col, dtype=np.int32).copy()
        self.variant = variant
        self.hops = hops
        self.F = [x & 0xFFFFFFFFFFFFFFFF for x in static_counts(self.row_ptr, self.col, variant)]

    def apply(self, ins, dels):
        r = fdgc_step(self.row_ptr, self.col, ins, dels, self.F, self.hops, self.variant)
        self.F = r["F"]
        self.row_ptr, self.col = r["row_ptr"], r["col"]
        return r
