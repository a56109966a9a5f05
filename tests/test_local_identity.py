"""The identity behind the edge-local delta, checked on the CPU.

The CUDA library can update the counts of a batch from the terms that the
batch can change: per-edge terms of the edges with an endpoint in V_X (the
endpoints of the changed pairs), per-vertex terms of V_X, and the 4-cliques
and 4-cycles that hold a changed pair, each counted once at its smallest
changed pair.  This file restates that rule in plain Python and checks it
against the oracle's full recount (Sec. 3 closed forms; the delta of
Lemma 2) on small random graphs and batches, including batches whose pairs
share cliques and cycles.  It pins the reasoning, not the kernels (the GPU
parity tests pin those).
"""
import itertools

import numpy as np

import oracle
from gc_testutil import csr_from_edges


def _adj(n, edges):
    a = [set() for _ in range(n)]
    for u, v in edges:
        a[u].add(v)
        a[v].add(u)
    return a


def _c2(x):
    return x * (x - 1) // 2


def _c3(x):
    return x * (x - 1) * (x - 2) // 6


def local_delta_sums(n, edges_b, ins, dels):
    """Delta of the non-induced sums (P, S, TT, D, K, Q) by the local rule."""
    Gb = _adj(n, edges_b)
    eb = {(min(u, v), max(u, v)) for u, v in edges_b}
    A = {(min(u, v), max(u, v)) for u, v in ins} - eb
    D = {(min(u, v), max(u, v)) for u, v in dels} & eb
    both = A & D
    A, D = A - both, D - both
    Ga = _adj(n, (eb - D) | A)
    VX = {x for p in A | D for x in p}
    delta = [0] * 6
    for G, sign in ((Ga, 1), (Gb, -1)):
        d = [len(G[v]) for v in range(n)]
        P = S = TT2 = Dm = 0
        for u in VX:
            S += _c3(d[u])
            for w in G[u]:
                if w in VX and w < u:
                    continue
                t = len(G[u] & G[w])
                P += (d[u] - 1) * (d[w] - 1) - t
                TT2 += t * (d[u] + d[w] - 4)
                Dm += _c2(t)
        delta[0] += sign * P
        delta[1] += sign * S
        delta[2] += sign * TT2
        delta[3] += sign * Dm
    # subgraphs holding a changed pair, at their smallest such pair
    for G, X, sign in ((Ga, A, 1), (Gb, D, -1)):
        for p in sorted(X):
            u, v = p
            T = sorted(G[u] & G[v])
            for w, z in itertools.combinations(T, 2):
                if z in G[w]:
                    es = [(min(a, b), max(a, b)) for a, b in ((u, w), (v, w), (u, z), (v, z), (w, z))]
                    if all(not (e in X and e < p) for e in es):
                        delta[4] += sign
            for w in G[v] - {u}:
                for z in (G[u] & G[w]) - {v}:
                    es = [(min(a, b), max(a, b)) for a, b in ((v, w), (w, z), (z, u))]
                    if all(not (e in X and e < p) for e in es):
                        delta[5] += sign
    delta[2] //= 2
    return delta, (eb - D) | A


def _sums(n, edges):
    rp, col = csr_from_edges(n, edges)
    return [int(x) for x in oracle.sums_literal(rp, col)]


def test_local_rule_equals_full_recount():
    rng = np.random.default_rng(31)
    for trial in range(60):
        n = int(rng.integers(5, 26))
        p = float(rng.uniform(0.1, 0.7))
        edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p]
        all_pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
        k = int(rng.integers(1, 9))
        pick = rng.choice(len(all_pairs), size=min(2 * k, len(all_pairs)), replace=False)
        ins = [all_pairs[i] for i in pick[:k]]
        dels = [all_pairs[i] for i in pick[k:]]
        if trial % 3 == 0 and edges:  # deletions that share cliques and cycles
            dels = [edges[i] for i in rng.choice(len(edges), size=min(k, len(edges)), replace=False)]
        delta, after = local_delta_sums(n, edges, ins, dels)
        before_s = _sums(n, edges)
        after_s = _sums(n, sorted(after))
        assert delta == [a - b for a, b in zip(after_s, before_s)], trial


def test_local_rule_on_dense_cliques():
    # every 4-clique and 4-cycle of K_9 holds several changed pairs at once
    n = 9
    full = [(a, b) for a in range(n) for b in range(a + 1, n)]
    rng = np.random.default_rng(5)
    for trial in range(10):
        drop = {full[i] for i in rng.choice(len(full), size=12, replace=False)}
        base = [e for e in full if e not in drop]
        delta, after = local_delta_sums(n, base, sorted(drop), [])
        assert delta == [a - b for a, b in zip(_sums(n, sorted(after)), _sums(n, base))]
        delta, after = local_delta_sums(n, full, [], sorted(drop))
        assert delta == [a - b for a, b in zip(_sums(n, sorted(after)), _sums(n, full))]


def local_delta_sums_t2(n, edges_b, ins, dels):
    """The same delta with maintained triangle sums T2(x) = sum of t_e at x:
    only the triangles through changed pairs are listed (once, at their
    smallest changed pair), TT in vertex form, D on the edges whose t
    changes; P from degree products at V_X and the change of sum t."""
    Gb = _adj(n, edges_b)
    eb = {(min(u, v), max(u, v)) for u, v in edges_b}
    A = {(min(u, v), max(u, v)) for u, v in ins} - eb
    D = {(min(u, v), max(u, v)) for u, v in dels} & eb
    both = A & D
    A, D = A - both, D - both
    ea = (eb - D) | A
    Ga = _adj(n, ea)
    X = A | D
    VX = {x for p in X for x in p}
    T2b = [sum(len(Gb[x] & Gb[w]) for w in Gb[x]) for x in range(n)]
    U = [Ga[x] | Gb[x] for x in range(n)]
    dt = {}      # change of t per edge
    dtri2 = {}   # change of T2 per vertex
    for p in sorted(X):
        a, b = p
        for w in sorted(U[a] & U[b]):
            es = [(min(a, w), max(a, w)), (min(b, w), max(b, w))]
            if any(e in X and e < p for e in es):
                continue
            tri = [p] + es
            d = int(all(e in ea for e in tri)) - int(all(e in eb for e in tri))
            for e in tri:
                dt[e] = dt.get(e, 0) + d
            for x in (a, b, w):
                dtri2[x] = dtri2.get(x, 0) + 2 * d
    s3 = sum(dt.values())
    delta = [0] * 6
    da = [len(Ga[v]) for v in range(n)]
    db = [len(Gb[v]) for v in range(n)]
    at_vx = {e for e in ea | eb if e[0] in VX or e[1] in VX}
    for e in at_vx:
        u, w = e
        if e in ea:
            delta[0] += (da[u] - 1) * (da[w] - 1)
        if e in eb:
            delta[0] -= (db[u] - 1) * (db[w] - 1)
        d = dt.get(e, 0)
        if e in ea and e in eb:
            tb = len(Gb[u] & Gb[w])
            delta[3] += _c2(tb + d) - _c2(tb)
        elif e in ea:
            delta[3] += _c2(d)
        else:
            delta[3] -= _c2(-d)
    delta[0] -= s3
    tt2 = 0
    for x in VX | set(dtri2):
        tt2 += (T2b[x] + dtri2.get(x, 0)) * (da[x] - 2) - T2b[x] * (db[x] - 2)
        if x in VX:
            delta[1] += _c3(da[x]) - _c3(db[x])
    delta[2] = tt2 // 2
    full, _ = local_delta_sums(n, edges_b, ins, dels)   # K and Q as in the first form
    delta[4], delta[5] = full[4], full[5]
    T2a = [sum(len(Ga[x] & Ga[w]) for w in Ga[x]) for x in range(n)]
    assert all(T2a[x] == T2b[x] + dtri2.get(x, 0) for x in range(n))
    return delta, ea


def test_triangle_sum_form_equals_full_recount():
    rng = np.random.default_rng(77)
    for trial in range(60):
        n = int(rng.integers(5, 26))
        p = float(rng.uniform(0.1, 0.8))
        edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p]
        all_pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
        k = int(rng.integers(1, 10))
        pick = rng.choice(len(all_pairs), size=min(2 * k, len(all_pairs)), replace=False)
        ins = [all_pairs[i] for i in pick[:k]]
        dels = [all_pairs[i] for i in pick[k:]]
        if trial % 3 == 0 and edges:
            dels = [edges[i] for i in rng.choice(len(edges), size=min(k, len(edges)), replace=False)]
        delta, after = local_delta_sums_t2(n, edges, ins, dels)
        assert delta == [a - b for a, b in zip(_sums(n, sorted(after)), _sums(n, edges))], trial
