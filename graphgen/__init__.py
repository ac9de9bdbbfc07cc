"""Seeded synthetic graph generators and CSR plumbing.

This module produces the inputs shared by the CPU oracle, the tests and the
benchmark.  It holds none of the eigensolver arithmetic: it only builds simple
undirected graphs (Section 2 of the paper: no multi-edges, no self-loops,
positive weights) and stores their adjacency matrix A in CSR form with both
triangles present.

Every generator is deterministic in its seed (numpy PCG64).  The synthetic
families stand in for the paper's four networks (Section 4, Table 1), which are
not available here:

* ``ba_graph``      -- Barabasi-Albert preferential attachment
  (protein-sized stand-in, n=2,000, m=2).
* ``chung_lu``      -- power-law expected-degree graph, fast edge-sampling
  variant (internet/www/dblp-shaped stand-ins), largest component kept,
  nodes relabelled at random so hubs are not contiguous.
* ``grid_graph``    -- 2-D grid P_a x P_b.
* closed-form families (path, cycle, star, complete, complete bipartite,
  hypercube) whose Laplacian spectra are known exactly.
"""
from __future__ import annotations

import hashlib
import math
from dataclasses import dataclass

import numpy as np


@dataclass
class CSRGraph:
    """Adjacency matrix of a simple undirected graph, both triangles stored.

    rowptr  int64 [n+1], colidx int32 [nnz] sorted and unique within a row,
    weights float64 [nnz] or None for unit weights.  nnz = 2|E|.
    """

    n: int
    rowptr: np.ndarray
    colidx: np.ndarray
    weights: np.ndarray | None = None
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    @property
    def n_edges(self) -> int:
        return self.nnz // 2

    def degree_counts(self) -> np.ndarray:
        return np.diff(self.rowptr)

    def digest(self) -> str:
        h = hashlib.sha256()
        h.update(np.int64(self.n).tobytes())
        h.update(np.ascontiguousarray(self.rowptr, dtype=np.int64).tobytes())
        h.update(np.ascontiguousarray(self.colidx, dtype=np.int32).tobytes())
        if self.weights is not None:
            h.update(np.ascontiguousarray(self.weights, dtype=np.float64).tobytes())
        return h.hexdigest()[:16]


# ----------------------------------------------------------------------------
# CSR construction
# ----------------------------------------------------------------------------

def csr_from_edges(n: int, src, dst, weights=None, name: str = "") -> CSRGraph:
    """Symmetrise an edge list, drop self-loops and duplicates, build CSR.

    Duplicate edges keep the first weight seen (the graph is simple).
    """
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    w = None if weights is None else np.asarray(weights, dtype=np.float64)[keep]
    lo = np.minimum(src, dst)
    hi = np.maximum(src, dst)
    key = lo * n + hi
    key, first = np.unique(key, return_index=True)
    lo, hi = key // n, key % n
    if w is not None:
        w = w[first]
    rows = np.concatenate([lo, hi])
    cols = np.concatenate([hi, lo])
    ww = None if w is None else np.concatenate([w, w])
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    if ww is not None:
        ww = ww[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSRGraph(n, rowptr, cols.astype(np.int32), ww, name)


def edges_of(g: CSRGraph):
    """Upper-triangle edge list (i < j) with weights (or None)."""
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rowptr))
    cols = g.colidx.astype(np.int64)
    up = rows < cols
    w = None if g.weights is None else g.weights[up]
    return rows[up], cols[up], w


def components(g: CSRGraph) -> np.ndarray:
    """Connected-component label of every node (label = smallest node id)."""
    parent = np.arange(g.n, dtype=np.int64)
    s, d, _ = edges_of(g)
    # Vectorised label propagation with pointer jumping.
    while True:
        ps, pd = parent[s], parent[d]
        m = np.minimum(ps, pd)
        changed = False
        upd = m < parent[s]
        if upd.any():
            np.minimum.at(parent, s[upd], m[upd])
            changed = True
        upd = m < parent[d]
        if upd.any():
            np.minimum.at(parent, d[upd], m[upd])
            changed = True
        while True:
            pp = parent[parent]
            if np.array_equal(pp, parent):
                break
            parent = pp
        if not changed:
            break
    return parent


def induced_subgraph(g: CSRGraph, nodes: np.ndarray, name: str = "") -> CSRGraph:
    nodes = np.asarray(nodes, dtype=np.int64)
    newid = -np.ones(g.n, dtype=np.int64)
    newid[nodes] = np.arange(nodes.size)
    s, d, w = edges_of(g)
    keep = (newid[s] >= 0) & (newid[d] >= 0)
    return csr_from_edges(nodes.size, newid[s[keep]], newid[d[keep]],
                          None if w is None else w[keep], name or g.name)


def largest_component(g: CSRGraph) -> CSRGraph:
    lab = components(g)
    vals, counts = np.unique(lab, return_counts=True)
    big = vals[np.argmax(counts)]
    nodes = np.nonzero(lab == big)[0]
    if nodes.size == g.n:
        return g
    return induced_subgraph(g, nodes, g.name)


def relabel(g: CSRGraph, perm: np.ndarray) -> CSRGraph:
    """Node i of ``g`` becomes node perm[i]."""
    s, d, w = edges_of(g)
    return csr_from_edges(g.n, perm[s], perm[d], w, g.name)


def disjoint_union(*gs: CSRGraph) -> CSRGraph:
    srcs, dsts, ws, off = [], [], [], 0
    weighted = any(x.weights is not None for x in gs)
    for x in gs:
        s, d, w = edges_of(x)
        srcs.append(s + off)
        dsts.append(d + off)
        ws.append(np.ones(s.size) if w is None else w)
        off += x.n
    return csr_from_edges(off, np.concatenate(srcs), np.concatenate(dsts),
                          np.concatenate(ws) if weighted else None, "union")


def with_random_weights(g: CSRGraph, seed: int, lo: float = 0.5, hi: float = 4.0) -> CSRGraph:
    """Same pattern, symmetric positive weights drawn uniformly in [lo, hi)."""
    rng = np.random.default_rng(seed)
    s, d, _ = edges_of(g)
    return csr_from_edges(g.n, s, d, rng.uniform(lo, hi, size=s.size), g.name + "+w")


# ----------------------------------------------------------------------------
# Random graph families
# ----------------------------------------------------------------------------

def ba_graph(n: int, m: int, seed: int) -> CSRGraph:
    """Barabasi-Albert graph: start from K_{m+1}; each new node attaches to m
    distinct existing nodes chosen with probability proportional to degree
    (uniform draws from the running endpoint list).  Connected by construction."""
    rng = np.random.default_rng(seed)
    m0 = m + 1
    src, dst = [], []
    for i in range(m0):
        for j in range(i + 1, m0):
            src.append(i)
            dst.append(j)
    ends = np.empty(2 * (m0 * (m0 - 1) // 2 + (n - m0) * m), dtype=np.int64)
    ne = 0
    for a, b in zip(src, dst):
        ends[ne] = a
        ends[ne + 1] = b
        ne += 2
    src = list(src)
    dst = list(dst)
    u = rng.random(size=(n, 4 * m))
    for v in range(m0, n):
        chosen = []
        t = 0
        row = u[v]
        while len(chosen) < m:
            if t < row.size:
                x = row[t]
            else:
                x = rng.random()
            t += 1
            c = int(ends[int(x * ne)])
            if c not in chosen:
                chosen.append(c)
        for c in chosen:
            src.append(v)
            dst.append(c)
            ends[ne] = v
            ends[ne + 1] = c
            ne += 2
    return csr_from_edges(n, np.array(src), np.array(dst), None, f"ba(n={n},m={m},seed={seed})")


def chung_lu_weights(n: int, gamma: float, dbar: float, cap: float | None) -> np.ndarray:
    """Expected degrees w_i = c (i + i0)^(-1/(gamma-1)), i = 0..n-1, with c and
    i0 chosen so that mean(w) = dbar and max(w) = w_0 = cap."""
    if cap is None:
        cap = math.sqrt(n * dbar)
    alpha = 1.0 / (gamma - 1.0)
    idx = np.arange(n, dtype=np.float64)

    def mean_for(i0):
        # c fixed by w_0 = cap
        c = cap * i0 ** alpha
        return np.mean(c * (idx + i0) ** (-alpha))

    lo, hi = 1e-6, 1e12
    # mean_for is increasing in i0 (flatter distribution); bisection in log space
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if mean_for(mid) < dbar:
            lo = mid
        else:
            hi = mid
    i0 = math.sqrt(lo * hi)
    c = cap * i0 ** alpha
    return c * (idx + i0) ** (-alpha)


def chung_lu(n: int, gamma: float, dbar: float, seed: int, cap: float | None = None,
             keep_lcc: bool = True) -> CSRGraph:
    """Power-law expected-degree graph (fast Chung-Lu edge sampling).

    Draw M ~ Poisson(sum(w)/2) edges whose two endpoints are each chosen with
    probability w_i / sum(w); collapse duplicates and drop self-loops.  Keep the
    largest connected component and relabel nodes by a seeded permutation."""
    rng = np.random.default_rng(seed)
    w = chung_lu_weights(n, gamma, dbar, cap)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    M = int(rng.poisson(w.sum() / 2.0))
    a = np.minimum(np.searchsorted(cdf, rng.random(M), side="right"), n - 1)
    b = np.minimum(np.searchsorted(cdf, rng.random(M), side="right"), n - 1)
    g = csr_from_edges(n, a, b, None, f"chung_lu(n={n},gamma={gamma},dbar={dbar},seed={seed})")
    if keep_lcc:
        g = largest_component(g)
    perm = rng.permutation(g.n)
    return relabel(g, perm)


def grid_graph(a: int, b: int) -> CSRGraph:
    """2-D grid P_a x P_b, node (i, j) -> i*b + j."""
    ids = np.arange(a * b).reshape(a, b)
    s = np.concatenate([ids[:, :-1].ravel(), ids[:-1, :].ravel()])
    d = np.concatenate([ids[:, 1:].ravel(), ids[1:, :].ravel()])
    return csr_from_edges(a * b, s, d, None, f"grid({a}x{b})")


# ----------------------------------------------------------------------------
# Closed-form families
# ----------------------------------------------------------------------------

def path_graph(n: int) -> CSRGraph:
    return csr_from_edges(n, np.arange(n - 1), np.arange(1, n), None, f"path({n})")


def cycle_graph(n: int) -> CSRGraph:
    return csr_from_edges(n, np.arange(n), (np.arange(n) + 1) % n, None, f"cycle({n})")


def star_graph(n: int) -> CSRGraph:
    return csr_from_edges(n, np.zeros(n - 1, dtype=np.int64), np.arange(1, n), None, f"star({n})")


def complete_graph(n: int) -> CSRGraph:
    i, j = np.triu_indices(n, 1)
    return csr_from_edges(n, i, j, None, f"complete({n})")


def complete_bipartite(a: int, b: int) -> CSRGraph:
    i, j = np.meshgrid(np.arange(a), a + np.arange(b), indexing="ij")
    return csr_from_edges(a + b, i.ravel(), j.ravel(), None, f"K({a},{b})")


def hypercube(d: int) -> CSRGraph:
    n = 1 << d
    s, t = [], []
    for bit in range(d):
        v = np.arange(n)
        u = v ^ (1 << bit)
        keep = v < u
        s.append(v[keep])
        t.append(u[keep])
    return csr_from_edges(n, np.concatenate(s), np.concatenate(t), None, f"hypercube({d})")


# ----------------------------------------------------------------------------
# The benchmark workloads (synthetic stand-ins for the paper's networks)
# ----------------------------------------------------------------------------

WORKLOADS = {
    # protein-sized: BA n=2,000, 2 edges per new node, k=10, FP64 JD
    "c1": dict(kind="ba", n=2000, m=2, seed=1, k=10),
    # internet-shaped: Chung-Lu gamma=2.2, n=22,000, mean degree 4.2, LCC, k=20
    "c2": dict(kind="cl", n=22000, gamma=2.2, dbar=4.2, cap=None, seed=2, k=20),
    # www-shaped: Chung-Lu gamma=2.1, n=325,000, mean degree 7, max ~10^4, LCC, k=10
    "c3": dict(kind="cl", n=325000, gamma=2.1, dbar=7.0, cap=1.0e4, seed=3, k=10),
    # dblp-scale: Chung-Lu gamma=2.5, n=10^6, mean degree 6, LCC, k=10
    "c5": dict(kind="cl", n=1000000, gamma=2.5, dbar=6.0, cap=None, seed=5, k=10),
}


def workload_graph(name: str) -> CSRGraph:
    spec = WORKLOADS[name]
    if spec["kind"] == "ba":
        g = ba_graph(spec["n"], spec["m"], spec["seed"])
    else:
        g = chung_lu(spec["n"], spec["gamma"], spec["dbar"], spec["seed"], spec["cap"])
    g.name = name
    return g


def batch_specs(count: int = 256, seed: int = 1000, n_lo: int = 500, n_hi: int = 50000):
    """The batched workload: `count` graphs with n log-uniform in [n_lo, n_hi],
    thirds BA (m in {2,3,4}), Chung-Lu (gamma in U[2.0,2.8], mean degree in
    U[3,8]) and 2-D grids (aspect ratio in [1,4])."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        kind = i % 3
        if kind == 0:
            specs.append(dict(kind="ba", n=n, m=int(rng.integers(2, 5)), seed=seed + i))
        elif kind == 1:
            specs.append(dict(kind="cl", n=n, gamma=float(rng.uniform(2.0, 2.8)),
                              dbar=float(rng.uniform(3.0, 8.0)), cap=None, seed=seed + i))
        else:
            r = float(rng.uniform(1.0, 4.0))
            a = max(2, int(round(math.sqrt(n * r))))
            b = max(2, int(round(n / a)))
            specs.append(dict(kind="grid", a=a, b=b, seed=seed + i))
    return specs


def graph_from_spec(spec) -> CSRGraph:
    if spec["kind"] == "ba":
        return ba_graph(spec["n"], spec["m"], spec["seed"])
    if spec["kind"] == "cl":
        return chung_lu(spec["n"], spec["gamma"], spec["dbar"], spec["seed"], spec.get("cap"))
    if spec["kind"] == "grid":
        return grid_graph(spec["a"], spec["b"])
    raise ValueError(spec["kind"])


def random_block(n: int, b: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Seeded uniform(-1, 1) n x b block (row-major), for kernel-level tests."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(n, b)).astype(dtype)
