"""The C ABI library loads, exports every symbol include/lapeig.h declares, and
rejects invalid input with the documented status codes (host-side checks
only: no GPU work is started by these calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

import graphgen as G
import paper_1311_1695_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "lapeig.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lap_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(pkg.LIB_PATH):
        from paper_1311_1695_gb300 import build
        build.build()
    return pkg.lib()


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) <= set(pkg.exported_symbols()) | {"lap_opts_default"}


def test_opts_default_and_strerror(lib):
    o = pkg.lap_opts()
    lib.lap_opts_default(ctypes.byref(o))
    assert o.struct_size == ctypes.sizeof(pkg.lap_opts)
    assert o.inner_maxit == 20 and o.inner_tol == 1e-2  # ITMAX, delta_PCG (Section 4)
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7, -8, -9):
        assert lib.lap_strerror(code)


def _call(g, k=3, tol=1e-8, **kw):
    with pytest.raises(pkg.LapError) as e:
        pkg.lap_eigs(g, k, tol, **kw)
    return e.value.status


def test_rejects_self_loop(lib):
    g = G.path_graph(6)
    g.colidx = g.colidx.copy()
    g.colidx[0] = 0  # row 0: (0,0)
    assert _call(g) in (pkg.LAP_ESELFLOOP, pkg.LAP_EUNSORTED, pkg.LAP_ENOTSYM)


def test_rejects_asymmetric(lib):
    g = G.csr_from_edges(5, [0, 1, 2, 3], [1, 2, 3, 4])
    rp = g.rowptr.copy()
    ci = g.colidx.copy()
    # drop the (1, 0) entry: shift row 1
    keep = np.ones(ci.size, bool)
    keep[rp[1]] = False
    ci2 = ci[keep]
    rp2 = rp.copy()
    rp2[2:] -= 1
    bad = G.CSRGraph(5, rp2, ci2, None)
    assert _call(bad) == pkg.LAP_ENOTSYM


def test_rejects_asymmetric_values_and_counts(lib):
    """The symmetry check (a binary search for (j, i) per nonzero (i, j)):
    equal patterns with unequal weights, and a row with an extra one-way edge
    whose row counts still add up, are both rejected; a symmetric weighted
    graph passes the host checks."""
    g = G.with_random_weights(G.cycle_graph(8), 3)
    g.weights = g.weights.copy()
    g.weights[0] *= 2.0  # (0, 1) no longer equals (1, 0)
    assert _call(g) == pkg.LAP_ENOTSYM
    # edges 0->1, 1->2, 2->0 only one way: every row has one entry, the sum
    # matches, the transpose does not
    one_way = G.CSRGraph(3, np.array([0, 1, 2, 3]), np.array([1, 2, 0], dtype=np.int32), None)
    assert _call(one_way, k=1) == pkg.LAP_ENOTSYM
    # a hub row with a missing reverse entry
    star = G.csr_from_edges(6, [0, 0, 0, 0, 0], [1, 2, 3, 4, 5])
    rp, ci = star.rowptr.copy(), star.colidx.copy()
    keep = np.ones(ci.size, bool)
    keep[rp[3]] = False  # drop (3, 0)
    rp2 = rp.copy()
    rp2[4:] -= 1
    assert _call(G.CSRGraph(6, rp2, ci[keep], None)) == pkg.LAP_ENOTSYM


def test_validation_of_large_graphs_split_over_threads(lib):
    """Graphs large enough for the host checks to run on several threads
    (row ranges of equal nonzero count): a fault in any range is found, and
    when several rows are faulty the first one in row order decides the
    status."""
    g = G.with_random_weights(G.grid_graph(300, 300), 5)  # 358,800 nonzeros
    n, rp = g.n, g.rowptr
    late = rp[n - 10]  # a nonzero in the last range
    # one-way weight change near the end
    w = g.weights.copy()
    w[late] *= 3.0
    assert _call(G.CSRGraph(n, rp, g.colidx, w)) == pkg.LAP_ENOTSYM
    # a missing reverse entry in the middle: drop (i, j), keep (j, i)
    mid = n // 2
    keep = np.ones(g.colidx.size, bool)
    keep[rp[mid]] = False
    rp2 = rp.copy()
    rp2[mid + 1:] -= 1
    assert _call(G.CSRGraph(n, rp2, g.colidx[keep], w[keep])) == pkg.LAP_ENOTSYM
    # an unsorted row late and a non-positive weight early: the earlier row decides
    ci = g.colidx.copy()
    ci[late], ci[late + 1] = ci[late + 1], ci[late]
    w2 = g.weights.copy()
    w2[rp[100]] = 0.0
    assert _call(G.CSRGraph(n, rp, ci, w2)) == pkg.LAP_EWEIGHT
    assert _call(G.CSRGraph(n, rp, ci, g.weights)) == pkg.LAP_EUNSORTED


def test_rejects_bad_weight(lib):
    g = G.with_random_weights(G.cycle_graph(8), 1)
    g.weights = g.weights.copy()
    g.weights[3] = -1.0
    assert _call(g) == pkg.LAP_EWEIGHT
    g.weights[3] = np.nan
    assert _call(g) == pkg.LAP_EWEIGHT


def test_rejects_unsorted(lib):
    g = G.complete_graph(5)
    ci = g.colidx.copy()
    ci[0], ci[1] = ci[1], ci[0]
    assert _call(G.CSRGraph(5, g.rowptr, ci, None)) == pkg.LAP_EUNSORTED


def test_rejects_bad_k_and_tol(lib):
    g = G.cycle_graph(10)
    assert _call(g, k=0) == pkg.LAP_EINVAL
    assert _call(g, k=10) == pkg.LAP_EINVAL  # k > n - 1
    assert _call(g, k=2, tol=0.0) == pkg.LAP_EINVAL
    assert _call(g, k=2, method=7) == pkg.LAP_EINVAL


def test_rejects_out_of_range_column(lib):
    g = G.path_graph(4)
    ci = g.colidx.copy()
    ci[-1] = 9
    assert _call(G.CSRGraph(4, g.rowptr, ci, None)) == pkg.LAP_EINVAL
