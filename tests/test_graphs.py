"""Input generators: determinism, simple-graph structure, connectivity."""
import numpy as np
import pytest

import graphgen as G


def _check_simple(g):
    n = g.n
    assert g.rowptr[0] == 0 and g.rowptr[-1] == g.colidx.size
    rows = np.repeat(np.arange(n), np.diff(g.rowptr))
    assert np.all(rows != g.colidx), "self-loop"
    for i in range(0, n, max(1, n // 200)):
        c = g.colidx[g.rowptr[i]:g.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0), "row not sorted/unique"
    key = rows * n + g.colidx
    keyt = g.colidx.astype(np.int64) * n + rows
    assert np.array_equal(np.sort(key), np.sort(keyt)), "not symmetric"


@pytest.mark.parametrize("make", [
    lambda: G.ba_graph(500, 3, 11),
    lambda: G.chung_lu(3000, 2.2, 4.2, 5),
    lambda: G.grid_graph(7, 9),
    lambda: G.hypercube(5),
    lambda: G.complete_bipartite(3, 5),
])
def test_simple_symmetric(make):
    g = make()
    _check_simple(g)
    assert g.digest() == make().digest(), "generator not deterministic"


def test_ba_edge_count_and_connected():
    g = G.ba_graph(2000, 2, 1)
    assert g.n_edges == 3 + (2000 - 3) * 2
    assert np.unique(G.components(g)).size == 1


def test_chung_lu_lcc_connected_and_heavy_tailed():
    g = G.chung_lu(20000, 2.2, 4.2, 2)
    assert np.unique(G.components(g)).size == 1
    deg = g.degree_counts()
    assert deg.max() > 20 * np.median(deg)
    assert 2.5 < deg.mean() < 6.0


def test_components_and_union():
    u = G.disjoint_union(G.path_graph(4), G.cycle_graph(5), G.star_graph(3))
    assert np.unique(G.components(u)).size == 3
    assert u.n == 12


def test_weighted_copy_keeps_symmetry():
    g = G.with_random_weights(G.ba_graph(200, 2, 3), 9)
    _check_simple(g)
    A = np.zeros((g.n, g.n))
    for i in range(g.n):
        for p in range(g.rowptr[i], g.rowptr[i + 1]):
            A[i, g.colidx[p]] = g.weights[p]
    assert np.array_equal(A, A.T) and A.min() >= 0


def test_batch_specs_mix():
    specs = G.batch_specs(30)
    kinds = [s["kind"] for s in specs]
    assert kinds.count("ba") == kinds.count("cl") == kinds.count("grid") == 10
