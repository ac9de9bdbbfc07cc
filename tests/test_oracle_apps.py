"""Pins of the oracle's applications of the computed pairs (Section 2):
bisection and ordering from the Fiedler vector, and centralities from the
approximated pseudo-inverse, against the relaxation identities the paper
derives, brute-force edge sums, closed forms, and library routines (numpy's
pseudo-inverse, networkx's current-flow centralities)."""
import itertools

import numpy as np
import pytest

import graphgen as G
from oracle import centrality, dense, fiedler
from oracle.laplacian import Laplacian


def _barbell(m):
    """Two complete graphs K_m joined by the edge (m - 1, m)."""
    src, dst = [], []
    for base in (0, m):
        for i, j in itertools.combinations(range(m), 2):
            src.append(base + i)
            dst.append(base + j)
    src.append(m - 1)
    dst.append(m)
    return G.csr_from_edges(2 * m, np.array(src), np.array(dst))


@pytest.mark.parametrize("g", [G.ba_graph(120, 2, 4), G.grid_graph(7, 11), G.with_random_weights(G.ba_graph(90, 3, 2), 6)])
@pytest.mark.parametrize("frac", [0.5, 0.3])
def test_relaxed_bisection_identities(g, frac):
    """x = (n1 - n2)/(2n) e + sqrt(n1 n2 / n) v2 satisfies both constraints,
    x^T x = n/4 and e^T x = (n1 - n2)/2, and reaches x^T L x = n1 n2 lambda2 / n;
    every discrete bisection of the same sizes cuts at least that much."""
    ev, V = dense.smallest_eigpairs(g, 1)
    n = g.n
    n1 = int(frac * n)
    n2 = n - n1
    x = fiedler.relaxed_bisection(V[:, 0], n1)
    lap = Laplacian(g)
    assert np.isclose(x @ x, n / 4, rtol=1e-12)
    assert np.isclose(x.sum(), (n1 - n2) / 2, rtol=1e-12, atol=1e-9)
    assert np.isclose(x @ lap.matvec(x), n1 * n2 * ev[0] / n, rtol=1e-10)
    side, cut = fiedler.fiedler_partition(g, V[:, 0], n1)
    assert (side == 0).sum() == n1
    assert cut >= n1 * n2 * ev[0] / n * (1 - 1e-12)
    # cut size is Eq. 1 at x_i = +-1/2
    xs = np.where(side == 0, -0.5, 0.5)
    assert np.isclose(cut, xs @ lap.matvec(xs), rtol=1e-12)


def test_bisection_of_a_barbell_cuts_the_bridge():
    g = _barbell(10)
    ev, V = dense.smallest_eigpairs(g, 1)
    side, cut = fiedler.fiedler_partition(g, V[:, 0], 10)
    assert cut == 1.0
    assert len(set(side[:10])) == 1 and len(set(side[10:])) == 1


def test_fiedler_order_of_a_path_is_monotone():
    n = 60
    g = G.path_graph(n)
    ev, V = dense.smallest_eigpairs(g, 1)
    perm = fiedler.fiedler_order(V[:, 0])
    assert list(perm) in (list(range(n)), list(range(n))[::-1])
    assert fiedler.bandwidth_profile(g, perm) == (1, n - 1)
    # a scrambled labelling has a larger bandwidth; the Fiedler order of the
    # relabelled path restores bandwidth 1
    rng = np.random.default_rng(3)
    q = rng.permutation(n)
    h = G.relabel(g, q)
    assert fiedler.bandwidth_profile(h, np.arange(n))[0] > 1
    evh, Vh = dense.smallest_eigpairs(h, 1)
    assert fiedler.bandwidth_profile(h, fiedler.fiedler_order(Vh[:, 0]))[0] == 1


def test_order_ties_by_index():
    v = np.array([0.5, -1.0, 0.5, -1.0, 0.0])
    assert list(fiedler.fiedler_order(v)) == [1, 3, 4, 0, 2]


# ---------------------------------------------------------------- pseudo-inverse and centralities

def _pairs(g):
    lap = Laplacian(g)
    w, V = np.linalg.eigh(lap.dense())
    return w, V, lap


def test_partial_sums_with_every_pair_are_the_pseudo_inverse():
    g = G.with_random_weights(G.ba_graph(40, 2, 7), 1)
    w, V, lap = _pairs(g)
    Gp = centrality.pseudo_inverse(g)
    T = centrality.pinv_partial(w[1:], V[:, 1:], "T")
    assert np.allclose(T, Gp, atol=1e-10)
    for sigma in (w[5], 0.5 * (w[5] + w[-1])):
        S = centrality.pinv_partial(w[1:], V[:, 1:], "S", sigma)
        assert np.allclose(S, Gp, atol=1e-10)


@pytest.mark.parametrize("k", [3, 10])
def test_S_closed_form_equals_the_sum_with_sigma_for_the_rest(k):
    """S = T + sum_{j > k} v_j v_j^T / sigma (the definition, with every
    eigenvector) equals the closed form that needs only the k pairs."""
    g = G.grid_graph(5, 7)
    w, V, lap = _pairs(g)
    sigma = w[k]
    T = centrality.pinv_partial(w[1:k + 1], V[:, 1:k + 1], "T")
    S_def = T + sum(np.outer(V[:, j], V[:, j]) for j in range(k + 1, g.n)) / sigma
    S = centrality.pinv_partial(w[1:k + 1], V[:, 1:k + 1], "S", sigma)
    assert np.allclose(S, S_def, atol=1e-12)
    X = np.random.default_rng(1).standard_normal((g.n, 3))
    assert np.allclose(centrality.apply_partial(w[1:k + 1], V[:, 1:k + 1], X, "S", sigma), S @ X, atol=1e-12)
    assert np.allclose(centrality.apply_partial(w[1:k + 1], V[:, 1:k + 1], X, "T"), T @ X, atol=1e-12)


def _nx(g):
    nx = pytest.importorskip("networkx")
    H = nx.Graph()
    H.add_nodes_from(range(g.n))
    for i in range(g.n):
        for p in range(g.rowptr[i], g.rowptr[i + 1]):
            j = int(g.colidx[p])
            if j > i:
                H.add_edge(i, j, weight=1.0 if g.weights is None else float(g.weights[p]))
    return nx, H


@pytest.mark.parametrize("g", [G.ba_graph(30, 2, 5), G.with_random_weights(G.grid_graph(4, 6), 9)])
def test_centralities_with_the_exact_pseudo_inverse_match_networkx(g):
    nx, H = _nx(g)
    Gp = centrality.pseudo_inverse(g)
    c = centrality.closeness(Gp)
    ref = nx.current_flow_closeness_centrality(H, weight="weight")
    assert np.allclose(c, [ref[i] for i in range(g.n)], rtol=1e-9)
    pairs = list(itertools.combinations(range(g.n), 2))
    b = centrality.betweenness(g, Gp, pairs)
    refb = nx.current_flow_betweenness_centrality(H, normalized=False, weight="weight")
    assert np.allclose(b, [refb[i] for i in range(g.n)], rtol=1e-9, atol=1e-9)
