"""The applications of the computed pairs on the device (Section 2) against
the oracle on the same pairs: the Fiedler ordering (exact permutation, ties by
index), its bandwidth and profile, the bisection and its cut size, the
pseudo-inverse approximations T and S applied to a block, and the
current-flow closeness and betweenness."""
import numpy as np
import pytest

import graphgen as G
from oracle import centrality, dense, fiedler

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    import paper_1311_1695_gb300 as p
    from paper_1311_1695_gb300 import build
    build.build()
    return p


GRAPHS = [
    lambda: G.grid_graph(70, 53),                                   # 3,710 nodes: four sort blocks, ragged
    lambda: G.with_random_weights(G.ba_graph(5000, 2, 3), 4),       # weighted, hubs
    lambda: G.path_graph(1000),                                     # a single sort block
]


@pytest.mark.parametrize("make", GRAPHS)
def test_fiedler_order_and_bisection(pkg, make):
    g = make()
    ev, V = dense.smallest_eigpairs(g, 1)
    v2 = V[:, 0].copy()
    Gd = pkg.Graph(g)
    app = pkg.Applications(Gd)
    v2d = torch.from_numpy(v2).cuda()
    perm, stats = app.fiedler_order(v2d)
    ref = fiedler.fiedler_order(v2)
    assert np.array_equal(perm.cpu().numpy(), ref)
    assert (stats["bandwidth"], stats["profile"]) == fiedler.bandwidth_profile(g, ref)
    assert (stats["bandwidth0"], stats["profile0"]) == fiedler.bandwidth_profile(g, np.arange(g.n))
    for n1 in (g.n // 2, g.n // 3):
        side, cut, bound = app.fiedler_bisect(v2d, ev[0], n1)
        rside, rcut = fiedler.fiedler_partition(g, v2, n1)
        assert np.array_equal(side.cpu().numpy(), rside)
        assert np.isclose(cut, rcut, rtol=1e-12)
        assert np.isclose(bound, n1 * (g.n - n1) * ev[0] / g.n, rtol=1e-14)
        assert cut >= bound * (1 - 1e-12)
    Gd.close()


def test_fiedler_order_ties_go_by_index(pkg):
    g = G.grid_graph(40, 40)  # symmetric: repeated Fiedler entries
    v2 = np.round(G.random_block(g.n, 1, 5)[:, 0], 1)  # many exact ties
    Gd = pkg.Graph(g)
    perm, _ = pkg.Applications(Gd).fiedler_order(torch.from_numpy(v2).cuda())
    assert np.array_equal(perm.cpu().numpy(), fiedler.fiedler_order(v2))
    Gd.close()


@pytest.mark.parametrize("mode", ["T", "S"])
def test_pseudo_inverse_and_centralities(pkg, mode):
    g = G.with_random_weights(G.ba_graph(600, 3, 8), 2)
    k = 12
    ev, V = dense.smallest_eigpairs(g, k)
    sigma = ev[-1] if mode == "S" else 0.0
    Gd = pkg.Graph(g)
    app = pkg.Applications(Gd)
    Vd = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    X = G.random_block(g.n, 5, 9)
    Y = app.pinv_apply(ev, Vd, torch.from_numpy(X).cuda(), mode, sigma).cpu().numpy()
    refY = centrality.apply_partial(ev, V, X, mode, sigma if mode == "S" else None)
    assert np.abs(Y - refY).max() <= 1e-12 * np.abs(refY).max()
    P = centrality.pinv_partial(ev, V, mode, sigma if mode == "S" else None)
    c = app.closeness(ev, Vd, mode, sigma).cpu().numpy()
    assert np.allclose(c, centrality.closeness(P), rtol=1e-10)
    rng = np.random.default_rng(4)
    pairs = [tuple(rng.choice(g.n, 2, replace=False)) for _ in range(45)]  # two chunks of pairs
    b = app.betweenness(ev, Vd, pairs, mode, sigma).cpu().numpy()
    refb = centrality.betweenness(g, P, pairs)
    assert np.allclose(b, refb, rtol=1e-10, atol=1e-12 * np.abs(refb).max())
    Gd.close()


def test_fiedler_order_at_scale(pkg):
    """The dblp-scale graph (950,816 nodes): the GPU sort of a seeded vector is
    the oracle's order exactly."""
    g = G.workload_graph("c5")
    v2 = G.random_block(g.n, 1, 11)[:, 0]
    Gd = pkg.Graph(g)
    perm, stats = pkg.Applications(Gd).fiedler_order(torch.from_numpy(v2).cuda())
    assert np.array_equal(perm.cpu().numpy(), fiedler.fiedler_order(v2))
    Gd.close()
