"""Solves on a handle's degree-ordered copy (lap_graph_set_reorder): the
eigenpairs come back in the caller's numbering and match the oracle's dense
definition, for every method, a batch, and start blocks given in the
caller's numbering (host and device)."""
import numpy as np
import pytest

import graphgen as G
from parity import all_pairs, check_eigpairs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1311_1695_gb300 as p
    from paper_1311_1695_gb300 import build
    build.build()
    return p


def _blocks(V, nrows, k):
    """Graph s's column-major n_s x k block at offset row0[s] * k."""
    Vh = V.cpu().numpy()
    out, off = [], 0
    for n in nrows:
        out.append(Vh[off * k:(off + n) * k].reshape(k, n).T)
        off += n
    return out


@pytest.mark.parametrize("method,precision,k", [("jd", "fp64", 10), ("jd", "mixed", 10), ("dacg", "fp64", 5),
                                                ("irlm", "fp64", 5)])
def test_degree_order_matches_definition(pkg, method, precision, k):
    import torch
    g = G.chung_lu(3000, 2.2, 5.0, 71)
    Gd = pkg.Graph(g)
    Gd.set_reorder("degree")
    V = torch.zeros(g.n * k, dtype=torch.float64, device="cuda")
    ev, infos = Gd.eigs(k, 1e-8, method=method, evecs=V, precision=precision)
    assert infos[0]["status"] == 0, infos[0]
    ev_ref, V_ref = all_pairs(g)
    check_eigpairs(g, ev[0], _blocks(V, [g.n], k)[0], ev_ref, V_ref, k=k)
    # the same handle back on the graph as numbered: the same pairs
    Gd.set_reorder("none")
    ev2, infos2 = Gd.eigs(k, 1e-8, method=method, evecs=V, precision=precision)
    assert infos2[0]["status"] == 0
    check_eigpairs(g, ev2[0], _blocks(V, [g.n], k)[0], ev_ref, V_ref, k=k)
    Gd.close()


def test_batched_degree_order(pkg):
    """Every graph of a batch relabelled on its own rows; blocks returned at
    the caller's offsets."""
    import torch
    gs = [G.ba_graph(400, 2, 61), G.grid_graph(18, 25), G.chung_lu(1500, 2.4, 5.0, 62),
          G.with_random_weights(G.ba_graph(700, 3, 63), 64)]
    k = 4
    nrows = [g.n for g in gs]
    Gd = pkg.Graph(gs)
    Gd.set_reorder("degree")
    V = torch.zeros(sum(nrows) * k, dtype=torch.float64, device="cuda")
    evs, infos = Gd.eigs(k, 1e-8, evecs=V, precision="mixed")
    for g, ev, Vb, info in zip(gs, evs, _blocks(V, nrows, k), infos):
        assert info["status"] == 0, info
        ev_ref, V_ref = all_pairs(g)
        check_eigpairs(g, ev, Vb, ev_ref, V_ref, k=k)
    Gd.close()


@pytest.mark.parametrize("where", ["host", "device"])
def test_start_block_in_caller_numbering(pkg, where):
    """The oracle's eigenvectors, in the caller's numbering, as the start
    block: the solve on the relabelled copy must see them as eigenvectors
    (converged within a few outer iterations; a start left in the wrong
    order is a random block and takes far more)."""
    import torch
    g = G.chung_lu(3000, 2.2, 5.0, 72)
    k = 6
    ev_ref, V_ref = all_pairs(g)
    Gd = pkg.Graph(g)
    Gd.set_reorder("degree")
    V = torch.zeros(g.n * k, dtype=torch.float64, device="cuda")
    x0 = np.ascontiguousarray(V_ref[:, :k])
    kw = dict(x0=x0) if where == "host" else dict(x0_dev=torch.from_numpy(x0).cuda())
    ev, infos = Gd.eigs(k, 1e-8, evecs=V, precision="fp64", **kw)
    assert infos[0]["status"] == 0, infos[0]
    assert infos[0]["outer_its"] <= 3, infos[0]
    check_eigpairs(g, ev[0], _blocks(V, [g.n], k)[0], ev_ref, V_ref, k=k)
    # the random start on the same handle needs clearly more iterations
    ev2, infos2 = Gd.eigs(k, 1e-8, evecs=V, precision="fp64")
    assert infos2[0]["outer_its"] > infos[0]["outer_its"] + 3, (infos[0], infos2[0])
    Gd.close()


def test_reorder_mode_validation(pkg):
    g = G.ba_graph(300, 2, 5)
    Gd = pkg.Graph(g)
    with pytest.raises(pkg.LapError):
        Gd.set_reorder(2)
    Gd.set_reorder("auto")
    Gd.close()
