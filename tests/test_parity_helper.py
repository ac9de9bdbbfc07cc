"""The parity checker itself, on the CPU: it accepts the oracle's own pairs,
rejects a wrong eigenvalue, a vector from the wrong eigenspace and a
non-orthogonal block, and refuses to judge a cluster that runs past the end
of a truncated oracle list."""
import numpy as np
import pytest

import graphgen as G
from oracle import dense
from parity import all_pairs, check_eigpairs


def test_accepts_exact_pairs_and_rejects_wrong_ones():
    g = G.ba_graph(200, 2, 8)
    ev_ref, V_ref = all_pairs(g)
    k = 5
    check_eigpairs(g, ev_ref[:k], V_ref[:, :k], ev_ref, V_ref, k=k)
    with pytest.raises(AssertionError):  # eigenvalue off by 1e-6 relative
        check_eigpairs(g, ev_ref[:k] * (1 + 1e-6), V_ref[:, :k], ev_ref, V_ref, k=k, tol=1e-3)
    W = V_ref[:, :k].copy()
    W[:, 2] = V_ref[:, k + 3]  # a vector of another eigenspace with the wrong value claimed
    with pytest.raises(AssertionError, match="residual"):
        check_eigpairs(g, ev_ref[:k], W, ev_ref, V_ref, k=k)
    # the same vector with its own value: the value check catches it
    e = ev_ref[:k].copy()
    e[2] = ev_ref[k + 3]
    with pytest.raises(AssertionError, match="eigenvalue"):
        check_eigpairs(g, e, W, ev_ref, V_ref, k=k)
    W = V_ref[:, :k] + 1e-4 * V_ref[:, k:2 * k]
    with pytest.raises(AssertionError):
        check_eigpairs(g, ev_ref[:k], W, ev_ref, V_ref, k=k)


def test_refuses_a_cluster_past_a_truncated_list():
    g = G.cycle_graph(40)  # doubly degenerate pairs
    ev_ref, V_ref = dense.smallest_eigpairs(g, 4)  # ends inside the pair 3, 4 ... (5 is its partner)
    ev, V = ev_ref[:3], V_ref[:, :3]
    with pytest.raises(AssertionError, match="more oracle pairs"):
        check_eigpairs(g, ev, V, ev_ref[:3], V_ref[:, :3], k=3)
    ev_all, V_all = all_pairs(g)
    check_eigpairs(g, ev_all[:4], V_all[:, :4], ev_all, V_all, k=4)


def test_value_based_check_certifies_and_rejects():
    g = G.grid_graph(9, 14)
    ev_ref, V_ref = all_pairs(g)
    from parity import check_against_values
    k = 6
    out = check_against_values(g, ev_ref[:k], V_ref[:, :k], ev_ref[:12])
    assert out["angle_bound"] < 1e-6
    # a missed eigenvalue: the pairs 0, 1, 2, 3, 4, 6 claimed as the six smallest
    idx = [0, 1, 2, 3, 4, 6]
    with pytest.raises(AssertionError, match="eigenvalue"):
        check_against_values(g, ev_ref[idx], V_ref[:, idx], ev_ref[:12])
    # a list that ends inside a cluster holding one of the pairs
    # a list that ends inside a cluster holding one of the pairs: no
    # per-cluster angle is certified, the k-subspace bound still is
    fake = np.r_[ev_ref[:k], ev_ref[k - 1] + 1e-13]
    out = check_against_values(g, ev_ref[:k], V_ref[:, :k], fake)
    assert out["angle_bound"] is None
    out = check_against_values(g, ev_ref[:k], V_ref[:, :k], ev_ref[:12])
    assert out["subspace_bound"] < 1e-10
