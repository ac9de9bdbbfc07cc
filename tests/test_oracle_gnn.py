"""Pins of the warm-start network's FP64 definition: finite differences for
every parameter gradient, and the subspace loss's invariances."""
import numpy as np

import graphgen as G
from oracle import dense, gnn


def test_backward_matches_finite_differences():
    g = G.with_random_weights(G.ba_graph(40, 2, 3), 5)
    k = 3
    F = gnn.features(g, 7, nfeat=6)
    params = gnn.init_params(k, seed=1, nfeat=6, width=5)
    _, U = dense.smallest_eigpairs(g, k)

    def loss_of(ps):
        X, _ = gnn.forward(g, F, ps)
        return gnn.subspace_loss(X, U)[0]

    X, cache = gnn.forward(g, F, params)
    loss, dX = gnn.subspace_loss(X, U)
    grads = gnn.backward(g, cache, params, dX)
    h = 1e-6
    rng = np.random.default_rng(0)
    for pi, P in enumerate(params):
        flat = P.reshape(-1)
        for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = loss_of(params)
            flat[idx] = old - h
            lm = loss_of(params)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - grads[pi].reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd)), (pi, idx, fd)


def test_subspace_loss_invariances():
    rng = np.random.default_rng(2)
    U, _ = np.linalg.qr(rng.standard_normal((50, 4)))
    # without the ridge: zero on span(U), for any invertible recombination
    X = U @ rng.standard_normal((4, 4))
    assert abs(gnn.subspace_loss(X, U, eps=0.0)[0]) < 1e-12
    # invariant under X -> X R and under U -> U Q (orthogonal Q)
    Y = rng.standard_normal((50, 4))
    R = rng.standard_normal((4, 4))
    Q, _ = np.linalg.qr(rng.standard_normal((4, 4)))
    l0 = gnn.subspace_loss(Y, U, eps=0.0)[0]
    assert abs(gnn.subspace_loss(Y @ R, U, eps=0.0)[0] - l0) < 1e-10
    assert abs(gnn.subspace_loss(Y, U @ Q, eps=0.0)[0] - l0) < 1e-10
    # still invariant under U -> U Q with the ridge
    assert abs(gnn.subspace_loss(Y, U @ Q)[0] - gnn.subspace_loss(Y, U)[0]) < 1e-10
    # one for a block orthogonal to span(U)
    Z = Y - U @ (U.T @ Y)
    assert abs(gnn.subspace_loss(Z, U, eps=0.0)[0] - 1.0) < 1e-12
    # with the ridge, X = U gives 1 - 1/(1 + eps) exactly; a rank-deficient X
    # stays finite
    assert abs(gnn.subspace_loss(U, U)[0] - gnn.EPS_RIDGE / (1 + gnn.EPS_RIDGE)) < 1e-14
    Xd = np.column_stack([X[:, :3], X[:, 0]])
    assert np.isfinite(gnn.subspace_loss(Xd, U)[0])


def test_ridge_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    U, _ = np.linalg.qr(rng.standard_normal((30, 3)))
    X = rng.standard_normal((30, 3))
    _, dX = gnn.subspace_loss(X, U, eps=1e-2)
    h = 1e-6
    for (i, j) in [(0, 0), (7, 2), (29, 1)]:
        Xp, Xm = X.copy(), X.copy()
        Xp[i, j] += h
        Xm[i, j] -= h
        fd = (gnn.subspace_loss(Xp, U, eps=1e-2)[0] - gnn.subspace_loss(Xm, U, eps=1e-2)[0]) / (2 * h)
        assert abs(fd - dX[i, j]) <= 1e-7 * max(1.0, abs(fd))


def test_output_is_centred():
    g = G.ba_graph(60, 2, 4)
    F = gnn.features(g, 3)
    X, _ = gnn.forward(g, F, gnn.init_params(4, seed=2))
    assert np.abs(X.sum(axis=0)).max() < 1e-10


def test_features_shape_and_range():
    g = G.ba_graph(30, 2, 1)
    F = gnn.features(g, 3)
    assert F.shape == (30, gnn.NFEAT)
    assert np.all(F[:, 0] == 1.0) and F[:, 1].max() == 1.0
    assert np.abs(F[:, 2:]).max() < 1.0


def test_bf16_rounding_against_known_values():
    """The oracle's BF16 rounding: 8 significant bits, ties to even."""
    from oracle.gnn import round_bf16
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 2.0 ** -9, 1.0 + 3 * 2.0 ** -9, -3.14159, 65504.0, 1e-40])
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 (the spacing at 1): ties to even
    ref = np.array([1.0, 1.0, 1.0, 1.0 + 2.0 ** -7, -3.140625, 65536.0, 0.0])
    got = round_bf16(x)
    assert np.array_equal(got[:6], ref[:6])
    assert abs(got[6]) < 1e-38  # a float32 subnormal keeps its top bits
    rng = np.random.default_rng(0)
    v = rng.standard_normal(1000) * 10.0 ** rng.integers(-5, 5, 1000)
    r = round_bf16(v)
    assert np.all(np.abs(r - v) <= 2.0 ** -8 * np.abs(v) * (1 + 1e-6))
    assert np.array_equal(round_bf16(r), r)  # idempotent
