"""The warm-start network's device forward and backward against the FP64
oracle definition (same BF16-rounded weights), and the gain of the trained
network over the random start."""
import os

import numpy as np
import pytest

import graphgen as G
from oracle import dense
from oracle import gnn as ognn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    import paper_1311_1695_gb300 as p
    from paper_1311_1695_gb300 import build
    build.build()
    return p


def _graphs():
    return [G.with_random_weights(G.chung_lu(1500, 2.4, 6.0, 3), 2), G.ba_graph(900, 3, 4)]


def test_forward_backward_match_oracle(pkg):
    """Each stage against the FP64 definition on the same BF16 weights, the
    oracle rounding its stored activations to BF16 where the kernels store
    them: forward X; loss and dX (the oracle evaluated on the GPU's X, since
    dX involves (X^T X)^{-1}, which amplifies rounding of X by its condition
    number); backward fed with the oracle's dX.  Tolerances from the
    arithmetic: a stored activation can land one BF16 step (2^-8 relative)
    from the oracle's when an FP32 sum and the FP64 one straddle a rounding
    boundary, and the weight gradients round dZ to BF16 for the tensor-core
    product (2^-9 relative per term)."""
    from paper_1311_1695_gb300 import gnn
    gs = _graphs()
    k = 6
    params = gnn.init_params(k, seed=3)
    pb = [gnn.to_bf16(p) for p in params]
    H = pkg.Graph(gs)
    net = gnn.Net(H, k)
    U = [dense.smallest_eigpairs(g, k)[1] for g in gs]
    net.set_targets(torch.from_numpy(np.vstack(U)).float().cuda())
    X = net.forward(params, seed=11).cpu().double().numpy()
    losses = net.loss()
    dX_gpu = net.dX[:, :k].cpu().double().numpy()
    ref_grads = [np.zeros_like(p) for p in params]
    dX_ref_all = []
    off = 0
    for s_, (g, Ug) in enumerate(zip(gs, U)):
        F = ognn.features(g, 11, nfeat=gnn.NFEAT)
        Xr, cache = ognn.forward(g, F, pb, store=ognn.round_bf16)
        Xg = X[off:off + g.n]
        err = np.abs(Xg - Xr)
        assert err.max() <= 2.0 ** -5 * np.abs(Xr).max(), err.max()
        assert err.mean() <= 2.0 ** -10 * np.abs(Xr).max(), err.mean()
        # loss and dX on the GPU's X
        lg, dXg = ognn.subspace_loss(Xg, Ug)
        assert abs(losses[s_] - lg) <= 1e-5
        dXg = dXg / len(gs)
        assert np.abs(dX_gpu[off:off + g.n] - dXg).max() <= 1e-3 * np.abs(dXg).max()
        # backward on the oracle's exact dX
        _, dXr = ognn.subspace_loss(Xr, Ug)
        dXr = dXr / len(gs)
        dX_ref_all.append(dXr)
        for a, b in zip(ref_grads, ognn.backward(g, cache, pb, dXr)):
            a += b
        off += g.n
    net.dX[:, :k] = torch.from_numpy(np.vstack(dX_ref_all)).float()
    grads = net.backward()
    names = [f"{nm}{l}" for l in range(3) for nm in ("W", "U", "b")] + ["Wout"]
    errs = {nm: float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-8)) for nm, a, b in zip(names, grads, ref_grads)}
    assert max(errs.values()) <= 2e-2, errs
    H.close()


def test_trained_warm_start_beats_random(pkg):
    from paper_1311_1695_gb300 import gnn
    if not os.path.exists(gnn.WEIGHTS):
        pytest.skip("no trained weights committed")
    params, meta = gnn.load_params()
    k = params[-1].shape[1]
    gains = []
    for seed in (901, 902, 903):
        g = G.chung_lu(30000, 2.5, 6.0, seed)
        H = pkg.Graph(g)
        x0 = gnn.warm_start(H, params)
        _, infos_r = H.eigs(k, 1e-8, precision="mixed")
        ev_w, infos_w = H.eigs(k, 1e-8, precision="mixed", x0_dev=x0)
        assert infos_w[0]["status"] == 0 and infos_r[0]["status"] == 0
        gains.append(infos_r[0]["n_matvec"] / infos_w[0]["n_matvec"])
        H.close()
    assert np.median(gains) > 1.0, gains


def test_native_warm_start_matches_driver(pkg):
    """lap_gnn_warm_start (the forward pass orchestrated in the library) gives
    the Python-driven forward's proposal on the same handle and seed: the
    same kernels in the same order, so equal up to the order of the FP32
    atomic sums in the centring (a few FP32 ulps of the column means)."""
    from paper_1311_1695_gb300 import gnn
    params = gnn.init_params(10, seed=7)
    for g in _graphs():
        H = pkg.Graph(g)
        Xp = gnn.warm_start(H, params, seed=99).cpu().numpy()
        Xn = gnn.warm_start_native(H, params, seed=99).cpu().numpy()
        H.close()
        assert Xn.shape == Xp.shape
        assert np.abs(Xn - Xp).max() <= 1e-5 * np.abs(Xp).max()


def test_use_gnn_option_solves_and_falls_back(pkg):
    """lap_opts.use_gnn: the solve starts from the network's proposal and
    returns the definition's pairs; a batch of graphs, or another method,
    takes the random start without error."""
    from paper_1311_1695_gb300 import gnn
    from parity import all_pairs, check_eigpairs
    if not os.path.exists(gnn.WEIGHTS):
        pytest.skip("no trained weights committed")
    params, _ = gnn.load_params()
    g = G.chung_lu(3000, 2.5, 6.0, 11)
    ev_ref, V_ref = all_pairs(g)
    ev, V, info = pkg.lap_eigs(g, 10, tol=1e-8, precision="mixed", use_gnn=True, gnn_params=params)
    assert info["status"] == 0, info
    check_eigpairs(g, ev, V, ev_ref, V_ref, k=10)
    ev2, V2, info2 = pkg.lap_eigs(g, 10, tol=1e-8, method="dacg", use_gnn=True, gnn_params=params)
    assert info2["status"] == 0
    check_eigpairs(g, ev2, V2, ev_ref, V_ref, k=10)
    evs, Vs, infos = pkg.lap_eigs_batched([g, G.ba_graph(800, 2, 5)], 6, tol=1e-8, use_gnn=True, gnn_params=params)
    assert all(i["status"] == 0 for i in infos)


def test_use_gnn_wall_time_gain_c5(pkg):
    """The learned start on the dblp-scale graph (n = 950,816, k = 10, mixed
    precision), through the C ABI: its wall time, forward pass included, is
    below the random start's, and its pairs are the oracle's (stored values,
    tests/golden/eigs_c5.txt)."""
    import sys
    import time
    from paper_1311_1695_gb300 import gnn
    from parity import check_against_values
    if not os.path.exists(gnn.WEIGHTS):
        pytest.skip("no trained weights committed")
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
    from make_golden import load
    params, _ = gnn.load_params()
    g = G.workload_graph("c5")
    digest, ev_ref = load("c5")
    assert digest == g.digest()
    H = pkg.Graph(g)
    V = torch.zeros(g.n * 10, dtype=torch.float64, device="cuda")
    times = {}
    for label, kw in (("random", {}), ("gnn", dict(use_gnn=True, gnn_params=params))):
        H.eigs(10, 1e-8, evecs=V, precision="mixed", **kw)  # warm-up (the first solve autotunes the handle)
        ts = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ev, infos = H.eigs(10, 1e-8, evecs=V, precision="mixed", **kw)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
            assert infos[0]["status"] == 0, infos[0]
        times[label] = float(np.median(ts))
        if label == "gnn":
            Vh = V.cpu().numpy().reshape(10, g.n).T
            check_against_values(g, ev[0], Vh, ev_ref)
    H.close()
    assert times["gnn"] < times["random"], times


def test_adam_step_matches_definition(pkg):
    """lap_adam_step over three steps against Adam written out (Kingma and
    Ba's bias-corrected moments) in FP64."""
    from paper_1311_1695_gb300 import gnn
    rng = np.random.default_rng(5)
    params = [rng.standard_normal((7, 3)), rng.standard_normal(11)]
    ref = [p.copy() for p in params]
    m = [np.zeros_like(p) for p in ref]
    v = [np.zeros_like(p) for p in ref]
    opt = gnn.Adam(params, lr=0.01)
    for t in range(1, 4):
        grads = [rng.standard_normal(p.shape) for p in params]
        opt.step(params, grads)
        for p, g_, mm, vv in zip(ref, grads, m, v):
            mm[...] = 0.9 * mm + 0.1 * g_
            vv[...] = 0.999 * vv + 0.001 * g_ * g_
            p -= 0.01 * (mm / (1 - 0.9 ** t)) / (np.sqrt(vv / (1 - 0.999 ** t)) + 1e-8)
    for p, r in zip(params, ref):
        assert np.abs(p - r).max() <= 1e-13 * (1 + np.abs(r).max())
