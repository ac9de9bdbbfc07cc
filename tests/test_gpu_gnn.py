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
