"""Failure detection on the device, made on purpose without any fault: a grid
barrier whose wait limit is set below the time the other CTAs need to arrive
gives up, the kernel ends early and the call returns LAP_ETIMEOUT; the same
handle then gives correct results.  Also the wall-clock cap (LAP_ETIMEOUT
with a partial result) and a NaN in the iteration (LAP_ENUMERIC: weights
finite in FP64 that overflow FP32 in the mixed-precision phase)."""
import numpy as np
import pytest

import graphgen as G
from oracle import blockops, dense
from oracle.laplacian import Laplacian

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    import paper_1311_1695_gb300 as p
    from paper_1311_1695_gb300 import build
    build.build()
    return p


def _graph():
    # 4,435 rows after the largest component: a single graph cut into 304 tiles, hub rows
    return G.chung_lu(5000, 2.2, 5.0, 7)


def _block(g, b):
    lap = Laplacian(g)
    X = np.linalg.qr(blockops.project(G.random_block(g.n, b, 3), None))[0]
    theta, Yr = np.linalg.eigh(X.T @ lap.matvec(X))
    X = X @ Yr
    return X, theta, lap.matvec(X) - X * theta[None, :]


def test_barrier_wait_limit_then_recovery(pkg):
    g = _graph()
    Gd = pkg.Graph(g)
    assert Gd.info()["nlong"] > 0
    b, iters = 6, 6
    X, theta, R = _block(g, b)
    Xd = torch.from_numpy(X).cuda()
    Rd = torch.from_numpy(R).cuda()
    th = torch.from_numpy(theta[None, :]).cuda()
    # a limit of 1 ns: the first CTA to reach the first barrier gives up
    Gd.set_launch(device_timeout_ms=1e-6)
    with pytest.raises(pkg.LapError) as e:
        Gd.pcg_correction(Xd, th, Rd, iters)
    assert e.value.status == pkg.LAP_ETIMEOUT
    # the same handle, default limit: the fixed-step correction is the oracle's
    Gd.set_launch(device_timeout_ms=0.0)
    T = Gd.pcg_correction(Xd, th, Rd, iters).cpu().numpy()
    ref = blockops.pcg_correction(g, theta, R, X, iters)
    assert (np.abs(T - ref).max(axis=0) / np.abs(ref).max(axis=0)).max() <= 1e-8
    # a whole solve with the tiny limit stops with LAP_ETIMEOUT ...
    k = 5
    for precision in ("fp64", "mixed"):
        ev, infos = Gd.eigs(k, 1e-8, precision=precision, device_timeout_ms=1e-6)
        assert infos[0]["status"] == pkg.LAP_ETIMEOUT, infos[0]
    # ... and the next one on the same handle converges to the oracle's values
    V = torch.zeros(g.n * k, dtype=torch.float64, device="cuda")
    ev, infos = Gd.eigs(k, 1e-8, evecs=V, precision="mixed")
    assert infos[0]["status"] == 0, infos[0]
    ev_ref = dense.smallest_eigpairs(g, k)[0]
    assert np.all(np.abs(ev[0] - ev_ref) <= 1e-7 * ev_ref)
    Vh = V.cpu().numpy().reshape(k, g.n).T
    lap = Laplacian(g)
    assert np.linalg.norm(lap.matvec(Vh) - Vh * ev[0][None, :], axis=0).max() <= 1e-8 * lap.norm1
    Gd.close()


def test_wall_clock_cap_gives_partial_result(pkg):
    g = G.workload_graph("c1")
    ev, V, info = pkg.lap_eigs(g, 10, tol=1e-8, max_seconds=1e-9)
    assert info["status"] == pkg.LAP_ETIMEOUT
    assert 0 <= info["n_converged"] < 10
    assert np.all(np.isfinite(ev)) and np.all(np.isfinite(V))


def test_overflow_in_the_fp32_phase_is_a_numeric_error(pkg):
    g = G.ba_graph(500, 3, 9)
    g.weights = np.full(g.colidx.size, 1e39)  # finite in FP64, infinite in FP32
    with pytest.raises(pkg.LapError) as e:
        pkg.lap_eigs(g, 4, tol=1e-8, precision="mixed")
    assert e.value.status == pkg.LAP_ENUMERIC
    # the library stays usable: an ordinary solve right after
    g1 = G.ba_graph(500, 3, 9)
    ev, V, info = pkg.lap_eigs(g1, 4, tol=1e-8, precision="mixed")
    assert info["status"] == 0
    assert np.allclose(ev, dense.smallest_eigpairs(g1, 4)[0], rtol=1e-7)
