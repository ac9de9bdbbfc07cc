"""Step-level parity: each kernel of the Jacobi-Davidson outer loop, called
through the C ABI on device blocks, against the oracle's definition on the
same seeded inputs.  Sizes span several row tiles with a ragged tail; graphs
include power-law hubs (the one-CTA-per-row path), weights and batches."""
import numpy as np
import pytest

import graphgen as G
from oracle import blockops, dense
from oracle.laplacian import Laplacian

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
EPS = {torch.float64: np.finfo(np.float64).eps, torch.float32: np.finfo(np.float32).eps}


@pytest.fixture(scope="module")
def pkg():
    import paper_1311_1695_gb300 as p
    from paper_1311_1695_gb300 import build
    build.build()
    return p


GRAPHS = {
    "ba": lambda: G.ba_graph(3001, 2, 5),
    "cl_hubs": lambda: G.chung_lu(20000, 2.1, 7.0, 3, cap=2000.0),
    "weighted": lambda: G.with_random_weights(G.chung_lu(5000, 2.3, 5.0, 4), 8),
    "grid": lambda: G.grid_graph(37, 41),
}


def _dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dt).cuda()


def _abs_bound(g, X):
    """|L| |X| row by row and the row lengths, for a rounding bound."""
    lap = Laplacian(g)
    absL = abs(lap.L)
    return absL @ np.abs(X), np.diff(g.rowptr) + 2


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("b", [1, 3, 10, 20, 33])
def test_spmm(pkg, name, dt, b):
    g = GRAPHS[name]()
    Gd = pkg.Graph(g)
    X = G.random_block(g.n, b, 11).astype(np.float32 if dt == torch.float32 else np.float64)
    Xd = _dev(X, dt)
    Yd = torch.empty_like(Xd)
    Gd.spmm(Xd, Yd)
    Y = Yd.cpu().double().numpy()
    ref = blockops.lap_spmm(g, X.astype(np.float64))
    S, deg = _abs_bound(g, X.astype(np.float64))
    bound = 2 * EPS[dt] * deg[:, None] * S + 1e-300
    assert np.all(np.abs(Y - ref) <= bound), np.max(np.abs(Y - ref) / bound)
    Gd.close()


@pytest.mark.parametrize("team", [4, 8, 16, 32])
def test_spmm_schedules_agree(pkg, team):
    g = GRAPHS["cl_hubs"]()
    Gd = pkg.Graph(g)
    X = _dev(G.random_block(g.n, 8, 3), torch.float64)
    Y0 = torch.empty_like(X)
    Gd.spmm(X, Y0)
    Gd.set_schedule(team=team, long_thresh=16)
    assert Gd.info()["nlong"] > 0
    Y1 = torch.empty_like(X)
    Gd.spmm(X, Y1)
    assert torch.allclose(Y0, Y1, rtol=1e-12, atol=1e-12 * Y0.abs().max().item())
    Gd.close()


def test_spmm_batched_block_diagonal(pkg):
    gs = [G.ba_graph(700, 3, 1), G.grid_graph(20, 30), G.chung_lu(3000, 2.5, 4.0, 9)]
    Gd = pkg.Graph(gs)
    n = sum(x.n for x in gs)
    X = G.random_block(n, 6, 2)
    Yd = torch.empty((n, 6), dtype=torch.float64, device="cuda")
    Gd.spmm(_dev(X, torch.float64), Yd)
    Y = Yd.cpu().numpy()
    off = 0
    for x in gs:
        ref = blockops.lap_spmm(x, X[off:off + x.n])
        assert np.abs(Y[off:off + x.n] - ref).max() <= 1e-12 * np.abs(ref).max()
        off += x.n
    Gd.close()


def test_spmm_empty_rows_and_tiny(pkg):
    # a star has one hub and n-1 rows of length 1; a 2-node path the smallest graph
    for g in (G.star_graph(5000), G.path_graph(2)):
        Gd = pkg.Graph(g)
        X = G.random_block(g.n, 4, 1)
        Yd = torch.empty((g.n, 4), dtype=torch.float64, device="cuda")
        Gd.spmm(_dev(X, torch.float64), Yd)
        ref = blockops.lap_spmm(g, X)
        assert np.abs(Yd.cpu().numpy() - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max())
        Gd.close()


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("p,q,ones", [(0, 5, 1), (7, 3, 0), (12, 12, 1), (40, 10, 0), (63, 20, 1)])
def test_gram(pkg, dt, p, q, ones):
    g = GRAPHS["cl_hubs"]()
    Gd = pkg.Graph(g)
    A = G.random_block(g.n, max(p, 1), 1)[:, :p] if p else None
    B = G.random_block(g.n, q, 2)
    npdt = np.float32 if dt == torch.float32 else np.float64
    Ad = None if A is None else _dev(A.astype(npdt), dt)
    Gm = Gd.gram(Ad, _dev(B.astype(npdt), dt), ones=bool(ones)).cpu().numpy()[0]
    A64 = np.zeros((g.n, 0)) if A is None else A.astype(npdt).astype(np.float64)
    B64 = B.astype(npdt).astype(np.float64)
    ref = blockops.gram(A64, B64)
    if ones:
        ref = np.vstack([B64.mean(axis=0, keepdims=True), ref])
    tol = (64 if dt == torch.float64 else 64 * 32) * EPS[dt] * g.n
    assert np.abs(Gm - ref).max() <= tol, np.abs(Gm - ref).max()
    Gd.close()


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_project(pkg, dt):
    g = GRAPHS["weighted"]()
    Gd = pkg.Graph(g)
    Q, _ = np.linalg.qr(blockops.project(G.random_block(g.n, 6, 5), None))
    X = G.random_block(g.n, 9, 6)
    npdt = np.float32 if dt == torch.float32 else np.float64
    Xd = _dev(X.astype(npdt), dt)
    Gd.project(_dev(Q.astype(npdt), dt), Xd)
    ref = blockops.project(X.astype(npdt).astype(np.float64), Q.astype(npdt).astype(np.float64))
    tol = 1e-12 if dt == torch.float64 else 2e-5
    assert np.abs(Xd.cpu().double().numpy() - ref).max() <= tol * np.abs(X).max() * 10
    Gd.close()


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("m,b", [(0, 4), (6, 10), (20, 12)])
def test_cgs2(pkg, dt, m, b):
    g = GRAPHS["ba"]()
    Gd = pkg.Graph(g)
    V = np.linalg.qr(blockops.project(G.random_block(g.n, max(m, 1), 4), None))[0][:, :m]
    T = G.random_block(g.n, b, 8)
    npdt = np.float32 if dt == torch.float32 else np.float64
    Td = _dev(T.astype(npdt), dt)
    kept = Gd.cgs2(_dev(V.astype(npdt), dt) if m else None, Td)
    assert kept.all()
    U = Td.cpu().double().numpy()
    ref, _ = blockops.orthonormalize(V.astype(npdt).astype(np.float64) if m else None, T.astype(npdt).astype(np.float64))
    tol = 1e-10 if dt == torch.float64 else 2e-4
    assert np.abs(U - ref).max() <= tol
    assert np.abs(U.T @ U - np.eye(b)).max() <= (1e-12 if dt == torch.float64 else 2e-6)
    Gd.close()


def test_cgs2_drops_dependent_columns(pkg):
    g = GRAPHS["grid"]()
    Gd = pkg.Graph(g)
    V = np.linalg.qr(blockops.project(G.random_block(g.n, 5, 4), None))[0]
    T = G.random_block(g.n, 6, 9)
    T[:, 2] = V @ np.arange(1, 6)  # inside span(V)
    T[:, 4] = 2 * T[:, 1] - T[:, 0]  # dependent on earlier columns
    T[:, 5] = 0.0  # empty
    Td = _dev(T, torch.float64)
    kept = Gd.cgs2(_dev(V, torch.float64), Td)
    assert list(kept[0]) == [1, 1, 0, 1, 0, 0]
    U = Td.cpu().numpy()
    assert np.abs(U[:, [2, 4, 5]]).max() == 0.0
    ref, _ = blockops.orthonormalize(V, T[:, [0, 1, 3]])
    assert np.abs(U[:, [0, 1, 3]] - ref).max() <= 1e-10
    Gd.close()


@pytest.mark.parametrize("m", [1, 2, 7, 24, 44, 64])
def test_syev(pkg, m):
    rng = np.random.default_rng(m)
    H = rng.standard_normal((4, m, m))
    H = H + H.transpose(0, 2, 1)
    H[1] = np.diag(np.arange(m, dtype=float)) + 1e-3 * H[1]  # nearly diagonal
    H[2] = np.kron(np.eye((m + 1) // 2), np.ones((2, 2)))[:m, :m]  # repeated eigenvalues
    # graded spectrum over six decades (the spread of a Laplacian's Ritz values)
    Q = np.linalg.qr(rng.standard_normal((m, m)))[0]
    H[3] = (Q * np.logspace(-6, 0, m)[None, :]) @ Q.T
    H[3] = 0.5 * (H[3] + H[3].T)
    ev, Y = pkg.lap_syev_batched(torch.from_numpy(H).cuda())
    ev, Y = ev.cpu().numpy(), Y.cpu().numpy()
    for i in range(4):
        ref = np.linalg.eigvalsh(H[i])
        assert np.abs(ev[i] - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max()) * m
        assert np.abs(Y[i].T @ Y[i] - np.eye(m)).max() <= 1e-13 * m
        assert np.abs(H[i] @ Y[i] - Y[i] * ev[i][None, :]).max() <= 1e-13 * m * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_rayleigh_ritz_and_residuals(pkg, dt):
    g = GRAPHS["ba"]()
    Gd = pkg.Graph(g)
    ev, U = dense.smallest_eigpairs(g, 12)
    # a basis whose span contains the 8 smallest eigenvectors exactly, plus noise directions
    B = np.column_stack([U[:, :8], blockops.project(G.random_block(g.n, 4, 3), U[:, :8])])
    B = np.linalg.qr(B)[0] @ np.linalg.qr(G.random_block(12, 12, 4))[0]
    npdt = np.float32 if dt == torch.float32 else np.float64
    Vd = _dev(B.astype(npdt), dt)
    theta = Gd.rayleigh_ritz(Vd)
    th = theta.cpu().numpy()[0]
    tol = 1e-10 if dt == torch.float64 else 1e-4
    assert np.abs(th[:8] - ev[:8]).max() <= tol * max(1, ev[7])
    rn = Gd.residual_norms(Vd[:, :8].contiguous(), theta[:, :8].contiguous()).cpu().numpy()[0]
    ref = blockops.residual_norms(g, Vd[:, :8].cpu().double().numpy(), th[:8])
    assert np.abs(rn - ref).max() <= (1e-11 if dt == torch.float64 else 1e-4) * Laplacian(g).norm1
    Gd.close()


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("name", ["ba", "weighted"])
def test_pcg_correction_fixed_steps(pkg, dt, name):
    g = GRAPHS[name]()
    Gd = pkg.Graph(g)
    ev, U = dense.smallest_eigpairs(g, 6) if g.n <= 4000 else (None, None)
    if U is None:
        U = np.linalg.qr(blockops.project(G.random_block(g.n, 6, 1), None))[0]
        lap = Laplacian(g)
        th0 = np.einsum("ij,ij->j", U, lap.matvec(U))
    else:
        th0 = ev
    # perturbed Ritz-like block: X orthonormal, theta its Rayleigh quotients, R its residuals
    X = np.linalg.qr(blockops.project(U + 1e-2 * G.random_block(g.n, 6, 2), None))[0]
    lap = Laplacian(g)
    # Ritz vectors of span(X): the residuals are then orthogonal to [e, X]
    theta, Yr = np.linalg.eigh(X.T @ lap.matvec(X))
    X = X @ Yr
    R = lap.matvec(X) - X * theta[None, :]
    npdt = np.float32 if dt == torch.float32 else np.float64
    X, R = X.astype(npdt), R.astype(npdt)
    iters = 8
    Td = Gd.pcg_correction(_dev(X, dt), torch.from_numpy(theta[None, :]).cuda(), _dev(R, dt), iters)
    T = Td.cpu().double().numpy()
    ref = blockops.pcg_correction(g, theta, R.astype(np.float64), X.astype(np.float64), iters)
    scale = np.abs(ref).max(axis=0)
    err = (np.abs(T - ref).max(axis=0) / scale).max()
    assert err <= (1e-8 if dt == torch.float64 else 5e-3), err
    Gd.close()


@pytest.mark.parametrize("p,q,ld_in,beta,ones", [(4, 32, 4, 0.0, 0), (6, 32, 6, 1.0, 1), (32, 16, 32, 0.0, 0),
                                                 (65 - 1, 24, 64, 0.0, 1)])
def test_block_update(pkg, p, q, ld_in, beta, ones):
    """lap_block_update: Y = beta Y + [1 | A] S, including p < q."""
    import ctypes
    g = GRAPHS["grid"]()
    Gd = pkg.Graph(g)
    A = G.random_block(g.n, ld_in, 3).astype(np.float32)
    Y0 = G.random_block(g.n, q, 4).astype(np.float32)
    S = np.random.default_rng(5).standard_normal((p + ones, q))
    Ad, Yd = _dev(A, torch.float32), _dev(Y0, torch.float32)
    Sd = torch.from_numpy(S).cuda()
    st = pkg.lib().lap_block_update(Gd.h, pkg.LAP_F32, ctypes.c_void_p(Yd.data_ptr()), q, q, beta, 1.0,
                                    ctypes.c_void_p(Ad.data_ptr()), ld_in, p, ones, ctypes.c_void_p(Sd.data_ptr()), q, 0,
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    A64 = A[:, :p].astype(np.float64)
    ref = beta * Y0 + (np.hstack([np.ones((g.n, 1)), A64]) if ones else A64) @ S
    assert np.abs(Yd.cpu().double().numpy() - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max())
    Gd.close()


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_pcg_correction_batched_with_hubs(pkg, dt):
    """The fused correction solve on a batch handle: per-graph scalars and
    hub rows (chunked; several graphs' hubs) against the oracle graph by graph."""
    # (no star graph here: its eigenvalue 1 of multiplicity n - 2 makes the
    # shifted system at theta ~ 1 singular and both solves diverge)
    gs = [G.chung_lu(4000, 2.1, 6.0, 21, cap=900.0), G.grid_graph(25, 30), G.ba_graph(1500, 4, 23),
          G.with_random_weights(G.chung_lu(2500, 2.3, 5.0, 22), 5)]
    Gd = pkg.Graph(gs)
    assert Gd.info()["nlong"] > 0
    b, iters = 5, 7
    npdt = np.float32 if dt == torch.float32 else np.float64
    Xs, Rs, ths = [], [], []
    for i, g in enumerate(gs):
        lap = Laplacian(g)
        X = np.linalg.qr(blockops.project(G.random_block(g.n, b, 30 + i), None))[0]
        theta, Yr = np.linalg.eigh(X.T @ lap.matvec(X))
        X = X @ Yr
        R = lap.matvec(X) - X * theta[None, :]
        Xs.append(X.astype(npdt)); Rs.append(R.astype(npdt)); ths.append(theta)
    Td = Gd.pcg_correction(_dev(np.vstack(Xs), dt), torch.from_numpy(np.vstack(ths)).cuda(),
                           _dev(np.vstack(Rs), dt), iters)
    T = Td.cpu().double().numpy()
    off = 0
    for g, X, R, th in zip(gs, Xs, Rs, ths):
        ref = blockops.pcg_correction(g, th, R.astype(np.float64), X.astype(np.float64), iters)
        err = (np.abs(T[off:off + g.n] - ref).max(axis=0) / np.abs(ref).max(axis=0)).max()
        assert err <= (1e-8 if dt == torch.float64 else 5e-3), err
        off += g.n
    Gd.close()


_WIDE = {}


def _wide_graph():
    """A weighted BA graph (3,001 nodes, hubs) and its 30 smallest eigenvectors, once."""
    if not _WIDE:
        g = G.with_random_weights(G.ba_graph(3001, 2, 5), 8)
        _WIDE["g"] = g
        _WIDE["U"] = dense.smallest_eigpairs(g, 30)[1]
    return _WIDE["g"], _WIDE["U"]


def _ritz_block(g, U, b, seed):
    """X: b Ritz vectors of a block near the smallest eigenvectors U (orthonormal,
    orthogonal to e), theta their Ritz values, R their residuals (orthogonal to
    [e, X]), as in a JD outer iteration."""
    lap = Laplacian(g)
    U = U[:, :b]
    X = np.linalg.qr(blockops.project(U + 1e-2 * G.random_block(g.n, b, seed), None))[0]
    theta, Yr = np.linalg.eigh(X.T @ lap.matvec(X))
    X = X @ Yr
    R = lap.matvec(X) - X * theta[None, :]
    return X, theta, R


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("b", [12, 20, 22, 30])
@pytest.mark.parametrize("max_ctas", [0, 16, 2])
def test_pcg_correction_wide_blocks_and_tiles_per_cta(pkg, dt, b, max_ctas):
    """The correction solve at the block widths the benchmarked solves use
    (b = 12: 16-lane row groups; b = 20, 22: the 24-column instantiation;
    b = 30: 32 columns) and with several row tiles per CTA: max_ctas = 0 gives
    one tile per CTA (X rows resident), 16 gives about three per CTA (resident
    where shared memory allows, else re-staged per tile and phase), 2 gives
    more than twenty (re-staged), against the oracle's fixed-step projected
    PCG.  Weighted edges and hub rows included."""
    g, U = _wide_graph()
    Gd = pkg.Graph(g)
    assert Gd.info()["nlong"] > 0
    Gd.set_launch(max_ctas=max_ctas)
    X, theta, R = _ritz_block(g, U, b, 40 + b)
    npdt = np.float32 if dt == torch.float32 else np.float64
    X, R = X.astype(npdt), R.astype(npdt)
    if dt == torch.float32:
        # FP32: a shift below the spectrum on the complement of [e, X] (an SPD
        # system), so the FP32 iterates follow the FP64 ones to rounding; at
        # the Ritz values of the wide blocks the shifted system is nearly
        # singular in some columns and 8 FP32 steps drift from the FP64 ones
        theta = np.full_like(theta, 0.5 * theta[0])
    iters = 8
    Td = Gd.pcg_correction(_dev(X, dt), torch.from_numpy(theta[None, :]).cuda(), _dev(R, dt), iters)
    T = Td.cpu().double().numpy()
    ref = blockops.pcg_correction(g, theta, R.astype(np.float64), X.astype(np.float64), iters)
    err = (np.abs(T - ref).max(axis=0) / np.abs(ref).max(axis=0)).max()
    assert err <= (1e-8 if dt == torch.float64 else 5e-3), err
    Gd.close()


def _kernel_names(pkg, run):
    pkg.lap_profile_read()
    pkg.lap_profile_enable(True)
    try:
        run()
        return set(pkg.lap_profile_read())
    finally:
        pkg.lap_profile_enable(False)


@pytest.mark.parametrize("dt,b", [(torch.float32, 4), (torch.float32, 8), (torch.float32, 12), (torch.float32, 16),
                                  (torch.float64, 2), (torch.float64, 4), (torch.float64, 8)])
@pytest.mark.parametrize("max_ctas", [0, 7])
def test_pcg_correction_per_phase_form(pkg, dt, b, max_ctas):
    """The per-phase correction solve (one launch per PCG phase, row tiles
    staged by bulk copies), forced on from the first row, against the
    oracle's fixed-step projected PCG; with 7 CTAs each walks many tiles."""
    g, U = _wide_graph()
    Gd = pkg.Graph(g)
    Gd.set_launch(max_ctas=max_ctas, split_rows=1)
    X, theta, R = _ritz_block(g, U, b, 70 + b)
    npdt = np.float32 if dt == torch.float32 else np.float64
    X, R = X.astype(npdt), R.astype(npdt)
    iters = 8
    out = {}

    def run():
        out["T"] = Gd.pcg_correction(_dev(X, dt), torch.from_numpy(theta[None, :]).cuda(), _dev(R, dt), iters)
    names = _kernel_names(pkg, run)
    assert "pcg_split" in names and "pcg_fused" not in names, names
    T = out["T"].cpu().double().numpy()
    ref = blockops.pcg_correction(g, theta, R.astype(np.float64), X.astype(np.float64), iters)
    err = (np.abs(T - ref).max(axis=0) / np.abs(ref).max(axis=0)).max()
    assert err <= (1e-8 if dt == torch.float64 else 5e-3), err
    Gd.close()


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_pcg_per_phase_form_batched_with_hubs(pkg, dt):
    """The per-phase form on a batch handle (per-graph accumulators and hub
    rows of several graphs) against the oracle graph by graph."""
    gs = [G.chung_lu(4000, 2.1, 6.0, 21, cap=900.0), G.grid_graph(25, 30), G.ba_graph(1500, 4, 23),
          G.with_random_weights(G.chung_lu(2500, 2.3, 5.0, 22), 5)]
    Gd = pkg.Graph(gs)
    Gd.set_launch(split_rows=1)
    b, iters = 8 if dt == torch.float32 else 4, 7
    npdt = np.float32 if dt == torch.float32 else np.float64
    Xs, Rs, ths = [], [], []
    for i, g in enumerate(gs):
        lap = Laplacian(g)
        X = np.linalg.qr(blockops.project(G.random_block(g.n, b, 30 + i), None))[0]
        theta, Yr = np.linalg.eigh(X.T @ lap.matvec(X))
        X = X @ Yr
        R = lap.matvec(X) - X * theta[None, :]
        Xs.append(X.astype(npdt)); Rs.append(R.astype(npdt)); ths.append(theta)
    out = {}

    def run():
        out["T"] = Gd.pcg_correction(_dev(np.vstack(Xs), dt), torch.from_numpy(np.vstack(ths)).cuda(),
                                     _dev(np.vstack(Rs), dt), iters)
    assert "pcg_split" in _kernel_names(pkg, run)
    T = out["T"].cpu().double().numpy()
    off = 0
    for g, X, R, th in zip(gs, Xs, Rs, ths):
        ref = blockops.pcg_correction(g, th, R.astype(np.float64), X.astype(np.float64), iters)
        err = (np.abs(T[off:off + g.n] - ref).max(axis=0) / np.abs(ref).max(axis=0)).max()
        assert err <= (1e-8 if dt == torch.float64 else 5e-3), err
        off += g.n
    Gd.close()


@pytest.mark.parametrize("dt,b", [(torch.float32, 12), (torch.float32, 4), (torch.float64, 8)])
def test_pcg_correction_with_approximate_inverse(pkg, dt, b):
    """The correction solve with the factored approximate inverse G^T G
    (two sparse products per step) against the oracle's fixed-step projected
    PCG with the oracle's own FSAI factor."""
    from oracle import precond as pc
    g, U = _wide_graph()
    Gd = pkg.Graph(g)
    Gd.set_precond("fsai")
    X, theta, R = _ritz_block(g, U, b, 90 + b)
    npdt = np.float32 if dt == torch.float32 else np.float64
    X, R = X.astype(npdt), R.astype(npdt)
    if dt == torch.float32:
        theta = np.full_like(theta, 0.5 * theta[0])  # SPD shift: FP32 follows FP64 to rounding
    iters = 8
    out = {}

    def run():
        out["T"] = Gd.pcg_correction(_dev(X, dt), torch.from_numpy(theta[None, :]).cuda(), _dev(R, dt), iters)
    names = _kernel_names(pkg, run)
    assert "pcg_split" in names and "pcg_fused" not in names, names
    T = out["T"].cpu().double().numpy()
    M = pc.make_preconditioner(Laplacian(g), "fsai")
    ref = blockops.pcg_correction(g, theta, R.astype(np.float64), X.astype(np.float64), iters, precond=M)
    err = (np.abs(T - ref).max(axis=0) / np.abs(ref).max(axis=0)).max()
    assert err <= (1e-8 if dt == torch.float64 else 5e-3), err
    Gd.close()


@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
@pytest.mark.parametrize("b", [2, 12])
def test_autotuned_schedule_matches_oracle(pkg, dt, b):
    """The autotuner picks among its candidates and the SpMM it leaves in
    place gives the oracle's L X (hub rows included)."""
    g = GRAPHS["cl_hubs"]()
    Gd = pkg.Graph(g)
    u, h = Gd.autotune("f32" if dt == torch.float32 else "f64", b)
    assert h in (32, 64, 128, 256, 1 << 30)
    assert u in ((2, 4, 8, 102, 104) if b >= 3 else (4, 8, 16, 32))
    X = G.random_block(g.n, b, 21).astype(np.float32 if dt == torch.float32 else np.float64)
    Xd = _dev(X, dt)
    Yd = torch.empty_like(Xd)
    Gd.spmm(Xd, Yd)
    ref = blockops.lap_spmm(g, X.astype(np.float64))
    S, deg = _abs_bound(g, X.astype(np.float64))
    assert np.all(np.abs(Yd.cpu().double().numpy() - ref) <= 2 * EPS[dt] * deg[:, None] * S + 1e-300)
    Gd.close()


@pytest.mark.parametrize("gathers", [2, 4, 8, 102, 104])
@pytest.mark.parametrize("dt,b", [(torch.float32, 12), (torch.float32, 5), (torch.float64, 6)])
def test_every_vectorised_form_matches_oracle(pkg, gathers, dt, b):
    """Each form of the vectorised SpMM the autotuner chooses among (lanes
    per row with 2/4/8 gathers in flight, or a lane per row with 2/4
    neighbours in flight) gives the oracle's L X, hub rows included."""
    g = GRAPHS["cl_hubs"]()
    Gd = pkg.Graph(g)
    Gd.set_gathers(gathers)
    X = G.random_block(g.n, b, 23).astype(np.float32 if dt == torch.float32 else np.float64)
    Xd = _dev(X, dt)
    Yd = torch.empty_like(Xd)
    Gd.spmm(Xd, Yd)
    ref = blockops.lap_spmm(g, X.astype(np.float64))
    S, deg = _abs_bound(g, X.astype(np.float64))
    assert np.all(np.abs(Yd.cpu().double().numpy() - ref) <= 2 * EPS[dt] * deg[:, None] * S + 1e-300)
    Gd.close()
