"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: closed-form spectra, Eq. 1,
L e = 0, trace and component-count invariants, brute-force loops on tiny
inputs, and the dense definition (LAPACK) for the iterative solvers.
"""
import math

import numpy as np
import pytest

import graphgen as G
from oracle import blockops, dacg, dense, irlm, jd
from oracle.laplacian import Laplacian, dense_laplacian_loops, quadratic_form_edges
from oracle.rng import splitmix64, uniform_block


# ---------------------------------------------------------------- Laplacian

@pytest.mark.parametrize("g", [G.ba_graph(60, 2, 3), G.with_random_weights(G.chung_lu(200, 2.3, 4.0, 1), 4)])
def test_laplacian_matches_entrywise_assembly(g):
    lap = Laplacian(g)
    assert np.array_equal(lap.dense(), dense_laplacian_loops(g))


@pytest.mark.parametrize("weighted", [False, True])
def test_quadratic_form_eq1_and_null_vector(weighted):
    g = G.ba_graph(80, 3, 5)
    if weighted:
        g = G.with_random_weights(g, 2)
    lap = Laplacian(g)
    x = np.random.default_rng(0).standard_normal(g.n)
    # Eq. 1: x^T L x = 1/2 sum A_ij (x_i - x_j)^2  (Section 2)
    assert math.isclose(x @ lap.matvec(x), quadratic_form_edges(g, x), rel_tol=1e-12)
    # L e = 0 (Section 2)
    assert np.abs(lap.matvec(np.ones(g.n))).max() < 1e-12
    # ||L||_1 = max column abs sum = 2 max_i d_i
    Lm = lap.dense()
    assert math.isclose(np.abs(Lm).sum(axis=0).max(), lap.norm1, rel_tol=1e-14)


def test_laplacian_rejects_bad_input():
    g = G.path_graph(4)
    g.weights = np.array([1.0, -1.0, -1.0, 1.0, 1.0, 1.0])
    with pytest.raises(ValueError):
        Laplacian(g)


# ---------------------------------------------------------------- closed forms

def _path(n):
    return np.sort(2 - 2 * np.cos(np.pi * np.arange(n) / n))


CLOSED = [
    (G.path_graph(30), _path(30)),
    (G.cycle_graph(24), np.sort(2 - 2 * np.cos(2 * np.pi * np.arange(24) / 24))),
    (G.star_graph(17), np.array([0.0] + [1.0] * 15 + [17.0])),
    (G.complete_graph(12), np.array([0.0] + [12.0] * 11)),
    (G.complete_bipartite(4, 7), np.sort([0.0] + [4.0] * 6 + [7.0] * 3 + [11.0])),
    (G.grid_graph(5, 8), np.sort((_path(5)[:, None] + _path(8)[None, :]).ravel())),
    (G.hypercube(5), np.sort(np.concatenate([[2.0 * i] * math.comb(5, i) for i in range(6)]))),
]


@pytest.mark.parametrize("g,spec", CLOSED, ids=[c[0].name for c in CLOSED])
def test_dense_spectrum_closed_forms(g, spec):
    assert np.allclose(dense.full_spectrum(g), spec, atol=1e-12)
    # the k smallest on the complement of e: drop the single zero
    ev, V = dense.smallest_eigpairs(g, 5)
    assert np.allclose(ev, spec[1:6], atol=1e-12)
    assert np.abs(V.sum(axis=0)).max() < 1e-10
    assert np.allclose(V.T @ V, np.eye(5), atol=1e-12)


def test_components_multiplicity_and_trace():
    u = G.disjoint_union(G.path_graph(6), G.cycle_graph(7), G.complete_graph(4))
    spec = dense.full_spectrum(u)
    # multiplicity of 0 = number of connected components (Section 2)
    assert np.sum(np.abs(spec) < 1e-10) == 3
    # multiset union of the parts' spectra
    parts = np.sort(np.concatenate([_path(6), 2 - 2 * np.cos(2 * np.pi * np.arange(7) / 7), [0, 4, 4, 4]]))
    assert np.allclose(spec, parts, atol=1e-12)
    # trace L = sum of degrees = 2|E| = sum of eigenvalues
    assert math.isclose(spec.sum(), 2 * u.n_edges, rel_tol=1e-12)
    # on the complement of e the c - 1 extra zeros come first
    ev, _ = dense.smallest_eigpairs(u, 4)
    assert np.allclose(ev[:2], 0, atol=1e-12) and ev[2] > 0.1


def test_include_null_prepends_constant_pair():
    g = G.path_graph(10)
    ev, V = dense.smallest_eigpairs(g, 3, include_null=True)
    assert ev[0] == 0.0 and np.allclose(V[:, 0], 1 / np.sqrt(10))
    assert np.allclose(ev[1:], _path(10)[1:3])


def test_weyl_monotone_under_edge_addition():
    g = G.ba_graph(50, 2, 1)
    s, d, _ = G.edges_of(g)
    g2 = G.csr_from_edges(g.n, np.append(s, 0), np.append(d, 49))
    assert np.all(dense.full_spectrum(g2) >= dense.full_spectrum(g) - 1e-12)


# ---------------------------------------------------------------- iterative solvers

def _check_pairs(g, ev, V, ev_ref, tol):
    lap = Laplacian(g)
    assert np.allclose(ev, ev_ref, rtol=1e-7, atol=1e-10 * lap.norm1)
    R = lap.matvec(V) - V * ev[None, :]
    assert np.linalg.norm(R, axis=0).max() <= tol * lap.norm1
    assert np.abs(V.sum(axis=0)).max() < 1e-8
    assert np.allclose(V.T @ V, np.eye(V.shape[1]), atol=1e-8)


SOLVER_GRAPHS = [
    G.path_graph(120),
    G.grid_graph(9, 13),
    G.ba_graph(300, 2, 21),
    G.chung_lu(600, 2.3, 4.0, 8),
    G.with_random_weights(G.ba_graph(250, 3, 2), 17),
]


@pytest.mark.parametrize("g", SOLVER_GRAPHS, ids=[x.name for x in SOLVER_GRAPHS])
def test_jd_matches_definition(g):
    k = 6
    ev_ref, _ = dense.smallest_eigpairs(g, k)
    ev, V, info = jd.jd_smallest(g, k, tol=1e-8)
    _check_pairs(g, ev, V, ev_ref, 1e-8)
    assert info["outer"] > 0 and info["n_matvec"] > 0


def test_jd_ic0_same_result():
    g = G.ba_graph(200, 2, 4)
    ev_ref, _ = dense.smallest_eigpairs(g, 4)
    ev, V, _ = jd.jd_smallest(g, 4, precond="ic0")
    _check_pairs(g, ev, V, ev_ref, 1e-8)


def test_jd_closed_form_path_eigenvalues():
    n = 200
    ev, V, _ = jd.jd_smallest(G.path_graph(n), 4)
    assert np.allclose(ev, 2 - 2 * np.cos(np.pi * np.arange(1, 5) / n), rtol=1e-9)


@pytest.mark.parametrize("g", SOLVER_GRAPHS[1:4], ids=[x.name for x in SOLVER_GRAPHS[1:4]])
def test_dacg_matches_definition(g):
    k = 4
    ev_ref, _ = dense.smallest_eigpairs(g, k)
    ev, V, info = dacg.dacg_smallest(g, k)
    _check_pairs(g, ev, V, ev_ref, 1e-8)


@pytest.mark.parametrize("g", SOLVER_GRAPHS[1:4] + [SOLVER_GRAPHS[4]], ids=[x.name for x in SOLVER_GRAPHS[1:5]])
def test_irlm_matches_definition(g):
    k = 5
    ev_ref, _ = dense.smallest_eigpairs(g, k)
    ev, V, info = irlm.irlm_smallest(g, k)
    _check_pairs(g, ev, V, ev_ref, 1e-8)


def test_irlm_ncv_table():
    # ncv = 15, 30, 60, 120 for 1, 5, 20, 50 pairs (Section 4)
    assert [irlm.ncv_for(k) for k in (1, 5, 20, 50)] == [15, 30, 60, 120]


# ---------------------------------------------------------------- per-step definitions

def test_spmm_brute_force():
    g = G.with_random_weights(G.ba_graph(40, 2, 9), 3)
    X = uniform_block(5, g.n, 3)
    sh = np.array([0.5, -1.0, 2.0])
    Lm = dense_laplacian_loops(g)
    assert np.allclose(blockops.lap_spmm(g, X, sh), Lm @ X - X * sh, atol=1e-13)


def test_gram_brute_force():
    A = uniform_block(1, 17, 4)
    B = uniform_block(2, 17, 3)
    ref = np.array([[sum(A[r, i] * B[r, j] for r in range(17)) for j in range(3)] for i in range(4)])
    assert np.allclose(blockops.gram(A, B), ref, atol=1e-14)


def test_project_properties():
    n = 50
    Q, _ = np.linalg.qr(blockops.project(uniform_block(3, n, 4), None))
    X = uniform_block(4, n, 3)
    P = blockops.project(X, Q)
    assert np.abs(Q.T @ P).max() < 1e-13 and np.abs(P.sum(axis=0)).max() < 1e-12
    assert np.allclose(blockops.project(P, Q), P, atol=1e-13)
    # X - P lies in span{e, Q}
    B = np.column_stack([np.ones(n) / np.sqrt(n), Q])
    D = X - P
    assert np.allclose(B @ (B.T @ D), D, atol=1e-13)


def test_orthonormalize_is_gram_schmidt():
    n = 40
    Q, _ = np.linalg.qr(blockops.project(uniform_block(6, n, 3), None))
    T = uniform_block(7, n, 4)
    U, R = blockops.orthonormalize(Q, T)
    assert np.allclose(U.T @ U, np.eye(4), atol=1e-13)
    assert np.abs(Q.T @ U).max() < 1e-13 and np.abs(U.sum(axis=0)).max() < 1e-12
    assert np.allclose(np.triu(R), R) and np.all(np.diag(R) > 0)
    # classical Gram-Schmidt written out column by column gives the same U
    P = blockops.project(T, Q)
    cols = []
    for j in range(4):
        v = P[:, j].copy()
        for u in cols:
            v -= (u @ P[:, j]) * u
        cols.append(v / np.linalg.norm(v))
    assert np.allclose(np.column_stack(cols), U, atol=1e-12)


def test_rayleigh_ritz_exact_on_invariant_subspace():
    g = G.grid_graph(6, 7)
    ev, V = dense.smallest_eigpairs(g, 6)
    M = np.linalg.qr(V @ uniform_block(3, 6, 6))[0]  # same span, rotated
    th, X = blockops.rayleigh_ritz(g, M, 3)
    assert np.allclose(th, ev[:3], atol=1e-12)
    assert blockops.residual_norms(g, X, th).max() < 1e-11


def test_pcg_correction_solves_projected_system():
    g = G.ba_graph(120, 2, 5)
    ev, V = dense.smallest_eigpairs(g, 3)
    Q = V[:, :1]
    theta = np.array([0.5 * ev[0], 0.2 * ev[0]])  # below the spectrum on the complement: SPD case
    R = blockops.project(uniform_block(9, g.n, 2), Q)
    T = blockops.pcg_correction(g, theta, R, Q, iters=400)
    lap = Laplacian(g)
    B = np.column_stack([np.ones(g.n) / np.sqrt(g.n), Q])
    for j in range(2):
        # direct solve on the complement: Z^T (L - theta) Z y = -Z^T r, t = Z y
        Z = np.linalg.svd(np.eye(g.n) - B @ B.T)[0][:, :g.n - 2]
        y = np.linalg.solve(Z.T @ (lap.dense() - theta[j] * np.eye(g.n)) @ Z, -Z.T @ R[:, j])
        assert np.allclose(T[:, j], Z @ y, atol=1e-9)


def test_projected_product_identity_of_the_two_phase_step():
    """The reading behind the correction solve's two-phase step: with L e = 0
    and Q = [e/sqrt(n), X] orthonormal, for any z and theta
        (L - theta)(I - QQ^T) z = (L z - theta z) + theta g0 e - (LX - theta X) g,
    g0 = mean(z), g = X^T z; so the product of the new search direction needs
    only the SpMM of z and the fixed block LX."""
    g = G.with_random_weights(G.ba_graph(90, 3, 4), 2)
    lap = Laplacian(g)
    Q = np.linalg.qr(blockops.project(uniform_block(5, g.n, 4), None))[0]
    X = Q
    LX = lap.matvec(X)
    z = uniform_block(6, g.n, 1)[:, 0]
    B = np.column_stack([np.ones(g.n) / np.sqrt(g.n), X])
    for theta in (0.0, 0.37, 2.5):
        lhs = lap.matvec((z - B @ (B.T @ z))[:, None])[:, 0] - theta * (z - B @ (B.T @ z))
        g0, gx = z.mean(), X.T @ z
        rhs = (lap.matvec(z[:, None])[:, 0] - theta * z) + theta * g0 * np.ones(g.n) - (LX - theta * X) @ gx
        assert np.allclose(lhs, rhs, atol=1e-12)


# ---------------------------------------------------------------- generator

def test_splitmix64_reference_vector():
    rows = [l.split() for l in open(__file__.replace("test_oracle.py", "golden/splitmix64.txt"))
            if l.strip() and not l.startswith("#")]
    for r in rows:
        got = splitmix64(int(r[0]), np.arange(3, dtype=np.uint64))
        assert [int(v) for v in got] == [int(x, 16) for x in r[1:]]
    u = uniform_block(0, 100, 3)
    assert u.min() >= -1 and u.max() < 1 and abs(u.mean()) < 0.2


# ---------------------------------------------------------------- pins of the correction solve, IC(0), signs

def _cg_krylov_minimiser(A, M, rhs, j):
    """The j-th iterate of preconditioned CG from t = 0, by its defining
    property and not by its recurrences: on an SPD operator A with SPD
    preconditioner M, t_j minimises (t* - t)^T A (t* - t) over the Krylov space
    K_j(M A, M rhs), so t_j = K (K^T A K)^{-1} K^T rhs for any basis K of it."""
    cols = [M @ rhs]
    for _ in range(j - 1):
        cols.append(M @ (A @ cols[-1]))
    K = np.linalg.qr(np.column_stack(cols))[0]  # orthonormal basis of the same span
    return K @ np.linalg.solve(K.T @ A @ K, K.T @ rhs)


@pytest.mark.parametrize("weighted,kind", [(False, "jacobi"), (True, "jacobi"), (False, "fsai"), (True, "fsai")])
def test_pcg_correction_iterates_are_cg_optimal(weighted, kind):
    """Algorithm 2 step 8 after j steps (not only at convergence): with Q =
    [e/sqrt(n), X] and theta below the spectrum of L on the complement of Q
    (the SPD case), the projected operator A = Pi (L - theta) Pi and the
    projected preconditioner M = Pi D^{-1} Pi (Section 3.2.1 with P = D^{-1})
    are SPD on range(Pi), and the oracle's iterate after j steps must be the
    A-norm minimiser over K_j(M A, M rhs), rhs = -Pi r.  A dropped outer
    projection, a wrong beta or alpha, or a missing preconditioner changes the
    Krylov space or the minimiser and fails this."""
    g = G.ba_graph(48, 2, 11)
    if weighted:
        g = G.with_random_weights(g, 5)
    lap = Laplacian(g)
    n = g.n
    X = np.linalg.qr(blockops.project(uniform_block(21, n, 3), None))[0]
    B = np.column_stack([np.ones(n) / np.sqrt(n), X])
    Pi = np.eye(n) - B @ B.T
    Lm = lap.dense()
    # smallest eigenvalue of L on range(Pi)
    Z = np.linalg.svd(Pi)[0][:, :n - 4]
    lam = np.linalg.eigvalsh(Z.T @ Lm @ Z)[0]
    theta = np.array([0.5 * lam, 0.1 * lam, 0.9 * lam])
    R = uniform_block(22, n, 3)
    from oracle import precond as pc
    if kind == "jacobi":
        Mfull, fn = np.diag(1.0 / lap.d), None
    else:
        Gf = pc.fsai_factor(lap.L).toarray()
        Mfull = Gf.T @ Gf
        fn = pc.make_preconditioner(lap, "fsai")
    M = Pi @ Mfull @ Pi
    for j in (1, 2, 3, 5, 8):
        T = blockops.pcg_correction(g, theta, R, X, iters=j, precond=fn)
        for c in range(3):
            A = Pi @ (Lm - theta[c] * np.eye(n)) @ Pi
            ref = _cg_krylov_minimiser(A, M, -Pi @ R[:, c], j)
            assert np.allclose(T[:, c], ref, rtol=0, atol=1e-10 * np.abs(ref).max()), (j, c)


def test_ic0_factor_reproduces_the_pattern_entries():
    """IC(0) (Section 4, Section 3.1.1): F is lower triangular with exactly the
    pattern of tril(M), M = L + alpha diag(L), and (F F^T)_ij = M_ij on that
    pattern (no fill-in is kept, the kept entries are exact)."""
    g = G.with_random_weights(G.chung_lu(150, 2.3, 4.0, 6), 3)
    lap = Laplacian(g)
    alpha = 1e-3
    from oracle import precond
    F = precond.ic0_factor(lap.L, alpha)
    assert F is not None
    M = (lap.L + alpha * __import__("scipy.sparse", fromlist=["diags"]).diags(lap.L.diagonal())).toarray()
    Fd = F.toarray()
    pat = np.tril(M) != 0
    assert np.array_equal(Fd != 0, pat)
    FF = Fd @ Fd.T
    assert np.allclose(FF[pat], M[pat], rtol=0, atol=1e-12 * np.abs(M).max())
    # off the pattern F F^T differs from M (fill-in was dropped), so the test is not vacuous
    assert np.abs(FF[~pat & np.tri(g.n, dtype=bool)]).max() > 1e-6


def test_canonical_signs_convention():
    """Sign reading: the entry of largest magnitude of each returned vector is
    positive, the first such entry on an exact tie."""
    V = np.array([[0.1, 0.5, -0.5, 0.0],
                  [-0.9, -0.5, 0.5, -0.2],
                  [0.3, 0.1, 0.1, 0.0]])
    W = dense.canonical_signs(V)
    assert np.array_equal(W[:, 0], -V[:, 0])
    assert np.array_equal(W[:, 1], V[:, 1])
    assert np.array_equal(W[:, 2], -V[:, 2])
    assert np.array_equal(W[:, 3], -V[:, 3])
    assert np.array_equal(V[0], [0.1, 0.5, -0.5, 0.0])  # input untouched



@pytest.mark.parametrize("cap", [32, 2])
def test_fsai_factor_defining_conditions(cap):
    """Factored approximate inverse (Section 5's product of sparse matrices):
    G lower triangular on the pattern of tril(A) (rows over the cap keep
    their diagonal), (G A)_ij = 0 for j < i in the row's pattern, and
    (G A G^T)_ii = 1, A = L + alpha diag(L)."""
    from oracle import precond as pc
    import scipy.sparse as sp
    g = G.with_random_weights(G.chung_lu(200, 2.3, 4.0, 3), 5)
    lap = Laplacian(g)
    alpha = 1e-3
    Gm = pc.fsai_factor(lap.L, alpha, cap).toarray()
    A = (lap.L + alpha * sp.diags(lap.L.diagonal())).toarray()
    assert np.allclose(np.triu(Gm, 1), 0.0)
    low = np.tril(A) != 0
    capped = low.sum(axis=1) > cap
    pat = low.copy()
    pat[capped] = np.eye(g.n, dtype=bool)[capped]
    assert np.array_equal(Gm != 0, pat)
    GA = Gm @ A
    off = pat & ~np.eye(g.n, dtype=bool)
    assert np.abs(GA[off]).max() < 1e-12 * np.abs(A).max()
    assert np.allclose(np.diag(Gm @ A @ Gm.T), 1.0, atol=1e-12)
    if cap == 2:
        assert capped.any()


def test_fsai_with_a_full_pattern_is_the_exact_inverse():
    """On a complete graph tril(A) is full: G is the inverse Cholesky factor
    and G^T G = A^{-1} exactly."""
    from oracle import precond as pc
    import scipy.sparse as sp
    g = G.complete_graph(9)
    lap = Laplacian(g)
    Gm = pc.fsai_factor(lap.L, 1e-3).toarray()
    A = (lap.L + 1e-3 * sp.diags(lap.L.diagonal())).toarray()
    assert np.allclose(Gm.T @ Gm, np.linalg.inv(A), atol=1e-10)


@pytest.mark.parametrize("g", [G.ba_graph(300, 2, 21), G.chung_lu(600, 2.3, 4.0, 8)], ids=["ba300", "cl600"])
def test_jd_with_fsai_reaches_the_same_pairs(g):
    """The preconditioner changes the iteration counts, not the pairs.  (Like
    any single-vector JD with locking, the oracle can skip an eigenvalue and
    lock the next one first; ba(200, 2, 4) does so with this preconditioner,
    which is why the GPU solver works on a block.)"""
    ev_ref, _ = dense.smallest_eigpairs(g, 4)
    ev, V, _ = jd.jd_smallest(g, 4, precond="fsai")
    _check_pairs(g, ev, V, ev_ref, 1e-8)
