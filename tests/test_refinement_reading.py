"""The small eigensolver's fast mode (CPU check of the reading, no GPU): FP32
Jacobi eigenvectors of the projected matrix H, then one refinement step in
the form of Ogita and Aishima ("Iterative refinement for symmetric eigenvalue
decomposition", 2018) with first-order corrections bounded by 1e-3 of the gap
(closer pairs, and equal Ritz values, kept as a cluster) and a Newton-Schulz
orthonormalisation.  Written here in numpy from that description: it must
take FP32-accurate vectors of separated eigenvalues to FP64 accuracy, and it
must not produce 0/0 for exactly equal eigenvalues."""
import numpy as np


def refine(H, X, lam, nr):
    """One refinement step of the first nr columns of X (FP64 arrays)."""
    m = H.shape[0]
    Xr = X[:, :nr]
    Z = H @ Xr
    S = X.T @ Z
    R = np.eye(m)[:, :nr] - X.T @ Xr
    lam = lam.copy()
    lam[:nr] = np.diag(S[:nr, :nr]) / (1.0 - np.diag(R[:nr, :nr]))
    E = 0.5 * R
    for i in range(m):
        for j in range(nr):
            if i == j:
                continue
            num = S[i, j] + lam[j] * R[i, j]
            gap = lam[j] - lam[i]
            if abs(num) < 1e-3 * abs(gap):  # strict: gap 0 is a cluster
                E[i, j] = num / gap
    Xn = Xr + X @ E
    for _ in range(3):
        G = Xn.T @ Xn
        if np.abs(G - np.eye(nr)).max() <= 4e-16:
            break
        Xn = Xn @ (1.5 * np.eye(nr) - 0.5 * G)
    return Xn, lam[:nr]


def fp32_eig(H):
    w, V = np.linalg.eigh(H.astype(np.float32))
    o = np.argsort(w)
    return w[o].astype(np.float64), V[:, o].astype(np.float64)


def test_separated_eigenvalues_reach_fp64_accuracy():
    rng = np.random.default_rng(3)
    m, nr = 46, 24
    Q = np.linalg.qr(rng.standard_normal((m, m)))[0]
    ev = np.sort(rng.uniform(0.05, 8.0, m))
    ev[:nr] = 0.08 + 0.004 * np.arange(nr)  # the restart's closely spaced kept values
    H = (Q * ev) @ Q.T
    H = 0.5 * (H + H.T)
    lam0, X0 = fp32_eig(H)
    res0 = np.abs(H @ X0[:, :nr] - X0[:, :nr] * lam0[:nr]).max()
    Xn, lam = refine(H, X0, lam0, nr)
    nH = np.linalg.norm(H)
    res = np.abs(H @ Xn - Xn * lam).max()
    assert res0 > 1e-10 * nH  # an FP32-level start (about 3e-9 here)
    assert res < 2e-14 * nH
    assert np.abs(Xn.T @ Xn - np.eye(nr)).max() < 1e-14
    assert np.allclose(lam, ev[:nr], rtol=0, atol=1e-13 * nH)


def test_equal_eigenvalues_are_a_cluster_not_nan():
    rng = np.random.default_rng(4)
    m, nr = 20, 8
    Q = np.linalg.qr(rng.standard_normal((m, m)))[0]
    ev = np.concatenate([np.full(6, 2.0), np.linspace(4.0, 9.0, m - 6)])
    H = (Q * ev) @ Q.T
    H = 0.5 * (H + H.T)
    # exact eigenvectors of the degenerate block (any basis of it): equal
    # Ritz values, num = 0 and gap = 0 for every pair inside the cluster
    X = Q.copy()
    Xn, lam = refine(H, X, ev.copy(), nr)
    assert np.all(np.isfinite(Xn)) and np.all(np.isfinite(lam))
    assert np.abs(H @ Xn - Xn * lam).max() < 1e-13 * np.linalg.norm(H)
    # an FP32 start keeps the cluster's span to FP32 level and stays finite
    lam0, X0 = fp32_eig(H)
    Xn, lam = refine(H, X0, lam0, nr)
    assert np.all(np.isfinite(Xn))
    U = Q[:, :6]
    assert np.linalg.norm(Xn[:, :6] - U @ (U.T @ Xn[:, :6]), 2) < 1e-5
