"""Per-step definitions of the Jacobi-Davidson hot path, in FP64.

Each function is the plain mathematical definition of one step the GPU library
performs, so a GPU result can be compared element by element:

* ``lap_spmm``        -- Y = L X - X diag(shift): the matrix-vector product
  (Section 3 item 1; Algorithm 2 step 3) on a block, with an optional
  per-column shift (the (A - theta I) of Eq. 4/5).
* ``project``         -- Pi_Q X = X - Q (Q^T X) with Q = [e/sqrt(n), Q_lock]:
  the deflation of Eq. 5.
* ``gram``            -- A^T B (the V^T w column of H, Algorithm 2 step 4).
* ``orthonormalize``  -- the block that Gram-Schmidt against Q and then
  within itself produces (Algorithm 2 step 2 applied to a block): the unique
  orthonormal Q-factor of (I - Q Q^T) T with a positive triangular factor.
* ``rayleigh_ritz``   -- smallest eigenpairs of H = V^T L V and the Ritz
  vectors V Y (Algorithm 2 steps 5-6).
* ``residual_norms``  -- ||L x_j - theta_j x_j|| per column (step 6-7).
* ``pcg_correction``  -- a fixed number of projected, preconditioned CG steps
  on (I - QQ^T)(L - theta I)(I - QQ^T) t = -r (Eq. 5, step 8; the
  preconditioner (I - QQ^T) P (I - QQ^T) of Section 3.2.1 with P = D^{-1}).
"""
from __future__ import annotations

import numpy as np

from .laplacian import Laplacian


def lap_spmm(g, X: np.ndarray, shift=None) -> np.ndarray:
    lap = Laplacian(g)
    Y = lap.matvec(X)
    if shift is not None:
        Y = Y - X * np.asarray(shift)[None, :]
    return Y


def project(X: np.ndarray, Q: np.ndarray | None, null: bool = True) -> np.ndarray:
    """X - e (e^T X)/n - Q (Q^T X); Q has orthonormal columns orthogonal to e."""
    Y = X.astype(np.float64).copy()
    if null:
        Y = Y - Y.mean(axis=0, keepdims=True)
    if Q is not None and Q.shape[1] > 0:
        Y = Y - Q @ (Q.T @ Y)
    return Y


def gram(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    return A.T.astype(np.float64) @ B.astype(np.float64)


def orthonormalize(Q: np.ndarray | None, T: np.ndarray, null: bool = True):
    """Orthonormal basis of the part of span(T) orthogonal to [e, Q], by the
    unique QR factorisation with positive diagonal.  Returns (U, R)."""
    P = project(T, Q, null)
    U, R = np.linalg.qr(P)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return U * s[None, :], R * s[:, None]


def rayleigh_ritz(g, V: np.ndarray, k: int):
    """(theta [k], X = V Y [n, k]) from H = V^T L V, V orthonormal."""
    lap = Laplacian(g)
    H = V.T @ lap.matvec(V)
    H = 0.5 * (H + H.T)
    w, Y = np.linalg.eigh(H)
    return w[:k], V @ Y[:, :k]


def residual_norms(g, X: np.ndarray, theta: np.ndarray) -> np.ndarray:
    lap = Laplacian(g)
    R = lap.matvec(X) - X * theta[None, :]
    return np.linalg.norm(R, axis=0)


def pcg_correction(g, theta: np.ndarray, R: np.ndarray, Q: np.ndarray, iters: int,
                   null: bool = True, precond=None):
    """``iters`` steps of projected preconditioned CG, column by column, on
    Pi (L - theta_j I) Pi t_j = -r_j with Pi = I - [e/sqrt(n), Q][.]^T,
    starting from t_j = 0, preconditioner Pi M Pi with M = D^{-1} (Jacobi) or
    the callable ``precond`` (x -> M x).  No early exit, so the iterates are
    defined exactly.  Returns T (n x b)."""
    lap = Laplacian(g)
    d = lap.d
    apply = (lambda x: x / d) if precond is None else precond
    n, b = R.shape
    T = np.zeros((n, b))
    for j in range(b):
        th = theta[j]
        res = project(-R[:, j:j + 1], Q, null)[:, 0]
        t = np.zeros(n)
        z = project(apply(res)[:, None], Q, null)[:, 0]
        p = z.copy()
        rho = res @ z
        for _ in range(iters):
            q = project((lap.L @ p - th * p)[:, None], Q, null)[:, 0]
            pq = p @ q
            if pq == 0.0 or rho == 0.0:
                break
            alpha = rho / pq
            t = t + alpha * p
            res = res - alpha * q
            z = project(apply(res)[:, None], Q, null)[:, 0]
            rho_new = res @ z
            beta = rho_new / rho
            rho = rho_new
            p = z + beta * p
        T[:, j] = t
    return T
