"""Implicitly restarted Lanczos on L^+ (Algorithm 1 right, Section 3.1).

Lanczos is run on the inverse operator so that the smallest eigenvalues of L
become the largest of the operator: every step solves L w_j = v_j by PCG
(Section 3.1.1) to ||v_j - L w_j|| / ||v_j|| <= delta_PCG = 1e-2 * tol
(Section 4).  L is singular; the whole process is kept in the complement of e
(v_j orthogonal to e makes L w = v consistent and w is projected back), which
turns L^{-1} into the pseudo-inverse L^+ there (reading).

Recurrence (Algorithm 1): alpha_j = w_j^T v_j, w_j -= alpha_j v_j + beta_j
v_{j-1}, beta_{j+1} = ||w_j||, v_{j+1} = w_j / beta_{j+1}, with full
reorthogonalisation of w_j against V (applied twice) to keep V orthonormal in
finite precision.  After ncv steps the factorisation is implicitly restarted
(ARPACK's IRLM, which the paper uses but does not spell out): the ncv - k'
unwanted Ritz values are applied as exact shifts by shifted QR steps on the
tridiagonal T, which compresses it to the k' wanted directions.  ncv follows
the paper's table (15, 30, 60, 120 for 1, 5, 20, 50 pairs), linearly
interpolated in between.
"""
from __future__ import annotations

import numpy as np

from .laplacian import Laplacian
from .precond import make_preconditioner
from .rng import uniform_block
from .jd import NotConverged


def ncv_for(k: int) -> int:
    table = [(1, 15), (5, 30), (20, 60), (50, 120)]
    if k <= 1:
        return 15
    for (k0, c0), (k1, c1) in zip(table, table[1:]):
        if k <= k1:
            return int(round(c0 + (k - k0) * (c1 - c0) / (k1 - k0)))
    return int(round(120 + (k - 50) * 70 / 30))


def _proj_e(x):
    return x - x.mean()


def pcg_solve(lap, P, v, rtol, maxit=100000):
    """PCG for L w = v with v orthogonal to e; iterates kept orthogonal to e."""
    v = _proj_e(v)
    w = np.zeros_like(v)
    res = v.copy()
    z = _proj_e(P(res))
    p = z.copy()
    rho = res @ z
    nv = np.linalg.norm(v)
    its = 0
    while np.linalg.norm(res) > rtol * nv:
        if its >= maxit:
            raise NotConverged("inner PCG")
        its += 1
        q = lap.matvec(p)
        alpha = rho / (p @ q)
        w = w + alpha * p
        res = res - alpha * q
        z = _proj_e(P(res))
        rho_new = res @ z
        p = z + (rho_new / rho) * p
        rho = rho_new
    return _proj_e(w), its


def _shifted_qr_step(T, mu):
    """One explicit shifted QR step on symmetric T: T - mu I = QR, T <- RQ + mu I."""
    m = T.shape[0]
    Qm, R = np.linalg.qr(T - mu * np.eye(m))
    return R @ Qm + mu * np.eye(m), Qm


def irlm_smallest(g, k: int, tol: float = 1e-8, ncv: int | None = None, precond: str = "jacobi",
                  seed: int = 0, max_restarts: int = 300, margin: float = 0.1):
    lap = Laplacian(g)
    n = g.n
    P = make_preconditioner(lap, precond)
    m = ncv or ncv_for(k)
    m = min(m, n - 1)
    kw = min(k + max(2, k // 2), m - 1)  # wanted directions kept at restart
    rtol = 1e-2 * tol  # delta_PCG = 1e-2 * delta (Section 4)
    V = np.zeros((n, m + 1))
    alpha = np.zeros(m)
    beta = np.zeros(m + 1)
    v = _proj_e(uniform_block(seed, n, 1)[:, 0])
    V[:, 0] = v / np.linalg.norm(v)
    j0 = 0
    inner = 0
    solves = 0
    for restart in range(max_restarts):
        for j in range(j0, m):
            w, its = pcg_solve(lap, P, V[:, j], rtol)
            inner += its
            solves += 1
            alpha[j] = w @ V[:, j]
            w = w - alpha[j] * V[:, j]
            if j > 0:
                w = w - beta[j] * V[:, j - 1]
            for _ in range(2):
                w = _proj_e(w - V[:, :j + 1] @ (V[:, :j + 1].T @ w))
            beta[j + 1] = np.linalg.norm(w)
            V[:, j + 1] = w / beta[j + 1]
        T = np.diag(alpha[:m]) + np.diag(beta[1:m], 1) + np.diag(beta[1:m], -1)
        mu, S = np.linalg.eigh(T)
        # largest of L^+ = smallest of L
        order = np.argsort(-mu)
        mu, S = mu[order], S[:, order]
        ritz_est = np.abs(beta[m] * S[m - 1, :k])
        if np.all(ritz_est <= margin * tol * mu[:k]):
            X = V[:, :m] @ S[:, :k]
            X = X / np.linalg.norm(X, axis=0)
            LX = lap.matvec(X)
            lam = np.einsum("ij,ij->j", X, LX)
            R = LX - X * lam[None, :]
            if np.all(np.linalg.norm(R, axis=0) <= margin * tol * lap.norm1):
                o = np.argsort(lam, kind="stable")
                return lam[o], X[:, o], dict(restarts=restart, solves=solves, inner=inner,
                                              n_matvec=lap.n_matvec, ncv=m, norm1=lap.norm1)
        # implicit restart with the m - kw unwanted Ritz values as exact shifts
        Qacc = np.eye(m)
        Tm = T.copy()
        for s in mu[kw:]:
            Tm, Qs = _shifted_qr_step(Tm, s)
            Qacc = Qacc @ Qs
        f = V[:, m] * beta[m]
        fk = V[:, :m] @ Qacc[:, kw] * Tm[kw, kw - 1] + f * Qacc[m - 1, kw - 1]
        Vk = V[:, :m] @ Qacc[:, :kw]
        V[:, :kw] = Vk
        alpha[:kw] = np.diag(Tm)[:kw]
        beta[1:kw] = np.diag(Tm, 1)[:kw - 1]
        beta[kw] = np.linalg.norm(fk)
        fk = fk - V[:, :kw] @ (V[:, :kw].T @ fk)
        beta[kw] = np.linalg.norm(fk)
        V[:, kw] = fk / beta[kw]
        j0 = kw
    raise NotConverged(f"IRLM: {max_restarts} restarts")
