"""Jacobi-Davidson for the smallest eigenpairs of L (Algorithm 2, Section 3.2).

One eigenpair at a time, in the paper's order:

  for each wanted pair j (deflation, Eq. 5):
    repeat (outer iteration k):
      step 2  orthogonalise the new vector v against the locked vectors
              Q = [e/sqrt(n), u_1..u_{j-1}] and the search basis V by modified
              Gram-Schmidt (applied twice);
      step 3  normalise v; w = L v;
      step 4  grow H = V^T L V by the new row and column; V = [V v], W = [W w];
      step 5  smallest eigenpair (theta, y) of H;
      step 6  u = V y, r = W y - theta u  (= L u - theta u);
      step 7  stop when ||r|| is small (reading below);
      restart when dim H reaches m_max: keep the m_min Ritz vectors with the
              smallest Ritz values (thick restart);
      step 8  solve (I - Q'Q'^T)(L - theta I)(I - Q'Q'^T) v = -r,  Q' = [Q, u],
              approximately by PCG (at most ITMAX steps or a relative residual
              drop of delta_PCG), preconditioner (I - Q'Q'^T) P (I - Q'Q'^T)
              (Section 3.2.1), P = D^{-1} (Jacobi) or IC(0) of L.
    lock (theta, u); the remaining Ritz vectors of V seed the next pair.

Readings where the paper is silent:
* stop test: ||L u - theta u||_2 <= tol * ||L||_1, checked on a freshly
  computed L u (the paper's theta-relative test divides by theta; Section 4);
* restart keeps the m_min smallest Ritz vectors (the paper says "the last
  m_min columns of V");
* P = D^{-1} by default; IC(0) of L + alpha diag(L) is available
  (``precond='ic0'``); the preconditioner changes iteration counts only;
* start vector: SplitMix64 uniform(-1, 1) (``oracle.rng``), projected and
  normalised.
Defaults m_min=5, m_max=10, ITMAX=20, delta_PCG=1e-2 are the paper's (Section 4).
"""
from __future__ import annotations

import numpy as np

from .laplacian import Laplacian
from .rng import uniform_block
from .precond import make_preconditioner


class NotConverged(RuntimeError):
    pass


def _mgs(v: np.ndarray, bases) -> np.ndarray:
    """Modified Gram-Schmidt of v against the columns of each basis, twice."""
    for _ in range(2):
        for B in bases:
            for c in range(B.shape[1]):
                v = v - (B[:, c] @ v) * B[:, c]
    return v


def _project(x: np.ndarray, Q: np.ndarray) -> np.ndarray:
    return x - Q @ (Q.T @ x)


def pcg_correction(lap: Laplacian, P, theta: float, r: np.ndarray, Qc: np.ndarray,
                   itmax: int, delta: float):
    """Step 8: projected PCG on (I-QQ^T)(L-theta I)(I-QQ^T) t = -r (Notay:
    CG is applicable although the projected operator may be indefinite)."""
    res = _project(-r, Qc)
    t = np.zeros_like(res)
    z = _project(P(res), Qc)
    p = z.copy()
    rho = res @ z
    res0 = np.linalg.norm(res)
    its = 0
    for its in range(1, itmax + 1):
        q = _project(lap.matvec(p) - theta * p, Qc)
        pq = p @ q
        if pq == 0.0 or rho == 0.0:
            break
        alpha = rho / pq
        t = t + alpha * p
        res = res - alpha * q
        if np.linalg.norm(res) <= delta * res0:
            break
        z = _project(P(res), Qc)
        rho_new = res @ z
        p = z + (rho_new / rho) * p
        rho = rho_new
    return t, its


def jd_smallest(g, k: int, tol: float = 1e-8, m_min: int = 5, m_max: int = 10,
                itmax: int = 20, delta_pcg: float = 1e-2, precond: str = "jacobi",
                seed: int = 0, max_outer: int = 400, margin: float = 0.1,
                include_null: bool = False):
    """Return (evals [k], evecs [n, k], info dict)."""
    lap = Laplacian(g)
    n = g.n
    P = make_preconditioner(lap, precond)
    stop = margin * tol * lap.norm1
    Q = np.full((n, 1), 1.0 / np.sqrt(n))  # locked vectors, e/sqrt(n) first
    evals = []
    kk = k - 1 if include_null else k
    V = np.zeros((n, 0))
    W = np.zeros((n, 0))
    H = np.zeros((0, 0))
    v = uniform_block(seed, n, 1)[:, 0]
    outer_total = 0
    inner_total = 0
    while len(evals) < kk:
        outer = 0
        while True:
            outer += 1
            outer_total += 1
            if outer > max_outer:
                raise NotConverged(f"pair {len(evals) + 1}: no convergence in {max_outer} outer iterations")
            if v is not None:
                # steps 2-4
                v = _mgs(v, [Q, V])
                nv = np.linalg.norm(v)
                if nv < 1e-10:
                    v = _mgs(uniform_block(seed + outer_total, n, 1)[:, 0], [Q, V])
                    nv = np.linalg.norm(v)
                v = v / nv
                w = lap.matvec(v)
                h = V.T @ w
                H = np.block([[H, h[:, None]], [h[None, :], np.array([[v @ w]])]])
                V = np.column_stack([V, v])
                W = np.column_stack([W, w])
            # step 5
            Hs = 0.5 * (H + H.T)
            thetas, Y = np.linalg.eigh(Hs)
            theta = thetas[0]
            # step 6
            u = V @ Y[:, 0]
            r = W @ Y[:, 0] - theta * u
            # step 7 (checked on an explicit L u)
            if np.linalg.norm(r) <= stop:
                nu = np.linalg.norm(u)
                u = u / nu
                theta = u @ lap.matvec(u)
                r_exp = lap.matvec(u) - theta * u
                if np.linalg.norm(r_exp) <= stop:
                    evals.append(theta)
                    Q = np.column_stack([Q, u])
                    # the other Ritz vectors seed the next pair
                    V = V @ Y[:, 1:]
                    W = W @ Y[:, 1:]
                    H = np.diag(thetas[1:])
                    v = None if V.shape[1] > 0 else uniform_block(seed + 7919 * len(evals), n, 1)[:, 0]
                    break
            # restart
            if V.shape[1] >= m_max:
                V = V @ Y[:, :m_min]
                W = W @ Y[:, :m_min]
                H = np.diag(thetas[:m_min])
            # step 8
            Qc = np.column_stack([Q, u])
            v, its = pcg_correction(lap, P, theta, r, Qc, itmax, delta_pcg)
            inner_total += its
    evals = np.array(evals)
    evecs = Q[:, 1:].copy()
    order = np.argsort(evals, kind="stable")
    evals, evecs = evals[order], evecs[:, order]
    if include_null:
        evals = np.concatenate([[0.0], evals])
        evecs = np.column_stack([np.full(n, 1.0 / np.sqrt(n)), evecs])
    info = dict(outer=outer_total, inner=inner_total, n_matvec=lap.n_matvec, norm1=lap.norm1)
    return evals, evecs, info
