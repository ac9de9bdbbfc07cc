"""Deflation-accelerated conjugate gradient (Algorithm 3, Section 3.3).

For j = 1..p the Rayleigh quotient q(x) = x^T L x / x^T x is minimised over
x orthogonal to U = [e/sqrt(n), u_1, .., u_{j-1}] by a nonlinear preconditioned
conjugate gradient; then lambda_j = q(x), u_j = x / sqrt(eta) with
eta = x^T x, and u_j joins U.

The paper gives only "nonlinear preconditioned CG" (step 2).  The reading
implemented here is the standard Rayleigh-quotient NLCG:
  g = 2 (L x - q x) / (x^T x)                gradient of q at x
  z = (I - U U^T) P g                        preconditioned, deflated gradient
  beta = (g^T z) / (g_prev^T z_prev)          (0 on the first step)
  p = -z + beta p, then p = (I - U U^T) p    search direction orthogonal to U
  x <- x + alpha p, with alpha minimising q(x + alpha p) exactly (the smaller
  root of the 2 x 2 Rayleigh-Ritz problem on span{x, p}).
Each iteration costs one matrix-vector product (L p), one preconditioner
application and the orthogonalisation against U (Section 3.3.1).
Stop test (reading): ||L x - q x|| / ||x|| <= tol * ||L||_1.
"""
from __future__ import annotations

import numpy as np

from .laplacian import Laplacian
from .precond import make_preconditioner
from .rng import uniform_block
from .jd import NotConverged


def _proj(x, U):
    return x - U @ (U.T @ x)


def _line_min(a11, a12, a22, b11, b12, b22):
    """Smallest generalised eigenpair of [[a11,a12],[a12,a22]] c = mu [[b11,b12],[b12,b22]] c.
    Returns alpha = c2 / c1 (the step along p from x)."""
    # det(A - mu B) = 0:  (b11 b22 - b12^2) mu^2 - (a11 b22 + a22 b11 - 2 a12 b12) mu + (a11 a22 - a12^2) = 0
    A2 = b11 * b22 - b12 * b12
    A1 = -(a11 * b22 + a22 * b11 - 2.0 * a12 * b12)
    A0 = a11 * a22 - a12 * a12
    disc = max(A1 * A1 - 4.0 * A2 * A0, 0.0)
    # smaller root, computed stably
    sq = np.sqrt(disc)
    if A1 <= 0:
        mu = (2.0 * A0) / (-A1 + sq) if (-A1 + sq) != 0 else 0.0
    else:
        mu = (-A1 - sq) / (2.0 * A2)
    # (a11 - mu b11) c1 + (a12 - mu b12) c2 = 0
    r1 = a11 - mu * b11
    r2 = a12 - mu * b12
    if abs(r2) < 1e-300:
        return 0.0
    return -r1 / r2


def dacg_smallest(g, k: int, tol: float = 1e-8, precond: str = "jacobi", seed: int = 0,
                  max_iter: int = 20000, margin: float = 0.1):
    lap = Laplacian(g)
    n = g.n
    P = make_preconditioner(lap, precond)
    stop = margin * tol * lap.norm1
    U = np.full((n, 1), 1.0 / np.sqrt(n))
    evals = []
    its_total = 0
    for j in range(k):
        x = _proj(uniform_block(seed + 104729 * j, n, 1)[:, 0], U)
        x = x / np.linalg.norm(x)
        Ax = lap.matvec(x)
        p = np.zeros(n)
        Ap = np.zeros(n)
        gz_prev = None
        for it in range(max_iter + 1):
            xx = x @ x
            q = (x @ Ax) / xx
            res = Ax - q * x
            if np.linalg.norm(res) / np.sqrt(xx) <= stop:
                break
            if it == max_iter:
                raise NotConverged(f"DACG pair {j + 1}: {max_iter} iterations")
            its_total += 1
            gvec = 2.0 * res / xx
            z = _proj(P(gvec), U)
            gz = gvec @ z
            beta = 0.0 if gz_prev is None else gz / gz_prev
            gz_prev = gz
            p = -z + beta * p
            p = _proj(p, U)
            Ap = lap.matvec(p)
            alpha = _line_min(x @ Ax, x @ Ap, p @ Ap, xx, x @ p, p @ p)
            x = x + alpha * p
            Ax = Ax + alpha * Ap
            # keep the scale of x bounded; L x is rescaled with it
            nx = np.linalg.norm(x)
            x, Ax = x / nx, Ax / nx
            # refresh L x now and then against drift of the recurrence
            if it % 50 == 49:
                Ax = lap.matvec(x)
        eta = x @ x
        u = x / np.sqrt(eta)
        lam = u @ lap.matvec(u)
        evals.append(lam)
        U = np.column_stack([U, u])
    evals = np.array(evals)
    evecs = U[:, 1:]
    order = np.argsort(evals, kind="stable")
    return evals[order], evecs[:, order], dict(iters=its_total, n_matvec=lap.n_matvec, norm1=lap.norm1)
