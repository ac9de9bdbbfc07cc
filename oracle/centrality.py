"""Centralities from the computed eigenpairs (Section 2): the pseudo-inverse
G^+ = sum_{i>=2} v_i v_i^T / lambda_i of the Laplacian, approximated from k
computed pairs by the partial sums T^(k) or by S^(k), which replaces the
missing eigenvalues by one constant sigma.  Test infrastructure only (the
CPU oracle): imported by tests/ and bench.py's CPU leg, never by the library.

Readings.  "The k computed pairs" are the solver's output (lambda_j, v_j),
j = 1..k, the k smallest eigenvalues on the complement of e; the paper's
T^(k) sums its pairs 2..k of the full spectrum, i.e. k - 1 of them, so the
library's T over k computed pairs is the paper's T^(k+1).  S keeps e/sqrt(n)
out: S = (I - e e^T / n) / sigma + sum_j (1/lambda_j - 1/sigma) v_j v_j^T.
Current-flow closeness of node i is 1 / sum_j R_ij with the effective
resistances R_ij = P_ii + P_jj - 2 P_ij of P = G^+ (or its approximation);
as P e = 0 the sum is n P_ii + tr P.  Current-flow betweenness sums, over
source-target pairs (s, t), the current through node i when a unit current
enters at s and leaves at t: the potentials are p = P (e_s - e_t) and node
i != s, t carries 1/2 sum_j A_ij |p_i - p_j|; the ends carry none.
"""
from __future__ import annotations

import numpy as np

from .laplacian import Laplacian


def pinv_partial(evals: np.ndarray, V: np.ndarray, mode: str = "T", sigma: float | None = None) -> np.ndarray:
    """Dense T (mode "T") or S (mode "S") from the computed pairs, as the
    sum of rank-one terms (small n)."""
    n, k = V.shape
    if mode == "T":
        P = np.zeros((n, n))
        for j in range(k):
            P += np.outer(V[:, j], V[:, j]) / evals[j]
        return P
    P = (np.eye(n) - np.ones((n, n)) / n) / sigma
    for j in range(k):
        P += (1.0 / evals[j] - 1.0 / sigma) * np.outer(V[:, j], V[:, j])
    return P


def apply_partial(evals, V, X, mode="T", sigma=None):
    """P X without forming P."""
    C = V.T @ X
    if mode == "T":
        return V @ (C / evals[:, None])
    Xc = X - X.mean(axis=0, keepdims=True)
    return Xc / sigma + V @ (C * (1.0 / evals - 1.0 / sigma)[:, None])


def closeness(P: np.ndarray) -> np.ndarray:
    """1 / sum_j R_ij, R_ij = P_ii + P_jj - 2 P_ij, summed pair by pair."""
    n = P.shape[0]
    d = np.diag(P)
    out = np.empty(n)
    for i in range(n):
        out[i] = 1.0 / sum(d[i] + d[j] - 2.0 * P[i, j] for j in range(n))
    return out


def betweenness(g, P: np.ndarray, pairs) -> np.ndarray:
    """Sum over the pairs of each node's throughput (ends excluded), edge by
    edge."""
    n = g.n
    out = np.zeros(n)
    for s, t in pairs:
        b = np.zeros(n)
        b[s], b[t] = 1.0, -1.0
        p = P @ b
        for i in range(n):
            if i == s or i == t:
                continue
            acc = 0.0
            for q in range(g.rowptr[i], g.rowptr[i + 1]):
                j = g.colidx[q]
                w = 1.0 if g.weights is None else float(g.weights[q])
                acc += w * abs(p[i] - p[j])
            out[i] += 0.5 * acc
    return out


def pseudo_inverse(g) -> np.ndarray:
    """G^+ by the library's dense pseudo-inverse (for pins only)."""
    return np.linalg.pinv(Laplacian(g).dense())
