"""The graph Laplacian L = D - A (Section 2 of the paper).

A is the weighted adjacency matrix of a simple undirected graph with positive
weights; D is the diagonal of generalised degrees d_i = sum_j A_ij.  The oracle
stores L explicitly, diagonal included, as a scipy CSR matrix (a library sparse
product is its only matvec primitive).

Residuals are normalised by ||L||_1 = max_j sum_i |L_ij| = 2 max_i d_i: the
diagonal contributes d_j and the off-diagonal column entries sum to d_j.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class Laplacian:
    def __init__(self, g):
        n = g.n
        self.n = n
        rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.rowptr))
        cols = g.colidx.astype(np.int64)
        w = np.ones(cols.size) if g.weights is None else np.asarray(g.weights, dtype=np.float64)
        if np.any(rows == cols):
            raise ValueError("self-loop in adjacency")
        if np.any(w <= 0) or not np.all(np.isfinite(w)):
            raise ValueError("weights must be positive and finite")
        # generalised degrees: sum of incident weights (Section 2)
        self.d = np.bincount(rows, weights=w, minlength=n).astype(np.float64)
        A = sp.csr_matrix((w, (rows, cols)), shape=(n, n))
        if (A - A.T).count_nonzero() != 0:
            raise ValueError("adjacency is not symmetric")
        self.A = A
        self.L = (sp.diags(self.d) - A).tocsr()
        self.norm1 = 2.0 * float(self.d.max()) if n > 0 else 0.0
        self.n_matvec = 0

    def matvec(self, X: np.ndarray) -> np.ndarray:
        """L X for a vector or an n x b block."""
        self.n_matvec += 1 if X.ndim == 1 else X.shape[1]
        return self.L @ X

    def dense(self) -> np.ndarray:
        return self.L.toarray()

    def trace(self) -> float:
        return float(self.d.sum())


def quadratic_form_edges(g, x: np.ndarray) -> float:
    """Eq. 1: x^T L x = 1/2 sum_{i,j} A_ij (x_i - x_j)^2, summed edge by edge."""
    total = 0.0
    for i in range(g.n):
        for p in range(g.rowptr[i], g.rowptr[i + 1]):
            j = g.colidx[p]
            w = 1.0 if g.weights is None else g.weights[p]
            total += 0.5 * w * (x[i] - x[j]) ** 2
    return total


def dense_laplacian_loops(g) -> np.ndarray:
    """D - A assembled entry by entry (brute force, tiny graphs only)."""
    Lm = np.zeros((g.n, g.n))
    for i in range(g.n):
        for p in range(g.rowptr[i], g.rowptr[i + 1]):
            j = g.colidx[p]
            w = 1.0 if g.weights is None else g.weights[p]
            Lm[i, j] -= w
            Lm[i, i] += w
    return Lm
