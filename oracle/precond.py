"""Preconditioners P ~ L^{-1} (Section 3, item 2; Section 3.1.1; Section 4).

* ``jacobi``: P = D^{-1}, the diagonal of L inverted.
* ``fsai``:   a factored sparse approximate inverse P = G^T G, the
  "approximate inverse ... as a product of sparse matrices" the paper's
  conclusion (Section 5) proposes for parallel machines.  G is lower
  triangular with the pattern of tril(A), A = L + alpha diag(L) (L itself is
  singular), row i from the small system A[P_i, P_i] y = e_i over its pattern
  P_i = {j <= i : A_ij != 0}, g_i = y / sqrt(y_i); so (G A)_ij = 0 for
  j in P_i, j != i, and (G A G^T)_ii = 1.  Reading: a row whose pattern holds
  more than FSAI_CAP entries keeps only its diagonal (g_ii = 1/sqrt(a_ii)),
  so the set-up stays local; alpha = 1e-3 as for IC(0).
* ``ic0``:    incomplete Cholesky with no fill-in, K^{-1} = (F F^T)^{-1}
  (Section 4), computed on L + alpha diag(L).  L is singular (L e = 0), so the
  last pivot of an exact factorisation vanishes; the paper does not discuss
  breakdown.  Reading: start with alpha = 1e-3 and multiply by 10 until every
  pivot is positive.  IC(0) changes iteration counts, never the eigenpairs.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import spsolve_triangular


def ic0_factor(Lmat: sp.csr_matrix, alpha: float):
    """Lower-triangular F with the pattern of tril(L), F F^T ~ L + alpha diag(L)."""
    n = Lmat.shape[0]
    M = (Lmat + alpha * sp.diags(Lmat.diagonal())).tocsr()
    low = sp.tril(M).tocsr()
    low.sort_indices()
    rows = [dict() for _ in range(n)]
    for i in range(n):
        for p in range(low.indptr[i], low.indptr[i + 1]):
            rows[i][int(low.indices[p])] = float(low.data[p])
    F = [dict() for _ in range(n)]
    for i in range(n):
        Fi = F[i]
        for kcol in sorted(rows[i]):
            a = rows[i][kcol]
            if kcol < i:
                Fk = F[kcol]
                s = a
                for j, fij in Fi.items():
                    if j < kcol and j in Fk:
                        s -= fij * Fk[j]
                Fi[kcol] = s / Fk[kcol]
            else:
                s = a - sum(v * v for j, v in Fi.items() if j < i)
                if s <= 0.0:
                    return None
                Fi[i] = np.sqrt(s)
    ri, ci, vi = [], [], []
    for i in range(n):
        for j, v in F[i].items():
            ri.append(i)
            ci.append(j)
            vi.append(v)
    return sp.csr_matrix((vi, (ri, ci)), shape=(n, n))


FSAI_CAP = 32


def fsai_factor(Lmat: sp.csr_matrix, alpha: float = 1e-3, cap: int = FSAI_CAP) -> sp.csr_matrix:
    """G (lower triangular, CSR) of the factored approximate inverse G^T G of
    A = L + alpha diag(L), row by row."""
    n = Lmat.shape[0]
    A = (Lmat + alpha * sp.diags(Lmat.diagonal())).tocsr()
    A.sort_indices()
    rows, cols, vals = [], [], []
    for i in range(n):
        lo, hi = A.indptr[i], A.indptr[i + 1]
        pat = [int(j) for j in A.indices[lo:hi] if j <= i]
        if len(pat) > cap:
            pat = [i]
        m = len(pat)
        sub = np.zeros((m, m))
        for a, ja in enumerate(pat):
            for c, jc in enumerate(pat):
                sub[a, c] = A[ja, jc]
        e = np.zeros(m)
        e[pat.index(i)] = 1.0
        y = np.linalg.solve(sub, e)
        y /= np.sqrt(y[pat.index(i)])
        rows += [i] * m
        cols += pat
        vals += list(y)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def make_preconditioner(lap, kind: str):
    if kind == "jacobi":
        dinv = 1.0 / lap.d
        return lambda x: x * dinv
    if kind == "ic0":
        alpha = 1e-3
        F = None
        while F is None:
            F = ic0_factor(lap.L, alpha)
            alpha *= 10.0
        Ft = F.T.tocsr()

        def apply(x):
            y = spsolve_triangular(F, x, lower=True)
            return spsolve_triangular(Ft, y, lower=False)
        return apply
    if kind == "fsai":
        G = fsai_factor(lap.L)
        Gt = G.T.tocsr()
        return lambda x: Gt @ (G @ x)
    if kind == "none":
        return lambda x: x
    raise ValueError(kind)
