"""The definition: k smallest eigenpairs of L on the complement of e.

Section 2: L is symmetric positive semidefinite, L e = 0, so lambda_1 = 0 with
eigenvector e / sqrt(n), and 0 has multiplicity equal to the number of
connected components.  Section 4 asks for the smallest strictly positive
eigenvalues of connected graphs; the reading used here for any graph is "the k
smallest eigenvalues of L restricted to the orthogonal complement of e"
(lambda_2 .. lambda_{k+1} when the graph is connected; on a graph with c
components the c - 1 extra zeros come first).

Computed exactly (up to rounding) as the k smallest eigenpairs of
L + sigma * e e^T / n with sigma > lambda_max: adding sigma e e^T / n moves the
eigenvalue of e from 0 to sigma and leaves every eigenpair orthogonal to e
unchanged.  The dense symmetric eigensolve is numpy's (LAPACK syevd).
"""
from __future__ import annotations

import numpy as np

from .laplacian import Laplacian


def full_spectrum(g) -> np.ndarray:
    """All n eigenvalues of L in ascending order (dense)."""
    return np.linalg.eigvalsh(Laplacian(g).dense())


def smallest_eigpairs(g, k: int, include_null: bool = False):
    """Return (evals [k] ascending, evecs [n, k]) of L on the complement of e.

    With include_null the pair (0, e / sqrt(n)) is prepended and k - 1 pairs
    follow."""
    lap = Laplacian(g)
    n = g.n
    Lm = lap.dense()
    sigma = lap.norm1 + 1.0  # Gershgorin: lambda_max <= 2 max d_i = ||L||_1
    M = Lm + (sigma / n) * np.ones((n, n))
    w, V = np.linalg.eigh(M)
    kk = k - 1 if include_null else k
    evals = w[:kk].copy()
    evecs = V[:, :kk].copy()
    if include_null:
        evals = np.concatenate([[0.0], evals])
        evecs = np.concatenate([np.full((n, 1), 1.0 / np.sqrt(n)), evecs], axis=1)
    return evals, canonical_signs(evecs)


def canonical_signs(V: np.ndarray) -> np.ndarray:
    """Sign convention: the entry of largest magnitude in each column is
    positive (ties: lowest index)."""
    V = V.copy()
    for c in range(V.shape[1]):
        i = int(np.argmax(np.abs(V[:, c])))
        if V[i, c] < 0:
            V[:, c] = -V[:, c]
    return V
