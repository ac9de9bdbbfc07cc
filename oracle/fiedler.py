"""Applications of the Fiedler pair (Section 2): graph bisection and the
profile-reducing ordering.  Test infrastructure only (the CPU oracle):
imported by tests/ and bench.py's CPU leg, never by the library.

* ``relaxed_bisection``: the relaxed minimiser of x^T L x with x^T x = n/4
  and e^T x = (n1 - n2)/2, x = (n1 - n2)/(2n) e + sqrt(n1 n2 / n) v2, whose
  value is n1 n2 lambda2 / n (Section 2).
* ``fiedler_partition``: the discrete bisection the relaxation suggests -- the
  n1 nodes with the smallest Fiedler-vector entries (ties by node index) form
  one side -- and its cut size, the sum of the weights of the edges between
  the sides (Eq. 1 with x_i = +-1/2).
* ``fiedler_order``: the ordering of the nodes by their Fiedler-vector
  entries (ties by node index), and the bandwidth and profile of A under an
  ordering.
"""
from __future__ import annotations

import numpy as np


def relaxed_bisection(v2: np.ndarray, n1: int) -> np.ndarray:
    n = v2.size
    n2 = n - n1
    return (n1 - n2) / (2.0 * n) * np.ones(n) + np.sqrt(n1 * n2 / n) * v2


def fiedler_order(v2: np.ndarray) -> np.ndarray:
    """perm[r] = the node at position r: ascending Fiedler entries, ties by index."""
    return np.lexsort((np.arange(v2.size), v2))


def fiedler_partition(g, v2: np.ndarray, n1: int):
    """(side [n] in {0, 1}, cut size): side 0 holds the n1 nodes first in the
    Fiedler order."""
    perm = fiedler_order(v2)
    side = np.ones(g.n, dtype=np.int32)
    side[perm[:n1]] = 0
    return side, cut_size(g, side)


def cut_size(g, side: np.ndarray) -> float:
    """Sum of the weights of the edges whose ends are on different sides
    (each undirected edge once), edge by edge."""
    total = 0.0
    for i in range(g.n):
        for p in range(g.rowptr[i], g.rowptr[i + 1]):
            j = g.colidx[p]
            if j > i and side[i] != side[j]:
                total += 1.0 if g.weights is None else float(g.weights[p])
    return total


def bandwidth_profile(g, perm: np.ndarray):
    """Bandwidth max |pos(i) - pos(j)| over the edges and profile
    sum_r (r - min(r, min_j pos(j))) over the rows r of the reordered matrix,
    pos the inverse of perm, row by row."""
    pos = np.empty(g.n, dtype=np.int64)
    pos[perm] = np.arange(g.n)
    bw = 0
    prof = 0
    for i in range(g.n):
        r = pos[i]
        lo = r
        for p in range(g.rowptr[i], g.rowptr[i + 1]):
            c = pos[g.colidx[p]]
            bw = max(bw, abs(int(r - c)))
            lo = min(lo, c)
        prof += int(r - lo)
    return bw, prof
