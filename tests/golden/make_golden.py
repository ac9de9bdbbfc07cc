"""Writes the stored reference eigenvalues of the large synthetic workloads
(tests/golden/eigs_<workload>.txt), computed by the CPU oracle only.

    python tests/golden/make_golden.py c2 c3 c5

c2 (18,080 nodes): the dense definition (oracle.dense, every eigenvalue of L
on the complement of e; the first 40 are stored).  c3 and c5 (275k and 951k
nodes): the oracle's single-vector Jacobi-Davidson (Algorithm 2 with
locking, pairs found in ascending order) to a residual of 1e-11 ||L||_1, so
that each stored value is within (residual)^2 / gap (Kato-Temple) of an
eigenvalue, far below a relative 1e-7 even for the closest pairs.
Each file records the graph's digest, so a test can check that it is
comparing the same seeded graph."""
from __future__ import annotations

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import graphgen  # noqa: E402
from oracle import dense, jd  # noqa: E402
from oracle.laplacian import Laplacian  # noqa: E402

PAIRS = {"c2": 40, "c3": 16, "c5": 14}


def write(name: str):
    g = graphgen.workload_graph(name)
    lap = Laplacian(g)
    t = time.perf_counter()
    if name == "c2":
        ev, V = dense.smallest_eigpairs(g, PAIRS[name])
        how = "dense definition (eigh of L + sigma e e^T / n)"
    else:
        ev, V, info = jd.jd_smallest(g, PAIRS[name], tol=1e-11, margin=1.0, max_outer=2000)
        how = f"oracle Jacobi-Davidson, tol 1e-11 ||L||_1, {info['outer']} outer its, {info['n_matvec']} MVPs"
    dt = time.perf_counter() - t
    res = np.linalg.norm(lap.matvec(V) - V * ev[None, :], axis=0) / lap.norm1
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"eigs_{name}.txt")
    with open(path, "w") as f:
        f.write(f"# workload {name}: n={g.n} nnz={g.nnz} digest={g.digest()}\n")
        f.write(f"# {how}; {dt:.0f} s on one CPU process\n")
        f.write("# columns: index, eigenvalue on the complement of e, ||L v - lambda v|| / ||L||_1\n")
        for i, (e, r) in enumerate(zip(ev, res)):
            f.write(f"{i} {float(e)!r} {float(r):.3e}\n")
    print(path, f"{dt:.0f} s")


def load(name: str):
    """(digest, eigenvalues) of a stored file."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"eigs_{name}.txt")
    digest, ev = None, []
    for line in open(path):
        if line.startswith("# workload"):
            digest = line.split("digest=")[1].strip()
        elif line.strip() and not line.startswith("#"):
            ev.append(float(line.split()[1]))
    return digest, np.array(ev)


if __name__ == "__main__":
    for name in sys.argv[1:] or ["c2", "c3", "c5"]:
        write(name)
