"""The paper's experiment grid (Section 4, Tables 2-5): the N_eig smallest
strictly positive eigenpairs of each test network, for N_eig in {1, 5, 20, 50}
and exit tolerances delta in {1e-3, 1e-6} of the relative residual
||L u - theta u|| / theta, with the three solvers (DACG, JD, IRLM), reporting
matrix-vector products (MVP), outer iterations (linear-system solutions for
JD and IRLM) and wall time.

    python -m paper_1311_1695_gb300.sweep --workloads c1,c2 --json sweep.jsonl

Differences from the paper's runs, stated per record:
  * the networks are the seeded synthetic stand-ins of `graphgen`
    (c1 protein-sized, c2 internet-shaped, c3 www-shaped, c5 dblp-scale);
  * the preconditioner is D^{-1} (Jacobi) or the factored sparse approximate
    inverse G^T G (`--precond fsai`, JD's correction solve) instead of IC(0);
  * JD is the block method of this library: it holds every wanted pair in its
    block (b = N_eig + 2 <= 32), so N_eig = 50 is reported as not run for JD;
  * times are GB300 wall times of one solve on a resident graph (the first
    solve of each configuration is an untimed warm-up).
Each record also carries the largest ||L u - theta u|| / ||L||_1 and the
status, so a row that did not converge is visible as such.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NEIG = (1, 5, 20, 50)
DELTAS = (1e-3, 1e-6)
METHODS = ("dacg", "jd", "irlm")
JD_MAX_PAIRS = 30


def run_one(G, k: int, delta: float, method: str, precond: str = "jacobi", precision: str = "fp64",
            warmup: bool = True, **extra) -> dict:
    """One solve of the grid on the resident graph handle G; returns a record."""
    import torch

    rec = dict(n_eig=k, delta=delta, method=method, precond=precond if method == "jd" else "jacobi",
               precision=precision if method == "jd" else "fp64")
    if method == "jd" and k > JD_MAX_PAIRS:
        rec["skipped"] = f"JD holds at most {JD_MAX_PAIRS} pairs in its block"
        return rec
    opts = dict(tol_mode="theta", precision=rec["precision"], **extra)
    if method == "jd":
        opts["precond"] = precond
    if warmup:
        G.eigs(k, delta, method=method, **opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev, infos = G.eigs(k, delta, method=method, **opts)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    i = infos[0]
    rec.update(mvp=int(i["n_matvec"]), outer_its=int(i["outer_its"]), seconds=round(dt, 4),
               status=int(i["status"]), n_converged=int(i["n_converged"]),
               max_rel_residual=float(i["max_rel_residual"]), lambda_2=float(ev[0][0]),
               lambda_k=float(ev[0][k - 1]))
    return rec


def table(records) -> str:
    """Markdown table in the layout of the paper's Tables 2-5: one row per
    (N_eig, delta), per method MVP, seconds and outer iterations."""
    rows = {}
    for r in records:
        rows.setdefault((r["n_eig"], r["delta"]), {})[r["method"]] = r
    head = "| N_eig | delta | " + " | ".join(f"{m} MVP | {m} s | {m} outer" for m in METHODS) + " |"
    sep = "|" + "---|" * (2 + 3 * len(METHODS))
    out = [head, sep]
    for (k, d), by in sorted(rows.items(), key=lambda x: (x[0][1] < 1e-4, x[0][0])):
        cells = []
        for m in METHODS:
            r = by.get(m)
            if r is None or "skipped" in r:
                cells += ["—", "—", "—"]
            else:
                flag = "" if r["status"] == 0 else f" (status {r['status']})"
                cells += [f"{r['mvp']}{flag}", f"{r['seconds']:.3f}", str(r["outer_its"]) if m != "dacg" else "—"]
        out.append(f"| {k} | {d:.0e} | " + " | ".join(cells) + " |")
    return "\n".join(out)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workloads", default="c1,c2")
    ap.add_argument("--neig", default=",".join(map(str, NEIG)))
    ap.add_argument("--delta", default=",".join(f"{d:g}" for d in DELTAS))
    ap.add_argument("--methods", default=",".join(METHODS))
    ap.add_argument("--precond", default="jacobi", choices=["jacobi", "fsai"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--json", default=None, help="append one JSON line per record to this file")
    a = ap.parse_args(argv)

    import torch  # noqa: F401  (device memory for the resident graph)

    import graphgen
    import paper_1311_1695_gb300 as pkg
    from paper_1311_1695_gb300 import build

    build.build()
    records = []
    for wl in a.workloads.split(","):
        g = graphgen.workload_graph(wl)
        G = pkg.Graph([g])
        if a.precond == "fsai":
            G.set_precond("fsai")
        print(f"## {wl}: n = {g.n}, nnz = {int(g.nnz)}", flush=True)
        recs = []
        for d in (float(x) for x in a.delta.split(",")):
            for k in (int(x) for x in a.neig.split(",")):
                for m in a.methods.split(","):
                    r = run_one(G, k, d, m, precond=a.precond, precision=a.precision)
                    r["workload"] = wl
                    recs.append(r)
                    if a.json:
                        with open(a.json, "a") as f:
                            f.write(json.dumps(r) + "\n")
        print(table(recs), flush=True)
        records += recs
    return records


if __name__ == "__main__":
    main()
