"""Time one hot-path kernel in isolation through the C ABI (and give ncu a
short, self-contained command to capture it).

    python -m paper_1311_1695_gb300.kernel_bench --workload c3 --kernel pcg --b 12
    python -m paper_1311_1695_gb300.kernel_bench --workload c3 --kernel spmm --b 12 --dtype f64

The graph is numbered by decreasing degree by default, as the solvers'
copy of a large graph is (--order as-numbered keeps the generator's order).

kernel: spmm (degree-fused L X), pcg (the fused projected-PCG correction solve,
--iters steps), syev (the small eigensolver on --nmat random m x m matrices).
Inputs are seeded and synthetic: X is an orthonormal block orthogonal to the
constant vector, R a random block orthogonal to [e, X], theta = --theta.
Each kernel runs --warmup times untimed, then --reps times between CUDA
events; the script prints one JSON line with the mean time per call.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--kernel", default="pcg", choices=["spmm", "pcg", "syev"])
    ap.add_argument("--b", type=int, default=12)
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--theta", type=float, default=0.1)
    ap.add_argument("--m", type=int, default=46)
    ap.add_argument("--nmat", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--order", default="degree", choices=["degree", "as-numbered"],
                    help="node numbering of the graph: by decreasing degree (the numbering the solvers use for a "
                         "large graph, lap_graph_set_reorder) or as generated")
    a = ap.parse_args(argv)

    import torch
    import graphgen
    import paper_1311_1695_gb300 as pkg
    from paper_1311_1695_gb300 import build
    build.build()
    dt = torch.float32 if a.dtype == "f32" else torch.float64
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"kernel": a.kernel, "workload": a.workload, "dtype": a.dtype}
    if a.kernel == "syev":
        rng = np.random.default_rng(0)
        H = rng.standard_normal((a.nmat, a.m, a.m))
        H = torch.from_numpy(H + H.transpose(0, 2, 1)).cuda()
        run = lambda: pkg.lap_syev_batched(H)
        out.update(m=a.m, nmat=a.nmat)
    else:
        g = graphgen.workload_graph(a.workload)
        if a.order == "degree":  # the solvers' copy: nodes by decreasing degree, ties by number
            deg = np.diff(g.rowptr)
            perm = np.empty(g.n, dtype=np.int64)
            perm[np.argsort(-deg, kind="stable")] = np.arange(g.n)
            g = graphgen.relabel(g, perm)
        G = pkg.Graph(g)
        rng = np.random.default_rng(0)
        X = rng.standard_normal((g.n, a.b))
        X -= X.mean(axis=0)
        X = np.linalg.qr(X)[0]
        R = rng.standard_normal((g.n, a.b))
        R -= R.mean(axis=0)
        R -= X @ (X.T @ R)
        Xd = torch.from_numpy(np.ascontiguousarray(X)).to(dt).cuda()
        Rd = torch.from_numpy(np.ascontiguousarray(R)).to(dt).cuda()
        Yd = torch.empty_like(Xd)
        th = torch.full((1, a.b), a.theta, dtype=torch.float64, device="cuda")
        if a.kernel == "spmm":
            run = lambda: G.spmm(Xd, Yd)
        else:
            run = lambda: G.pcg_correction(Xd, th, Rd, a.iters)
        info = G.info()
        out.update(n=int(g.n), nnz=int(g.rowptr[-1]), b=a.b, hubs=int(info["nlong"]), team=int(info["team"]),
                   order=a.order)
        if a.kernel == "pcg":
            out["iters"] = a.iters
    for _ in range(a.warmup):
        run()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    out["us_per_call"] = round(e0.elapsed_time(e1) / a.reps * 1e3, 2)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
