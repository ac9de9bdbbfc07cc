"""Train the warm-start network on eigenvectors computed by this library.

    python -m paper_1311_1695_gb300.train_gnn [--graphs 10000] [--k 10]
        [--batch 32] [--epochs 3] [--lr 1e-3] [--out gnn_weights.json]

Training set: Chung-Lu graphs (largest component), n log-uniform in
[1,000, 20,000], degree exponent uniform in [2.2, 2.8], mean degree 6, seeds
100000 + i.  Targets: the k smallest eigenvectors from lap_eigs_batched
(mixed precision, tol 1e-6: a start block needs no more).  Loss: the subspace
loss of gnn.Net, Adam on the FP64 master weights (BF16 in every kernel).
Graph generation runs in a spawn process pool before any CUDA call.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def spec_of(i: int):
    rng = np.random.default_rng(100000 + i)
    n = int(round(math.exp(rng.uniform(math.log(1000), math.log(20000)))))
    return dict(n=n, gamma=float(rng.uniform(2.2, 2.8)), dbar=6.0, seed=100000 + i)


def make_graph(i: int):
    import graphgen
    s = spec_of(i)
    g = graphgen.chung_lu(s["n"], s["gamma"], s["dbar"], s["seed"])
    return g.n, g.rowptr, g.colidx


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--graphs", type=int, default=10000)
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--workers", type=int, default=min(16, os.cpu_count() or 4))
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    t0 = time.time()
    ctx = mp.get_context("spawn")
    with ctx.Pool(a.workers) as pool:
        raw = pool.map(make_graph, range(a.graphs), chunksize=16)
    t_gen = time.time() - t0

    import torch
    import graphgen
    from paper_1311_1695_gb300 import Graph, build, lap_eigs_batched
    from paper_1311_1695_gb300 import gnn
    build.build()
    graphs = [graphgen.CSRGraph(n, rp, ci, None) for n, rp, ci in raw]
    # targets, solved in lock-step batches
    t1 = time.time()
    targets, nconv = [], 0
    for s in range(0, len(graphs), 64):
        chunk = graphs[s:s + 64]
        _, Vs, infos = lap_eigs_batched(chunk, a.k, tol=1e-6, precision="mixed")
        targets += [V.astype(np.float32) for V in Vs]
        nconv += sum(1 for i in infos if i["status"] == 0)
    t_solve = time.time() - t1
    params = gnn.init_params(a.k, seed=0)
    opt = gnn.Adam(params, lr=a.lr)
    order = np.arange(len(graphs))
    rng = np.random.default_rng(0)
    curve = []
    t2 = time.time()
    for ep in range(a.epochs):
        rng.shuffle(order)
        ep_loss = []
        for s in range(0, len(order), a.batch):
            idx = order[s:s + a.batch]
            H = Graph([graphs[i] for i in idx])
            net = gnn.Net(H, a.k)
            net.set_targets(torch.from_numpy(np.vstack([targets[i] for i in idx])).cuda())
            net.forward(params, seed=int(rng.integers(1 << 31)))
            losses = net.loss()
            grads = net.backward()
            opt.step(params, grads)
            ep_loss.append(float(np.mean(losses)))
            H.close()
        curve.append(float(np.mean(ep_loss)))
        print(f"epoch {ep}: mean subspace loss {curve[-1]:.4f}", flush=True)
    t_train = time.time() - t2
    meta = dict(graphs=len(graphs), k=a.k, batch=a.batch, epochs=a.epochs, lr=a.lr, loss_curve=curve,
                targets_converged=nconv, seconds=dict(generate=t_gen, solve=t_solve, train=t_train),
                recipe="Chung-Lu LCC, n log-uniform [1000, 20000], gamma U[2.2, 2.8], mean degree 6, seeds 100000+i")
    gnn.save_params(params, a.out or gnn.WEIGHTS, meta)
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
