"""The warm-start message-passing network and its subspace loss, in FP64.

The paper has no learned component; this is the definition the GPU's
training and inference kernels are checked against.  Network (width w = 32,
s = HOPS aggregation steps per layer):

  H_0 = F                                   (n x f node features)
  Z_l = (M^s H_l) W_l + H_l U_l + 1 b_l^T   M = D^{-1} A (mean over neighbours)
  H_{l+1} = tanh(Z_l),  l = 0, 1, 2
  X = C H_3 W_out,   C = I - 1 1^T / n      (n x k proposed start block,
                                             centred: the wanted eigenvectors
                                             are orthogonal to 1)

Loss, invariant to the sign and rotation of the target eigenvectors U
(n x k, orthonormal) and, for eps = 0, to any invertible recombination of X's
columns:

  loss(X) = 1 - tr(G^{-1} X^T U U^T X) / k,   G = X^T X + eps (tr(X^T X) / k) I

which is 0 exactly when span(X) = span(U) (eps = 0).  The small ridge eps
keeps the loss and its gradient finite when X is nearly rank deficient.
With A = G^{-1} (X^T U U^T X) G^{-1}, its gradient is
  dloss/dX = -(2/k) (U U^T X G^{-1} - X A - (eps / k) tr(A) X).

Node features: column 0 = 1, column 1 = log(1 + d_i) / log(1 + d_max), the
rest uniform(-1, 1) from SplitMix64 (counter node * f + column).
"""
from __future__ import annotations

import numpy as np

from .laplacian import Laplacian
from .rng import splitmix64

WIDTH = 32
LAYERS = 3
NFEAT = 16
HOPS = 4
EPS_RIDGE = 1e-6


def features(g, seed: int, nfeat: int = NFEAT) -> np.ndarray:
    lap = Laplacian(g)
    d = lap.d
    F = np.empty((g.n, nfeat))
    F[:, 0] = 1.0
    F[:, 1] = np.log1p(d) / np.log1p(d.max())
    z = splitmix64(seed, np.arange(g.n * nfeat, dtype=np.uint64)).reshape(g.n, nfeat)
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    F[:, 2:] = (2.0 * u - 1.0)[:, 2:]
    return F


def param_shapes(k: int, nfeat: int = NFEAT, width: int = WIDTH):
    shapes = []
    fin = nfeat
    for _ in range(LAYERS):
        shapes += [("W", (fin, width)), ("U", (fin, width)), ("b", (width,))]
        fin = width
    shapes.append(("Wout", (width, k)))
    return shapes


def init_params(k: int, seed: int = 0, nfeat: int = NFEAT, width: int = WIDTH):
    rng = np.random.default_rng(seed)
    out = []
    for name, shp in param_shapes(k, nfeat, width):
        if name == "b":
            out.append(np.zeros(shp))
        else:
            out.append(rng.standard_normal(shp) / np.sqrt(shp[0]))
    return out


def _mean_agg(g, H):
    lap = Laplacian(g)
    return (lap.A @ H) / lap.d[:, None]


def _mean_agg_T(g, H):
    lap = Laplacian(g)
    return lap.A @ (H / lap.d[:, None])


def round_bf16(x) -> np.ndarray:
    """Nearest BFloat16 value (8-bit significand, ties to even) of each
    entry, as FP64: the float32 bit pattern with its low 16 bits rounded
    away (values and their FP32 rounding: the stored activations are FP32
    sums rounded once)."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(x))


def forward(g, F, params, store=None):
    """store: None (FP64 throughout) or a rounding applied to every stored
    activation -- the features, each aggregation hop, each layer's output --
    as the BF16 inference and training kernels store them."""
    keep = (lambda v: v) if store is None else store
    H = keep(F)
    cache = []
    for l in range(LAYERS):
        W, U, b = params[3 * l: 3 * l + 3]
        MH = H
        for _ in range(HOPS):
            MH = keep(_mean_agg(g, MH))
        Z = MH @ W + H @ U + b[None, :]
        Hn = keep(np.tanh(Z))
        cache.append((H, MH, Hn))
        H = Hn
    X = H @ params[-1]
    X = X - X.mean(axis=0)[None, :]
    return X, cache


def backward(g, cache, params, dX):
    grads = [None] * len(params)
    H3 = cache[-1][2]
    dX = dX - dX.mean(axis=0)[None, :]   # the centring is its own adjoint
    grads[-1] = H3.T @ dX
    dH = dX @ params[-1].T
    for l in reversed(range(LAYERS)):
        H, MH, Hn = cache[l]
        W, U, b = params[3 * l: 3 * l + 3]
        dZ = dH * (1.0 - Hn * Hn)
        grads[3 * l] = MH.T @ dZ
        grads[3 * l + 1] = H.T @ dZ
        grads[3 * l + 2] = dZ.sum(axis=0)
        T = dZ @ W.T
        for _ in range(HOPS):
            T = _mean_agg_T(g, T)
        dH = T + dZ @ U.T
    return grads


def subspace_loss(X, U, eps: float = EPS_RIDGE):
    k = U.shape[1]
    Gm = X.T @ X
    Gm = Gm + eps * (np.trace(Gm) / k) * np.eye(k)
    Gi = np.linalg.inv(Gm)
    UX = U.T @ X
    M = UX.T @ UX
    loss = 1.0 - np.trace(Gi @ M) / k
    A = Gi @ M @ Gi
    dX = -(2.0 / k) * (U @ UX @ Gi - X @ A - (eps / k) * np.trace(A) * X)
    return loss, dX
