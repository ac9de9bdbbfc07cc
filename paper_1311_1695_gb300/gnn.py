"""Learned warm start: a 3-layer message-passing network (width 32) that
proposes the initial Jacobi-Davidson block, trained on eigenvectors the
solver itself computed.  The paper has no learned component.

Every forward and backward step runs in the library's kernels; this module
only lays out the device buffers and marshals the small parameter matrices.
Storage and arithmetic: the node features, every aggregation hop and every
layer's output are BF16 (lap_gnn_features_bf16, lap_gnn_aggregate_bf16);
the dense layers [M^s H | H] [W; U] + b are BF16 tensor-core products with
FP32 accumulation and the tanh fused (lap_gnn_dense_bf16); the weight
gradients [M^s H | H]^T dZ are BF16 tensor-core products over the rows with
FP32 accumulation within a CTA and FP64 across CTAs (lap_gnn_wgrad_bf16);
the output X, the loss gradient dX and the back-propagated dH are FP32.
Weights are FP64 masters rounded to BF16 for every use.

Network, for a batch handle of graphs (each graph its own segment):
    H_0 = F (features),  tanh([M^s H_l | H_l] [W_l; U_l] + b_l) -> H_{l+1},
    X = C H_3 W_out,     M = D^{-1} A,  s = HOPS,  C = per-graph centring.
Loss per graph: 1 - tr(G^{-1} X^T U U^T X) / k with G = X^T X + eps tr(X^T X)/k I
(U = solver eigenvectors); its k x k algebra (lap_gnn_loss) and the Adam update
(lap_adam_step) run in the library too.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

from . import LAP_F32, LAP_F64, Graph, _check, _stream, lib

WIDTH = 32
NFEAT = 16
LAYERS = 3
HOPS = 4
EPS_RIDGE = 1e-6
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gnn_weights.json")


def to_bf16(x: np.ndarray) -> np.ndarray:
    """Round FP64 values to the nearest BF16 (ties to even), returned as FP64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def param_shapes(k: int):
    shapes, fin = [], NFEAT
    for _ in range(LAYERS):
        shapes += [("W", (fin, WIDTH)), ("U", (fin, WIDTH)), ("b", (WIDTH,))]
        fin = WIDTH
    shapes.append(("Wout", (WIDTH, k)))
    return shapes


def init_params(k: int, seed: int = 0):
    rng = np.random.default_rng(seed)
    out = []
    for name, shp in param_shapes(k):
        out.append(np.zeros(shp) if name == "b" else rng.standard_normal(shp) / np.sqrt(shp[0]))
    return out


def save_params(params, path=WEIGHTS, meta=None):
    json.dump({"k": int(params[-1].shape[1]), "params": [p.tolist() for p in params], "meta": meta or {}},
              open(path, "w"))


def load_params(path=WEIGHTS):
    d = json.load(open(path))
    return [np.asarray(p, dtype=np.float64) for p in d["params"]], d.get("meta", {})


class Net:
    """Device buffers of one batch handle; forward/backward on them."""

    def __init__(self, G: Graph, k: int):
        import torch
        self.G, self.k = G, k
        n = G.n
        dev = "cuda"
        f32, b16 = torch.float32, torch.bfloat16
        # AH_l = [M^s H_l | H_l] in BF16; layer 0 holds the features in its right half
        self.AH = [torch.zeros((n, 2 * NFEAT), dtype=b16, device=dev)] + \
                  [torch.zeros((n, 2 * WIDTH), dtype=b16, device=dev) for _ in range(LAYERS)]
        self.tmp = [torch.zeros((n, WIDTH), dtype=b16, device=dev) for _ in range(2)]
        self.UX = torch.zeros((n, 2 * k), dtype=f32, device=dev)  # [U | X]
        self.dX = torch.zeros((n, WIDTH), dtype=f32, device=dev)  # k columns used, the rest zero
        self.dH = torch.zeros((n, WIDTH), dtype=f32, device=dev)
        self.T1 = torch.zeros((n, WIDTH), dtype=f32, device=dev)
        self.dHn = torch.zeros((n, WIDTH), dtype=f32, device=dev)
        self.ftmp = [torch.zeros((n, WIDTH), dtype=f32, device=dev) for _ in range(2)]
        self.nseg = G.nseg
        self.rows = np.diff(G.row0)

    # -- helpers
    def _S(self, mats, nseg=1):
        import torch
        S = np.concatenate([np.atleast_2d(m) for m in mats], axis=0)
        # row-major (C order) whatever the layout of the inputs (a transposed
        # weight is an F-ordered view): the kernel reads S[i * lds + j]
        S = np.array(np.broadcast_to(S, (nseg,) + S.shape), dtype=np.float64, order="C", copy=True)
        return torch.from_numpy(S).cuda().contiguous(), S.shape[-1], S.shape[-2] * S.shape[-1]

    def _update(self, Y, ldy, q, beta, A, lda, p, ones, S, lds, ss):
        _check(lib().lap_block_update(self.G.h, LAP_F32, ctypes.c_void_p(Y), ldy, q, beta, 1.0,
                                      None if A is None else ctypes.c_void_p(A), lda, p, ones,
                                      ctypes.c_void_p(S.data_ptr()), lds, ss, _stream()), "lap_block_update")

    def _gram(self, A, lda, p, B, ldb, q, ones):
        import torch
        Gm = torch.zeros((self.nseg, p + ones, q), dtype=torch.float64, device="cuda")
        _check(lib().lap_gram(self.G.h, LAP_F32, None if A is None else ctypes.c_void_p(A), lda, p,
                              ctypes.c_void_p(B), ldb, q, ones, ctypes.c_void_p(Gm.data_ptr()), _stream()), "lap_gram")
        return Gm

    def _weights_bf16(self, mats, cols=WIDTH):
        """Stacked BF16 weights (rows of the inputs, `cols` columns, zero padded)."""
        import torch
        W = np.concatenate([np.atleast_2d(m) for m in mats], axis=0)
        Wp = np.zeros((W.shape[0], cols))
        Wp[:, :W.shape[1]] = W
        # the values are BF16 already (to_bf16): the conversion is exact
        return torch.from_numpy(Wp).to(torch.float32).to(torch.bfloat16).cuda().contiguous()

    def _aggregate16(self, src, lds, dst, ldd, w):
        """dst = M^s src, every hop stored in BF16 (s = HOPS)."""
        cur, ldc = src, lds
        for h in range(HOPS):
            last = h == HOPS - 1
            out, ldo = (dst, ldd) if last else (self.tmp[h % 2].data_ptr(), WIDTH)
            _check(lib().lap_gnn_aggregate_bf16(self.G.h, 0, ctypes.c_void_p(cur), ldc, ctypes.c_void_p(out), ldo, w,
                                                _stream()), "lap_gnn_aggregate_bf16")
            cur, ldc = out, ldo

    def _aggregate_T32(self, src, lds, dst, ldd, w):
        """dst = (M^T)^s src on FP32 blocks (back-propagation)."""
        cur, ldc = src, lds
        for h in range(HOPS):
            last = h == HOPS - 1
            out, ldo = (dst, ldd) if last else (self.ftmp[h % 2].data_ptr(), WIDTH)
            _check(lib().lap_gnn_aggregate(self.G.h, 1, ctypes.c_void_p(cur), ldc, ctypes.c_void_p(out), ldo, w,
                                           _stream()), "lap_gnn_aggregate")
            cur, ldc = out, ldo

    def _dense(self, K, A, lda, W, bias, Y, ldy, ncols, act, out_bf16):
        _check(lib().lap_gnn_dense_bf16(self.G.h, K, ctypes.c_void_p(A), lda, ctypes.c_void_p(W.data_ptr()),
                                        None if bias is None else ctypes.c_void_p(bias.data_ptr()), ctypes.c_void_p(Y),
                                        ldy, ncols, act, out_bf16, _stream()), "lap_gnn_dense_bf16")

    def _wgrad(self, K, A, lda, dZ, ldz):
        import torch
        Gw = torch.zeros((K, WIDTH), dtype=torch.float64, device="cuda")
        _check(lib().lap_gnn_wgrad_bf16(self.G.h, K, ctypes.c_void_p(A), lda, ctypes.c_void_p(dZ), ldz,
                                        ctypes.c_void_p(Gw.data_ptr()), _stream()), "lap_gnn_wgrad_bf16")
        return Gw.cpu().numpy()

    def _centre(self, Y, ldy, q):
        """Subtract each graph's column means from Y (n x q, FP32)."""
        Gm = self._gram(None, 0, 0, Y, ldy, q, 1)  # per-graph column means
        S = (-Gm).contiguous()
        self._update(Y, ldy, q, 1.0, None, 0, 0, 1, S, q, q)

    # -- forward: returns X (view of UX[:, k:])
    def forward(self, params, seed: int):
        import torch
        P = [to_bf16(p) for p in params]
        AH = self.AH
        e2 = 2  # bytes per BF16 value
        _check(lib().lap_gnn_features_bf16(self.G.h, seed, NFEAT, ctypes.c_void_p(AH[0].data_ptr() + e2 * NFEAT),
                                           2 * NFEAT, _stream()), "lap_gnn_features_bf16")
        fin = NFEAT
        self._dev_w = []
        for l in range(LAYERS):
            A = AH[l]
            # left half = M^s H_l
            self._aggregate16(A.data_ptr() + e2 * fin, 2 * fin, A.data_ptr(), 2 * fin, fin)
            W, U, b = P[3 * l: 3 * l + 3]
            Wd = self._weights_bf16([W, U])
            bd = torch.from_numpy(b).float().cuda()
            self._dev_w.append((Wd, bd))
            Hn = AH[l + 1].data_ptr() + e2 * WIDTH
            self._dense(2 * fin, A.data_ptr(), 2 * fin, Wd, bd, Hn, 2 * WIDTH, WIDTH, 1, 1)
            fin = WIDTH
        Wo = self._weights_bf16([P[-1]])
        self._dev_w.append((Wo, None))
        X = self.UX.data_ptr() + 4 * self.k
        self._dense(WIDTH, AH[LAYERS].data_ptr() + e2 * WIDTH, 2 * WIDTH, Wo, None, X, 2 * self.k, self.k, 0, 0)
        self._centre(X, 2 * self.k, self.k)
        self._P = P
        return self.UX[:, self.k:]

    def set_targets(self, U):
        """U: float32 CUDA tensor n x k (each graph's solver eigenvectors in its rows)."""
        self.UX[:, :self.k] = U

    # -- loss per graph and dX
    def loss(self):
        """Per-graph losses (numpy) and dX on the device; the k x k algebra runs
        in the library (lap_gnn_loss)."""
        import torch
        k = self.k
        UXp = self.UX.data_ptr()
        P = self._gram(UXp, 2 * k, k, UXp + 4 * k, 2 * k, k, 0).contiguous()
        Q = self._gram(UXp + 4 * k, 2 * k, k, UXp + 4 * k, 2 * k, k, 0).contiguous()
        losses = torch.zeros(self.nseg, dtype=torch.float64, device="cuda")
        St = torch.zeros((self.nseg, 2 * k, k), dtype=torch.float64, device="cuda")
        _check(lib().lap_gnn_loss(self.nseg, k, EPS_RIDGE, ctypes.c_void_p(P.data_ptr()), ctypes.c_void_p(Q.data_ptr()),
                                  ctypes.c_void_p(losses.data_ptr()), ctypes.c_void_p(St.data_ptr()), _stream()),
               "lap_gnn_loss")
        self._update(self.dX.data_ptr(), WIDTH, k, 0.0, UXp, 2 * k, 2 * k, 0, St, k, 2 * k * k)
        return losses.cpu().numpy()

    # -- backward: gradients (summed over the graphs of the batch), FP64 numpy
    def backward(self):
        P, k, AH = self._P, self.k, self.AH
        e2 = 2
        grads = [None] * len(P)
        self._centre(self.dX.data_ptr(), WIDTH, k)  # the centring is its own adjoint
        H3 = AH[LAYERS].data_ptr() + e2 * WIDTH
        grads[-1] = self._wgrad(WIDTH, H3, 2 * WIDTH, self.dX.data_ptr(), WIDTH)[:, :k]
        S, lds, _ = self._S([P[-1].T])
        self._update(self.dH.data_ptr(), WIDTH, WIDTH, 0.0, self.dX.data_ptr(), WIDTH, k, 0, S, lds, 0)
        fin_of = [NFEAT] + [WIDTH] * (LAYERS - 1)
        for l in reversed(range(LAYERS)):
            fin = fin_of[l]
            Hn = AH[l + 1].data_ptr() + e2 * WIDTH
            dZ = self.dH.data_ptr()
            _check(lib().lap_gnn_tanh_back_bf16(self.G.h, ctypes.c_void_p(dZ), WIDTH, ctypes.c_void_p(Hn), 2 * WIDTH,
                                                WIDTH, _stream()), "lap_gnn_tanh_back_bf16")
            Gw = self._wgrad(2 * fin, AH[l].data_ptr(), 2 * fin, dZ, WIDTH)
            grads[3 * l] = Gw[:fin]
            grads[3 * l + 1] = Gw[fin:]
            Gm = self._gram(None, 0, 0, dZ, WIDTH, WIDTH, 1).cpu().numpy()
            # the ones row is a per-graph mean: back to a sum
            grads[3 * l + 2] = (Gm[:, 0, :] * self.rows[:, None]).sum(axis=0)
            if l > 0:
                W, U = P[3 * l], P[3 * l + 1]
                S, lds, _ = self._S([W.T])
                self._update(self.T1.data_ptr(), WIDTH, fin, 0.0, dZ, WIDTH, WIDTH, 0, S, lds, 0)
                self._aggregate_T32(self.T1.data_ptr(), WIDTH, self.dHn.data_ptr(), WIDTH, fin)
                S, lds, _ = self._S([U.T])
                self._update(self.dHn.data_ptr(), WIDTH, fin, 1.0, dZ, WIDTH, WIDTH, 0, S, lds, 0)
                self.dH, self.dHn = self.dHn, self.dH
        return grads


class Adam:
    """Adam over the parameter list; the update runs in the library
    (lap_adam_step) on a flat device copy of the parameters and moments."""

    def __init__(self, params, lr=3e-3, b1=0.9, b2=0.999, eps=1e-8):
        import torch
        n = sum(p.size for p in params)
        self.m = torch.zeros(n, dtype=torch.float64, device="cuda")
        self.v = torch.zeros(n, dtype=torch.float64, device="cuda")
        self.t, self.lr, self.b1, self.b2, self.eps = 0, lr, b1, b2, eps

    def step(self, params, grads):
        import torch
        self.t += 1
        p = torch.from_numpy(np.concatenate([x.ravel() for x in params])).cuda()
        g = torch.from_numpy(np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in grads])).cuda()
        _check(lib().lap_adam_step(p.numel(), ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                   ctypes.c_void_p(self.m.data_ptr()), ctypes.c_void_p(self.v.data_ptr()), self.t,
                                   self.lr, self.b1, self.b2, self.eps, _stream()), "lap_adam_step")
        flat = p.cpu().numpy()
        o = 0
        for x in params:
            x[...] = flat[o:o + x.size].reshape(x.shape)
            o += x.size


def warm_start(G: Graph, params, seed: int = 0x5EED):
    """The network's proposal for graph handle G as a float64 CUDA tensor
    (n x k), ready for lap_eigs_graph's x0_dev."""
    k = params[-1].shape[1]
    net = Net(G, k)
    X = net.forward(params, seed)
    return X.double().contiguous()


def warm_start_native(G: Graph, params, seed: int = 0x5EED):
    """The same proposal from the library's own forward pass
    (lap_gnn_warm_start): float64 CUDA tensor n x k."""
    import torch
    k = int(params[-1].shape[1])
    flat = np.ascontiguousarray(np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in params]))
    X = torch.zeros((G.n, k), dtype=torch.float64, device="cuda")
    _check(lib().lap_gnn_warm_start(G.h, flat.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), flat.size, k, seed,
                                    ctypes.c_void_p(X.data_ptr()), k, _stream()), "lap_gnn_warm_start")
    return X
