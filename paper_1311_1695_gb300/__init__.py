"""Python binding of liblapeig.so: the k smallest eigenpairs of a sparse graph
Laplacian L = D - A on one GB300 (Bergamaschi, Bozzo, Franceschet, arXiv
1311.1695).

This module only marshals arguments into the C ABI declared in
include/lapeig.h; every step of the computation runs in the library's CUDA
kernels.  There is no CPU fallback: if the shared library has not been built,
every call raises.  Device blocks are passed as torch CUDA tensors (row-major,
unit stride along a row); PyTorch is used only for device memory and streams.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblapeig.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "lapeig.h")

LAP_OK, LAP_ENOCONV = 0, 1
LAP_EINVAL, LAP_ENOTSYM, LAP_EWEIGHT, LAP_ESELFLOOP = -1, -2, -3, -4
LAP_ENUMERIC, LAP_ENOMEM, LAP_ETIMEOUT, LAP_ECUDA, LAP_EUNSORTED = -5, -6, -7, -8, -9
LAP_JD, LAP_DACG, LAP_IRLM = 0, 1, 2
LAP_PREC_FP64, LAP_PREC_MIXED = 0, 1
LAP_F64, LAP_F32 = 0, 1
LAP_PRECOND_JACOBI, LAP_PRECOND_FSAI = 0, 1
_PRECONDS = {"jacobi": LAP_PRECOND_JACOBI, "fsai": LAP_PRECOND_FSAI}
LAP_REORDER_AUTO, LAP_REORDER_NONE, LAP_REORDER_DEGREE = -1, 0, 1
_REORDERS = {"auto": LAP_REORDER_AUTO, "none": LAP_REORDER_NONE, "degree": LAP_REORDER_DEGREE}
LAP_TOL_NORM1, LAP_TOL_THETA = 0, 1
_TOL_MODES = {"norm1": LAP_TOL_NORM1, "theta": LAP_TOL_THETA}

_METHODS = {"jd": LAP_JD, "dacg": LAP_DACG, "irlm": LAP_IRLM}
_PRECISIONS = {"fp64": LAP_PREC_FP64, "mixed": LAP_PREC_MIXED}


class LapError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status}: {detail}")
        self.status = status


class lap_opts(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("block", ctypes.c_int),
        ("m_keep", ctypes.c_int),
        ("inner_maxit", ctypes.c_int),
        ("inner_tol", ctypes.c_double),
        ("max_outer", ctypes.c_int),
        ("ncv", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("include_null", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("x0", ctypes.POINTER(ctypes.c_double)),
        ("k0", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("max_seconds", ctypes.c_double),
        ("team", ctypes.c_int),
        ("verbose", ctypes.c_int),
        ("x0_dev", ctypes.c_void_p),
        ("ldx0", ctypes.c_int),
        ("cuda_graph", ctypes.c_int),
        ("device_timeout_ms", ctypes.c_double),
        ("max_ctas", ctypes.c_int),
        ("precond", ctypes.c_int),
        ("precond_alpha", ctypes.c_double),
        ("ev_rtol", ctypes.c_double),
        ("tol_mode", ctypes.c_int),
        ("use_gnn", ctypes.c_int),
        ("gnn_k", ctypes.c_int),
        ("gnn_params", ctypes.POINTER(ctypes.c_double)),
    ]


class lap_info(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("n_converged", ctypes.c_int),
        ("outer_its", ctypes.c_int),
        ("inner_its", ctypes.c_int),
        ("n_matvec", ctypes.c_int64),
        ("norm_L", ctypes.c_double),
        ("max_rel_residual", ctypes.c_double),
        ("elapsed_ms", ctypes.c_double),
        ("phase1_outer", ctypes.c_int),
        ("spmm_team", ctypes.c_int),
        ("spmm_unroll", ctypes.c_int),
        ("hub_threshold", ctypes.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None

_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_PI = ctypes.POINTER(ctypes.c_int)
_PI64 = ctypes.POINTER(ctypes.c_int64)
_PI32 = ctypes.POINTER(ctypes.c_int32)

_SIGNATURES = {
    "lap_opts_default": (None, [ctypes.POINTER(lap_opts)]),
    "lap_strerror": (ctypes.c_char_p, [_I]),
    "lap_last_error": (ctypes.c_char_p, []),
    "lap_eigs": (_I, [_I64, _PI64, _PI32, _PD, _I, _D, _I, ctypes.POINTER(lap_opts), _PD, _PD,
                      ctypes.POINTER(lap_info)]),
    "lap_eigs_batched": (_I, [_I, _PI64, ctypes.POINTER(_PI64), ctypes.POINTER(_PI32), ctypes.POINTER(_PD), _PI, _D,
                              _I, ctypes.POINTER(lap_opts), ctypes.POINTER(_PD), ctypes.POINTER(_PD),
                              ctypes.POINTER(lap_info)]),
    "lap_eigs_graph": (_I, [_P, _I, _D, _I, ctypes.POINTER(lap_opts), _PD, _P, ctypes.POINTER(lap_info)]),
    "lap_profile_enable": (_I, [_I]),
    "lap_profile_read": (_I, [_I, ctypes.c_char_p, _I, _PD, _PD, _PI64, _PI]),
    "lap_graph_create": (_I, [_I64, _PI64, _PI32, _PD, ctypes.POINTER(_P)]),
    "lap_graph_create_batched": (_I, [_I, _PI64, ctypes.POINTER(_PI64), ctypes.POINTER(_PI32), ctypes.POINTER(_PD),
                                      ctypes.POINTER(_P)]),
    "lap_graph_destroy": (None, [_P]),
    "lap_graph_info": (_I, [_P, _PI64, _PI, _PD, _PI, _PI]),
    "lap_graph_set_schedule": (_I, [_P, _I, _I]),
    "lap_graph_set_launch": (_I, [_P, _I, _D, _I]),
    "lap_graph_set_precond": (_I, [_P, _I, _D]),
    "lap_spmm": (_I, [_P, _I, _P, _I, _P, _I, _I, _P]),
    "lap_gram": (_I, [_P, _I, _P, _I, _I, _P, _I, _I, _I, _P, _P]),
    "lap_gram_noalloc": (_I, [_I64, _I, _P, _I, _I, _P, _I, _I, _I, _P, _P]),
    "lap_gnn_features": (_I, [_P, ctypes.c_uint64, _I, _P, _I, _P]),
    "lap_gnn_aggregate": (_I, [_P, _I, _P, _I, _P, _I, _I, _P]),
    "lap_gnn_tanh": (_I, [_P, _I, _P, _I, _P, _I, _I, _P]),
    "lap_block_update": (_I, [_P, _I, _P, _I, _I, _D, _D, _P, _I, _I, _I, _P, _I, _I64, _P]),
    "lap_gnn_features_bf16": (_I, [_P, ctypes.c_uint64, _I, _P, _I, _P]),
    "lap_gnn_aggregate_bf16": (_I, [_P, _I, _P, _I, _P, _I, _I, _P]),
    "lap_gnn_dense_bf16": (_I, [_P, _I, _P, _I, _P, _P, _P, _I, _I, _I, _I, _P]),
    "lap_gnn_wgrad_bf16": (_I, [_P, _I, _P, _I, _P, _I, _P, _P]),
    "lap_gnn_tanh_back_bf16": (_I, [_P, _P, _I, _P, _I, _I, _P]),
    "lap_graph_set_gathers": (_I, [_P, _I]),
    "lap_graph_set_reorder": (_I, [_P, _I]),
    "lap_gnn_warm_start": (_I, [_P, _PD, ctypes.c_int64, _I, ctypes.c_uint64, _P, _I, _P]),
    "lap_gnn_param_count": (ctypes.c_int64, [_I]),
    "lap_gnn_loss": (_I, [_I, _I, _D, _P, _P, _P, _P, _P]),
    "lap_adam_step": (_I, [ctypes.c_int64, _P, _P, _P, _P, _I, _D, _D, _D, _D, _P]),
    "lap_graph_autotune": (_I, [_P, _I, _I, _PI, _PI, _P]),
    "lap_project": (_I, [_P, _I, _P, _I, _I, _P, _I, _I, _P]),
    "lap_cgs2": (_I, [_P, _I, _P, _I, _I, _P, _I, _I, _PI, _P]),
    "lap_syev_batched": (_I, [_I, _I, _P, _I, _P, _P, _I, _P]),
    "lap_rayleigh_ritz": (_I, [_P, _I, _P, _I, _I, _P, _P]),
    "lap_residual_norms": (_I, [_P, _I, _P, _I, _P, _I, _P, _P]),
    "lap_pcg_correction": (_I, [_P, _I, _P, _I, _P, _P, _I, _P, _I, _I, _I, _D, _P]),
    "lap_fiedler_order": (_I, [_P, _P, _P, _PI64, _PI64, _PI64, _PI64, _P]),
    "lap_fiedler_bisect": (_I, [_P, _P, _D, _I64, _P, _PD, _PD, _P]),
    "lap_pinv_apply": (_I, [_P, _I, _PD, _P, _I, _I, _D, _P, _I, _P, _I, _I, _P]),
    "lap_cf_closeness": (_I, [_P, _I, _PD, _P, _I, _I, _D, _P, _P]),
    "lap_cf_betweenness": (_I, [_P, _I, _PD, _P, _I, _I, _D, _I64, _PI64, _P, _P]),
}


def lib() -> ctypes.CDLL:
    """The loaded shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1311_1695_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGNATURES)


def _check(status: int, where: str, allow_partial: bool = False) -> int:
    if status == LAP_OK or (allow_partial and status in (LAP_ENOCONV, LAP_ETIMEOUT)):
        return status
    detail = lib().lap_last_error().decode()
    raise LapError(status, where, f"{lib().lap_strerror(status).decode()} ({detail})")


def _csr_args(g):
    """(n, rowptr int64, colidx int32, weights float64 or None) from a CSRGraph-like."""
    n = int(g.n)
    rp = np.ascontiguousarray(g.rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(g.colidx, dtype=np.int32)
    w = None if g.weights is None else np.ascontiguousarray(g.weights, dtype=np.float64)
    return n, rp, ci, w


def _ptr(a, ct):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ct))


def make_opts(block=0, m_keep=0, inner_maxit=20, inner_tol=1e-2, max_outer=1000, ncv=0, precision="fp64",
              include_null=False, seed=0x5EED, x0=None, stream=None, max_seconds=0.0, team=0, verbose=False,
              x0_dev=None, cuda_graph=True, device_timeout_ms=0.0, max_ctas=0, ev_rtol=0.0, precond="jacobi",
              precond_alpha=0.0, tol_mode="norm1", use_gnn=False, gnn_params=None):
    o = lap_opts()
    lib().lap_opts_default(ctypes.byref(o))
    o.block, o.m_keep, o.inner_maxit, o.inner_tol = block, m_keep, inner_maxit, inner_tol
    o.max_outer, o.ncv = max_outer, ncv
    o.precision = _PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.include_null = int(bool(include_null))
    o.seed = seed
    o.max_seconds, o.team, o.verbose = max_seconds, team, int(verbose)
    o.stream = stream
    o.cuda_graph = 0 if cuda_graph else -1
    o.device_timeout_ms, o.max_ctas, o.ev_rtol = device_timeout_ms, max_ctas, ev_rtol
    o.precond = _PRECONDS[precond] if isinstance(precond, str) else int(precond)
    o.precond_alpha = precond_alpha
    o.tol_mode = _TOL_MODES[tol_mode] if isinstance(tol_mode, str) else int(tol_mode)
    keep = None
    if x0_dev is not None:  # a row-major float64 CUDA tensor n x k0
        o.x0_dev = ctypes.c_void_p(x0_dev.data_ptr())
        o.ldx0 = x0_dev.stride(0)
        o.k0 = x0_dev.shape[1]
    if x0 is not None:
        keep = np.asfortranarray(x0, dtype=np.float64)
        o.x0 = keep.ctypes.data_as(_PD)
        o.k0 = keep.shape[1]
    if use_gnn:
        # the network's parameters, flattened in their order (gnn.param_shapes);
        # default: the trained weights shipped with the package
        if gnn_params is None:
            from . import gnn as _gnn
            gnn_params, _ = _gnn.load_params()
        flat = np.ascontiguousarray(np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in gnn_params]))
        o.use_gnn, o.gnn_k = 1, int(np.asarray(gnn_params[-1]).shape[1])
        o.gnn_params = flat.ctypes.data_as(_PD)
        keep = (keep, flat)
    return o, keep


def lap_eigs(g, k: int, tol: float = 1e-8, method: str = "jd", want_vectors: bool = True, **opts):
    """k smallest eigenpairs of L on the complement of e.  Returns
    (evals [k], evecs [n, k] or None, info dict); raises LapError on errors;
    partial results (LAP_ENOCONV / LAP_ETIMEOUT) are returned with info['status']."""
    n, rp, ci, w = _csr_args(g)
    o, _keep = make_opts(**opts)
    evals = np.zeros(k)
    evecs = np.zeros((k, n)) if want_vectors else None  # column-major n x k == row-major k x n
    info = lap_info()
    st = lib().lap_eigs(n, _ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32), _ptr(w, ctypes.c_double), k, tol,
                        _METHODS[method] if isinstance(method, str) else int(method), ctypes.byref(o),
                        _ptr(evals, ctypes.c_double), _ptr(evecs, ctypes.c_double), ctypes.byref(info))
    _check(st, "lap_eigs", allow_partial=True)
    return evals, (None if evecs is None else evecs.T), info.as_dict()  # n x k (a column-major view)


def lap_eigs_batched(graphs, k, tol: float = 1e-8, method: str = "jd", want_vectors: bool = True, **opts):
    """Many graphs: lock-step block JD (or DACG / IRLM one graph after
    another).  k: one count for all graphs or one per graph.  Returns lists
    (evals, evecs, infos)."""
    nb = len(graphs)
    args = [_csr_args(g) for g in graphs]
    ks = np.ascontiguousarray(np.broadcast_to(np.asarray(k, dtype=np.int32), (nb,)))
    ns = np.array([a[0] for a in args], dtype=np.int64)
    rps = (_PI64 * nb)(*[_ptr(a[1], ctypes.c_int64) for a in args])
    cis = (_PI32 * nb)(*[_ptr(a[2], ctypes.c_int32) for a in args])
    ws = (_PD * nb)(*[_ptr(a[3], ctypes.c_double) for a in args])
    evals = [np.zeros(int(kk)) for kk in ks]
    evecs = [np.zeros((int(kk), a[0])) for kk, a in zip(ks, args)] if want_vectors else None
    ev_p = (_PD * nb)(*[_ptr(e, ctypes.c_double) for e in evals])
    vv_p = (_PD * nb)(*[_ptr(v, ctypes.c_double) for v in evecs]) if want_vectors else None
    infos = (lap_info * nb)()
    o, _keep = make_opts(**opts)
    st = lib().lap_eigs_batched(nb, _ptr(ns, ctypes.c_int64), rps, cis, ws, ks.ctypes.data_as(_PI), tol,
                                _METHODS[method] if isinstance(method, str) else int(method), ctypes.byref(o), ev_p,
                                vv_p, infos)
    _check(st, "lap_eigs_batched", allow_partial=True)
    return evals, ([v.T for v in evecs] if want_vectors else None), [i.as_dict() for i in infos]  # column-major views


# ---------------------------------------------------------------- device-level API

def _dtype_of(t):
    import torch
    if t.dtype == torch.float64:
        return LAP_F64
    if t.dtype == torch.float32:
        return LAP_F32
    raise TypeError("blocks must be float32 or float64")


def _blk(t):
    """(pointer, leading dimension) of a row-major 2-D CUDA tensor."""
    if t is None:
        return None, 0
    if not t.is_cuda or t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("expected a 2-D CUDA tensor with unit stride along rows")
    return ctypes.c_void_p(t.data_ptr()), t.stride(0)


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Graph:
    """A graph (or batch of graphs) resident on the device (lap_graph handle)."""

    def __init__(self, graphs):
        if not isinstance(graphs, (list, tuple)):
            graphs = [graphs]
        h = ctypes.c_void_p()
        args = [_csr_args(g) for g in graphs]
        if len(args) == 1:
            n, rp, ci, w = args[0]
            st = lib().lap_graph_create(n, _ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32),
                                        _ptr(w, ctypes.c_double), ctypes.byref(h))
        else:
            nb = len(args)
            ns = np.array([a[0] for a in args], dtype=np.int64)
            rps = (_PI64 * nb)(*[_ptr(a[1], ctypes.c_int64) for a in args])
            cis = (_PI32 * nb)(*[_ptr(a[2], ctypes.c_int32) for a in args])
            ws = (_PD * nb)(*[_ptr(a[3], ctypes.c_double) for a in args])
            st = lib().lap_graph_create_batched(nb, _ptr(ns, ctypes.c_int64), rps, cis, ws, ctypes.byref(h))
        _check(st, "lap_graph_create")
        self.h = h
        self._keep = args
        self.row0 = np.concatenate([[0], np.cumsum([a[0] for a in args])])
        self.nseg = len(args)
        self.n = int(self.row0[-1])

    def close(self):
        if getattr(self, "h", None):
            lib().lap_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        nt, ns, team, nl = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        norm1 = np.zeros(self.nseg)
        _check(lib().lap_graph_info(self.h, ctypes.byref(nt), ctypes.byref(ns), _ptr(norm1, ctypes.c_double),
                                    ctypes.byref(team), ctypes.byref(nl)), "lap_graph_info")
        return dict(n_total=nt.value, nseg=ns.value, norm1=norm1, team=team.value, nlong=nl.value)

    def set_schedule(self, team=0, long_thresh=0):
        _check(lib().lap_graph_set_schedule(self.h, team, long_thresh), "lap_graph_set_schedule")

    def autotune(self, dtype="f32", b=12):
        """Time the SpMM schedules on this handle and keep the fastest
        (lap_graph_autotune); returns (gathers in flight or lanes per row,
        hub threshold)."""
        t, h = ctypes.c_int(), ctypes.c_int()
        _check(lib().lap_graph_autotune(self.h, LAP_F32 if dtype == "f32" else LAP_F64, b, ctypes.byref(t),
                                        ctypes.byref(h), _stream()), "lap_graph_autotune")
        return t.value, h.value

    def set_precond(self, kind="fsai", alpha=0.0):
        """Correction-solve preconditioner of the handle (lap_graph_set_precond)."""
        _check(lib().lap_graph_set_precond(self.h, _PRECONDS[kind] if isinstance(kind, str) else int(kind), alpha),
               "lap_graph_set_precond")

    def set_gathers(self, gathers):
        """Form of the vectorised SpMM (lap_graph_set_gathers): 2, 4, 8, 102 or 104."""
        _check(lib().lap_graph_set_gathers(self.h, gathers), "lap_graph_set_gathers")

    def set_reorder(self, mode="auto"):
        """Node order of the solves (lap_graph_set_reorder): "auto", "none" or "degree"."""
        _check(lib().lap_graph_set_reorder(self.h, _REORDERS[mode] if isinstance(mode, str) else int(mode)),
               "lap_graph_set_reorder")

    def set_launch(self, max_ctas=0, device_timeout_ms=0.0, split_rows=0):
        """CTA cap, device wait limit, and the row count from which the
        correction solve runs as per-phase launches (lap_graph_set_launch)."""
        _check(lib().lap_graph_set_launch(self.h, max_ctas, device_timeout_ms, split_rows), "lap_graph_set_launch")

    def eigs(self, k: int, tol: float = 1e-8, method: str = "jd", evecs=None, **opts):
        """Solve on the resident graph(s) (lap_eigs_graph).  evecs: optional
        float64 CUDA tensor of n_total * k elements receiving each graph's
        column-major eigenvector block at offset row0[s] * k.  Returns
        (evals [nseg, k] numpy, infos list)."""
        o, _keep = make_opts(**opts)
        evals = np.zeros(self.nseg * k)
        infos = (lap_info * self.nseg)()
        pv = None if evecs is None else ctypes.c_void_p(evecs.data_ptr())
        st = lib().lap_eigs_graph(self.h, k, tol, _METHODS[method] if isinstance(method, str) else int(method),
                                  ctypes.byref(o), _ptr(evals, ctypes.c_double), pv, infos)
        _check(st, "lap_eigs_graph", allow_partial=True)
        return evals.reshape(self.nseg, k), [i.as_dict() for i in infos]

    # Steps of the outer loop (device tensors in, device tensors out)
    def spmm(self, X, Y):
        px, ldx = _blk(X)
        py, ldy = _blk(Y)
        _check(lib().lap_spmm(self.h, _dtype_of(X), px, ldx, py, ldy, X.shape[1], _stream()), "lap_spmm")
        return Y

    def gram(self, A, B, ones=False):
        import torch
        pa, lda = _blk(A)
        pb, ldb = _blk(B)
        p = 0 if A is None else A.shape[1]
        q = B.shape[1]
        G = torch.zeros((self.nseg, p + int(ones), q), dtype=torch.float64, device=B.device)
        _check(lib().lap_gram(self.h, _dtype_of(B), pa, lda, p, pb, ldb, q, int(ones), ctypes.c_void_p(G.data_ptr()),
                              _stream()), "lap_gram")
        return G

    def project(self, Q, X):
        pq, ldq = _blk(Q)
        px, ldx = _blk(X)
        nq = 0 if Q is None else Q.shape[1]
        _check(lib().lap_project(self.h, _dtype_of(X), pq, ldq, nq, px, ldx, X.shape[1], _stream()), "lap_project")
        return X

    def cgs2(self, V, T):
        pv, ldv = _blk(V)
        pt, ldt = _blk(T)
        m = 0 if V is None else V.shape[1]
        kept = np.zeros(self.nseg * T.shape[1], dtype=np.int32)
        _check(lib().lap_cgs2(self.h, _dtype_of(T), pv, ldv, m, pt, ldt, T.shape[1], _ptr(kept, ctypes.c_int),
                              _stream()), "lap_cgs2")
        return kept.reshape(self.nseg, T.shape[1])

    def rayleigh_ritz(self, V):
        import torch
        pv, ldv = _blk(V)
        theta = torch.zeros((self.nseg, V.shape[1]), dtype=torch.float64, device=V.device)
        _check(lib().lap_rayleigh_ritz(self.h, _dtype_of(V), pv, ldv, V.shape[1], ctypes.c_void_p(theta.data_ptr()),
                                       _stream()), "lap_rayleigh_ritz")
        return theta

    def residual_norms(self, X, theta):
        import torch
        px, ldx = _blk(X)
        theta = theta.contiguous()
        out = torch.zeros((self.nseg, X.shape[1]), dtype=torch.float64, device=X.device)
        _check(lib().lap_residual_norms(self.h, _dtype_of(X), px, ldx, ctypes.c_void_p(theta.data_ptr()), X.shape[1],
                                        ctypes.c_void_p(out.data_ptr()), _stream()), "lap_residual_norms")
        return out

    def pcg_correction(self, X, theta, R, iters, delta=0.0):
        import torch
        px, ldx = _blk(X)
        pr, ldr = _blk(R)
        b = R.shape[1]
        T = torch.zeros((R.shape[0], b), dtype=R.dtype, device=R.device)
        theta = theta.contiguous()
        _check(lib().lap_pcg_correction(self.h, _dtype_of(R), px, ldx, ctypes.c_void_p(theta.data_ptr()), pr, ldr,
                                        ctypes.c_void_p(T.data_ptr()), b, b, iters, delta, _stream()),
               "lap_pcg_correction")
        return T


def _evals_arg(evals):
    e = np.ascontiguousarray(evals, dtype=np.float64)
    return e, _ptr(e, ctypes.c_double)


_MODES = {"T": 0, "S": 1}


class Applications:
    """The computed pairs put to use (Section 2): Fiedler ordering and
    bisection, and the pseudo-inverse approximations with the current-flow
    centralities, on a single-graph handle.  v2 and V are float64 CUDA
    tensors (n, and n x k row-major)."""

    def __init__(self, graph: "Graph"):
        self.G = graph

    def fiedler_order(self, v2):
        import torch
        perm = torch.empty(self.G.n, dtype=torch.int32, device=v2.device)
        bw, pr, bw0, pr0 = (ctypes.c_int64() for _ in range(4))
        _check(lib().lap_fiedler_order(self.G.h, ctypes.c_void_p(v2.data_ptr()), ctypes.c_void_p(perm.data_ptr()),
                                       ctypes.byref(bw), ctypes.byref(pr), ctypes.byref(bw0), ctypes.byref(pr0),
                                       _stream()), "lap_fiedler_order")
        return perm, dict(bandwidth=bw.value, profile=pr.value, bandwidth0=bw0.value, profile0=pr0.value)

    def fiedler_bisect(self, v2, lambda2: float, n1: int):
        import torch
        side = torch.empty(self.G.n, dtype=torch.int32, device=v2.device)
        cut, bound = ctypes.c_double(), ctypes.c_double()
        _check(lib().lap_fiedler_bisect(self.G.h, ctypes.c_void_p(v2.data_ptr()), float(lambda2), int(n1),
                                        ctypes.c_void_p(side.data_ptr()), ctypes.byref(cut), ctypes.byref(bound),
                                        _stream()), "lap_fiedler_bisect")
        return side, cut.value, bound.value

    def pinv_apply(self, evals, V, X, mode="T", sigma=0.0):
        import torch
        e, pe = _evals_arg(evals)
        Y = torch.empty_like(X)
        pv, ldv = _blk(V)
        px, ldx = _blk(X)
        py, ldy = _blk(Y)
        _check(lib().lap_pinv_apply(self.G.h, e.size, pe, pv, ldv, _MODES[mode], float(sigma), px, ldx, py, ldy,
                                    X.shape[1], _stream()), "lap_pinv_apply")
        return Y

    def closeness(self, evals, V, mode="T", sigma=0.0):
        import torch
        e, pe = _evals_arg(evals)
        out = torch.empty(self.G.n, dtype=torch.float64, device=V.device)
        pv, ldv = _blk(V)
        _check(lib().lap_cf_closeness(self.G.h, e.size, pe, pv, ldv, _MODES[mode], float(sigma),
                                      ctypes.c_void_p(out.data_ptr()), _stream()), "lap_cf_closeness")
        return out

    def betweenness(self, evals, V, pairs, mode="T", sigma=0.0):
        import torch
        e, pe = _evals_arg(evals)
        pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int64).reshape(-1, 2))
        out = torch.empty(self.G.n, dtype=torch.float64, device=V.device)
        pv, ldv = _blk(V)
        _check(lib().lap_cf_betweenness(self.G.h, e.size, pe, pv, ldv, _MODES[mode], float(sigma), pr.shape[0],
                                        _ptr(pr, ctypes.c_int64), ctypes.c_void_p(out.data_ptr()), _stream()),
               "lap_cf_betweenness")
        return out


def lap_syev_batched(H):
    """Eigen-decomposition of a batch of small symmetric FP64 device matrices
    H [nmat, m, m] -> (evals [nmat, m] ascending, Y [nmat, m, m])."""
    import torch
    H = H.contiguous()
    nmat, m, _ = H.shape
    ev = torch.zeros((nmat, m), dtype=torch.float64, device=H.device)
    Y = torch.zeros((nmat, m, m), dtype=torch.float64, device=H.device)
    _check(lib().lap_syev_batched(nmat, m, ctypes.c_void_p(H.data_ptr()), m, ctypes.c_void_p(ev.data_ptr()),
                                  ctypes.c_void_p(Y.data_ptr()), m, _stream()), "lap_syev_batched")
    return ev, Y


def lap_profile_enable(on: bool = True):
    _check(lib().lap_profile_enable(int(bool(on))), "lap_profile_enable")


def lap_profile_read(max_entries: int = 64):
    """{kernel name: dict(ms, bytes, launches)} accumulated since the last read
    (synchronises the device)."""
    L = 48
    names = ctypes.create_string_buffer(max_entries * L)
    ms = np.zeros(max_entries)
    by = np.zeros(max_entries)
    la = np.zeros(max_entries, dtype=np.int64)
    cnt = ctypes.c_int()
    _check(lib().lap_profile_read(max_entries, names, L, _ptr(ms, ctypes.c_double), _ptr(by, ctypes.c_double),
                                  _ptr(la, ctypes.c_int64), ctypes.byref(cnt)), "lap_profile_read")
    out = {}
    for i in range(cnt.value):
        nm = names.raw[i * L:(i + 1) * L].split(b"\0")[0].decode()
        out[nm] = dict(ms=float(ms[i]), bytes=float(by[i]), launches=int(la[i]))
    return out
