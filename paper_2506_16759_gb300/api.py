"""Python binding of the h2gb C ABI.

Thin wrappers that pass device pointers of torch CUDA tensors and the current
stream to libh2gb; the construction itself runs in the CUDA library.  Panels
(N x d) are handed over column-major: a tensor of shape (N, d) with strides
(1, N).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import BuildOpts, Stats, TreeInfo, check, lib

KERNELS = {"exp": 0, "matern32": 1, "gauss": 2, "laplace_ie": 3, "poly": 4, "h2sum": 5,
           "helmholtz_ie": 6}
PREC = {"fp64": 0, "mixed": 1, "mixed_simt": 2}
SKETCH = {"ksum": 0, "dense": 1, "callback": 2, "h2sum": 3}


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def colmajor(x: torch.Tensor) -> torch.Tensor:
    """(N, d) tensor with column-major storage (ld = N)."""
    if x.dim() == 1:
        return x.contiguous()
    return x.t().contiguous().t()


def _kid(kernel) -> int:
    return KERNELS[kernel] if isinstance(kernel, str) else int(kernel)


def _params(params, n=4) -> np.ndarray:
    p = np.zeros(n, dtype=np.float64)
    vals = list(params)
    p[:len(vals)] = vals
    return p


class ClusterTree:
    """KD cluster tree and block lists (h2_build_cluster_tree)."""

    def __init__(self, points: torch.Tensor, leaf_size: int = 64, eta: float = 0.7,
                 stream=None):
        if not points.is_cuda or points.dtype != torch.float64 or points.dim() != 2:
            raise ValueError("points must be a CUDA float64 tensor of shape (n, dim)")
        self.points = points.contiguous()
        n, dim = self.points.shape
        h = C.c_void_p()
        check(lib().h2_build_cluster_tree(self.points.data_ptr(), n, dim, leaf_size, eta,
                                          _stream(stream), C.byref(h)),
              "h2_build_cluster_tree")
        self.handle = h
        self._info = None

    @property
    def info(self) -> TreeInfo:
        if self._info is None:
            inf = TreeInfo()
            check(lib().h2_tree_info(self.handle, C.byref(inf)), "h2_tree_info")
            self._info = inf
        return self._info

    def export(self) -> dict:
        inf = self.info
        n, nn, dim = inf.n, inf.n_nodes, inf.dim
        perm = np.zeros(n, dtype=np.int32)
        begin = np.zeros(nn, dtype=np.int64)
        end = np.zeros(nn, dtype=np.int64)
        lo = np.zeros((nn, dim))
        hi = np.zeros((nn, dim))
        check(lib().h2_tree_export(self.handle, perm.ctypes.data, begin.ctypes.data,
                                   end.ctypes.data, lo.ctypes.data, hi.ctypes.data),
              "h2_tree_export")
        return {"perm": perm, "begin": begin, "end": end, "lo": lo, "hi": hi}

    def block_list(self, which: str, depth: int) -> dict:
        """{node: sorted partner list} for the far ('far') or near ('near') list."""
        inf = self.info
        rows = 1 << depth
        nnz = inf.near_nnz if which == "near" else inf.far_nnz[depth]
        ptr = np.zeros(rows + 1, dtype=np.int64)
        cols = np.zeros(max(nnz, 1), dtype=np.int32)
        check(lib().h2_tree_export_list(self.handle, 1 if which == "near" else 0, depth,
                                        ptr.ctypes.data, cols.ctypes.data),
              "h2_tree_export_list")
        first = rows - 1
        out = {}
        for r in range(rows):
            if ptr[r + 1] > ptr[r]:
                out[first + r] = cols[ptr[r]:ptr[r + 1]].tolist()
        return out

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib._lib is not None:
            lib().h2_tree_destroy(h)
            self.handle = None


def make_opts(d0=32, d_inc=16, d_max=256, prec="fp64", omega=None, seed=0, sketch="ksum",
              dense_a=None, timing=False, sampler=None, operands=None, ksum_tile=0,
              lowrank=None, bsr_engine=0, tc_cols=0, ksum_split=0, nonsym=False, psi=None,
              sampler_t=None, queue_order=0, sum_engine=0):
    o = BuildOpts()
    lib().h2_default_opts(C.byref(o))
    o.d0, o.d_inc, o.d_max = d0, d_inc, d_max
    o.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    keep = []
    if omega is not None:
        om = colmajor(omega)
        keep.append(om)
        o.omega_mode = 1
        o.omega_stored = om.data_ptr()
    o.seed = seed
    o.sketch = SKETCH[sketch] if isinstance(sketch, str) else int(sketch)
    if dense_a is not None:
        a = colmajor(dense_a)
        keep.append(a)
        o.dense_a = a.data_ptr()
    if sampler is not None:
        cb = _lib.SAMPLER_FN(sampler)
        keep.append(cb)
        o.sampler = cb
    if operands:
        arr = (C.c_void_p * len(operands))(*[op.handle.value for op in operands])
        keep.append(arr)
        o.operands = C.cast(arr, C.c_void_p)
        o.n_operands = len(operands)
    o.timing = 1 if timing else 0
    o.ksum_tile = ksum_tile
    o.bsr_engine, o.tc_cols, o.ksum_split = bsr_engine, tc_cols, ksum_split
    o.queue_order = queue_order
    o.sum_engine = sum_engine
    if nonsym:
        # separate row and column bases: Psi (stored mode) and A^T x (callback)
        o.nonsym = 1
        if psi is not None:
            ps = colmajor(psi)
            keep.append(ps)
            o.psi_stored = ps.data_ptr()
        if sampler_t is not None:
            cbt = _lib.SAMPLER_FN(sampler_t)
            keep.append(cbt)
            o.sampler_t = cbt
    if lowrank is not None:
        # (U, V): the operator gets the symmetric term U V^T
        u, v = (colmajor(x.to(torch.float64)) for x in lowrank)
        keep += [u, v]
        o.lowrank_u, o.lowrank_v, o.lowrank_rank = u.data_ptr(), v.data_ptr(), u.shape[1]
    return o, keep


class H2Matrix:
    """An H2 matrix built by h2_build / h2_build_batched."""

    def __init__(self, handle, status, trees, keep):
        self.handle = handle
        self.status = status
        self.trees = trees
        self._keep = keep

    @property
    def converged(self) -> bool:
        return self.status == _lib.H2_OK

    @classmethod
    def build(cls, tree: ClusterTree, kernel, params, tol: float, stream=None, **kw):
        lr = kw.get("lowrank")
        if lr is not None:
            # the library reads N x rank from each factor: check the shapes here
            u, v = lr
            n = tree.info.n
            if u.dim() != 2 or tuple(u.shape) != tuple(v.shape) or u.shape[0] != n:
                raise ValueError(f"low-rank factors must both be ({n}, rank), got "
                                 f"{tuple(u.shape)} and {tuple(v.shape)}")
        o, keep = make_opts(**kw)
        p = _params(params)
        h = C.c_void_p()
        st = lib().h2_build(tree.handle, _kid(kernel), p.ctypes.data, 4, float(tol), C.byref(o),
                            _stream(stream), C.byref(h))
        check(st, "h2_build", allow=(_lib.H2_OK, _lib.H2_ERR_NOT_CONVERGED))
        return cls(h, st, [tree], keep)

    @classmethod
    def build_batched(cls, trees, kernels, params, tols, stream=None, **kw):
        o, keep = make_opts(**kw)
        k = np.array([_kid(x) for x in kernels], dtype=np.int32)
        p = np.stack([_params(x) for x in params]).astype(np.float64)
        t = np.asarray(tols, dtype=np.float64)
        arr = (C.c_void_p * len(trees))(*[tr.handle.value for tr in trees])
        h = C.c_void_p()
        st = lib().h2_build_batched(C.cast(arr, C.c_void_p), len(trees), k.ctypes.data,
                                    p.ctypes.data, t.ctypes.data, C.byref(o), _stream(stream),
                                    C.byref(h))
        check(st, "h2_build_batched", allow=(_lib.H2_OK, _lib.H2_ERR_NOT_CONVERGED))
        return cls(h, st, list(trees), keep)

    def matvec(self, x: torch.Tensor, stream=None) -> torch.Tensor:
        squeeze = x.dim() == 1
        X = colmajor(x[:, None] if squeeze else x).to(torch.float64)
        Y = colmajor(torch.empty_like(X))
        check(lib().h2_matvec(self.handle, X.data_ptr(), Y.data_ptr(), X.shape[1],
                              _stream(stream)), "h2_matvec")
        return Y[:, 0] if squeeze else Y

    def stats(self) -> dict:
        st = Stats()
        check(lib().h2_stats(self.handle, C.byref(st)), "h2_stats")
        return {name: getattr(st, name) for name, _ in Stats._fields_}

    def export_col_level(self, level: int, inst: int = 0):
        """Column side of a non-symmetric build: (ranks, column skeletons as
        original indices)."""
        tree = self.trees[inst]
        nl = 1 << (tree.info.depth - level + 1)
        ranks = np.zeros(nl, dtype=np.int32)
        skel = np.zeros(nl * 512, dtype=np.int32)
        check(lib().h2_export_col_level(self.handle, inst, level, ranks.ctypes.data,
                                        skel.ctypes.data), "h2_export_col_level")
        return ranks, skel[:int(ranks.sum())]

    def export_level(self, level: int, inst: int = 0):
        """(ranks per cluster in heap order, skeleton original indices, eps_l, d_l)."""
        tree = self.trees[inst]
        depth = tree.info.depth - level + 1
        nl = 1 << depth
        ranks = np.zeros(nl, dtype=np.int32)
        skel = np.zeros(nl * 512, dtype=np.int32)
        eps = C.c_double()
        d = C.c_int32()
        check(lib().h2_export_level(self.handle, inst, level, ranks.ctypes.data, skel.ctypes.data,
                                    C.byref(eps), C.byref(d)), "h2_export_level")
        return ranks, skel[:int(ranks.sum())], eps.value, d.value

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib._lib is not None:
            lib().h2_matrix_destroy(h)
            self.handle = None


def autotune(tree: ClusterTree, kernel, params, tol: float, stream=None, **kw) -> tuple:
    """(best build keyword arguments, build ms) over the sample schedules,
    sketch engines and launch shapes h2_autotune tries."""
    o, keep = make_opts(**kw)
    best = BuildOpts()
    ms = C.c_double()
    p = _params(params)
    check(lib().h2_autotune(tree.handle, _kid(kernel), p.ctypes.data, 4, float(tol), C.byref(o),
                            _stream(stream), C.byref(best), C.byref(ms)), "h2_autotune")
    inv = {v: k for k, v in PREC.items()}
    out = dict(kw)
    out.update(d0=best.d0, d_inc=best.d_inc, prec=inv[best.prec], bsr_engine=best.bsr_engine,
               tc_cols=best.tc_cols, ksum_split=best.ksum_split, queue_order=best.queue_order,
               sum_engine=best.sum_engine)
    return out, ms.value


def ksum_sketch(points: torch.Tensor, kernel, params, omega: torch.Tensor, prec="fp64",
                stream=None) -> torch.Tensor:
    pts = points.contiguous()
    om = colmajor(omega)
    n, d = om.shape
    y = colmajor(torch.empty_like(om))
    p = _params(params)
    check(lib().h2_ksum_sketch(pts.data_ptr(), n, pts.shape[1], _kid(kernel), p.ctypes.data, 4,
                               om.data_ptr(), n, y.data_ptr(), n, d,
                               PREC[prec] if isinstance(prec, str) else prec, _stream(stream)),
          "h2_ksum_sketch")
    return y


def entry_block(points: torch.Tensor, kernel, params, rows: torch.Tensor, cols: torch.Tensor,
                stream=None) -> torch.Tensor:
    pts = points.contiguous()
    r = rows.to(torch.int32).contiguous()
    c = cols.to(torch.int32).contiguous()
    out = colmajor(torch.empty((r.numel(), c.numel()), dtype=torch.float64, device=pts.device))
    p = _params(params)
    check(lib().h2_entry_block(pts.data_ptr(), pts.shape[0], pts.shape[1], _kid(kernel),
                               p.ctypes.data, 4, r.data_ptr(), r.numel(), c.data_ptr(), c.numel(),
                               out.data_ptr(), _stream(stream)), "h2_entry_block")
    return out


def dense_sketch(a: torch.Tensor, omega: torch.Tensor, stream=None) -> torch.Tensor:
    A = colmajor(a)
    om = colmajor(omega)
    n, d = om.shape
    y = colmajor(torch.empty_like(om))
    check(lib().h2_dense_sketch(A.data_ptr(), n, n, om.data_ptr(), n, y.data_ptr(), n, d,
                                _stream(stream)), "h2_dense_sketch")
    return y


def _pack_panels(panels):
    dev = panels[0].device
    ms = np.array([p.shape[0] for p in panels], dtype=np.int32)
    ds = np.array([p.shape[1] for p in panels], dtype=np.int32)
    offs = np.zeros(len(panels), dtype=np.int64)
    offs[1:] = np.cumsum(ms.astype(np.int64) * ds)[:-1]
    flat = torch.cat([colmajor(p.to(torch.float64)).t().reshape(-1) for p in panels])
    return (torch.from_numpy(ms).to(dev), torch.from_numpy(ds).to(dev),
            torch.from_numpy(offs).to(dev), flat, ms, ds)


def batched_qr_mindiag(panels, stream=None) -> torch.Tensor:
    m, d, off, flat, _, _ = _pack_panels(panels)
    out = torch.zeros(len(panels), dtype=torch.float64, device=flat.device)
    check(lib().h2_batched_qr_mindiag(len(panels), m.data_ptr(), d.data_ptr(), off.data_ptr(),
                                      flat.data_ptr(), out.data_ptr(), _stream(stream)),
          "h2_batched_qr_mindiag")
    return out


def batched_row_id(panels, eps, stream=None):
    """Returns (ranks, [J_i], [E_i]) for sample panels Y_i (m_i x d_i)."""
    m, d, off, flat, ms, ds = _pack_panels(panels)
    dev = flat.device
    cap = ms.astype(np.int64) * np.minimum(ms, ds)
    eoff = np.zeros(len(panels), dtype=np.int64)
    eoff[1:] = np.cumsum(cap)[:-1]
    ldj = int(max(ms.max(), 1))
    k = torch.zeros(len(panels), dtype=torch.int32, device=dev)
    J = torch.zeros(len(panels) * ldj, dtype=torch.int32, device=dev)
    E = torch.zeros(int(max(cap.sum(), 1)), dtype=torch.float64, device=dev)
    ep = torch.as_tensor(np.asarray(eps, dtype=np.float64), device=dev)
    eo = torch.from_numpy(eoff).to(dev)
    check(lib().h2_batched_row_id(len(panels), m.data_ptr(), d.data_ptr(), off.data_ptr(),
                                  flat.data_ptr(), ep.data_ptr(), k.data_ptr(), J.data_ptr(), ldj,
                                  eo.data_ptr(), E.data_ptr(), _stream(stream)),
          "h2_batched_row_id")
    ks = k.cpu().numpy()
    Jh = J.cpu().numpy().reshape(len(panels), ldj)
    Eh = E.cpu().numpy()
    Js, Es = [], []
    for i, kk in enumerate(ks):
        Js.append(Jh[i, :kk].copy())
        Es.append(Eh[eoff[i]:eoff[i] + ms[i] * kk].reshape(kk, ms[i]).T.copy())
    return ks, Js, Es


def trim_memory() -> None:
    """Return the device blocks the library caches for reuse to CUDA."""
    lib().h2_trim_memory()
