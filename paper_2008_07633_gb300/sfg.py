"""Thin Python binding of libsfg (include/sfg.h): argument marshalling only.

Every function has the name of the C entry point it calls. Tensors are PyTorch CUDA tensors used
as device memory; the context queues work on a CUDA stream (by default PyTorch's current stream at
creation). No computation happens here: a missing or unloadable libsfg.so raises immediately.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("SFG_LIB", os.path.join(_HERE, "libsfg.so"))

SFG_F32, SFG_BF16 = 0, 1
SFG_SCORE_RATIO, SFG_SCORE_G, SFG_SCORE_P = 0, 1, 2
STATUS = {0: "SFG_OK", 1: "SFG_EINVAL", 2: "SFG_ENOMEM", 3: "SFG_ECUDA", 4: "SFG_ETIMEOUT",
          5: "SFG_ECAPACITY", 6: "SFG_EUNSUPPORTED"}

# Every symbol declared in include/sfg.h.
EXPORTS = ["sfg_ctx_create", "sfg_ctx_destroy", "sfg_ctx_trim", "sfg_ctx_set_stream", "sfg_last_error",
           "sfg_ctx_timing", "sfg_ctx_kernel_time", "sfg_ctx_launches", "sfg_laplacian", "sfg_graph_destroy",
           "sfg_graph_info", "sfg_graph_edges", "sfg_graph_csr", "sfg_graph_subgraph", "sfg_smooth",
           "sfg_jacobi", "sfg_score_edges", "sfg_select_topk", "sfg_spanning_tree", "sfg_affinity",
           "sfg_affinity_noalloc", "sfg_filter_score", "sfg_sparsify_batched", "sfg_mlp_create",
           "sfg_mlp_destroy", "sfg_mlp_params", "sfg_mlp_set_params", "sfg_mlp_forward",
           "sfg_mlp_gradient", "sfg_mlp_train", "sfg_edge_features", "sfg_sparsify_learned",
           "sfg_autotune", "sfg_tune_set", "sfg_tune_set_score", "sfg_tune_table",
           "sfg_coarsen", "sfg_backward_map", "sfg_sparsify", "sfg_kappa",
           "sfg_sparsify_to_kappa", "sfg_smooth_gs", "sfg_coloring", "sfg_solve_pcg",
           "sfg_hierarchy_levels", "sfg_hierarchy_graph", "sfg_hierarchy_map",
           "sfg_hierarchy_mask", "sfg_hierarchy_destroy", "sfg_batch_create", "sfg_batch_info",
           "sfg_batch_run", "sfg_batch_destroy", "sfg_mlp_check"]


class SfgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class sfg_params(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("steps", ctypes.c_int), ("levels", ctypes.c_int),
                ("omega", ctypes.c_double), ("seed", ctypes.c_uint64), ("mode", ctypes.c_int),
                ("budget_frac", ctypes.c_double), ("budget_unit", ctypes.c_int),
                ("storage", ctypes.c_int), ("smoother", ctypes.c_int)]


SFG_SMOOTH_JACOBI, SFG_SMOOTH_GAUSS_SEIDEL = 0, 1


_lib = None
_vp = ctypes.c_void_p
_i32, _i64, _int, _dbl, _u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
_pi32, _pi64, _pdbl = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)


def lib():
    """Load libsfg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2008_07633_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "sfg_ctx_create": [ctypes.POINTER(_vp), _int, _vp],
            "sfg_ctx_destroy": [_vp],
            "sfg_ctx_trim": [_vp],
            "sfg_ctx_set_stream": [_vp, _vp],
            "sfg_last_error": [_vp],
            "sfg_ctx_timing": [_vp, _int],
            "sfg_ctx_kernel_time": [_vp, ctypes.c_char_p, _pi64, _pdbl],
            "sfg_ctx_launches": [_vp, _pi64],
            "sfg_laplacian": [_vp, _i32, _i64, _vp, _vp, _vp, ctypes.POINTER(_vp)],
            "sfg_graph_destroy": [_vp],
            "sfg_graph_info": [_vp, _pi32, _pi64],
            "sfg_graph_edges": [_vp, _vp, _vp, _vp, _vp],
            "sfg_graph_csr": [_vp, _vp, _vp, _vp, _vp, _vp, _vp],
            "sfg_graph_subgraph": [_vp, _vp, _vp, ctypes.POINTER(_vp)],
            "sfg_smooth": [_vp, _vp, _int, _int, _dbl, _u64, _int, _vp],
            "sfg_jacobi": [_vp, _vp, _int, _int, _dbl, _int, _vp],
            "sfg_smooth_gs": [_vp, _vp, _int, _int, _dbl, _u64, _int, _vp],
            "sfg_coloring": [_vp, _vp, _vp, _pi32],
            "sfg_score_edges": [_vp, _vp, _vp, _vp, _int, _int, _vp, _i64, _int, _vp],
            "sfg_select_topk": [_vp, _vp, _vp, _i64, _i64, _vp],
            "sfg_filter_score": [_vp, _vp, _vp, _int, _int, _dbl, _u64, _int, _vp, _i64, _int, _vp],
            "sfg_spanning_tree": [_vp, _vp, _vp, _vp, _pi64],
            "sfg_affinity": [_vp, _vp, _vp, _int, _vp],
            "sfg_affinity_noalloc": [_vp, _vp, _vp, _int, _vp],
            "sfg_coarsen": [_vp, _vp, _vp, _int, _int, _vp, _vp, _pi32, ctypes.POINTER(_vp)],
            "sfg_backward_map": [_vp, _vp, _vp, _vp, _vp, _vp, _vp],
            "sfg_sparsify": [_vp, _vp, ctypes.POINTER(sfg_params), _vp, _pi64, ctypes.POINTER(_vp)],
            "sfg_hierarchy_levels": [_vp, ctypes.POINTER(_int)],
            "sfg_hierarchy_graph": [_vp, _int, ctypes.POINTER(_vp)],
            "sfg_hierarchy_map": [_vp, _vp, _int, _vp, _vp],
            "sfg_hierarchy_mask": [_vp, _vp, _int, _vp],
            "sfg_hierarchy_destroy": [_vp],
            "sfg_batch_create": [_vp, _int, ctypes.POINTER(_vp), ctypes.POINTER(sfg_params), _int,
                                 ctypes.POINTER(_vp)],
            "sfg_batch_info": [_vp, ctypes.POINTER(_int), _pi64, _pi64, _pi64],
            "sfg_batch_run": [_vp, _vp, _u64, _vp],
            "sfg_batch_destroy": [_vp],
            "sfg_sparsify_batched": [_vp, _int, ctypes.POINTER(_vp), ctypes.POINTER(sfg_params),
                                     ctypes.POINTER(_vp), _pi64],
            "sfg_kappa": [_vp, _vp, _vp, _int, _u64, _pdbl, _pdbl],
            "sfg_solve_pcg": [_vp, _vp, _vp, _vp, _dbl, _int, _vp, ctypes.POINTER(_int), _pdbl],
            "sfg_sparsify_to_kappa": [_vp, _vp, ctypes.POINTER(sfg_params), _dbl, _dbl, _int, _int,
                                      _vp, _pi64, _pdbl, ctypes.POINTER(_int)],
            "sfg_mlp_create": [_vp, _u64, ctypes.POINTER(_vp)],
            "sfg_autotune": [_vp, _vp, _int, _int, ctypes.POINTER(_int), _pdbl],
            "sfg_tune_set": [_vp, _int, _int, _int, _int],
            "sfg_tune_set_score": [_vp, _int, _int, _int, _int],
            "sfg_tune_table": [_vp, ctypes.c_char_p, _i64, _pi64],
            "sfg_mlp_destroy": [_vp],
            "sfg_mlp_params": [_vp, _vp, _vp],
            "sfg_mlp_set_params": [_vp, _vp, _vp],
            "sfg_mlp_forward": [_vp, _vp, _vp, _i64, _vp],
            "sfg_mlp_check": [_vp, _vp],
            "sfg_mlp_gradient": [_vp, _vp, _vp, _vp, _i64, _vp, _pdbl],
            "sfg_mlp_train": [_vp, _vp, _vp, _vp, _i64, _i64, _int, _dbl, _pdbl],
            "sfg_edge_features": [_vp, _vp, _vp, _int, _int, _dbl, _u64, _int, _vp, _i64, _vp],
            "sfg_sparsify_learned": [_vp, _vp, ctypes.POINTER(sfg_params), _vp, _int, _dbl, _vp,
                                     _pi64],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = None if name in ("sfg_ctx_destroy", "sfg_graph_destroy",
                                         "sfg_mlp_destroy", "sfg_hierarchy_destroy",
                                         "sfg_batch_destroy") else _int
        L.sfg_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dt(dtype):
    if dtype in (torch.float32, SFG_F32):
        return SFG_F32
    if dtype in (torch.bfloat16, SFG_BF16):
        return SFG_BF16
    raise ValueError(f"unsupported storage {dtype}")


def _tdt(code):
    return torch.float32 if code == SFG_F32 else torch.bfloat16


class Context:
    def __init__(self, device=0, stream=None):
        self.device = torch.device("cuda", device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._stream = s
        h = _vp()
        st = lib().sfg_ctx_create(ctypes.byref(h), device, _vp(s.cuda_stream))
        if st != 0:
            raise SfgError(st, "sfg_ctx_create failed")
        self.h = h

    def check(self, st):
        if st != 0:
            raise SfgError(st, lib().sfg_last_error(self.h).decode())

    def trim(self):
        """Return the context pool's unused device memory to the device."""
        self.check(lib().sfg_ctx_trim(self.h))

    def set_stream(self, stream):
        self._stream = stream
        self.check(lib().sfg_ctx_set_stream(self.h, _vp(stream.cuda_stream)))

    def close(self):
        if getattr(self, "h", None):
            lib().sfg_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Graph:
    """Owner of an sfg_graph handle."""

    def __init__(self, ctx, h):
        self.ctx = ctx
        self.h = h
        n, m = _i32(), _i64()
        lib().sfg_graph_info(h, ctypes.byref(n), ctypes.byref(m))
        self.n, self.m = n.value, m.value

    def close(self):
        if getattr(self, "h", None):
            lib().sfg_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sfg_ctx_create(device=0, stream=None) -> Context:
    return Context(device, stream)


def sfg_ctx_timing(ctx, on=True):
    ctx.check(lib().sfg_ctx_timing(ctx.h, 1 if on else 0))


def sfg_ctx_kernel_time(ctx, prefix):
    n, ms = _i64(), _dbl()
    ctx.check(lib().sfg_ctx_kernel_time(ctx.h, prefix.encode(), ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def sfg_ctx_launches(ctx):
    n = _i64()
    ctx.check(lib().sfg_ctx_launches(ctx.h, ctypes.byref(n)))
    return n.value


def sfg_laplacian(ctx, n, u, v, w) -> Graph:
    u, v, w = u.contiguous(), v.contiguous(), w.contiguous()
    assert u.dtype == torch.int32 and v.dtype == torch.int32 and w.dtype == torch.float32
    h = _vp()
    ctx.check(lib().sfg_laplacian(ctx.h, int(n), int(u.numel()), _ptr(u), _ptr(v), _ptr(w),
                                  ctypes.byref(h)))
    return Graph(ctx, h)


def sfg_graph_info(g):
    return g.n, g.m


def sfg_graph_edges(ctx, g):
    dev = ctx.device
    u = torch.empty(g.m, dtype=torch.int32, device=dev)
    v = torch.empty(g.m, dtype=torch.int32, device=dev)
    w = torch.empty(g.m, dtype=torch.float32, device=dev)
    ctx.check(lib().sfg_graph_edges(ctx.h, g.h, _ptr(u), _ptr(v), _ptr(w)))
    return u, v, w


def sfg_graph_csr(ctx, g):
    dev = ctx.device
    rp = torch.empty(g.n + 1, dtype=torch.int32, device=dev)
    col = torch.empty(2 * g.m, dtype=torch.int32, device=dev)
    val = torch.empty(2 * g.m, dtype=torch.float32, device=dev)
    eid = torch.empty(2 * g.m, dtype=torch.int32, device=dev)
    deg = torch.empty(g.n, dtype=torch.float64, device=dev)
    ctx.check(lib().sfg_graph_csr(ctx.h, g.h, _ptr(rp), _ptr(col), _ptr(val), _ptr(eid), _ptr(deg)))
    return rp, col, val, eid, deg


def sfg_graph_subgraph(ctx, g, mask) -> Graph:
    mask = mask.contiguous()
    assert mask.dtype == torch.uint8 and mask.numel() == g.m
    h = _vp()
    ctx.check(lib().sfg_graph_subgraph(ctx.h, g.h, _ptr(mask), ctypes.byref(h)))
    return Graph(ctx, h)


def sfg_smooth(ctx, g, K, steps, omega=0.7, seed=0, storage=torch.float32, out=None):
    code = _dt(storage)
    if out is None:
        out = torch.empty((g.n, K), dtype=_tdt(code), device=ctx.device)
    ctx.check(lib().sfg_smooth(ctx.h, g.h, K, steps, omega, seed & (2**64 - 1), code, _ptr(out)))
    return out


def sfg_smooth_gs(ctx, g, K, steps, omega=1.0, seed=0, storage=torch.float32, out=None):
    """Multicolour Gauss-Seidel smoothing; returns the projected n x K block."""
    if out is None:
        out = torch.empty((g.n, K), dtype=storage, device=ctx.device)
    ctx.check(lib().sfg_smooth_gs(ctx.h, g.h, K, steps, omega, seed & (2**64 - 1), _dt(storage),
                                  _ptr(out)))
    return out


def sfg_coloring(ctx, g):
    """(colour per node, number of colours) of the Gauss-Seidel colouring."""
    c = torch.empty(max(g.n, 1), dtype=torch.int32, device=ctx.device)
    nc = _i32()
    ctx.check(lib().sfg_coloring(ctx.h, g.h, _ptr(c), ctypes.byref(nc)))
    return c[:g.n], nc.value


def sfg_jacobi(ctx, g, X, steps, omega=0.7):
    assert X.is_contiguous()
    ctx.check(lib().sfg_jacobi(ctx.h, g.h, X.shape[1], steps, omega, _dt(X.dtype), _ptr(X)))
    return X


def sfg_score_edges(ctx, g, XG, XP, ids, mode=SFG_SCORE_RATIO, out=None):
    assert XG.dtype == XP.dtype and XG.shape == XP.shape
    ids = ids.contiguous()
    if out is None:
        out = torch.empty(ids.numel(), dtype=torch.float32, device=ctx.device)
    ctx.check(lib().sfg_score_edges(ctx.h, g.h, _ptr(XG), _ptr(XP), XG.shape[1], _dt(XG.dtype),
                                    _ptr(ids), ids.numel(), mode, _ptr(out)))
    return out


def sfg_filter_score(ctx, LG, LP, ids, K, steps, omega=0.7, seed=0, storage=torch.float32,
                     mode=SFG_SCORE_RATIO, out=None):
    ids = ids.contiguous()
    if out is None:
        out = torch.empty(ids.numel(), dtype=torch.float32, device=ctx.device)
    ctx.check(lib().sfg_filter_score(ctx.h, LG.h, LP.h, K, steps, omega, seed & (2**64 - 1),
                                     _dt(storage), _ptr(ids), ids.numel(), mode, _ptr(out)))
    return out


def sfg_select_topk(ctx, scores, ids, k, out=None):
    if out is None:
        out = torch.empty(max(int(k), 0), dtype=torch.int32, device=ctx.device)
    ctx.check(lib().sfg_select_topk(ctx.h, _ptr(scores.contiguous()), _ptr(ids.contiguous()),
                                    ids.numel(), int(k), _ptr(out)))
    return out


def sfg_spanning_tree(ctx, g, allow=None):
    mask = torch.empty(g.m, dtype=torch.uint8, device=ctx.device)
    nt = _i64()
    ctx.check(lib().sfg_spanning_tree(ctx.h, g.h, _ptr(allow), _ptr(mask), ctypes.byref(nt)))
    return mask, nt.value


def sfg_affinity(ctx, g, X):
    assert X.dtype == torch.float32 and X.is_contiguous()
    d = torch.empty(g.m, dtype=torch.float64, device=ctx.device)
    ctx.check(lib().sfg_affinity(ctx.h, g.h, _ptr(X), X.shape[1], _ptr(d)))
    return d


def sfg_affinity_noalloc(ctx, g, X, out=None):
    """sfg_affinity without any device allocation inside the library (see include/sfg.h)."""
    assert X.dtype == torch.float32 and X.is_contiguous()
    if out is None:
        out = torch.empty(g.m, dtype=torch.float64, device=ctx.device)
    ctx.check(lib().sfg_affinity_noalloc(ctx.h, g.h, _ptr(X), X.shape[1], _ptr(out)))
    return out


def sfg_coarsen(ctx, g, X):
    assert X.dtype in (torch.float32, torch.bfloat16) and X.is_contiguous()
    agg = torch.empty(g.n, dtype=torch.int32, device=ctx.device)
    f2c = torch.empty(g.m, dtype=torch.int32, device=ctx.device)
    nc = _i32()
    h = _vp()
    ctx.check(lib().sfg_coarsen(ctx.h, g.h, _ptr(X), X.shape[1], _dt(X.dtype), _ptr(agg), _ptr(f2c),
                                ctypes.byref(nc), ctypes.byref(h)))
    return agg, f2c, Graph(ctx, h)


def sfg_backward_map(ctx, fine, agg, f2c, coarse, pmask_c):
    out = torch.empty(fine.m, dtype=torch.uint8, device=ctx.device)
    ctx.check(lib().sfg_backward_map(ctx.h, fine.h, _ptr(agg), _ptr(f2c), coarse.h,
                                     _ptr(pmask_c.contiguous()), _ptr(out)))
    return out


class Hierarchy:
    """Owner of an sfg_hierarchy handle: the levels of one sfg_sparsify call."""

    def __init__(self, ctx, h, g0):
        self.ctx, self.h, self._g0 = ctx, h, g0
        lv = _int()
        ctx.check(lib().sfg_hierarchy_levels(h, ctypes.byref(lv)))
        self.levels = lv.value
        self.graphs = [g0]
        for lvl in range(1, self.levels + 1):
            gh = _vp()
            ctx.check(lib().sfg_hierarchy_graph(h, lvl, ctypes.byref(gh)))
            self.graphs.append(_BorrowedGraph(gh, self))

    def graph(self, level):
        """G_level (level 0 is the input graph)."""
        return self.graphs[level]

    def map(self, level):
        """H_level: (agg over G_{level-1}'s nodes, fine2coarse over G_{level-1}'s edges)."""
        f = self.graphs[level - 1]
        agg = torch.empty(f.n, dtype=torch.int32, device=self.ctx.device)
        f2c = torch.empty(max(f.m, 1), dtype=torch.int32, device=self.ctx.device)[:f.m]
        self.ctx.check(lib().sfg_hierarchy_map(self.ctx.h, self.h, level, _ptr(agg), _ptr(f2c)))
        return agg, f2c

    def mask(self, level):
        """P_level over G_level's canonical edges."""
        g = self.graphs[level]
        out = torch.empty(max(g.m, 1), dtype=torch.uint8, device=self.ctx.device)[:g.m]
        self.ctx.check(lib().sfg_hierarchy_mask(self.ctx.h, self.h, level, _ptr(out)))
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().sfg_hierarchy_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _BorrowedGraph(Graph):
    """A graph owned by a hierarchy (never destroyed through this handle)."""

    def __init__(self, h, owner):
        self.owner = owner
        super().__init__(owner.ctx, h)

    def close(self):
        self.h = None


def sfg_sparsify(ctx, g, K=8, steps=10, levels=0, omega=0.7, seed=0, mode=SFG_SCORE_RATIO,
                 budget_frac=0.1, budget_unit=1, storage=torch.float32, out=None,
                 smoother=SFG_SMOOTH_JACOBI, hierarchy=False):
    """Returns (mask, edges in P), plus a Hierarchy when hierarchy=True."""
    p = sfg_params(K, steps, levels, omega, seed & (2**64 - 1), mode, budget_frac, budget_unit,
                   _dt(storage), smoother)
    if out is None:
        out = torch.empty(g.m, dtype=torch.uint8, device=ctx.device)
    ns = _i64()
    hp = _vp()
    ctx.check(lib().sfg_sparsify(ctx.h, g.h, ctypes.byref(p), _ptr(out), ctypes.byref(ns),
                                 ctypes.byref(hp) if hierarchy else None))
    if hierarchy:
        return out, ns.value, Hierarchy(ctx, hp, g)
    return out, ns.value


def sfg_kappa(ctx, g, mask, steps=200, seed=1, info=False):
    """kappa(L_G, L_P) for P = the masked edges of g; returns (kappa, lambda_min, lambda_max), plus
    a dict (Lanczos steps, core CG iterations, ended on a failed core solve) when info=True."""
    mask = mask.contiguous()
    k = ctypes.c_double()
    inf = (ctypes.c_double * 6)()
    ctx.check(lib().sfg_kappa(ctx.h, g.h, _ptr(mask), steps, seed & (2**64 - 1), ctypes.byref(k),
                              ctypes.cast(inf, _pdbl)))
    out = (k.value, inf[0], inf[1])
    if info:
        return out + ({"steps": int(inf[2]), "cg_iterations": int(inf[3]),
                       "ended_on_failed_solve": bool(inf[4]), "lambda_min_exact": bool(inf[5])},)
    return out


def sfg_sparsify_to_kappa(ctx, g, kappa_target, batch_frac=0.01, max_rounds=20, kappa_steps=100,
                          K=8, steps=10, omega=0.7, seed=0, mode=SFG_SCORE_RATIO, budget_unit=0,
                          storage=torch.float32, smoother=SFG_SMOOTH_JACOBI):
    """Add edges in batches until kappa(L_G, L_P) <= kappa_target; returns (mask, n_selected,
    kappa trace, rounds of additions)."""
    p = sfg_params(K, steps, 0, omega, seed & (2**64 - 1), mode, 0.0, budget_unit, _dt(storage),
                   smoother)
    out = torch.empty(max(g.m, 1), dtype=torch.uint8, device=ctx.device)
    ns = _i64()
    trace = (ctypes.c_double * (max_rounds + 1))()
    rounds = _int()
    ctx.check(lib().sfg_sparsify_to_kappa(ctx.h, g.h, ctypes.byref(p), kappa_target, batch_frac,
                                          max_rounds, kappa_steps, _ptr(out), ctypes.byref(ns),
                                          ctypes.cast(trace, _pdbl), ctypes.byref(rounds)))
    return out[:g.m], ns.value, list(trace[:rounds.value + 1]), rounds.value


def sfg_solve_pcg(ctx, g, b, mask=None, tol=1e-8, maxit=1000, out=None):
    """x with L_G x = b (projected), by PCG preconditioned with the sparsifier `mask` (None:
    diagonal preconditioner); returns (x, iterations, relative residual)."""
    b = b.contiguous().to(torch.float64)
    if out is None:
        out = torch.empty(g.n, dtype=torch.float64, device=ctx.device)
    it = _int()
    rel = ctypes.c_double()
    ctx.check(lib().sfg_solve_pcg(ctx.h, g.h, None if mask is None else _ptr(mask.contiguous()),
                                  _ptr(b), tol, maxit, _ptr(out), ctypes.byref(it), ctypes.byref(rel)))
    return out, it.value, rel.value


def sfg_sparsify_batched(ctx, graphs, K=16, steps=15, omega=0.7, seed=0, mode=SFG_SCORE_RATIO,
                         budget_frac=0.05, budget_unit=0, storage=torch.float32):
    """Flat sparsification of a list of graphs in one batch; returns (masks, counts)."""
    ng = len(graphs)
    p = sfg_params(K, steps, 0, omega, seed & (2**64 - 1), mode, budget_frac, budget_unit,
                   _dt(storage))
    masks = [torch.empty(max(g.m, 1), dtype=torch.uint8, device=ctx.device) for g in graphs]
    hs = (_vp * ng)(*[g.h for g in graphs])
    outs = (_vp * ng)(*[m.data_ptr() for m in masks])
    counts = (ctypes.c_int64 * ng)()
    ctx.check(lib().sfg_sparsify_batched(ctx.h, ng, hs, ctypes.byref(p), outs, counts))
    return [m[:g.m] for m, g in zip(masks, graphs)], list(counts)


MLP_NPARAM, MLP_NFEAT = 5313, 16


class Mlp:
    """Owner of an sfg_mlp handle (the learned edge-proposal network)."""

    def __init__(self, ctx, seed=0):
        self.ctx = ctx
        h = _vp()
        ctx.check(lib().sfg_mlp_create(ctx.h, seed & (2**64 - 1), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().sfg_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sfg_mlp_create(ctx, seed=0):
    return Mlp(ctx, seed)


def sfg_mlp_params(ctx, net):
    out = torch.empty(MLP_NPARAM, dtype=torch.float32, device=ctx.device)
    ctx.check(lib().sfg_mlp_params(ctx.h, net.h, _ptr(out)))
    return out


def sfg_mlp_set_params(ctx, net, theta):
    theta = theta.contiguous().float()
    ctx.check(lib().sfg_mlp_set_params(ctx.h, net.h, _ptr(theta)))


def sfg_mlp_forward(ctx, net, feats, out=None):
    feats = feats.contiguous()
    if out is None:
        out = torch.empty(feats.shape[0], dtype=torch.float32, device=ctx.device)
    ctx.check(lib().sfg_mlp_forward(ctx.h, net.h, _ptr(feats), feats.shape[0], _ptr(out)))
    return out


def sfg_mlp_gradient(ctx, net, feats, targets):
    g = torch.empty(MLP_NPARAM, dtype=torch.float32, device=ctx.device)
    loss = _dbl()
    ctx.check(lib().sfg_mlp_gradient(ctx.h, net.h, _ptr(feats.contiguous()), _ptr(targets.contiguous()),
                                     feats.shape[0], _ptr(g), ctypes.byref(loss)))
    return g, loss.value


def sfg_mlp_train(ctx, net, feats, targets, batch=65536, epochs=1, lr=1e-3):
    loss = _dbl()
    ctx.check(lib().sfg_mlp_train(ctx.h, net.h, _ptr(feats.contiguous()), _ptr(targets.contiguous()),
                                  feats.shape[0], batch, epochs, lr, ctypes.byref(loss)))
    return loss.value


def sfg_edge_features(ctx, LG, LP, ids, K, steps, omega=0.7, seed=0, storage=torch.float32):
    ids = ids.contiguous()
    out = torch.empty((ids.numel(), MLP_NFEAT), dtype=torch.float32, device=ctx.device)
    ctx.check(lib().sfg_edge_features(ctx.h, LG.h, LP.h, K, steps, omega, seed & (2**64 - 1),
                                      _dt(storage), _ptr(ids), ids.numel(), _ptr(out)))
    return out


def sfg_sparsify_learned(ctx, g, net, K=32, steps=20, feat_steps=2, propose_frac=0.02, omega=0.7,
                         seed=0, mode=SFG_SCORE_RATIO, budget_frac=0.05, budget_unit=0,
                         storage=torch.float32):
    p = sfg_params(K, steps, 0, omega, seed & (2**64 - 1), mode, budget_frac, budget_unit,
                   _dt(storage))
    out = torch.empty(max(g.m, 1), dtype=torch.uint8, device=ctx.device)
    ns = _i64()
    ctx.check(lib().sfg_sparsify_learned(ctx.h, g.h, ctypes.byref(p), None if net is None else net.h,
                                         feat_steps, propose_frac, _ptr(out), ctypes.byref(ns)))
    return out[:g.m], ns.value


def sfg_autotune(ctx, g, K, storage=torch.float32):
    """Time the sweep's tile-shape variants on g; returns (variant, microseconds per sweep)."""
    v, us = _int(), _dbl()
    ctx.check(lib().sfg_autotune(ctx.h, g.h, K, _dt(storage), ctypes.byref(v), ctypes.byref(us)))
    return v.value, us.value


def sfg_tune_set(ctx, K, storage, degree_bucket, variant):
    ctx.check(lib().sfg_tune_set(ctx.h, K, _dt(storage), degree_bucket, variant))


def sfg_tune_set_score(ctx, K, storage, degree_bucket, shape):
    ctx.check(lib().sfg_tune_set_score(ctx.h, K, _dt(storage), degree_bucket, shape))


def sfg_tune_table(ctx):
    """The context's tuning table as a list of dicts (JSON from the library)."""
    import json

    n = _i64()
    ctx.check(lib().sfg_tune_table(ctx.h, None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value + 1)
    ctx.check(lib().sfg_tune_table(ctx.h, buf, n.value + 1, ctypes.byref(n)))
    return json.loads(buf.value.decode())


class Batch:
    """Owner of an sfg_batch plan (see include/sfg.h): build once, run many times."""

    def __init__(self, ctx, graphs, K=16, steps=15, omega=0.7, mode=SFG_SCORE_RATIO,
                 budget_frac=0.05, budget_unit=0, storage=torch.float32, autotune=False,
                 locality=False):
        self.ctx = ctx
        p = sfg_params(K, steps, 0, omega, 0, mode, budget_frac, budget_unit, _dt(storage),
                       SFG_SMOOTH_JACOBI)
        arr = (_vp * len(graphs))(*[g.h for g in graphs])
        h = _vp()
        flags = (1 if autotune else 0) | (2 if locality else 0)   # SFG_BATCH_AUTOTUNE, _LOCALITY
        ctx.check(lib().sfg_batch_create(ctx.h, len(graphs), arr, ctypes.byref(p), flags,
                                         ctypes.byref(h)))
        self.h = h
        ng, m = _int(), _i64()
        offs = (ctypes.c_int64 * (len(graphs) + 1))()
        cnt = (ctypes.c_int64 * len(graphs))()
        ctx.check(lib().sfg_batch_info(h, ctypes.byref(ng), ctypes.byref(m),
                                       ctypes.cast(offs, _pi64), ctypes.cast(cnt, _pi64)))
        self.ng, self.m = ng.value, m.value
        self.offsets = list(offs)
        self.counts = list(cnt)

    def run(self, seed, out=None):
        """All graphs' sparsifiers for one seed, as one mask over the concatenated edge lists."""
        if out is None:
            out = torch.empty(max(self.m, 1), dtype=torch.uint8, device=self.ctx.device)[:self.m]
        self.ctx.check(lib().sfg_batch_run(self.ctx.h, self.h, seed & (2**64 - 1), _ptr(out)))
        return out

    def split(self, mask):
        return [mask[self.offsets[g]:self.offsets[g + 1]] for g in range(self.ng)]

    def close(self):
        if getattr(self, "h", None):
            lib().sfg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sfg_mlp_check(ctx, net):
    """Synchronise; raise SfgError (SFG_ETIMEOUT) if a tensor-core wait of the network ran out."""
    ctx.check(lib().sfg_mlp_check(ctx.h, net.h))
