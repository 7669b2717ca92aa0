"""SF-GRASS oracle: plain FP64 CPU restatement of the method, for tests only.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package. The CUDA library never imports,
links or calls it, and it imports nothing from the CUDA library's package.

The arithmetic lives in ``sfg_oracle.cpp`` (single-threaded, FP64, no fused multiply-add), loaded
here through ctypes. This module adds the condition-number measurement of Sec. 2.2
(Eq. eqn:ineq): kappa(L_G, L_P) = lambda_max / lambda_min of the pencil (L_G, L_P) on the
complement of the common null space, from a dense generalised symmetric eigensolve (LAPACK through
scipy, a library primitive).

Parity status: pinned by ``tests/test_oracle_pins.py`` (closed-form spectra, invariants, brute
force). The end-to-end sparsifier edge set has no worked example in the paper: "parity unpinned"
against the paper, pinned only through kappa and the unit pins of its steps.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfg_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle_sfg.so")

# Score modes (same numbering as the CUDA library's public header, restated independently).
RATIO, G_ONLY, P_ONLY = 0, 1, 2
ETA = 1e-30


def build(force: bool = False) -> str:
    """Compile the oracle shared library with the host C++ compiler."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                               "-ffp-contract=off", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i32, _i64, _u64, _f64, _int = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int


def _declare(L):
    sig = {
        "orc_canonicalize": (_int, [_i32, _i64, _i32p, _i32p, _f32p, _i32p, _i32p, _f32p, _i64p]),
        "orc_laplacian": (None, [_i32, _i64, _i32p, _i32p, _f32p, _i64p, _i32p, _f64p, _i32p, _f64p]),
        "orc_laplacian_apply": (None, [_i32, _i64, _i32p, _i32p, _f32p, _int, _f64p, _f64p]),
        "orc_gaussian": (_f64, [_u64, _u64]),
        "orc_splitmix64": (_u64, [_u64]),
        "orc_init_vectors": (None, [_i32, _int, _u64, _f64p]),
        "orc_jacobi": (None, [_i32, _i64, _i32p, _i32p, _f32p, _int, _int, _f64, _f64p]),
        "orc_project": (None, [_i32, _int, _f64p]),
        "orc_smooth": (None, [_i32, _i64, _i32p, _i32p, _f32p, _int, _int, _f64, _u64, _f64p]),
        "orc_coloring": (_i32, [_i32, _i64, _i32p, _i32p, _f32p, _i32p]),
        "orc_gauss_seidel": (None, [_i32, _i64, _i32p, _i32p, _f32p, _int, _int, _f64, _f64p]),
        "orc_smooth_gs": (None, [_i32, _i64, _i32p, _i32p, _f32p, _int, _int, _f64, _u64, _f64p]),
        "orc_smooth_gs_colored": (None, [_i32, _i64, _i32p, _i32p, _f32p, _i32p, _i32, _int, _int,
                                         _f64, _u64, _f64p]),
        "orc_score_edges": (None, [_i32, _i64, _i32p, _i32p, _f32p, _f64p, _f64p, _int, _i32p,
                                   _i64, _int, _f64, _f64p]),
        "orc_topk": (None, [_f64p, _i32p, _i64, _i64, _i32p]),
        "orc_mst": (None, [_i32, _i64, _i32p, _i32p, _f32p, _u8p, _u8p]),
        "orc_components": (_i32, [_i32, _i64, _i32p, _i32p]),
        "orc_affinity": (None, [_i32, _i64, _i32p, _i32p, _f32p, _f64p, _int, _f64p]),
        "orc_aggregate": (_i32, [_i32, _i64, _i32p, _i32p, _f32p, _f64p, _i32p]),
        "orc_galerkin": (None, [_i32, _i64, _i32p, _i32p, _f32p, _i32p, _i32, _i32p, _i32p, _f32p,
                                _i64p, _i32p]),
        "orc_backward_map": (None, [_i32, _i64, _i32p, _i32p, _f32p, _i32p, _i32p, _i32, _i64,
                                    _i32p, _i32p, _f32p, _u8p, _u8p]),
        "orc_sparsify": (_int, [_i32, _i64, _i32p, _i32p, _f32p, _int, _int, _int, _f64, _u64, _int,
                                _f64, _int, _f64, _u8p]),
        "orc_sparsify_levels": (_int, [_i32, _i64, _i32p, _i32p, _f32p, _int, _int, _int, _f64, _u64,
                                       _int, _f64, _int, _f64, _u8p, _i64p, _i32p, _u8p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _p(a, t):
    return a.ctypes.data_as(t)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class Graph:
    """Canonical weighted undirected edge list (u < v, sorted, merged): edge id = position."""

    def __init__(self, n, u, v, w):
        self.n = int(n)
        self.u = _c(u, np.int32)
        self.v = _c(v, np.int32)
        self.w = _c(w, np.float32)

    @property
    def m(self):
        return int(self.u.shape[0])

    def args(self):
        return (self.n, self.m, _p(self.u, _i32p), _p(self.v, _i32p), _p(self.w, _f32p))

    def subgraph(self, mask):
        mask = np.asarray(mask).astype(bool)
        return Graph(self.n, self.u[mask], self.v[mask], self.w[mask])


def canonicalize(n, u, v, w) -> Graph:
    """Sec. 2.1 input convention: u < v, sorted, parallel edges summed in FP64, self-loops dropped."""
    u, v, w = _c(u, np.int32), _c(v, np.int32), _c(w, np.float32)
    m = u.shape[0]
    cu, cv, cw = np.empty(m, np.int32), np.empty(m, np.int32), np.empty(m, np.float32)
    mo = ctypes.c_int64(0)
    rc = lib().orc_canonicalize(int(n), m, _p(u, _i32p), _p(v, _i32p), _p(w, _f32p),
                                _p(cu, _i32p), _p(cv, _i32p), _p(cw, _f32p), ctypes.byref(mo))
    if rc != 0:
        raise ValueError("invalid edge list (id out of range or weight not finite and positive)")
    k = mo.value
    return Graph(n, cu[:k].copy(), cv[:k].copy(), cw[:k].copy())


def laplacian_csr(g: Graph):
    """CSR of L (Eq. formula_adjacency): row_ptr, col, A values (FP64), edge ids, degrees."""
    rp = np.empty(g.n + 1, np.int64)
    col = np.empty(2 * g.m, np.int32)
    val = np.empty(2 * g.m, np.float64)
    eid = np.empty(2 * g.m, np.int32)
    deg = np.empty(g.n, np.float64)
    lib().orc_laplacian(*g.args(), _p(rp, _i64p), _p(col, _i32p), _p(val, _f64p), _p(eid, _i32p),
                        _p(deg, _f64p))
    return rp, col, val, eid, deg


def laplacian_apply(g: Graph, x):
    x = _c(x, np.float64)
    K = 1 if x.ndim == 1 else x.shape[1]
    y = np.empty_like(x)
    lib().orc_laplacian_apply(*g.args(), K, _p(x, _f64p), _p(y, _f64p))
    return y


def gaussian(seed: int, j: int) -> float:
    return lib().orc_gaussian(seed & (2**64 - 1), j)


def splitmix64(x: int) -> int:
    return lib().orc_splitmix64(x & (2**64 - 1))


def init_vectors(n, K, seed):
    x = np.empty((n, K), np.float64)
    lib().orc_init_vectors(n, K, seed, _p(x, _f64p))
    return x


def jacobi(g: Graph, x, steps, omega=0.7):
    x = _c(x, np.float64).copy()
    K = 1 if x.ndim == 1 else x.shape[1]
    lib().orc_jacobi(*g.args(), K, steps, omega, _p(x, _f64p))
    return x


def project(x):
    x = _c(x, np.float64).copy()
    lib().orc_project(x.shape[0], x.shape[1], _p(x, _f64p))
    return x


def smooth(g: Graph, K, steps, omega=0.7, seed=0):
    x = np.empty((g.n, K), np.float64)
    lib().orc_smooth(*g.args(), K, steps, omega, seed, _p(x, _f64p))
    return x


def coloring(g: Graph):
    """Jones-Plassmann distance-1 colouring (priority splitmix64(0x636f6c6f72 ^ v)); returns
    (colour per node, number of colours)."""
    c = np.empty(g.n, np.int32)
    nc = lib().orc_coloring(*g.args(), _p(c, _i32p))
    return c, int(nc)


def gauss_seidel(g: Graph, x, steps, omega=1.0):
    """Gauss-Seidel sweeps on L x = 0 in colour order (Sec. 3.2), FP64."""
    x = _c(x, np.float64).copy()
    K = 1 if x.ndim == 1 else x.shape[1]
    lib().orc_gauss_seidel(*g.args(), K, steps, omega, _p(x, _f64p))
    return x


def smooth_gs(g: Graph, K, steps, omega=1.0, seed=0, coloring=None):
    """Gauss-Seidel smoothing in the order of g's own colouring, or of `coloring` = (colour per
    node, number of colours) when given (it must be proper for g)."""
    x = np.empty((g.n, K), np.float64)
    if coloring is None:
        lib().orc_smooth_gs(*g.args(), K, steps, omega, seed, _p(x, _f64p))
    else:
        c = _c(coloring[0], np.int32)
        lib().orc_smooth_gs_colored(*g.args(), _p(c, _i32p), int(coloring[1]), K, steps, omega, seed,
                                    _p(x, _f64p))
    return x


def score_edges(g: Graph, xg, xp, ids, mode=RATIO, eta=ETA):
    xg, xp = _c(xg, np.float64), _c(xp, np.float64)
    ids = _c(ids, np.int32)
    out = np.empty(ids.shape[0], np.float64)
    lib().orc_score_edges(*g.args(), _p(xg, _f64p), _p(xp, _f64p), xg.shape[1], _p(ids, _i32p),
                          ids.shape[0], mode, eta, _p(out, _f64p))
    return out


def topk(scores, ids, k):
    scores, ids = _c(scores, np.float64), _c(ids, np.int32)
    out = np.empty(k, np.int32)
    lib().orc_topk(_p(scores, _f64p), _p(ids, _i32p), ids.shape[0], k, _p(out, _i32p))
    return out


def mst(g: Graph, allow=None):
    """Maximum-weight spanning forest (Kruskal, order: weight desc, id asc) as a uint8 mask."""
    mask = np.empty(g.m, np.uint8)
    al = None if allow is None else _c(allow, np.uint8)
    lib().orc_mst(*g.args(), None if al is None else _p(al, _u8p), _p(mask, _u8p))
    return mask


def components(g: Graph) -> int:
    return lib().orc_components(g.n, g.m, _p(g.u, _i32p), _p(g.v, _i32p))


def affinity(g: Graph, x):
    x = _c(x, np.float64)
    d = np.empty(g.m, np.float64)
    lib().orc_affinity(*g.args(), _p(x, _f64p), x.shape[1], _p(d, _f64p))
    return d


def aggregate(g: Graph, delta):
    delta = _c(delta, np.float64)
    agg = np.empty(g.n, np.int32)
    nc = lib().orc_aggregate(*g.args(), _p(delta, _f64p), _p(agg, _i32p))
    return agg, int(nc)


def galerkin(g: Graph, agg, nc):
    agg = _c(agg, np.int32)
    cu, cv, cw = np.empty(g.m, np.int32), np.empty(g.m, np.int32), np.empty(g.m, np.float32)
    f2c = np.empty(g.m, np.int32)
    mo = ctypes.c_int64(0)
    lib().orc_galerkin(*g.args(), _p(agg, _i32p), nc, _p(cu, _i32p), _p(cv, _i32p), _p(cw, _f32p),
                       ctypes.byref(mo), _p(f2c, _i32p))
    k = mo.value
    return Graph(nc, cu[:k].copy(), cv[:k].copy(), cw[:k].copy()), f2c


def backward_map(g: Graph, agg, f2c, c: Graph, pmask_c):
    agg, f2c, pm = _c(agg, np.int32), _c(f2c, np.int32), _c(pmask_c, np.uint8)
    out = np.empty(g.m, np.uint8)
    lib().orc_backward_map(*g.args(), _p(agg, _i32p), _p(f2c, _i32p), c.n, c.m, _p(c.u, _i32p),
                           _p(c.v, _i32p), _p(c.w, _f32p), _p(pm, _u8p), _p(out, _u8p))
    return out


def sparsify(g: Graph, K=8, steps=10, levels=0, omega=0.7, seed=0, mode=RATIO, budget_frac=0.1,
             budget_unit=1, eta=ETA):
    """Algorithm 1: returns (mask over G's canonical edges, number of levels built)."""
    mask = np.empty(g.m, np.uint8)
    lf = lib().orc_sparsify(*g.args(), K, steps, levels, omega, seed, mode, budget_frac,
                            budget_unit, eta, _p(mask, _u8p))
    return mask, int(lf)


def sparsify_levels(g: Graph, K=8, steps=10, levels=0, omega=0.7, seed=0, mode=RATIO,
                    budget_frac=0.1, budget_unit=1, eta=ETA, hierarchy=False):
    """Algorithm 1 as `sparsify`, also returning per level l = 0..lf the row (N_l, M_l, c_l,
    edges of P_l before the level's edge recovery, edges after it). hierarchy=True adds the maps
    agg[l-1] (G_{l-1} -> G_l, l = 1..lf) and the level sparsifiers pmask[l] (over G_l's edges)."""
    mask = np.empty(g.m, np.uint8)
    stats = np.zeros((levels + 1, 5), np.int64)
    agg = np.zeros((max(levels, 1), g.n), np.int32)
    pm = np.zeros((levels + 1, max(g.m, 1)), np.uint8)
    lf = lib().orc_sparsify_levels(*g.args(), K, steps, levels, omega, seed, mode, budget_frac,
                                   budget_unit, eta, _p(mask, _u8p), _p(stats, _i64p),
                                   _p(agg, _i32p) if hierarchy else None,
                                   _p(pm, _u8p) if hierarchy else None)
    st = stats[:lf + 1]
    if not hierarchy:
        return mask, int(lf), st
    aggs = [agg[l - 1][:st[l - 1, 0]].copy() for l in range(1, lf + 1)]
    pms = [pm[l][:st[l, 1]].copy() for l in range(lf + 1)]
    return mask, int(lf), st, aggs, pms


# ------------------------------------------------------------------------------------------------
# Sec. 2.2 relative condition number (measurement, FP64 dense; tiny and small graphs only)
# ------------------------------------------------------------------------------------------------
def dense_laplacian(g: Graph, mask=None):
    L = np.zeros((g.n, g.n))
    sel = np.ones(g.m, bool) if mask is None else np.asarray(mask).astype(bool)
    for p, q, w in zip(g.u[sel], g.v[sel], g.w[sel].astype(np.float64)):
        L[p, q] -= w
        L[q, p] -= w
        L[p, p] += w
        L[q, q] += w
    return L


def kappa_dense(g: Graph, mask) -> float:
    """kappa(L_G, L_P) of Eq. eqn:ineq for P = edges of G with mask != 0, same weights.

    Both pencils share the null space spanned by the component indicators of G (when P spans G),
    so one node per component of G is grounded (its row and column removed). If P does not span
    G's components the reduced L_P is singular and kappa is infinite.
    """
    import scipy.linalg as sl

    LG = dense_laplacian(g)
    LP = dense_laplacian(g, mask)
    # ground the smallest node of each connected component of G
    parent = list(range(g.n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for p, q in zip(g.u, g.v):
        a, b = find(int(p)), find(int(q))
        if a != b:
            parent[max(a, b)] = min(a, b)
    keep = np.array([find(i) != i for i in range(g.n)])
    if keep.sum() == 0:
        return 1.0
    A = LG[np.ix_(keep, keep)]
    B = LP[np.ix_(keep, keep)]
    try:
        np.linalg.cholesky(B)
    except np.linalg.LinAlgError:
        return float("inf")
    ev = sl.eigh(A, B, eigvals_only=True)
    return float(ev[-1] / ev[0])


def _grounded_sparse(g: Graph, mask=None):
    """Sparse L_G (or L_P for mask) with one node per component of G grounded."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    sel = np.ones(g.m, bool) if mask is None else np.asarray(mask).astype(bool)
    u, v, w = g.u[sel], g.v[sel], g.w[sel].astype(np.float64)
    A = sp.coo_matrix((np.concatenate([w, w]), (np.concatenate([u, v]), np.concatenate([v, u]))),
                      shape=(g.n, g.n)).tocsr()
    L = sp.diags(np.asarray(A.sum(1)).ravel()) - A
    G = sp.coo_matrix((np.ones(g.m), (g.u, g.v)), shape=(g.n, g.n))
    _, lab = connected_components(G, directed=False)
    first = np.full(lab.max() + 1, g.n)
    np.minimum.at(first, lab, np.arange(g.n))
    keep = np.ones(g.n, bool)
    keep[first] = False
    return L.tocsc()[keep][:, keep]


def kappa_lanczos(g: Graph, mask) -> float:
    """kappa(L_G, L_P) of Eq. eqn:ineq for larger graphs: the extreme eigenvalues of the grounded
    pencil by implicitly restarted Lanczos (ARPACK through scipy, a library eigensolver), with
    sparse LU factorisations of the grounded Laplacians for the inner solves. lambda_max from the
    pencil (L_G, L_P), lambda_min as 1 / lambda_max of (L_P, L_G)."""
    from scipy.sparse.linalg import eigsh

    LG = _grounded_sparse(g)
    LP = _grounded_sparse(g, mask)
    if LG.shape[0] == 0:
        return 1.0
    hi = eigsh(LG, k=1, M=LP, which="LA", return_eigenvectors=False, tol=1e-8)[0]
    inv_lo = eigsh(LP, k=1, M=LG, which="LA", return_eigenvectors=False, tol=1e-8)[0]
    return float(hi * inv_lo)


def sparsify_to_kappa(g: Graph, kappa_target, batch_frac, max_rounds, K=8, steps=10, omega=0.7,
                      seed=0, mode=RATIO, budget_unit=0):
    """Flat sparsification to a target kappa (Sec. 2.2: kappa <= sigma^2; Sec. 3.4; Algorithm 1's
    sigma): P = maximum spanning forest; each round measures kappa (dense, exact), stops when it
    is <= kappa_target or after max_rounds rounds of additions, else embeds G and P from the same
    seed, scores the edges outside P and adds the top ones so that P holds
    round_half_up(r * batch_frac * base) edges beyond the forest after round r. Returns
    (mask, kappa trace, rounds of additions)."""
    mask = mst(g).astype(np.uint8)
    forest = int(mask.sum())
    base = g.n if budget_unit == 0 else g.m - forest
    trace = []
    r = 0
    while True:
        kap = kappa_dense(g, mask)
        trace.append(kap)
        if kap <= kappa_target or r == max_rounds:
            break
        target = int(np.floor((r + 1) * batch_frac * base + 0.5))
        k = min(target - (int(mask.sum()) - forest), g.m - int(mask.sum()))
        if k <= 0:
            break
        xg = smooth(g, K, steps, omega, seed)
        xp = smooth(g.subgraph(mask), K, steps, omega, seed)
        cand = np.nonzero(mask == 0)[0].astype(np.int32)
        sc = score_edges(g, xg, xp, cand, mode)
        mask[topk(sc, cand, k)] = 1
        r += 1
    return mask, trace, r


def sparsify_flat(g: Graph, K=8, steps=10, omega=0.7, seed=0, mode=RATIO, budget_frac=0.1,
                  budget_unit=1, smoother="jacobi"):
    """Flat Algorithm 1 (its scoring and selection steps on the spanning forest) with either smoother: P = maximum
    spanning forest; embed G and P from the same seed with weighted Jacobi or Gauss-Seidel (both in
    the order of G's colouring, which is proper for P), score the edges outside P, add the top
    round_half_up(beta * base) of them."""
    mask = mst(g).astype(np.uint8)
    forest = int(mask.sum())
    base = g.n if budget_unit == 0 else g.m - forest
    k = min(int(np.floor(budget_frac * base + 0.5)), g.m - forest)
    if k <= 0:
        return mask
    if smoother == "gs":  # P sweeps in G's colour order (proper for P, a subgraph of G)
        col = coloring(g)
        xg = smooth_gs(g, K, steps, omega, seed)
        xp = smooth_gs(g.subgraph(mask), K, steps, omega, seed, coloring=col)
    else:
        xg = smooth(g, K, steps, omega, seed)
        xp = smooth(g.subgraph(mask), K, steps, omega, seed)
    cand = np.nonzero(mask == 0)[0].astype(np.int32)
    mask[topk(score_edges(g, xg, xp, cand, mode), cand, k)] = 1
    return mask


def solve_laplacian(g: Graph, b):
    """x with L_G x = b (b first projected onto the range of L_G: its mean removed on every
    connected component) and mean zero on every component: grounded sparse direct solve (SuperLU
    through scipy, a library primitive), then the per-component mean removed."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    from scipy.sparse.linalg import spsolve

    b = np.asarray(b, np.float64).copy()
    A = sp.coo_matrix((np.ones(g.m), (g.u, g.v)), shape=(g.n, g.n))
    nc, lab = connected_components(A, directed=False)
    for c in range(nc):
        sel = lab == c
        b[sel] -= b[sel].mean()
    LG = _grounded_sparse(g)
    first = np.full(nc, g.n)
    np.minimum.at(first, lab, np.arange(g.n))
    keep = np.ones(g.n, bool)
    keep[first] = False
    x = np.zeros(g.n)
    if keep.any():
        x[keep] = spsolve(LG.tocsc(), b[keep])
    for c in range(nc):
        sel = lab == c
        x[sel] -= x[sel].mean()
    return x
