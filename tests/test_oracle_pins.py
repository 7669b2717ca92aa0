"""Pins of the CPU oracle against facts fixed by the paper and by mathematics (no GPU).

Each test ties one oracle step to something other than itself: closed-form spectra, invariants,
identities the paper states (quadratic form Sec. 2.1, perturbation Eq. formula_eig_perturb1_conclusion,
effective resistance Eq. formula_Reff, condition number Eq. eqn:ineq), brute force on tiny graphs,
or an independent library routine. Each is chosen so that a plausible slip (dropped term, wrong
sign, wrong index, transposed operand) fails it.
"""
import itertools
import os

import numpy as np
import pytest

import oracle as O
from paper_2008_07633_gb300 import inputs as gen

HERE = os.path.dirname(os.path.abspath(__file__))


def G(n, u, v, w):
    return O.canonicalize(n, u, v, w)


def dense_from_csr(g):
    rp, col, val, eid, deg = O.laplacian_csr(g)
    L = np.zeros((g.n, g.n))
    for p in range(g.n):
        L[p, p] = deg[p]
        for j in range(rp[p], rp[p + 1]):
            L[p, col[j]] -= val[j]
    return L


# ---------------------------------------------------------------- RNG (reading of Sec. 3.2) ----
def test_splitmix64_published_vectors():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "splitmix64.txt"))
            if l.strip() and not l.startswith("#")]
    for idx, val in rows:
        n = int(idx)
        assert O.splitmix64(((n - 1) * 0x9E3779B97F4A7C15) % 2**64) == int(val, 16)


def test_gaussian_moments_and_columns_orthogonal_to_ones():
    x = O.init_vectors(20000, 8, 123)
    assert np.abs(x.sum(0)).max() < 1e-9          # orthogonal to the all-one vector (Sec. 3.2)
    z = np.array([O.gaussian(7, j) for j in range(200000)])
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.015
    assert abs((z ** 3).mean()) < 0.03 and abs((z ** 4).mean() - 3) < 0.06
    # distinct seeds and distinct counters give distinct streams
    assert O.gaussian(1, 5) != O.gaussian(2, 5) and O.gaussian(1, 5) != O.gaussian(1, 6)


# ------------------------------------------------------------ Laplacian (Sec. 2.1) --------------
def test_canonical_form_and_dense_accumulation():
    n, u, v, w = gen.random_graph(40, 160, seed=3, dup_frac=0.2, self_loops=5)
    g = G(n, u, v, w)
    assert np.all(g.u < g.v)
    key = g.u.astype(np.int64) * n + g.v
    assert np.all(np.diff(key) > 0)                    # sorted, no repeats
    # Laplacians add: the dense sum over the raw (unmerged) input equals L of the canonical list
    D = np.zeros((n, n))
    for a, b, c in zip(u, v, w.astype(np.float64)):
        if a == b:
            continue
        D[a, b] -= c; D[b, a] -= c; D[a, a] += c; D[b, b] += c
    assert np.allclose(dense_from_csr(g), D, rtol=1e-6, atol=1e-6)
    assert np.allclose(O.dense_laplacian(g), D, rtol=1e-6, atol=1e-6)


def test_canonicalize_rejects_bad_input():
    with pytest.raises(ValueError):
        O.canonicalize(3, [0, 1], [1, 3], [1.0, 1.0])
    with pytest.raises(ValueError):
        O.canonicalize(3, [0, 1], [1, 2], [1.0, 0.0])
    with pytest.raises(ValueError):
        O.canonicalize(3, [0, 1], [1, 2], [1.0, np.nan])


def test_L_ones_zero_and_quadratic_form():
    n, u, v, w = gen.random_graph(60, 300, seed=5)
    g = G(n, u, v, w)
    one = np.ones((n, 1))
    assert np.abs(O.laplacian_apply(g, one)).max() < 1e-12
    rng = np.random.default_rng(0)
    x = rng.standard_normal((n, 3))
    lx = O.laplacian_apply(g, x)
    for k in range(3):
        qf = sum(float(c) * (x[p, k] - x[q, k]) ** 2 for p, q, c in zip(g.u, g.v, g.w))
        assert abs(x[:, k] @ lx[:, k] - qf) < 1e-9 * qf


@pytest.mark.parametrize("kind", ["path", "cycle", "grid"])
def test_closed_form_spectra(kind):
    if kind == "path":
        n = 17
        g = G(*gen.path(n))
        ref = 2 - 2 * np.cos(np.pi * np.arange(n) / n)
    elif kind == "cycle":
        n = 15
        g = G(*gen.cycle(n))
        ref = 2 - 2 * np.cos(2 * np.pi * np.arange(n) / n)
    else:
        a, b = 5, 7
        g = G(*gen.grid2d(a, b, weights="unit"))
        la = 2 - 2 * np.cos(np.pi * np.arange(a) / a)
        lb = 2 - 2 * np.cos(np.pi * np.arange(b) / b)
        ref = (la[:, None] + lb[None, :]).ravel()
    ev = np.linalg.eigvalsh(dense_from_csr(g))
    assert np.allclose(np.sort(ev), np.sort(ref), atol=1e-10)


# ------------------------------------------------------- Smoothing (Sec. 3.2) ------------------
def test_jacobi_fourier_mode_closed_form_cycle():
    n, T, om = 24, 7, 0.7
    g = G(*gen.cycle(n))
    j = np.arange(n)
    for k in (1, 3, 5):
        lam = 2 - 2 * np.cos(2 * np.pi * k / n)
        x = np.stack([np.cos(2 * np.pi * k * j / n), np.sin(2 * np.pi * k * j / n)], 1)
        y = O.jacobi(g, x, T, om)
        assert np.allclose(y, (1 - om * lam / 2) ** T * x, atol=1e-12)


def test_jacobi_fourier_mode_closed_form_weighted_torus():
    # 2-D torus with weight c everywhere: D = 4c, lambda = c(4 - 2cos a - 2cos b)
    a, b, c, T, om = 6, 8, 2.5, 5, 0.7
    idx = np.arange(a * b).reshape(a, b)
    u = np.concatenate([idx.ravel(), idx.ravel()])
    v = np.concatenate([np.roll(idx, -1, 1).ravel(), np.roll(idx, -1, 0).ravel()])
    g = G(a * b, u, v, np.full(u.size, c, np.float32))
    i, jj = np.divmod(np.arange(a * b), b)
    ka, kb = 2, 3
    x = np.cos(2 * np.pi * (ka * i / a + kb * jj / b))[:, None]
    lam = c * (4 - 2 * np.cos(2 * np.pi * ka / a) - 2 * np.cos(2 * np.pi * kb / b))
    y = O.jacobi(g, x, T, om)
    assert np.allclose(y, (1 - om * lam / (4 * c)) ** T * x, atol=1e-12)


def test_jacobi_invariants():
    n, u, v, w = gen.random_graph(50, 200, seed=9)
    g = G(n, u, v, w)
    _, _, _, _, deg = O.laplacian_csr(g)
    rng = np.random.default_rng(1)
    x1, x2 = rng.standard_normal((n, 4)), rng.standard_normal((n, 4))
    y1, y2 = O.jacobi(g, x1, 6), O.jacobi(g, x2, 6)
    assert np.allclose(deg @ y1, deg @ x1, rtol=1e-10)          # D-weighted mean kept
    assert np.allclose(O.jacobi(g, 2 * x1 - 3 * x2, 6), 2 * y1 - 3 * y2, atol=1e-10)  # linear
    c = np.ones((n, 1)) * 3.0
    assert np.allclose(O.jacobi(g, c, 6), c)                     # constants are fixed points


def test_jacobi_zero_degree_node_unchanged():
    g = G(5, [0, 1], [1, 2], [1.0, 2.0])            # nodes 3, 4 isolated
    x = np.arange(10, dtype=np.float64).reshape(5, 2)
    y = O.jacobi(g, x, 4)
    assert np.array_equal(y[3:], x[3:])


def test_project_and_smooth_is_low_pass():
    g = G(*gen.grid2d(16, 16, seed=4))
    x = O.smooth(g, 8, 10, 0.7, seed=11)
    assert np.abs(x.mean(0)).max() < 1e-12
    assert np.allclose(np.sqrt((x ** 2).mean(0)), 1.0)
    # Rayleigh quotients drop far below those of the raw random vectors
    r0 = O.init_vectors(g.n, 8, 11)
    rq = lambda z: np.diag(z.T @ O.laplacian_apply(g, z)) / np.diag(z.T @ z)
    assert np.all(rq(x) < 0.1 * rq(r0))


# ------------------------------------------------ Scores (Sec. 3.5) ----------------------------
def _eig_embedding(g):
    L = O.dense_laplacian(g)
    lam, U = np.linalg.eigh(L)
    return L, lam, U


def test_score_with_effective_resistance_embedding():
    # Eq. formula_Reff: with X = U_eff = [u_i / sqrt(lambda_i)], ||X^T e_pq||^2 = R_eff(p, q)
    n, u, v, w = gen.random_graph(20, 60, seed=13)
    g = G(n, u, v, w)
    L, lam, U = _eig_embedding(g)
    Ueff = U[:, 1:] / np.sqrt(lam[1:])
    ids = np.arange(g.m, dtype=np.int32)
    s = O.score_edges(g, Ueff, Ueff, ids, mode=O.G_ONLY)
    Lp = np.linalg.pinv(L)
    reff = np.array([Lp[p, p] + Lp[q, q] - 2 * Lp[p, q] for p, q in zip(g.u, g.v)])
    assert np.allclose(s, g.w * reff, rtol=1e-9)
    assert abs(s.sum() - (n - 1)) < 1e-9                         # Foster's theorem


def test_score_on_tree_is_path_resistance():
    n, u, v, w = gen.random_graph(12, 11, seed=17)               # a random spanning tree
    g = G(n, u, v, w)
    L, lam, U = _eig_embedding(g)
    Ueff = U[:, 1:] / np.sqrt(lam[1:])
    import networkx as nx
    T = nx.Graph()
    for p, q, c in zip(g.u, g.v, g.w):
        T.add_edge(int(p), int(q), r=1.0 / float(c))
    pairs = np.array([(0, 5), (3, 11), (7, 2)], np.int32)
    for p, q in pairs:
        r = nx.shortest_path_length(T, int(p), int(q), weight="r")
        d = ((Ueff[p] - Ueff[q]) ** 2).sum()
        assert abs(d - r) < 1e-9 * r


def test_score_first_order_eigen_perturbation():
    # Eq. formula_eig_perturb1_conclusion: d lambda_i / dt of L_P + t w e e^T at t = 0 is w (u_i^T e)^2
    n, u, v, w = gen.random_graph(10, 9, seed=19, lo=1.0, hi=3.0)
    gp = G(n, u, v, w)
    Lp, lam, U = _eig_embedding(gp)
    p, q, wt = 2, 7, 1.7
    e = np.zeros(n); e[p], e[q] = 1, -1
    K = 4
    # the score in P_ONLY mode with X = the first K nontrivial eigenvectors is Delta_K (Eq. ...conclusion2)
    gq = G(n, np.array([p]), np.array([q]), np.array([wt], np.float32))
    s = O.score_edges(gq, U[:, 1:K + 1], U[:, 1:K + 1], np.array([0], np.int32), mode=O.P_ONLY)[0]
    h = 1e-6
    lam_h = np.linalg.eigvalsh(Lp + h * wt * np.outer(e, e))
    fd = ((lam_h - lam) / h)[1:K + 1].sum()
    assert abs(s - fd) < 1e-4 * abs(fd)


def test_score_modes_and_ratio():
    n, u, v, w = gen.random_graph(30, 90, seed=21)
    g = G(n, u, v, w)
    rng = np.random.default_rng(3)
    xg, xp = rng.standard_normal((n, 5)), rng.standard_normal((n, 5))
    ids = np.arange(g.m, dtype=np.int32)[::3]
    sg = O.score_edges(g, xg, xp, ids, O.G_ONLY)
    sp = O.score_edges(g, xg, xp, ids, O.P_ONLY)
    r = O.score_edges(g, xg, xp, ids, O.RATIO)
    assert np.allclose(r, sp / (sg + O.ETA))
    assert np.allclose(O.score_edges(g, xp, xg, ids, O.G_ONLY), sp)   # blocks not swapped
    # translation invariance of distances
    assert np.allclose(O.score_edges(g, xg + 5.0, xp, ids, O.G_ONLY), sg)


# ------------------------------------------------ Selection (Algorithm 1) ----------------------
def test_topk_brute_force_and_ties():
    rng = np.random.default_rng(4)
    s = rng.integers(0, 20, 300).astype(np.float64)       # many ties
    ids = rng.permutation(1000)[:300].astype(np.int32)
    for k in (0, 1, 17, 150, 300):
        out = O.topk(s, ids, k)
        order = sorted(range(300), key=lambda i: (-s[i], ids[i]))[:k]
        assert np.array_equal(out, np.sort(ids[order]))
    same = np.ones(50)
    ids2 = np.arange(50, dtype=np.int32)[::-1].copy()
    assert np.array_equal(O.topk(same, ids2, 7), np.arange(7))


# ------------------------------------------------ Spanning tree (Sec. 3.4) ---------------------
def _spanning_trees(n, edges):
    for sub in itertools.combinations(range(len(edges)), n - 1):
        par = list(range(n))

        def f(a):
            while par[a] != a:
                a = par[a]
            return a
        ok = True
        for e in sub:
            a, b = f(edges[e][0]), f(edges[e][1])
            if a == b:
                ok = False
                break
            par[a] = b
        if ok:
            yield sub


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_mst_brute_force_small(seed):
    n = 7
    _, u, v, w = gen.random_graph(n, 12, seed=seed)
    rng = np.random.default_rng(seed)
    if seed % 2:                                  # integer weights: ties broken by edge id
        w = rng.integers(1, 4, u.size).astype(np.float32)
    g = G(n, u, v, w)
    edges = list(zip(g.u.tolist(), g.v.tolist()))
    trees = list(_spanning_trees(n, edges))
    # Kirchhoff: number of spanning trees = any cofactor of L
    L = O.dense_laplacian(G(n, g.u, g.v, np.ones(g.m, np.float32)))
    assert len(trees) == round(np.linalg.det(L[1:, 1:]))
    # the unique maximum under (weight desc, id asc): lexicographically best sorted key list
    def key(t):
        return sorted(((-float(g.w[e]), e) for e in t))
    best = min(trees, key=key)
    mask = O.mst(g)
    assert sorted(np.nonzero(mask)[0].tolist()) == sorted(best)


def test_mst_vs_scipy_and_tree_returns_itself():
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import minimum_spanning_tree
    n, u, v, w = gen.random_graph(200, 900, seed=23)
    g = G(n, u, v, w)
    assert len(np.unique(g.w)) == g.m                   # distinct weights: MST unique
    M = coo_matrix((-g.w.astype(np.float64), (g.u, g.v)), shape=(n, n)).tocsr()
    T = minimum_spanning_tree(M).tocoo()
    ref = set(zip(np.minimum(T.row, T.col).tolist(), np.maximum(T.row, T.col).tolist()))
    mask = O.mst(g)
    got = set(zip(g.u[mask == 1].tolist(), g.v[mask == 1].tolist()))
    assert got == ref
    tg = g.subgraph(mask)
    assert np.all(O.mst(tg) == 1)


# ------------------------------------------------ Condition number (Sec. 2.2) ------------------
def test_kappa_pins():
    n = 9
    g = G(*gen.cycle(n))
    assert abs(O.kappa_dense(g, np.ones(g.m)) - 1.0) < 1e-10
    mask = np.ones(g.m, np.uint8)
    mask[3] = 0
    assert abs(O.kappa_dense(g, mask) - n) < 1e-9       # unit cycle minus one edge
    n2, u, v, w = gen.random_graph(25, 70, seed=29)
    g2 = G(n2, u, v, w)
    t = O.mst(g2)
    extra = np.nonzero(t == 0)[0]
    m2 = np.ones(g2.m, np.uint8)
    e = extra[0]
    m2[e] = 0                                            # single removed edge: rank one
    Lp = O.dense_laplacian(g2, m2)
    pinv = np.linalg.pinv(Lp)
    p, q = g2.u[e], g2.v[e]
    r = pinv[p, p] + pinv[q, q] - 2 * pinv[p, q]
    assert abs(O.kappa_dense(g2, m2) - (1 + float(g2.w[e]) * r)) < 1e-8 * (1 + g2.w[e] * r)
    broken = t.copy()
    broken[np.nonzero(t)[0][0]] = 0
    assert O.kappa_dense(g2, broken) == float("inf")


# ------------------------------------------------ Coarsening (Sec. 3.2) ------------------------
def test_affinity_properties():
    g = G(5, [0, 1, 2, 3], [1, 2, 3, 4], [1.0] * 4)
    x = np.array([[1.0, 2.0], [2.0, 4.0], [-4.0, 2.0], [0.3, -0.1], [3.0, -1.0]])
    d = O.affinity(g, x)
    assert abs(d[0]) < 1e-15                 # parallel rows
    assert abs(d[1] - 1.0) < 1e-15           # orthogonal rows
    assert abs(d[3]) < 1e-15                 # anti-parallel rows (squared inner product)
    c = (x[2] @ x[3]) ** 2 / ((x[2] @ x[2]) * (x[3] @ x[3]))
    assert abs(d[2] - (1 - c)) < 1e-15
    assert np.allclose(O.affinity(g, x * np.array([[2.0], [1], [3], [0.5], [7]])), d)
    rng = np.random.default_rng(0)
    assert np.allclose(O.affinity(g, rng.standard_normal((5, 1))), 0.0)   # K = 1


def test_aggregation_brute_force():
    import networkx as nx
    n, u, v, w = gen.random_graph(40, 100, seed=31)
    g = G(n, u, v, w)
    rng = np.random.default_rng(5)
    delta = rng.random(g.m)
    agg, nc = O.aggregate(g, delta)
    H = nx.Graph()
    H.add_nodes_from(range(n))
    for p in range(n):
        nb = [(delta[e], int(g.v[e] if g.u[e] == p else g.u[e])) for e in range(g.m)
              if g.u[e] == p or g.v[e] == p]
        if nb:
            H.add_edge(p, min(nb)[1])
    comps = sorted((sorted(c) for c in nx.connected_components(H)), key=lambda c: c[0])
    assert nc == len(comps)
    for i, c in enumerate(comps):
        assert np.all(agg[c] == i)
    Gx = nx.Graph(list(zip(g.u.tolist(), g.v.tolist())))
    for c in comps:                            # every aggregation set is connected in G
        assert nx.is_connected(Gx.subgraph(c))


def test_galerkin_identities():
    n, u, v, w = gen.random_graph(60, 200, seed=37)
    g = G(n, u, v, w)
    rng = np.random.default_rng(6)
    agg, nc = O.aggregate(g, rng.random(g.m))
    c, f2c = O.galerkin(g, agg, nc)
    Lc = O.dense_laplacian(c)
    assert np.abs(Lc.sum(1)).max() < 1e-9
    Hp = np.zeros((n, nc))
    Hp[np.arange(n), agg] = 1.0                 # H^+ of Sec. 3.2
    y = rng.standard_normal(nc)
    L = O.dense_laplacian(g)
    # coarse weights are rounded once to float32, so the identity holds to float32 precision
    assert abs((Hp @ y) @ L @ (Hp @ y) - y @ Lc @ y) < 1e-6 * abs(y @ Lc @ y)
    inter = agg[g.u] != agg[g.v]
    assert abs(g.w[inter].astype(np.float64).sum() - c.w.astype(np.float64).sum()) < 1e-3
    assert np.all((f2c >= 0) == inter)
    a, b = agg[g.u[inter]], agg[g.v[inter]]
    assert np.array_equal(np.minimum(a, b), c.u[f2c[inter]])
    assert np.array_equal(np.maximum(a, b), c.v[f2c[inter]])


def test_backward_map_tree_to_tree():
    n, u, v, w = gen.random_graph(80, 260, seed=41)
    g = G(n, u, v, w)
    x = O.smooth(g, 6, 5, seed=3)
    agg, nc = O.aggregate(g, O.affinity(g, x))
    c, f2c = O.galerkin(g, agg, nc)
    pc = O.mst(c)
    pf = O.backward_map(g, agg, f2c, c, pc)
    assert int(pf.sum()) == n - 1
    assert O.kappa_dense(g, pf) < float("inf")          # spans G


def _strict_before(g, a, b):
    """Edge a precedes edge b in the strict order of the spanning-forest reading (weight
    descending, then edge id ascending)."""
    return g.w[a] > g.w[b] or (g.w[a] == g.w[b] and a < b)


def _connected_by(n, edges, g, s, t):
    adj = {}
    for e in edges:
        adj.setdefault(int(g.u[e]), []).append(int(g.v[e]))
        adj.setdefault(int(g.v[e]), []).append(int(g.u[e]))
    seen, stack = {s}, [s]
    while stack:
        a = stack.pop()
        for b in adj.get(a, ()):
            if b not in seen:
                seen.add(b)
                stack.append(b)
    return t in seen


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_backward_map_choices_by_brute_force(seed):
    """Sec. 3.4 backward mapping, checked edge by edge on small graphs with many weight ties and
    arbitrary aggregation sets (not only connected ones):
    - inter-cluster: for each selected coarse edge (I, J), exactly the fine edge between S_I and S_J
      of largest weight, ties to the smallest id, found by scanning every fine edge;
    - inner-cluster: an edge inside an aggregate is kept iff its endpoints are not already joined
      inside that aggregate by edges that come before it in the strict order (the cycle property,
      which characterises the unique maximum spanning forest of each induced subgraph)."""
    rng = np.random.default_rng(seed)
    n = 40
    u = rng.integers(0, n, 160).astype(np.int32)
    v = rng.integers(0, n, 160).astype(np.int32)
    w = rng.integers(1, 4, 160).astype(np.float32)          # weights 1..3: many ties
    g = G(n, u, v, w)
    agg = rng.integers(0, 7, n).astype(np.int32)
    nc = int(agg.max()) + 1
    c, f2c = O.galerkin(g, agg, nc)
    pc = (rng.random(c.m) < 0.6).astype(np.uint8)
    pf = O.backward_map(g, agg, f2c, c, pc)
    for ce in range(c.m):
        I, J = int(c.u[ce]), int(c.v[ce])
        between = [e for e in range(g.m)
                   if {int(agg[g.u[e]]), int(agg[g.v[e]])} == {I, J}]
        best = between[0]
        for e in between[1:]:
            if g.w[e] > g.w[best]:
                best = e
        chosen = [e for e in between if pf[e]]
        assert chosen == ([best] if pc[ce] else []), (ce, chosen, best)
    for e in range(g.m):
        a = int(agg[g.u[e]])
        if a != int(agg[g.v[e]]):
            continue
        earlier = [f for f in range(g.m) if f != e and int(agg[g.u[f]]) == a
                   and int(agg[g.v[f]]) == a and _strict_before(g, f, e)]
        keep = not _connected_by(n, earlier, g, int(g.u[e]), int(g.v[e]))
        assert bool(pf[e]) == keep, e


@pytest.mark.parametrize("levels,unit,beta", [(1, 0, 0.05), (2, 0, 0.05), (2, 1, 0.08),
                                              (3, 0, 0.12)])
def test_multilevel_budget_per_level(levels, unit, beta):
    """Reading c13 of the per-level budget (the paper gives no split; only its figures mention
    per-level edge counts): at every level l the sparsifier ends with round_half_up(beta * base_l)
    edges beyond a spanning forest of G_l (N_l - c_l edges), base_l = N_l (unit 0) or the number of
    off-forest edges of G_l (unit 1); edges mapped back from the coarser level count, and nothing
    is added once they are already over. Every level's component count equals G's (aggregates are
    connected), checked against a union-find count of G itself."""
    g = G(*gen.grid2d(24, 24, seed=3, weights="logu", lo=-2, hi=2))
    comps = O.components(g)
    mask, lf, st = O.sparsify_levels(g, K=8, steps=10, levels=levels, seed=11, budget_frac=beta,
                                     budget_unit=unit)
    assert lf == levels and st.shape == (levels + 1, 5)
    assert st[0, 0] == g.n and st[0, 1] == g.m and int(mask.sum()) == st[0, 4]
    assert np.all(np.diff(st[:, 0]) < 0)                   # every level is coarser
    for l in range(lf + 1):
        nl, ml, cl, before, after = (int(x) for x in st[l])
        assert cl == comps
        forest = nl - cl
        base = nl if unit == 0 else ml - forest
        target = int(np.floor(beta * base + 0.5))
        assert before >= forest
        assert after == min(ml, max(before, forest + target)), (l, st[l], target)
    # the coarsest level starts from its spanning forest alone
    assert st[lf, 3] == st[lf, 0] - st[lf, 2]


# ------------------------------------------------ Algorithm 1 ----------------------------------
def test_sparsify_flat_properties():
    g = G(*gen.grid2d(32, 32, seed=1))
    tree = O.mst(g)
    mask, lf = O.sparsify(g, K=8, steps=10, levels=0, budget_frac=0.1, budget_unit=1, seed=5)
    assert lf == 0
    assert np.all(mask[tree == 1] == 1)
    off = g.m - (g.n - 1)
    assert int(mask.sum()) == g.n - 1 + int(np.floor(0.1 * off + 0.5))
    t = G(*gen.path(20, weights="uniform"))
    tm, _ = O.sparsify(t, K=4, steps=5)
    assert np.all(tm == 1)


def test_sparsify_flat_cuts_kappa_against_the_tree():
    # Sec. 3.5 / Table 2: the recovered off-tree edges bring kappa(L_G, L_P) far below the
    # spanning tree's. 48 x 48 grid, 10% of the off-tree edges: the tree's kappa is 3,257 and
    # the sparsifier's 111-172 over three seeds of the random vectors (0.034-0.053 of the tree's),
    # against the bar of 0.1. (On a 32 x 32 grid the ratio is 0.09-0.12 across seeds: the tree's
    # kappa grows faster with the graph than the sparsifier's, so the bar sits on the larger grid.)
    g = G(*gen.grid2d(48, 48, seed=1))
    tree = O.mst(g)
    kt = O.kappa_dense(g, tree)
    for s in (1, 5):
        mask, _ = O.sparsify(g, K=8, steps=10, levels=0, budget_frac=0.1, budget_unit=1, seed=s)
        assert O.kappa_dense(g, mask) < 0.1 * kt


def test_sparsify_beats_random_choice():
    # 64 x 64 grid, 10% of the off-tree edges: the spectral choice (averaged over two seeds of the
    # random vectors) beats random choices of the same number of off-tree edges (three draws).
    # On much smaller grids the spread over the random vectors hides the difference.
    g = G(*gen.grid2d(64, 64, seed=1))
    tree = O.mst(g)
    ks = [O.kappa_dense(g, O.sparsify(g, K=8, steps=10, levels=0, budget_frac=0.1,
                                      budget_unit=1, seed=s)[0]) for s in (1, 2)]
    rng = np.random.default_rng(0)
    off = np.nonzero(tree == 0)[0]
    kr = []
    for _ in range(3):
        rnd = tree.copy()
        rnd[rng.choice(off, int(np.floor(0.1 * off.size + 0.5)), replace=False)] = 1
        kr.append(O.kappa_dense(g, rnd))
    assert np.mean(ks) < 0.8 * np.mean(kr), (ks, kr)


def test_sparsify_multilevel_properties():
    g = G(*gen.grid2d(14, 14, seed=2))
    mask, lf = O.sparsify(g, K=8, steps=10, levels=2, budget_frac=0.05, budget_unit=0, seed=7)
    assert lf == 2
    k = O.kappa_dense(g, mask)
    assert np.isfinite(k)
    target = int(np.floor(0.05 * g.n + 0.5))
    assert int(mask.sum()) >= g.n - 1 + target


def test_kappa_lanczos_matches_dense():
    for spec in (gen.grid2d(20, 25, seed=3), gen.random_graph(400, 1500, seed=4),
                 gen.random_graph(300, 500, seed=6, connected=False)):
        g = G(*spec)
        tree = O.mst(g)
        mask, _ = O.sparsify(g, K=8, steps=10, budget_frac=0.1, budget_unit=1, seed=2)
        for mk in (tree, mask):
            kd, kl = O.kappa_dense(g, mk), O.kappa_lanczos(g, mk)
            assert abs(kd - kl) <= 1e-5 * kd, (kd, kl)


def test_lambda_min_is_one_when_dropped_edges_leave_extra_components():
    """L_G = L_P + L_Q >= L_P (Q = G minus P), and any vector constant on the components of Q but
    not on those of G has L_G x = L_P x != 0: lambda_min(L_G, L_P) = 1 exactly when Q has more
    components than G, and > 1 otherwise (checked on a cycle, where Q is a single edge and
    connects nothing)."""
    import scipy.linalg as sl
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components

    def ncomp(n, u, v):
        return connected_components(coo_matrix((np.ones(len(u)), (u, v)), shape=(n, n)),
                                    directed=False)[0]

    def lam_min(g, mask):
        LG, LP = O.dense_laplacian(g), O.dense_laplacian(g, mask)
        keep = np.arange(g.n) != 0  # connected graphs here: ground node 0
        return sl.eigh(LG[np.ix_(keep, keep)], LP[np.ix_(keep, keep)], eigvals_only=True)[0]

    seen_exact = 0
    for spec in (gen.grid2d(12, 14, seed=1), gen.random_graph(120, 400, seed=2), gen.knn3d(150, k=6, seed=3)):
        g = G(*spec)
        assert ncomp(g.n, g.u, g.v) == 1
        for mask in (O.mst(g), O.sparsify(g, K=8, steps=10, budget_frac=0.2, budget_unit=1, seed=4)[0]):
            q = ~mask.astype(bool)
            extra = ncomp(g.n, g.u[q], g.v[q]) > 1
            lm = lam_min(g, mask)
            if extra:
                assert abs(lm - 1.0) <= 1e-9
                seen_exact += 1
            else:
                assert lm > 1.0 + 1e-9
    assert seen_exact > 0
    n = 9  # cycle minus one edge: Q is one edge, Q has n - 1 components > 1, lambda_min = 1
    g = G(n, np.arange(n), (np.arange(n) + 1) % n, np.ones(n))
    mask = np.ones(g.m, np.uint8)
    mask[0] = 0
    assert abs(lam_min(g, mask) - 1.0) <= 1e-9
    # complete graph K5 with P = the star at node 0: Q is K4 on the other nodes, node 0 is left
    # alone in Q, so lambda_min = 1
    n = 5
    u, v = np.triu_indices(n, 1)
    g = G(n, u, v, np.ones(len(u)))
    star = ((g.u == 0) | (g.v == 0)).astype(np.uint8)
    q = ~star.astype(bool)
    assert ncomp(n, g.u[q], g.v[q]) == 2  # node 0 is isolated in Q
    assert abs(lam_min(g, star) - 1.0) <= 1e-9


def test_sparsify_to_kappa_loop_invariants():
    """The kappa-target loop (Sec. 2.2, Sec. 3.4): each round adds exactly the scheduled edges,
    lambda_max(L_G, L_P) never increases as edges join P (L_P' >= L_P), and the loop stops at the
    first kappa <= target."""
    import scipy.linalg as sl

    g = G(*gen.grid2d(24, 24, seed=5))
    tree = O.mst(g)
    k0 = O.kappa_dense(g, tree)
    target = k0 / 3.0
    mask, trace, rounds = O.sparsify_to_kappa(g, target, batch_frac=0.02, max_rounds=12, K=8,
                                              steps=10, seed=3)
    assert trace[0] == k0 and len(trace) == rounds + 1
    assert trace[-1] <= target and all(k > target for k in trace[:-1])
    forest = int(tree.sum())
    assert int(mask.sum()) - forest == int(np.floor(rounds * 0.02 * g.n + 0.5))
    assert np.all(mask[tree.astype(bool)] == 1)

    def lam_max(m):
        LG, LP = O.dense_laplacian(g), O.dense_laplacian(g, m)
        keep = np.arange(g.n) != 0
        return sl.eigh(LG[np.ix_(keep, keep)], LP[np.ix_(keep, keep)], eigvals_only=True)[-1]

    # replay the rounds: lambda_max is non-increasing along the sequence of sparsifiers
    prev = lam_max(tree)
    m = tree.astype(np.uint8).copy()
    for r in range(1, rounds + 1):
        mr, _, _ = O.sparsify_to_kappa(g, 1.0, batch_frac=0.02, max_rounds=r, K=8, steps=10, seed=3)
        assert np.all(mr[m.astype(bool)] == 1)  # rounds only add edges
        cur = lam_max(mr)
        assert cur <= prev * (1 + 1e-9)
        prev, m = cur, mr


def test_coloring_is_proper_and_grundy():
    for spec in (gen.grid2d(15, 17, seed=1), gen.knn3d(300, k=8, seed=2), gen.chung_lu(800, seed=3)):
        g = G(*spec)
        c, nc = O.coloring(g)
        assert c.min() == 0 and c.max() == nc - 1 and np.all(c[g.u] != c[g.v])
        c2, _ = O.coloring(g)
        assert np.array_equal(c, c2)
        nb = [set() for _ in range(g.n)]
        for a, b in zip(g.u, g.v):
            nb[a].add(int(c[b]))
            nb[b].add(int(c[a]))
        for v in range(g.n):  # every smaller colour is taken by some neighbour
            assert set(range(c[v])) <= nb[v]


def test_gauss_seidel_is_the_matrix_splitting():
    """One sweep in colour order, x <- (D - omega A_L)^-1 ((1 - omega) D + omega A_U) x, with
    A_L / A_U the parts of A below / above the diagonal in the (colour, id) node order; constants
    are fixed points; the energy x^T L x never increases for 0 < omega < 2."""
    g = G(*gen.random_graph(60, 200, seed=4))
    c, _ = O.coloring(g)
    order = np.lexsort((np.arange(g.n), c))
    pos = np.empty(g.n, int)
    pos[order] = np.arange(g.n)
    L = O.dense_laplacian(g)
    A = np.diag(np.diag(L)) - L
    D = np.diag(np.diag(L))
    P = np.eye(g.n)[order]                      # row i of P x = x[order[i]]
    Ao = P @ A @ P.T
    AL, AU, Do = np.tril(Ao, -1), np.triu(Ao, 1), P @ D @ P.T
    rng = np.random.default_rng(0)
    x = rng.standard_normal((g.n, 3))
    for om in (1.0, 0.7, 1.4):
        ref = P.T @ np.linalg.solve(Do - om * AL, ((1 - om) * Do + om * AU) @ (P @ x))
        got = O.gauss_seidel(g, x, 1, om)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
        e = [np.einsum("ik,ij,jk->k", x, L, x)]
        y = x
        for _ in range(4):
            y = O.gauss_seidel(g, y, 1, om)
            e.append(np.einsum("ik,ij,jk->k", y, L, y))
        assert np.all(np.diff(np.array(e), axis=0) <= 1e-9 * e[0])
    ones = np.ones((g.n, 2)) * 3.5
    assert np.allclose(O.gauss_seidel(g, ones, 3, 1.0), ones, rtol=0, atol=1e-13)


def test_gauss_seidel_conserves_the_ordered_weighted_sum():
    """A colour-ordered SOR sweep keeps y^T x with y_p = d_p - omega * (weight to nodes after p in
    (colour, id) order): y^T = 1^T (D - omega A_L) is the left fixed vector of the sweep matrix.
    (This is why the GPU removes the y-weighted mean before Gauss-Seidel sweeps.)"""
    g = G(*gen.chung_lu(600, seed=7))
    c, _ = O.coloring(g)
    rank = np.lexsort((np.arange(g.n), c))
    pos = np.empty(g.n, int)
    pos[rank] = np.arange(g.n)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((g.n, 4))
    for om in (1.0, 0.7, 1.4):
        y = np.zeros(g.n)
        for a, b, w in zip(g.u, g.v, g.w.astype(np.float64)):
            y[a] += w
            y[b] += w
            earlier = a if pos[a] < pos[b] else b  # its edge to the other endpoint goes later
            y[earlier] -= om * w
        before = y @ x
        after = y @ O.gauss_seidel(g, x, 3, om)
        assert np.allclose(after, before, rtol=1e-10, atol=1e-10 * np.abs(x).sum())


def test_solve_laplacian_closed_forms():
    """Unit path: L x = e_0 - e_{n-1} is solved by a ramp with slope -1 (flow 1 through unit
    resistors); weighted path: the drop across edge i is 1 / w_i; any b: L x = b - mean(b) on each
    component, x has mean zero on each component."""
    n = 9
    g = G(n, np.arange(n - 1), np.arange(1, n), np.ones(n - 1))
    b = np.zeros(n)
    b[0], b[-1] = 1.0, -1.0
    x = O.solve_laplacian(g, b)
    assert np.allclose(np.diff(x), -1.0, atol=1e-12) and abs(x.mean()) < 1e-12
    w = np.linspace(0.5, 4.0, n - 1)
    g = G(n, np.arange(n - 1), np.arange(1, n), w)
    x = O.solve_laplacian(g, b)
    assert np.allclose(-np.diff(x), 1.0 / g.w.astype(np.float64), rtol=1e-10)
    g = G(*gen.random_graph(200, 320, seed=9, connected=False))
    rng = np.random.default_rng(2)
    b = rng.standard_normal(g.n)
    x = O.solve_laplacian(g, b)
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    _, lab = connected_components(coo_matrix((np.ones(g.m), (g.u, g.v)), shape=(g.n, g.n)), directed=False)
    bp = b.copy()
    for c in np.unique(lab):
        bp[lab == c] -= bp[lab == c].mean()
        assert abs(x[lab == c].mean()) < 1e-12
    assert np.abs(O.laplacian_apply(g, x) - bp).max() < 1e-9 * np.abs(bp).max()
