"""Seeded synthetic graph generators (inputs only; none of the method's arithmetic lives here).

The paper measures on SuiteSparse-style matrices, thermal grids and power-grid benchmarks that are
not available here (Sec. 4, Tables 2-4). These generators stand in for them with graphs of the same
shape: 2-D/3-D meshes, a power-grid mesh with via edges, 3-D k-nearest-neighbour graphs and
Chung-Lu power-law graphs. Every generator is a pure function of its arguments and a seed
(numpy PCG64), so the CUDA path, the CPU oracle and the benchmark all see identical bytes.

Each returns ``(n, u, v, w)``: int32 endpoint arrays and float32 positive weights. The lists are
not canonical (no particular order, duplicates possible where stated); canonicalisation is part of
the method under test.
"""
from __future__ import annotations

import numpy as np


def _rng(seed):
    return np.random.default_rng(np.random.PCG64(seed))


def _weights(rng, m, kind, lo=1.0, hi=10.0):
    if kind == "uniform":
        return rng.uniform(lo, hi, m).astype(np.float32)
    if kind == "logu":          # 10^U[lo, hi)
        return np.power(10.0, rng.uniform(lo, hi, m)).astype(np.float32)
    if kind == "lognormal":     # LogNormal(mu=lo, sigma=hi)
        return rng.lognormal(lo, hi, m).astype(np.float32)
    if kind == "unit":
        return np.ones(m, np.float32)
    raise ValueError(kind)


def grid2d(a, b, seed=1, weights="uniform", lo=1.0, hi=10.0):
    """a x b 4-neighbour grid, node id = i*b + j."""
    idx = np.arange(a * b, dtype=np.int64).reshape(a, b)
    u = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    v = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    rng = _rng(seed)
    return a * b, u.astype(np.int32), v.astype(np.int32), _weights(rng, u.size, weights, lo, hi)


def grid3d(s, seed=2, weights="logu", lo=-2.0, hi=2.0):
    """s^3 6-neighbour grid, node id = (i*s + j)*s + k."""
    idx = np.arange(s ** 3, dtype=np.int64).reshape(s, s, s)
    u = np.concatenate([idx[:, :, :-1].ravel(), idx[:, :-1, :].ravel(), idx[:-1, :, :].ravel()])
    v = np.concatenate([idx[:, :, 1:].ravel(), idx[:, 1:, :].ravel(), idx[1:, :, :].ravel()])
    rng = _rng(seed)
    return s ** 3, u.astype(np.int32), v.astype(np.int32), _weights(rng, u.size, weights, lo, hi)


def thermal3d(nx, ny, nz, seed=10, k_lo=-1.0, k_hi=2.0, jitter=0.1):
    """Thermal-like layered 3-D mesh (a stand-in for finite-volume thermal grids of stacked
    materials): nx x ny x nz 6-neighbour grid, node id = (z*ny + y)*nx + x. Layer z has a
    conductivity k_z = 10^U[k_lo, k_hi); a lateral edge in layer z has conductance k_z and a vertical
    edge between layers z and z+1 the series value 2 k_z k_{z+1} / (k_z + k_{z+1}); every edge is
    then scaled by U[1 - jitter, 1 + jitter)."""
    rng = _rng(seed)
    k = np.power(10.0, rng.uniform(k_lo, k_hi, nz))
    idx = np.arange(nx * ny * nz, dtype=np.int64).reshape(nz, ny, nx)
    ux, vx = idx[:, :, :-1].ravel(), idx[:, :, 1:].ravel()
    uy, vy = idx[:, :-1, :].ravel(), idx[:, 1:, :].ravel()
    uz, vz = idx[:-1, :, :].ravel(), idx[1:, :, :].ravel()
    kx = np.repeat(k, ny * (nx - 1))
    ky = np.repeat(k, (ny - 1) * nx)
    kv = 2 * k[:-1] * k[1:] / (k[:-1] + k[1:])
    kz = np.repeat(kv, ny * nx)
    u = np.concatenate([ux, uy, uz])
    v = np.concatenate([vx, vy, vz])
    w = np.concatenate([kx, ky, kz]) * rng.uniform(1 - jitter, 1 + jitter, u.size)
    return nx * ny * nz, u.astype(np.int32), v.astype(np.int32), w.astype(np.float32)


def power_grid(side, seed=3, via_frac=0.01, radius=8, sigma=1.5):
    """Circuit-like power-grid mesh: side x side 4-neighbour grid plus round(via_frac*N) "via"
    edges joining a uniform node to a node at a uniform lattice offset inside the Euclidean disk of
    the given radius (offset 0, unit grid offsets, off-grid targets and repeats excluded). All
    weights LogNormal(0, sigma)."""
    n = side * side
    idx = np.arange(n, dtype=np.int64).reshape(side, side)
    gu = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    gv = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    rng = _rng(seed)
    nvia = int(np.floor(via_frac * n + 0.5))
    offs = np.array([(dx, dy) for dx in range(-radius, radius + 1) for dy in range(-radius, radius + 1)
                     if 0 < dx * dx + dy * dy <= radius * radius and abs(dx) + abs(dy) > 1])
    have = set()
    vu, vv = [], []
    while len(vu) < nvia:
        cnt = 2 * (nvia - len(vu)) + 64
        p = rng.integers(0, n, cnt)
        o = offs[rng.integers(0, len(offs), cnt)]
        pi, pj = p // side, p % side
        qi, qj = pi + o[:, 0], pj + o[:, 1]
        ok = (qi >= 0) & (qi < side) & (qj >= 0) & (qj < side)
        for a, b in zip(p[ok], (qi * side + qj)[ok]):
            key = (min(a, b), max(a, b))
            if key in have:
                continue
            have.add(key)
            vu.append(a)
            vv.append(b)
            if len(vu) == nvia:
                break
    u = np.concatenate([gu, np.array(vu, np.int64)])
    v = np.concatenate([gv, np.array(vv, np.int64)])
    return n, u.astype(np.int32), v.astype(np.int32), _weights(rng, u.size, "lognormal", 0.0, sigma)


def knn3d(n, k=10, seed=4):
    """Symmetrised k-nearest-neighbour graph of n uniform points in [0,1)^3, Gaussian-kernel
    weights exp(-d^2 / s^2) with s the mean k-NN distance of this graph."""
    from scipy.spatial import cKDTree

    rng = _rng(seed)
    pts = rng.random((n, 3))
    d, j = cKDTree(pts).query(pts, k=k + 1)
    d, j = d[:, 1:], j[:, 1:]
    s = float(d.mean())
    u = np.repeat(np.arange(n, dtype=np.int64), k)
    v = j.ravel().astype(np.int64)
    a, b = np.minimum(u, v), np.maximum(u, v)
    key = np.unique(a * n + b)
    a, b = key // n, key % n
    dist2 = ((pts[a] - pts[b]) ** 2).sum(1)
    w = np.exp(-dist2 / (s * s)).astype(np.float32)
    w = np.maximum(w, np.float32(1e-30))
    return n, a.astype(np.int32), b.astype(np.int32), w


def batch_sizes(ng=512, lo=1e3, hi=2e5, seed=3):
    """Node counts of a batch of graphs: n_g = round(exp(U[ln lo, ln hi)))."""
    rng = _rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), ng))).astype(np.int64)


def chung_lu(n, avg_deg=16.0, gamma=2.3, seed=5, i0=1.0, lcc=True):
    """Chung-Lu power-law graph: expected degrees theta_i proportional to (i + i0)^(-1/(gamma-1)),
    scaled to the given mean and capped at sqrt(sum theta); n*avg_deg/2 endpoint pairs drawn with
    probability proportional to theta; self-loops dropped, repeats merged (first weight kept),
    weights U[0.5, 2). With lcc=True only the largest connected component is kept, relabelled in
    increasing id order."""
    rng = _rng(seed)
    theta = np.power(np.arange(n, dtype=np.float64) + i0, -1.0 / (gamma - 1.0))
    theta *= avg_deg * n / theta.sum()
    theta = np.minimum(theta, np.sqrt(theta.sum()))
    pairs = int(round(n * avg_deg / 2))
    cdf = np.cumsum(theta)
    cdf /= cdf[-1]
    u = np.searchsorted(cdf, rng.random(pairs), side="right").astype(np.int64)
    v = np.searchsorted(cdf, rng.random(pairs), side="right").astype(np.int64)
    w = rng.uniform(0.5, 2.0, pairs).astype(np.float32)
    keep = u != v
    u, v, w = u[keep], v[keep], w[keep]
    a, b = np.minimum(u, v), np.maximum(u, v)
    key, first = np.unique(a * n + b, return_index=True)
    first.sort()
    a, b, w = a[first], b[first], w[first]
    if lcc:
        import scipy.sparse as sp
        from scipy.sparse.csgraph import connected_components

        A = sp.coo_matrix((np.ones(a.size), (a, b)), shape=(n, n))
        _, lab = connected_components(A, directed=False)
        big = np.bincount(lab).argmax()
        inl = lab == big
        newid = np.cumsum(inl) - 1
        ke = inl[a]
        a, b, w = newid[a[ke]], newid[b[ke]], w[ke]
        n = int(inl.sum())
    return n, a.astype(np.int32), b.astype(np.int32), w


def hub_graph(n=6000, m=15000, seed=31, hubs=None):
    """A sparse random graph (m endpoint pairs drawn uniformly, self-loops and repeats left to the
    Laplacian) plus star hubs whose degrees are exact: by default about 2000, 700, 384 (three whole
    128-entry segments), 257 and 256, one of them the last node. The random pairs avoid the hubs
    and the star leaves are drawn from the other nodes without repetition. Weights U[1, 10)."""
    rng = _rng(seed)
    if hubs is None:
        hubs = ((7, 2000), (n * 2 // 3, 700), (n - 1, 384), (100, 257), (200, 256))
    hub_ids = [h for h, _ in hubs]
    u0, v0 = rng.integers(0, n, m), rng.integers(0, n, m)
    keep = ~(np.isin(u0, hub_ids) | np.isin(v0, hub_ids))
    u, v = [u0[keep]], [v0[keep]]
    others = np.setdiff1d(np.arange(n), hub_ids)
    for hub, d in hubs:
        u.append(np.full(d, hub))
        v.append(rng.choice(others, d, replace=False))
    u = np.concatenate(u).astype(np.int32)
    v = np.concatenate(v).astype(np.int32)
    w = rng.uniform(1.0, 10.0, u.size).astype(np.float32)
    return n, u, v, w


def path(n, weights="unit", seed=6):
    u = np.arange(n - 1)
    return n, u.astype(np.int32), (u + 1).astype(np.int32), _weights(_rng(seed), n - 1, weights)


def cycle(n, weights="unit", seed=7):
    u = np.arange(n)
    return n, u.astype(np.int32), ((u + 1) % n).astype(np.int32), _weights(_rng(seed), n, weights)


def random_graph(n, m, seed=8, weights="uniform", lo=1.0, hi=10.0, connected=True,
                 dup_frac=0.0, self_loops=0):
    """Random multigraph: a random spanning tree (if connected) plus uniform extra pairs; a
    fraction of repeated pairs and a few self-loops can be planted to exercise canonicalisation."""
    rng = _rng(seed)
    us, vs = [], []
    if connected and n > 1:
        perm = rng.permutation(n)
        for i in range(1, n):
            us.append(perm[i])
            vs.append(perm[rng.integers(0, i)])
    extra = max(0, m - len(us))
    a = rng.integers(0, n, extra)
    b = rng.integers(0, n, extra)
    ok = a != b
    us.extend(a[ok].tolist())
    vs.extend(b[ok].tolist())
    u = np.array(us, np.int64)
    v = np.array(vs, np.int64)
    if dup_frac > 0 and u.size:
        nd = int(dup_frac * u.size)
        pick = rng.integers(0, u.size, nd)
        u, v = np.concatenate([u, v[pick]]), np.concatenate([v, u[pick]])
    if self_loops:
        s = rng.integers(0, n, self_loops)
        u = np.concatenate([u, s])
        v = np.concatenate([v, s])
    order = rng.permutation(u.size)
    u, v = u[order], v[order]
    return n, u.astype(np.int32), v.astype(np.int32), _weights(rng, u.size, weights, lo, hi)


def gaussian_block(n, K, seed=9):
    """A plain seeded N x K float32 Gaussian block (for tests that pass vectors in directly)."""
    return _rng(seed).standard_normal((n, K)).astype(np.float32)
