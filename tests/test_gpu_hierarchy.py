"""The coarsening hierarchy that sfg_sparsify returns (Algorithm 1's [G_1 .. G_lf; H_1 .. H_lf]
with every level's sparsifier P_l), against the oracle's own multilevel run.

The aggregation of each level is an argmin over the neighbours' algebraic distances, computed by
the GPU from FP32 embeddings and by the oracle from FP64 ones. On the graphs below every such
argmin is decided by a relative margin of at least 1e-3 in the oracle's own distances (checked
first, from oracle data only), far above what FP32 rounding can move, so the maps H_l and the
coarse graphs G_l must agree bit for bit. The level sparsifiers must have the same sizes; their
recovered edges come from a top-k over FP32 scores and are compared by overlap.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2008_07633_gb300 import inputs as gen

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def S():
    import paper_2008_07633_gb300.sfg as S

    S.lib()
    return S


@pytest.fixture(scope="module")
def ctx(S):
    c = S.sfg_ctx_create(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _level_seed(seed, level):
    return seed if level == 0 else O.splitmix64(seed ^ level)


def _min_relative_gap(og, x):
    """Smallest relative gap between the best and second-best delta over all nodes."""
    d = O.affinity(og, x)
    rp, _, _, eid, _ = O.laplacian_csr(og)
    gap = np.inf
    for p in range(og.n):
        ds = np.sort(d[eid[rp[p]:rp[p + 1]]])
        if ds.size >= 2:
            gap = min(gap, (ds[1] - ds[0]) / max(ds[1], 1e-300))
    return gap


CASES = [
    ("grid48_logu", lambda: gen.grid2d(48, 48, seed=4, weights="logu", lo=-2, hi=2), 2),
    ("grid24_logu", lambda: gen.grid2d(24, 24, seed=3, weights="logu", lo=-2, hi=2), 3),
    ("thermal", lambda: gen.thermal3d(12, 12, 6, seed=11), 2),
    ("grid3d12_logu", lambda: gen.grid3d(12, seed=5), 2),
]


@pytest.mark.parametrize("name,spec,levels", CASES, ids=[c[0] for c in CASES])
def test_hierarchy_matches_oracle(S, ctx, name, spec, levels):
    K, T, seed, beta = 8, 10, 17, 0.05
    n, u, v, w = spec()
    g = S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w))
    og = O.canonicalize(n, u, v, w)
    om, lf, st, aggs, pms = O.sparsify_levels(og, K=K, steps=T, levels=levels, seed=seed,
                                              budget_frac=beta, budget_unit=0, hierarchy=True)
    # oracle-side precondition: every aggregation decision has a margin of at least 1e-3
    levels_og = [og]
    for l in range(1, lf + 1):
        x = O.smooth(levels_og[-1], K, T, 0.7, _level_seed(seed, l - 1))
        assert _min_relative_gap(levels_og[-1], x) > 1e-3
        c, _ = O.galerkin(levels_og[-1], aggs[l - 1], int(aggs[l - 1].max()) + 1)
        levels_og.append(c)
    mask, nsel, H = S.sfg_sparsify(ctx, g, K=K, steps=T, levels=levels, seed=seed,
                                   budget_frac=beta, budget_unit=0, hierarchy=True)
    assert H.levels == lf == levels
    assert np.array_equal(host(H.mask(0)), host(mask))
    for l in range(1, lf + 1):
        agg, f2c = H.map(l)
        assert np.array_equal(host(agg), aggs[l - 1]), l
        oc, of2c = O.galerkin(levels_og[l - 1], aggs[l - 1], levels_og[l].n)
        gl = H.graph(l)
        assert (gl.n, gl.m) == (oc.n, oc.m) == (st[l, 0], st[l, 1])
        cu, cv, cw = (host(t) for t in S.sfg_graph_edges(ctx, gl))
        assert np.array_equal(cu, oc.u) and np.array_equal(cv, oc.v)
        assert np.array_equal(cw.view(np.uint32), oc.w.view(np.uint32))
        assert np.array_equal(host(f2c), of2c)
    for l in range(lf + 1):
        pm = host(H.mask(l))
        assert pm.shape == pms[l].shape
        assert int(pm.sum()) == int(pms[l].sum()) == st[l, 4], l
        tree = O.mst(levels_og[l])
        if l == lf:
            assert np.all(pm[tree == 1] == 1)          # the coarsest level keeps its forest
        extra_g, extra_o = pm.astype(bool), pms[l].astype(bool)
        both = (extra_g & extra_o).sum()
        assert both >= 0.95 * extra_o.sum(), (l, both, extra_o.sum())
    H.close()


def test_hierarchy_flat_and_lifetime(S, ctx):
    n, u, v, w = gen.grid2d(30, 30, seed=2)
    g = S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w))
    mask, nsel, H = S.sfg_sparsify(ctx, g, K=8, steps=10, levels=0, seed=3, budget_frac=0.1,
                                   hierarchy=True)
    assert H.levels == 0 and H.graph(0) is g
    assert np.array_equal(host(H.mask(0)), host(mask))
    with pytest.raises(S.SfgError):
        H.map(1)
    # the coarse graphs stay valid after the call and after other work on the context
    _, _, H2 = S.sfg_sparsify(ctx, g, K=8, steps=10, levels=2, seed=3, budget_frac=0.1,
                              hierarchy=True)
    g2 = H2.graph(2)
    S.sfg_sparsify(ctx, g, K=8, steps=10, levels=1, seed=4, budget_frac=0.1)
    x = S.sfg_smooth(ctx, g2, 8, 5, 0.7, seed=1)
    assert torch.isfinite(x).all()
    H2.close()
    H.close()


@pytest.mark.parametrize("K", [8, 32])
def test_coarsen_bf16_block(S, ctx, K):
    # a BF16 block is widened exactly: coarsening it equals coarsening its FP32 copy and the
    # oracle's aggregation of the same values, bit for bit
    n, u, v, w = gen.grid2d(40, 40, seed=6, weights="logu", lo=-2, hi=2)
    g = S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w))
    og = O.canonicalize(n, u, v, w)
    xb = dev(gen.gaussian_block(n, K, seed=7)).to(torch.bfloat16)
    agg_b, f2c_b, cb = S.sfg_coarsen(ctx, g, xb)
    agg_f, f2c_f, cf = S.sfg_coarsen(ctx, g, xb.float().contiguous())
    assert torch.equal(agg_b, agg_f) and torch.equal(f2c_b, f2c_f)
    oagg, nc = O.aggregate(og, O.affinity(og, host(xb.float()).astype(np.float64)))
    assert np.array_equal(host(agg_b), oagg) and cb.n == nc


def test_sparsify_multilevel_bf16_same_hierarchy(S, ctx):
    # BF16 blocks change only the edge-recovery scores: the aggregation is taken on FP32
    # embeddings, so the hierarchy is the FP32 run's bit for bit, and kappa stays within the
    # BF16 storage tolerance of the FP32 run's
    n, u, v, w = gen.grid2d(48, 48, seed=4, weights="logu", lo=-2, hi=2)
    g = S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w))
    og = O.canonicalize(n, u, v, w)
    kw = dict(K=16, steps=10, levels=2, seed=17, budget_frac=0.05, budget_unit=0)
    m32, n32, h32 = S.sfg_sparsify(ctx, g, hierarchy=True, **kw)
    m16, n16, h16 = S.sfg_sparsify(ctx, g, storage=torch.bfloat16, hierarchy=True, **kw)
    assert h32.levels == h16.levels == 2
    for l in (1, 2):
        a32, f32 = h32.map(l)
        a16, f16 = h16.map(l)
        assert torch.equal(a32, a16) and torch.equal(f32, f16)
    k32, k16 = O.kappa_dense(og, host(m32)), O.kappa_dense(og, host(m16))
    assert n32 == n16
    assert k16 <= 1.25 * k32, (k16, k32)
