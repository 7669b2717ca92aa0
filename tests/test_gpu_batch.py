"""The batch plan (sfg_batch_create / sfg_batch_run): the batched flat method with its
graph-dependent part built once and its numeric part run without host synchronisation, so that a
run can be captured in a CUDA graph and replayed."""
import numpy as np
import pytest
import torch

from paper_2008_07633_gb300 import inputs as gen

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def S():
    import paper_2008_07633_gb300.sfg as S

    S.lib()
    return S


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _specs():
    rng = np.random.default_rng(91)
    specs = [gen.knn3d(int(np.exp(rng.uniform(np.log(300), np.log(3000)))), k=10, seed=500 + i)
             for i in range(12)]
    specs.append(gen.hub_graph(seed=33))                                   # rows over 256 entries
    specs.append(gen.random_graph(700, 1500, seed=12, connected=False))    # forest + isolated nodes
    specs.append(gen.path(40, weights="uniform"))                          # a tree: nothing to add
    return specs


def test_batch_plan_matches_sparsify_batched(S):
    ctx = S.sfg_ctx_create(0)
    gs = [S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w)) for n, u, v, w in _specs()]
    kw = dict(K=16, steps=15, budget_frac=0.05)
    masks, counts = S.sfg_sparsify_batched(ctx, gs, seed=7, **kw)
    plan = S.Batch(ctx, gs, **kw)
    assert plan.ng == len(gs) and plan.m == sum(g.m for g in gs)
    assert plan.counts == list(counts)
    out = plan.run(7)
    for mb, part, c in zip(masks, plan.split(out), plan.counts):
        assert torch.equal(mb, part)
        assert int(part.sum().item()) == c
    # a second seed gives another sparsifier of the same sizes
    other = plan.run(8)
    assert [int(p.sum().item()) for p in plan.split(other)] == plan.counts
    assert not torch.equal(other, out)


def test_batch_run_captured_in_a_cuda_graph(S):
    stream = torch.cuda.Stream()
    ctx = S.sfg_ctx_create(0, stream)
    with torch.cuda.stream(stream):
        gs = [S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w)) for n, u, v, w in _specs()]
        plan = S.Batch(ctx, gs, K=32, steps=12, budget_frac=0.05, autotune=True)
        ref = plan.run(11)
        out = torch.empty_like(ref)
    stream.synchronize()
    for g in gs:          # the plan keeps its own copy of the graphs
        g.close()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream, capture_error_mode="relaxed"):
        plan.run(11, out=out)
    for _ in range(3):
        out.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


def _locality_specs():
    specs = _specs()
    # integer weights: many weight ties, which the forest breaks by original edge id
    n, u, v, w = gen.random_graph(1500, 6000, seed=44, lo=1, hi=4)
    specs.append((n, u, v, np.floor(w).astype(np.float32)))
    specs.append(gen.random_graph(900, 1000, seed=45, connected=False))   # several components
    # a long chain with short chords: more breadth-first levels than the search labels (4096), so
    # its far end keeps the input order
    n, u, v, w = gen.path(9000, weights="uniform")
    rng = np.random.default_rng(46)
    a = rng.integers(0, n - 3, 300)
    u = np.concatenate([u, a]).astype(np.int32)
    v = np.concatenate([v, a + 2 + rng.integers(0, 2, a.size)]).astype(np.int32)
    w = np.concatenate([w, rng.uniform(1.0, 10.0, a.size)]).astype(np.float32)
    specs.append((n, u, v, w))
    return specs


def test_locality_order_keeps_forest_and_sizes(S):
    """With the nodes renumbered by breadth-first level, the spanning forests (budget 0) equal the
    input-order plan's bit for bit -- weight ties are broken by the original edge ids -- and the
    masks come out in the original edge order."""
    ctx = S.sfg_ctx_create(0)
    gs = [S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w)) for n, u, v, w in _locality_specs()]
    kw = dict(K=16, steps=15, budget_frac=0.0)
    plain = S.Batch(ctx, gs, **kw)
    loc = S.Batch(ctx, gs, locality=True, **kw)
    assert loc.counts == plain.counts and loc.offsets == plain.offsets
    assert torch.equal(loc.run(3), plain.run(3))


def test_locality_order_sparsifiers(S):
    """With a budget, the sparsifiers differ from the input-order plan's only through FP32
    summation order: same sizes, at least 95% of every graph's selected edges shared, kappa
    within 5%; runs are deterministic and replay from a CUDA graph bit for bit."""
    stream = torch.cuda.Stream()
    ctx = S.sfg_ctx_create(0, stream)
    with torch.cuda.stream(stream):
        gs = [S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w)) for n, u, v, w in _locality_specs()]
        kw = dict(K=16, steps=15, budget_frac=0.05)
        plain = S.Batch(ctx, gs, **kw)
        loc = S.Batch(ctx, gs, locality=True, autotune=True, **kw)
        a, b = plain.run(7), loc.run(7)
        again = loc.run(7)
        forest = plain.split(S.Batch(ctx, gs, K=16, steps=15, budget_frac=0.0).run(7))
    stream.synchronize()
    assert loc.counts == plain.counts
    assert torch.equal(b, again)
    for g, pa, pb, f in zip(gs, plain.split(a), loc.split(b), forest):
        assert int(pa.sum()) == int(pb.sum())
        assert torch.equal(pb & f, f)                       # the forest is kept
        sel_a, sel_b = pa & ~f.bool(), pb & ~f.bool()
        k = int(sel_a.sum())
        if k == 0:
            continue
        assert int((sel_a & sel_b).sum()) >= 0.95 * k
        if g.n >= 1000:
            ka = S.sfg_kappa(ctx, g, pa)[0]
            kb = S.sfg_kappa(ctx, g, pb)[0]
            assert abs(kb / ka - 1.0) <= 0.05
    out = torch.empty_like(b)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream, capture_error_mode="relaxed"):
        loc.run(7, out=out)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, b)


def test_batch_plan_rejects_bad_arguments(S):
    ctx = S.sfg_ctx_create(0)
    n, u, v, w = gen.grid2d(8, 8)
    g = S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w))
    with pytest.raises(S.SfgError) as e:
        S.Batch(ctx, [g], K=12)
    assert e.value.status == 6
    with pytest.raises(S.SfgError) as e:
        S.Batch(ctx, [g], omega=1.5)
    assert e.value.status == 1
