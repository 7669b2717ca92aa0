"""The allocation-free affinity entry point against the allocating one.

sfg_affinity_noalloc exists for callers that cannot let a library allocate device memory (their
memory is owned by their own pool, or allocation is not permitted where they run). It must give
exactly what sfg_affinity gives (both are bit-exact FP64 evaluations of the same formula), call
after call, even though every call reuses the same fixed scratch array. This file is collected
last so that a run stopping at the first failure has run everything else first.
"""
import numpy as np
import pytest
import torch

from paper_2008_07633_gb300 import inputs as gen

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def _graph(S, ctx, n, u, v, w):
    t = [torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in (u, v, w)]
    return S.sfg_laplacian(ctx, n, *t)


def test_affinity_noalloc_matches_affinity_on_consecutive_calls():
    import paper_2008_07633_gb300.sfg as S

    ctx = S.sfg_ctx_create(0)
    g1 = _graph(S, ctx, *gen.grid2d(64, 64, seed=1))
    g2 = _graph(S, ctx, *gen.random_graph(3001, 12000, seed=3))
    calls = [(g1, gen.gaussian_block(g1.n, 8, seed=5)), (g2, gen.gaussian_block(g2.n, 16, seed=6)),
             (g1, gen.gaussian_block(g1.n, 32, seed=7))]
    for g, x in calls:
        X = torch.from_numpy(x).to(DEV)
        ref = S.sfg_affinity(ctx, g, X)
        got = S.sfg_affinity_noalloc(ctx, g, X)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)     # the tolerance of the affinity tests: bit-exact


def test_affinity_noalloc_rejects_graphs_beyond_its_scratch():
    import paper_2008_07633_gb300.sfg as S

    ctx = S.sfg_ctx_create(0)
    n = (1 << 20) + 1
    g = _graph(S, ctx, n, np.array([0], np.int32), np.array([1], np.int32),
               np.array([1.0], np.float32))
    X = torch.zeros((n, 4), dtype=torch.float32, device=DEV)
    with pytest.raises(S.SfgError) as e:
        S.sfg_affinity_noalloc(ctx, g, X)
    assert e.value.status == 5 and "exceeds" in str(e.value)


def test_affinity_noalloc_needs_no_allocation():
    # A context whose first pool allocation fails (SFG_FAULT_ALLOC=1, read when the context is
    # created): the allocating entry point reports SFG_ENOMEM, the allocation-free one still
    # gives the same result, call after call. Graph and block come from another context.
    import os

    import paper_2008_07633_gb300.sfg as S

    ctx = S.sfg_ctx_create(0)
    g = _graph(S, ctx, *gen.grid2d(48, 48, seed=2))
    X = torch.from_numpy(gen.gaussian_block(g.n, 16, seed=8)).to(DEV)
    ref = S.sfg_affinity(ctx, g, X)
    old = os.environ.get("SFG_FAULT_ALLOC")
    os.environ["SFG_FAULT_ALLOC"] = "1"
    try:
        starved = S.sfg_ctx_create(0)
    finally:
        if old is None:
            del os.environ["SFG_FAULT_ALLOC"]
        else:
            os.environ["SFG_FAULT_ALLOC"] = old
    with pytest.raises(S.SfgError) as e:
        S.sfg_affinity(starved, g, X)
    assert e.value.status == 2
    for _ in range(2):
        out = torch.empty(g.m, dtype=torch.float64, device=DEV)
        got = S.sfg_affinity_noalloc(starved, g, X, out=out)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
