"""Runtime behaviour on the GPU: the tile-shape autotuner, CUDA-graph capture of the filter+score
step, and error paths (an injected allocation failure, made on the host; no GPU fault)."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2008_07633_gb300 import inputs as gen

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def S():
    import paper_2008_07633_gb300.sfg as S

    S.lib()
    return S


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def test_autotune_variants_agree_bit_for_bit(S):
    ctx = S.sfg_ctx_create(0)
    n, u, v, w = gen.grid3d(40, seed=2)
    g = S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w))
    x0 = torch.from_numpy(gen.gaussian_block(n, 32, seed=3)).to(DEV)
    outs = []
    for var in range(6):
        S.sfg_tune_set(ctx, 32, torch.float32, 2, var)   # the 3-D grid's degree bucket (2m/n ~ 6)
        outs.append(S.sfg_jacobi(ctx, g, x0.clone(), 7, 0.7))
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    S.sfg_tune_set(ctx, 32, torch.float32, 2, -1)
    best, us = S.sfg_autotune(ctx, g, 32)
    assert 0 <= best < 6 and us > 0
    table = S.sfg_tune_table(ctx)
    assert len(table) == 1 and table[0]["score_shape"] in (0, 1, 2)
    assert table == [{"K": 32, "dtype": 0, "degree_bucket": 2, "variant": best,
                      "tiles_per_warp": [1, 2, 4, 1, 2, 4][best],
                      "ctas_per_sm": [4, 4, 4, 3, 3, 3][best],
                      "score_shape": table[0]["score_shape"]}]
    assert torch.equal(S.sfg_jacobi(ctx, g, x0.clone(), 7, 0.7), outs[0])


@pytest.mark.parametrize("K,dt", [(4, torch.float32), (32, torch.float32), (64, torch.float32),
                                  (8, torch.bfloat16), (64, torch.bfloat16)])
def test_score_shapes_agree_bit_for_bit(S, K, dt):
    # every launch shape of the scorer, on a mesh (degree bucket 2) and a denser graph (bucket 3)
    ctx = S.sfg_ctx_create(0)
    for n, u, v, w in (gen.grid3d(24, seed=2), gen.knn3d(6000, k=10, seed=3)):
        g = S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w))
        bucket = int(np.floor(np.log2(2 * g.m / g.n)))
        xg = torch.from_numpy(gen.gaussian_block(g.n, K, seed=5)).to(DEV).to(dt)
        xp = torch.from_numpy(gen.gaussian_block(g.n, K, seed=6)).to(DEV).to(dt)
        ids = dev(np.arange(g.m, dtype=np.int32)[::-1].copy())
        outs = []
        shapes = (0, 1, 2, -1)
        for shape in shapes:
            S.sfg_tune_set_score(ctx, K, dt, bucket, shape)
            for mode in (0, 1, 2):
                outs.append(S.sfg_score_edges(ctx, g, xg, xp, ids, mode=mode))
        for j in range(1, len(shapes)):
            for i in range(3):
                assert torch.equal(outs[i], outs[3 * j + i])
    with pytest.raises(S.SfgError):
        S.sfg_tune_set_score(ctx, K, dt, 2, 3)


def test_filter_score_and_select_capture_in_a_cuda_graph(S):
    stream = torch.cuda.Stream()
    ctx = S.sfg_ctx_create(0, stream)
    n, u, v, w = gen.knn3d(5000, k=10, seed=5)
    with torch.cuda.stream(stream):
        g = S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w))
        tree, _ = S.sfg_spanning_tree(ctx, g)
        p = S.sfg_graph_subgraph(ctx, g, tree)
        off = torch.nonzero(tree == 0).flatten().to(torch.int32)
        k = int(0.05 * n)
        ref_s = S.sfg_filter_score(ctx, g, p, off, 16, 15, 0.7, seed=9)
        ref_sel = S.sfg_select_topk(ctx, ref_s, off, k)
        scores = torch.empty_like(ref_s)
        sel = torch.empty_like(ref_sel)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream, capture_error_mode="relaxed"):
        S.sfg_filter_score(ctx, g, p, off, 16, 15, 0.7, seed=9, out=scores)
        S.sfg_select_topk(ctx, scores, off, k, out=sel)
    for _ in range(3):
        scores.zero_()
        sel.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(scores, ref_s) and torch.equal(sel, ref_sel)


_INJECT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
import paper_2008_07633_gb300.sfg as S
from paper_2008_07633_gb300 import inputs as gen
ctx = S.sfg_ctx_create(0)
n, u, v, w = gen.grid2d(30, 30)
t = [torch.from_numpy(a).cuda() for a in (u, v, w)]
try:
    S.sfg_laplacian(ctx, n, *t)
    print("NOFAIL")
except S.SfgError as e:
    print("STATUS", e.status, str(e).split(":", 1)[1].strip()[:60])
g = S.sfg_laplacian(ctx, n, *t)           # later calls work: the context stays usable
x = S.sfg_smooth(ctx, g, 8, 5, 0.7, 1)
torch.cuda.synchronize()
print("OK", bool(torch.isfinite(x).all()))
"""


@pytest.mark.parametrize("nth", [1, 3, 6])
def test_injected_allocation_failure_returns_enomem(nth):
    env = dict(os.environ, SFG_FAULT_ALLOC=str(nth))
    r = subprocess.run([sys.executable, "-c", _INJECT, ROOT], capture_output=True, text=True,
                       env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.split("\n")
    assert lines[0].startswith("STATUS 2"), r.stdout      # SFG_ENOMEM, not a crash
    assert "injected allocation failure" in lines[0]
    assert lines[1] == "OK True"


def test_argument_errors_leave_context_usable(S):
    ctx = S.sfg_ctx_create(0)
    n, u, v, w = gen.grid2d(10, 10)
    g = S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w))
    host_ptr = torch.zeros(g.m, dtype=torch.uint8)               # not device memory
    with pytest.raises(S.SfgError) as e:
        S.sfg_graph_subgraph(ctx, g, host_ptr)
    assert e.value.status == 1 and "device" in str(e.value)
    with pytest.raises(S.SfgError):
        S.sfg_sparsify(ctx, g, K=12)                              # unsupported K
    x = S.sfg_smooth(ctx, g, 8, 3)
    torch.cuda.synchronize()
    assert torch.isfinite(x).all()


def test_pool_trim_keeps_context_usable(S):
    ctx = S.sfg_ctx_create(0)
    n, u, v, w = gen.grid2d(40, 40, seed=2)
    g = S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w))
    a = S.sfg_smooth(ctx, g, 16, 5, 0.7, seed=4)
    torch.cuda.synchronize()
    ctx.trim()
    b = S.sfg_smooth(ctx, g, 16, 5, 0.7, seed=4)   # allocations after a trim map memory again
    assert torch.equal(a, b)
    del g
    ctx.close()



_WITHHOLD = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
import paper_2008_07633_gb300.sfg as S
ctx = S.sfg_ctx_create(0)                      # SFG_FAULT_MMA_WAIT=1: no MMA is ever issued
net = S.sfg_mlp_create(ctx, seed=1)
X = torch.randn(1000, 16, device="cuda")
y = S.sfg_mlp_forward(ctx, net, X)             # queued without synchronisation
try:
    S.sfg_mlp_check(ctx, net)
    print("NOFAIL")
except S.SfgError as e:
    print("STATUS", e.status)
try:
    S.sfg_mlp_gradient(ctx, net, X, torch.zeros(1000, device="cuda"))
    print("NOFAIL")
except S.SfgError as e:
    print("STATUS", e.status)
print("OK", bool(torch.isfinite(torch.ones(3, device="cuda")).all()))
"""


def test_tensor_core_wait_runs_out_and_reports_etimeout():
    # The bounded completion waits of the tensor-core kernels, run out on purpose by withholding
    # every MMA and commit (host switch read at context creation): nothing is in flight, so the
    # kernels give up after their time limit, release TMEM and return; the host sees SFG_ETIMEOUT
    # once per check and the process keeps using the GPU.
    env = dict(os.environ, SFG_FAULT_MMA_WAIT="1")
    r = subprocess.run([sys.executable, "-c", _WITHHOLD, ROOT], capture_output=True, text=True,
                       env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.split("\n")
    assert lines[0] == "STATUS 4" and lines[1] == "STATUS 4", r.stdout
    assert lines[2] == "OK True"


def test_entry_points_keep_the_callers_device(S):
    """Every call runs on its context's device and gives the caller's current device back. With one
    GPU this checks that nothing changes the current device; with two, the context lives on device
    0 while device 1 is current."""
    other = 1 if torch.cuda.device_count() > 1 else 0
    torch.cuda.set_device(other)
    try:
        ctx = S.sfg_ctx_create(0)
        assert torch.cuda.current_device() == other
        n, u, v, w = gen.grid2d(24, 24, seed=4)
        g = S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w))
        assert torch.cuda.current_device() == other
        tree, _ = S.sfg_spanning_tree(ctx, g)
        x = S.sfg_smooth(ctx, g, 8, 5, 0.7, 11)
        mask, _ = S.sfg_sparsify(ctx, g, K=8, steps=5, budget_frac=0.05, budget_unit=0)
        assert torch.cuda.current_device() == other
        assert x.device == DEV and mask.device == DEV and tree.device == DEV
        torch.cuda.synchronize(DEV)
        assert torch.isfinite(x).all()
        assert int(mask.sum()) >= n - 1
    finally:
        torch.cuda.set_device(0)
