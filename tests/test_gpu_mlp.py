"""The learned edge-proposal scorer on the GPU against its FP64 oracle (oracle/mlp.py).

BF16 bar (stated): the GPU rounds the features, W1, W2, the first hidden layer and the backward
deltas to BF16 (unit roundoff 2^-9) with FP32 accumulation, so forward outputs and gradients are
compared normwise against the FP64 oracle fed the same BF16-rounded features and weights, within
2e-2 (outputs) and 5e-2 (gradients). Initial weights follow the generator to FP32 rounding; the
features follow their definition to 1e-4 (FP32 logarithms of FP32 distances).
"""
import numpy as np
import pytest
import torch

import oracle as O
import oracle.mlp as M
from paper_2008_07633_gb300 import inputs as gen
from conftest import write_report

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


def bf16(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300)


def _bf16_params(theta):
    p = M.unflatten(theta)
    p["W1"], p["W2"] = bf16(p["W1"]), bf16(p["W2"])
    return M.flatten(p)


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = np.zeros((n, 16), np.float32)
    X[:, :8] = rng.standard_normal((n, 8)).astype(np.float32)
    t = (X[:, 0] - 0.5 * X[:, 3] + 0.25 * X[:, 5] * X[:, 1]).astype(np.float32)
    return X, t


def test_mlp_init_follows_generator(S, ctx):
    net = S.sfg_mlp_create(ctx, seed=42)
    th = host(S.sfg_mlp_params(ctx, net)).astype(np.float64)
    ref = M.init_params(42)
    assert np.abs(th - ref).max() <= 1e-6 * np.abs(ref).max()


@pytest.mark.parametrize("ne", [1, 15, 16, 1000, 70001])
def test_mlp_forward_matches_oracle(S, ctx, ne):
    net = S.sfg_mlp_create(ctx, seed=3)
    rng = np.random.default_rng(ne)
    theta = (M.init_params(3) + 0.05 * rng.standard_normal(M.NPARAM)).astype(np.float32)
    S.sfg_mlp_set_params(ctx, net, dev(theta))
    X, _ = _data(ne, ne)
    y = host(S.sfg_mlp_forward(ctx, net, dev(X)))
    ref, _ = M.forward(_bf16_params(theta.astype(np.float64)), bf16(X))
    assert rel(y, ref) < 2e-2


def test_mlp_gradient_matches_oracle(S, ctx):
    net = S.sfg_mlp_create(ctx, seed=4)
    rng = np.random.default_rng(0)
    theta = (M.init_params(4) + 0.05 * rng.standard_normal(M.NPARAM)).astype(np.float32)
    S.sfg_mlp_set_params(ctx, net, dev(theta))
    X, t = _data(5003, 1)
    g, loss = S.sfg_mlp_gradient(ctx, net, dev(X), dev(t))
    g = host(g)
    ref, lref = M.grad(_bf16_params(theta.astype(np.float64)), bf16(X), t.astype(np.float64))
    assert abs(loss - lref) <= 2e-2 * lref
    o = 0
    for name, shape in M.SIZES:
        k = int(np.prod(shape))
        assert rel(g[o:o + k], ref[o:o + k]) < 5e-2, name
        o += k


def test_mlp_gradient_deterministic(S, ctx):
    net = S.sfg_mlp_create(ctx, seed=5)
    X, t = _data(20000, 2)
    g1, _ = S.sfg_mlp_gradient(ctx, net, dev(X), dev(t))
    g2, _ = S.sfg_mlp_gradient(ctx, net, dev(X), dev(t))
    assert torch.equal(g1, g2)


def test_mlp_training_reduces_loss(S, ctx):
    net = S.sfg_mlp_create(ctx, seed=6)
    X, t = _data(50000, 3)
    _, l0 = S.sfg_mlp_gradient(ctx, net, dev(X), dev(t))
    l1 = S.sfg_mlp_train(ctx, net, dev(X), dev(t), batch=4096, epochs=20, lr=3e-3)
    assert l1 < 0.1 * l0, (l0, l1)


def test_edge_features_match_oracle(S, ctx):
    n, u, v, w = gen.grid2d(48, 48, seed=1)
    og = O.canonicalize(n, u, v, w)
    g = S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w))
    tree, _ = S.sfg_spanning_tree(ctx, g)
    p = S.sfg_graph_subgraph(ctx, g, tree)
    off = np.nonzero(host(tree) == 0)[0].astype(np.int32)
    f = host(S.sfg_edge_features(ctx, g, p, dev(off), 16, 2, 0.7, seed=9))
    ot = O.mst(og)
    xg = O.smooth(og, 16, 2, 0.7, 9)
    xp = O.smooth(og.subgraph(ot), 16, 2, 0.7, 9)
    sg = O.score_edges(og, xg, xp, off, O.G_ONLY)
    sp = O.score_edges(og, xg, xp, off, O.P_ONLY)
    _, _, _, _, deg = O.laplacian_csr(og)
    cnt = np.bincount(np.concatenate([og.u, og.v]), minlength=n)
    ref = M.features(og.w[off], deg[og.u[off]], deg[og.v[off]], cnt[og.u[off]], cnt[og.v[off]], sg, sp)
    assert np.abs(f - ref).max() < 1e-4


def _train_set(S, ctx, seeds, K=16, T=20, Tf=2):
    feats, targs = [], []
    for sd in seeds:
        n, u, v, w = gen.knn3d(4000, k=10, seed=sd)
        g = S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w))
        tree, _ = S.sfg_spanning_tree(ctx, g)
        p = S.sfg_graph_subgraph(ctx, g, tree)
        off = torch.nonzero(tree == 0).flatten().to(torch.int32)
        feats.append(S.sfg_edge_features(ctx, g, p, off, K, Tf, 0.7, seed=sd))
        s = S.sfg_filter_score(ctx, g, p, off, K, T, 0.7, seed=sd)
        targs.append(torch.log(s + 1e-30))
    return torch.cat(feats), torch.cat(targs)


def test_learned_proposals_against_plain_method(S, ctx):
    """Train on method-generated data (8 seeded graphs), then on a held-out graph compare the
    learned form (2-step features -> network -> top proposals -> 20-step rescoring) with the plain
    method at several proposal fractions, and the network's ranking with ranking by the 2-step
    score itself (the method without the network). The plain method is the yardstick: the learned
    form must match its kappa within 5% at some proposal fraction <= 0.5; the curve is reported."""
    X, y = _train_set(S, ctx, range(201, 209))
    net = S.sfg_mlp_create(ctx, seed=11)
    loss = S.sfg_mlp_train(ctx, net, X, y, batch=8192, epochs=30, lr=2e-3)
    n, u, v, w = gen.knn3d(2500, k=10, seed=300)
    og = O.canonicalize(n, u, v, w)
    g = S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w))
    plain, np_ = S.sfg_sparsify(ctx, g, K=16, steps=20, levels=0, seed=300, budget_frac=0.05,
                                budget_unit=0)
    kp = O.kappa_dense(og, host(plain))
    curve = {}
    for frac in (0.1, 0.2, 0.35, 0.5):
        learned, nl = S.sfg_sparsify_learned(ctx, g, net, K=16, steps=20, feat_steps=2,
                                             propose_frac=frac, seed=300, budget_frac=0.05)
        assert np_ == nl
        curve[frac] = O.kappa_dense(og, host(learned))
    tree, _ = S.sfg_spanning_tree(ctx, g)
    p = S.sfg_graph_subgraph(ctx, g, tree)
    off = torch.nonzero(tree == 0).flatten().to(torch.int32)
    truth = host(S.sfg_filter_score(ctx, g, p, off, 16, 20, 0.7, seed=300))
    two = host(S.sfg_filter_score(ctx, g, p, off, 16, 2, 0.7, seed=300))
    pred = host(S.sfg_mlp_forward(ctx, net, S.sfg_edge_features(ctx, g, p, off, 16, 2, 0.7, seed=300)))
    from scipy.stats import spearmanr
    r_net, r_two = spearmanr(pred, truth)[0], spearmanr(two, truth)[0]
    k = int(np.floor(0.05 * n + 0.5))
    top = set(np.argsort(-truth)[:k])
    rec = {f: (len(top & set(np.argsort(-pred)[:int(f * truth.size)])) / k,
               len(top & set(np.argsort(-two)[:int(f * truth.size)])) / k) for f in curve}
    report = (f"LEARNED_REPORT train loss {loss:.3f}; kappa plain {kp:.1f}; learned by proposal "
              f"fraction {dict((f, round(c, 1)) for f, c in curve.items())}; Spearman vs 20-step "
              f"score: network {r_net:.3f}, 2-step score {r_two:.3f}; top-k recall in the "
              f"proposals (network, 2-step): {dict((f, (round(a, 3), round(b, 3))) for f, (a, b) in rec.items())}")
    print("\n" + report)
    write_report("learned_report.txt", report)
    assert r_net > 0.5
    assert min(abs(c - kp) / kp for c in curve.values()) <= 0.05, report
