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
    score itself (the method without the network). What the network must gain over the method
    without it: a higher rank correlation with the 20-step score than the 2-step score has, and a
    higher recall of the 20-step top-k inside the top 20% of candidates. kappa at each proposal
    fraction is reported against the plain method's."""
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
    assert r_net > r_two, report
    assert rec[0.2][0] > rec[0.2][1], report


# ------------------------------------------------------------------ learned form vs its oracle --
def _oracle_trained_theta():
    """Network weights trained by the oracle alone (FP64 features and 20-step labels of three
    seeded k-NN graphs, full-batch Adam): a network that ranks like a trained one, with no GPU
    data in it. Rounded to FP32 (the library keeps FP32 master weights)."""
    Xs, ts = [], []
    for sd in (401, 402, 403):
        og = O.canonicalize(*gen.knn3d(1500, k=10, seed=sd))
        st = M.learned_stages(og, M.init_params(1), K=16, steps=20, feat_steps=2, propose_frac=1.0,
                              seed=sd, budget_frac=0.05)
        full = O.score_edges(og, st["xg"], st["xp"], st["cand"])
        Xs.append(st["feats"])
        ts.append(np.log(full + 1e-30))
    X, t = np.concatenate(Xs), np.concatenate(ts)
    theta = M.init_params(11)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    for step in range(1, 301):
        g, _ = M.grad(theta, X, t)
        theta, m, v = M.adam_step(theta, m, v, g, step, lr=3e-3)
    return theta.astype(np.float32).astype(np.float64)


def _agree_outside_band(got_ids, ref_ids, universe, value, threshold, band):
    """Membership of every id whose reference value lies farther than band from the threshold is
    the same in both selections; returns the number of ids inside the band."""
    gs, rs = np.isin(universe, got_ids), np.isin(universe, ref_ids)
    clear = np.abs(value - threshold) > band
    bad = np.nonzero(clear & (gs != rs))[0]
    assert bad.size == 0, (bad[:5], value[bad[:5]], threshold, band[bad[:5]] if np.ndim(band) else band)
    return int((~clear).sum())


def test_sparsify_learned_matches_oracle(S, ctx):
    """sfg_sparsify_learned against the oracle's restatement, stage by stage. Each stage is a
    selection decided by floating point, so ids must agree exactly outside a band around the
    selection threshold whose width is the stage's error bar: for the proposals, the network fed
    the oracle's own features against the oracle's forward in the kernel's precision (BF16
    features, weights and first hidden layer; band 1e-2); for the final top-k, the oracle's
    proposals rescored on the GPU against the oracle's scores (per-edge FP32 bar, times 2)."""
    from parity import score_bar, score_condition

    theta = _oracle_trained_theta()
    net = S.sfg_mlp_create(ctx, seed=0)
    S.sfg_mlp_set_params(ctx, net, dev(theta.astype(np.float32)))
    K, T, Tf, frac, seed = 16, 20, 2, 0.2, 300
    n, u, v, w = gen.knn3d(2500, k=10, seed=seed)
    og = O.canonicalize(n, u, v, w)
    g = S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w))
    st = M.learned_stages(og, theta, K=K, steps=T, feat_steps=Tf, propose_frac=frac, seed=seed,
                          budget_frac=0.05)
    k, nprop, cand = st["k"], st["nprop"], st["cand"]
    # the call itself, and the same stages through the public calls: bit-identical
    mask, nsel = S.sfg_sparsify_learned(ctx, g, net, K=K, steps=T, feat_steps=Tf,
                                        propose_frac=frac, seed=seed, budget_frac=0.05)
    tree, _ = S.sfg_spanning_tree(ctx, g)
    assert np.array_equal(host(tree), st["forest"])
    p = S.sfg_graph_subgraph(ctx, g, tree)
    dcand = dev(cand)
    feats = S.sfg_edge_features(ctx, g, p, dcand, K, Tf, 0.7, seed=seed)
    pred = S.sfg_mlp_forward(ctx, net, feats)
    prop = S.sfg_select_topk(ctx, pred, dcand, nprop)
    sc = S.sfg_filter_score(ctx, g, p, prop, K, T, 0.7, seed=seed)
    sel = S.sfg_select_topk(ctx, sc, prop, k)
    composed = tree.clone()
    composed[sel.long()] = 1
    assert torch.equal(composed, mask) and nsel == int(st["mask"].sum())
    # stage 1: features (definition, FP32 logarithms)
    assert np.abs(host(feats) - st["feats"]).max() < 1e-4
    # stage 2: the network on the oracle's features (the oracle's own output as input) against the
    # oracle's forward in the kernel's precision; per row within 1e-3 + 2^-8 |y| except for rows
    # where one BF16 rounding of H1 fell the other way (at most 0.1%); then the proposals = top
    # nprop predictions agree outside a band of 1e-2 around the threshold
    pref = M.forward_kernel_precision(theta, st["feats"])
    pg = host(S.sfg_mlp_forward(ctx, net, dev(st["feats"].astype(np.float32)))).astype(np.float64)
    off_rows = np.abs(pg - pref) > 1e-3 + 2.0 ** -8 * np.abs(pref)
    assert off_rows.mean() <= 1e-3, off_rows.sum()
    tau = np.sort(pref)[::-1][nprop - 1]
    amb_p = _agree_outside_band(host(S.sfg_select_topk(ctx, dev(pg.astype(np.float32)), dcand, nprop)),
                                O.topk(pref, cand, nprop), cand, pref, tau, 1e-2)
    # stage 3: the oracle's proposals rescored by the plain filter on the GPU, then top-k
    sc_o = S.sfg_filter_score(ctx, g, p, dev(st["prop"]), K, T, 0.7, seed=seed)
    sel_o = host(S.sfg_select_topk(ctx, sc_o, dev(st["prop"]), k))
    bar = score_bar(st["scores"], score_condition(og, st["xg"], st["xp"], st["prop"], 0))
    tau_s = np.sort(st["scores"])[::-1][k - 1]
    amb_s = _agree_outside_band(sel_o, st["sel"], st["prop"], st["scores"], tau_s, 2 * bar)
    final = host(mask).astype(bool)
    overlap = (final & st["mask"].astype(bool)).sum() - int(st["forest"].sum())
    write_report("learned_parity.txt",
                 f"knn3d n={og.n}: {cand.size} candidates, {nprop} proposals, k={k}; network rows "
                 f"off the 1e-3 bar {int(off_rows.sum())}; proposals in the 1e-2 band {amb_p}; "
                 f"rescored proposals in the FP32 band {amb_s}; final selection overlap with the "
                 f"oracle {overlap}/{k}")
    assert overlap >= 0.95 * k
