"""Oracle of the learned edge-proposal scorer: FP64 numpy restatement (test infrastructure only).

The paper has no learned part; this restates the specification the library implements: per
candidate edge e = (p, q) eight features from a short (feature) embedding,
    f0 = ln w,  f1 = ln d_p + ln d_q,  f2 = |ln d_p - ln d_q|,  f3 = ln(s_G + tiny),
    f4 = ln(s_P + tiny),  f5 = ln(s_P + tiny) - ln(s_G + eta),  f6 = ln(deg_p deg_q),
    f7 = ln(s_G + s_P + tiny),  f8..f15 = 0,
with d the weighted degree, deg the number of neighbours, s_G, s_P the projected-embedding
distances of Sec. 3.5 (w ||X^T e_pq||^2 on L_G and on L_P), tiny = 1e-30, eta = 1e-30; a network
16 -> 64 -> 64 -> 1 with ReLU (parameters W1 [16][64], b1, W2 [64][64], b2, w3 [64], b3, flat in
that order, 5313 values); loss L = mean((y - t)^2); Adam with bias correction. Initial weights
are Kaiming-uniform from the counter-based generator: u_j = (splitmix64(s0 + j gamma) >> 11) 2^-53,
s0 = splitmix64(seed), weight j = (2 u_j - 1) sqrt(6 / fan_in); biases 0.

Parity status: the forward pass and the analytic gradients are pinned by central finite
differences (tests/test_oracle_mlp.py); the features by their definition on hand-made inputs.
"""
from __future__ import annotations

import numpy as np

F, H = 16, 64
SIZES = [("W1", (F, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)   # 5313
TINY = 1e-30
GAMMA = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1


def _splitmix64(x):
    z = (x + GAMMA) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def unflatten(theta):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + n], np.float64).reshape(shape)
        o += n
    return out


def flatten(p):
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SIZES])


def init_params(seed):
    s0 = _splitmix64(seed & MASK)
    theta = np.zeros(NPARAM)
    fan = {"W1": F, "W2": H, "w3": H}
    o = 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        if name in fan:
            b = np.sqrt(6.0 / fan[name])
            for j in range(o, o + n):
                u = (_splitmix64((s0 + j * GAMMA) & MASK) >> 11) * 2.0 ** -53
                theta[j] = (2.0 * u - 1.0) * b
        o += n
    return theta


def features(w, dp, dq, degp, degq, sg, sp, eta=1e-30):
    """Feature rows (E x 16) from per-edge quantities (all 1-D arrays of length E)."""
    w, dp, dq, sg, sp = (np.asarray(a, np.float64) for a in (w, dp, dq, sg, sp))
    degp, degq = np.asarray(degp, np.float64), np.asarray(degq, np.float64)
    X = np.zeros((w.size, F))
    X[:, 0] = np.log(w)
    X[:, 1] = np.log(dp) + np.log(dq)
    X[:, 2] = np.abs(np.log(dp) - np.log(dq))
    X[:, 3] = np.log(sg + TINY)
    X[:, 4] = np.log(sp + TINY)
    X[:, 5] = np.log(sp + TINY) - np.log(sg + eta)
    X[:, 6] = np.log(degp * degq)
    X[:, 7] = np.log(sg + sp + TINY)
    return X


def forward(theta, X):
    p = unflatten(theta)
    z1 = X @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["w3"] + p["b3"][0]
    return y, (z1, h1, z2, h2)


def round_bf16(a):
    """Round to the nearest BF16 number, ties to even (the upper 16 bits of the FP32 pattern after
    adding 0x7fff plus the lowest kept bit), returned as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_kernel_precision(theta, X):
    """The network with the library's BF16 rounding points -- features, W1, W2 and the first
    hidden layer rounded to BF16, everything else exact: the precision in which the library's
    tensor-core kernels take the proposal decision."""
    p = unflatten(theta)
    z1 = round_bf16(X) @ round_bf16(p["W1"]) + p["b1"]
    h1 = round_bf16(np.maximum(z1, 0.0))
    z2 = h1 @ round_bf16(p["W2"]) + p["b2"]
    return np.maximum(z2, 0.0) @ p["w3"] + p["b3"][0]


def loss(theta, X, t):
    y, _ = forward(theta, X)
    return float(np.mean((y - t) ** 2))


def grad(theta, X, t):
    """Analytic gradient of loss() by backpropagation; returns (grad, loss)."""
    p = unflatten(theta)
    y, (z1, h1, z2, h2) = forward(theta, X)
    B = X.shape[0]
    d3 = 2.0 * (y - t) / B
    g = {"w3": h2.T @ d3, "b3": np.array([d3.sum()])}
    d2 = np.outer(d3, p["w3"]) * (z2 > 0)
    g["W2"] = h1.T @ d2
    g["b2"] = d2.sum(0)
    d1 = (d2 @ p["W2"].T) * (z1 > 0)
    g["W1"] = X.T @ d1
    g["b1"] = d1.sum(0)
    return flatten(g), float(np.mean((y - t) ** 2))


def adam_step(theta, m, v, g, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------------------------------------------------------------
# The learned-proposal form of the flat method (not in the paper; the plain method of Sec. 3.5 is
# its rescoring step and final arbiter), in the order the library specifies: spanning forest;
# features of every off-forest edge from a feat_steps embedding; network predictions; the top
# max(k, round_half_up(propose_frac * candidates)) predictions become proposals; the proposals are
# rescored by the plain filter (steps sweeps on L_G and L_P from the same seed); the top k
# rescored proposals join the forest.
# ------------------------------------------------------------------------------------------------
def learned_stages(og, theta, K, steps, feat_steps, propose_frac, seed, budget_frac=0.05,
                   budget_unit=0, omega=0.7, mode=0):
    """Returns a dict with every intermediate of the learned form: forest mask, candidate ids,
    budget k, feature rows, predictions, proposal ids (ascending), their rescored scores, the
    selected ids (ascending) and the final mask."""
    import oracle as O

    forest = O.mst(og).astype(np.uint8)
    cand = np.nonzero(forest == 0)[0].astype(np.int32)
    n_tree = int(forest.sum())
    base = og.n if budget_unit == 0 else cand.size
    k = min(max(int(np.floor(budget_frac * base + 0.5)), 0), cand.size)
    out = {"forest": forest, "cand": cand, "k": k}
    if k == 0:
        out["mask"] = forest
        return out
    nprop = min(max(int(np.floor(propose_frac * cand.size + 0.5)), k), cand.size)
    pg = og.subgraph(forest)
    xg_f = O.smooth(og, K, feat_steps, omega, seed)
    xp_f = O.smooth(pg, K, feat_steps, omega, seed)
    sg = O.score_edges(og, xg_f, xp_f, cand, O.G_ONLY)
    sp = O.score_edges(og, xg_f, xp_f, cand, O.P_ONLY)
    _, _, _, _, deg = O.laplacian_csr(og)
    cnt = np.bincount(np.concatenate([og.u, og.v]), minlength=og.n)
    feats = features(og.w[cand], deg[og.u[cand]], deg[og.v[cand]], cnt[og.u[cand]],
                     cnt[og.v[cand]], sg, sp)
    pred, _ = forward(theta, feats)
    prop = O.topk(pred, cand, nprop)
    xg = O.smooth(og, K, steps, omega, seed)
    xp = O.smooth(pg, K, steps, omega, seed)
    scores = O.score_edges(og, xg, xp, prop, mode)
    sel = O.topk(scores, prop, k)
    mask = forest.copy()
    mask[sel] = 1
    out.update(nprop=nprop, feats=feats, pred=pred, prop=prop, scores=scores, sel=sel, mask=mask,
               xg=xg, xp=xp)
    return out
