"""Per-edge parity bar for FP32 edge scores against the FP64 oracle.

The bar is 1e-5 relative per edge: |s - ref| <= 1e-5 * max(|ref|, 1e-6 * median |ref|) (the floor
covers scores that are zero in exact arithmetic). One class of edges cannot meet it in FP32 at
all: when the two endpoint rows of a block almost coincide (strongly coupled endpoints), the score
is a small difference of large numbers, and storing the oracle's own FP64 vectors once in FP32
already moves it by more than 1e-5. For an edge e = (p, q) and a block X, the first-order
relative change of w ||X_p - X_q||^2 when every entry moves by a relative u is at most
u * c_X(e), c_X(e) = 2 sum_k |X_pk - X_qk| (|X_pk| + |X_qk|) / sum_k (X_pk - X_qk)^2;
a RATIO score adds the condition numbers of its two blocks. With u = 2^-24 (FP32) an edge with
c(e) <= 16 loses at most 1e-6 to representation alone and keeps the plain 1e-5 bar; an edge with
a larger c(e) gets the bar scaled by c(e) / 16, i.e. about ten units of its own representation
error (the sweeps add a few roundings of the same size each). c(e) is computed from the
oracle's vectors only, never from the GPU's output.
"""
import numpy as np

TOL = 1e-5
C_PLAIN = 16.0


def block_condition(u, v, X, ids):
    p, q = u[ids], v[ids]
    D = X[p] - X[q]
    num = 2.0 * (np.abs(D) * (np.abs(X[p]) + np.abs(X[q]))).sum(1)
    den = (D * D).sum(1)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), np.inf)


def score_condition(og, xg, xp, ids, mode=0):
    """Condition number c(e) of each listed edge's score (mode 0 RATIO, 1 G, 2 P)."""
    ids = np.asarray(ids, np.int64)
    if mode == 1:
        return block_condition(og.u, og.v, xg, ids)
    if mode == 2:
        return block_condition(og.u, og.v, xp, ids)
    return block_condition(og.u, og.v, xg, ids) + block_condition(og.u, og.v, xp, ids)


def score_bar(ref, cond):
    floor = 1e-6 * np.median(np.abs(ref)) if ref.size else 0.0
    scale = np.maximum(np.abs(ref), max(floor, 1e-300))
    return TOL * scale * np.maximum(1.0, cond / C_PLAIN)


def check_scores(s, ref, cond):
    """Assert the per-edge bar; return a summary (edges, worst error over its bar, share of edges
    under the plain 1e-5 bar, share of edges whose bar is scaled)."""
    s = np.asarray(s, np.float64)
    ref = np.asarray(ref, np.float64)
    assert s.shape == ref.shape
    if ref.size == 0:
        return {"edges": 0}
    bar = score_bar(ref, cond)
    err = np.abs(s - ref)
    floor = 1e-6 * np.median(np.abs(ref))
    plain = err <= TOL * np.maximum(np.abs(ref), max(floor, 1e-300))
    worst = float((err / bar).max())
    bad = np.nonzero(err > bar)[0]
    assert bad.size == 0, (f"{bad.size} of {ref.size} edges over the per-edge bar; first "
                           f"{bad[:5].tolist()}: got {s[bad[:5]].tolist()} ref {ref[bad[:5]].tolist()} "
                           f"cond {cond[bad[:5]].tolist()}")
    return {"edges": int(ref.size), "worst_over_bar": worst, "plain_share": float(plain.mean()),
            "scaled_share": float((cond > C_PLAIN).mean())}
