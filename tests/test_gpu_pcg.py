"""Sparsifier-preconditioned conjugate gradients (sfg_solve_pcg) against the oracle's grounded
direct solve: solutions to the solver tolerance, P = G converging in one step, determinism, and a
report of iterations and time with the diagonal, spanning-tree and sparsifier preconditioners."""
import numpy as np
import pytest
import torch

import oracle as O
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


GRAPHS = {
    "grid2d": lambda: gen.grid2d(30, 30, seed=1),
    "disconnected": lambda: gen.random_graph(700, 1000, seed=2, connected=False),
    "knn": lambda: gen.knn3d(1500, k=8, seed=3),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_pcg_matches_direct_solve(S, ctx, name):
    n, u, v, w = GRAPHS[name]()
    og = O.canonicalize(n, u, v, w)
    g = S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w))
    b = np.random.default_rng(5).standard_normal(n)
    ref = O.solve_laplacian(og, b)
    spars, _ = S.sfg_sparsify(ctx, g, K=8, steps=10, seed=1, budget_frac=0.05, budget_unit=0)
    tree, _ = S.sfg_spanning_tree(ctx, g)
    its = {}
    for label, mask in (("sparsifier", spars), ("tree", tree), ("diagonal", None)):
        x, it, rel = S.sfg_solve_pcg(ctx, g, dev(b), mask=mask, tol=1e-10, maxit=20000)
        x = x.cpu().numpy()
        assert rel <= 1e-10, (label, rel)
        assert np.linalg.norm(x - ref) <= 1e-7 * np.linalg.norm(ref), label
        its[label] = it
    assert its["sparsifier"] <= its["tree"], its   # P contains the tree: at least as good


def test_pcg_exact_preconditioner_and_determinism(S, ctx):
    n, u, v, w = gen.grid2d(20, 24, seed=4)
    g = S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w))
    b = dev(np.random.default_rng(1).standard_normal(n))
    full = torch.ones(g.m, dtype=torch.uint8, device=DEV)
    x, it, rel = S.sfg_solve_pcg(ctx, g, b, mask=full, tol=1e-10)
    assert it == 1 and rel <= 1e-10          # P = G: the preconditioner is the inverse
    spars, _ = S.sfg_sparsify(ctx, g, K=8, steps=10, seed=1, budget_frac=0.05, budget_unit=0)
    x1, i1, _ = S.sfg_solve_pcg(ctx, g, b, mask=spars, tol=1e-10)
    x2, i2, _ = S.sfg_solve_pcg(ctx, g, b, mask=spars, tol=1e-10)
    assert i1 == i2 and torch.equal(x1, x2)
    tree, _ = S.sfg_spanning_tree(ctx, g)
    t = tree.clone()
    t[torch.nonzero(t).flatten()[0]] = 0
    with pytest.raises(S.SfgError):
        S.sfg_solve_pcg(ctx, g, b, mask=t)


def test_pcg_report(S, ctx):
    """64^3 grid with the bench's weights: iterations and time to 1e-8 (reported, not gated)."""
    import os
    import time
    n, u, v, w = gen.grid3d(64, seed=2)
    g = S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w))
    b = dev(np.random.default_rng(7).standard_normal(n))
    spars, ns = S.sfg_sparsify(ctx, g, K=32, steps=20, seed=1234, budget_frac=0.05, budget_unit=0)
    tree, _ = S.sfg_spanning_tree(ctx, g)
    rows = []
    for label, mask in (("sparsifier 5%", spars), ("spanning tree", tree), ("diagonal", None)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, it, rel = S.sfg_solve_pcg(ctx, g, b, mask=mask, tol=1e-8, maxit=5000)
        torch.cuda.synchronize()
        rows.append(f"{label}: {it} iterations, {time.perf_counter() - t0:.2f} s, relres {rel:.1e}")
    report = f"PCG_REPORT 64^3 grid (n={n}, m={g.m}): " + "; ".join(rows)
    print("\n" + report)
    write_report("pcg_report.txt", report)
