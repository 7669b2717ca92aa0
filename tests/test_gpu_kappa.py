"""sfg_kappa (Sec. 2.2, Eq. eqn:ineq) on the GPU against the oracle's kappa.

Small graphs: the Krylov dimension reaches n - (components), so the GPU Lanczos is exact up to
FP64 rounding and must match the dense generalised eigensolve to 1e-7. Mid-size graphs: 200 steps
against the oracle's ARPACK value, within the 5% kappa bar (the extreme Ritz values are reported).
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


def _setup(S, ctx, spec):
    n, u, v, w = spec
    og = O.canonicalize(n, u, v, w)
    g = S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w))
    return og, g


SMALL = {
    "grid": lambda: gen.grid2d(20, 25, seed=3),
    "random": lambda: gen.random_graph(300, 1200, seed=4),
    "disconnected": lambda: gen.random_graph(250, 420, seed=6, connected=False),
    "knn": lambda: gen.knn3d(400, k=8, seed=7),
}


@pytest.mark.parametrize("name", sorted(SMALL))
def test_kappa_small_exact(S, ctx, name):
    og, g = _setup(S, ctx, SMALL[name]())
    tree = O.mst(og)
    spars, _ = O.sparsify(og, K=8, steps=10, budget_frac=0.1, budget_unit=1, seed=2)
    for mask in (tree, spars):
        ref = O.kappa_dense(og, mask)
        k, lmin, lmax, info = S.sfg_kappa(ctx, g, dev(mask.astype(np.uint8)), steps=5000, seed=3,
                                          info=True)
        assert abs(k - ref) <= 1e-7 * ref, (name, k, ref, info)
        assert lmin >= 1.0 - 1e-9 and abs(lmax / lmin - k) <= 1e-12 * k


def test_kappa_closed_forms(S, ctx):
    # P = G: kappa = 1
    og, g = _setup(S, ctx, gen.grid2d(12, 9, seed=1))
    k, _, _ = S.sfg_kappa(ctx, g, torch.ones(g.m, dtype=torch.uint8, device=DEV), steps=500)
    assert abs(k - 1.0) <= 1e-10
    # unit cycle minus one edge: kappa = n
    n = 37
    u = np.arange(n, dtype=np.int32)
    v = ((u + 1) % n).astype(np.int32)
    og, g = _setup(S, ctx, (n, u, v, np.ones(n, np.float32)))
    mask = np.ones(og.m, np.uint8)
    mask[5] = 0
    k, _, _ = S.sfg_kappa(ctx, g, dev(mask), steps=500)
    assert abs(k - n) <= 1e-9 * n
    # P misses a component's spanning edge: kappa is infinite
    og, g = _setup(S, ctx, gen.grid2d(6, 6, seed=2))
    tree = O.mst(og).astype(np.uint8)
    tree[np.nonzero(tree)[0][0]] = 0
    k, _, _ = S.sfg_kappa(ctx, g, dev(tree), steps=50)
    assert k == float("inf")


def test_kappa_deterministic(S, ctx):
    og, g = _setup(S, ctx, gen.grid2d(40, 40, seed=5))
    mask, _ = S.sfg_sparsify(ctx, g, K=8, steps=10, seed=5, budget_frac=0.05, budget_unit=0)
    a = S.sfg_kappa(ctx, g, mask, steps=100, seed=9)
    b = S.sfg_kappa(ctx, g, mask, steps=100, seed=9)
    assert a == b


MID = {
    "grid3d_20": lambda: gen.grid3d(20, seed=2),
    "grid2d_160": lambda: gen.grid2d(160, 160, seed=8),
    "power_grid": lambda: gen.power_grid(120, seed=4),
}


@pytest.mark.parametrize("name", sorted(MID))
def test_kappa_midsize_lanczos(S, ctx, name):
    og, g = _setup(S, ctx, MID[name]())
    mask, _ = S.sfg_sparsify(ctx, g, K=16, steps=20, seed=11, budget_frac=0.05, budget_unit=0)
    m = mask.cpu().numpy()
    ref = O.kappa_lanczos(og, m)
    k, lmin, lmax, info = S.sfg_kappa(ctx, g, mask, steps=200, seed=1, info=True)
    print(f"\nKAPPA {name}: n={og.n} gpu={k:.6g} (lmin {lmin:.6g}, lmax {lmax:.6g}) oracle={ref:.6g}"
          f" {info}")
    assert abs(k - ref) <= 0.05 * ref


@pytest.mark.parametrize("spec", ["grid", "knn"])
def test_sparsify_to_kappa_matches_oracle(S, ctx, spec):
    n, u, v, w = gen.grid2d(28, 28, seed=5) if spec == "grid" else gen.knn3d(700, k=8, seed=9)
    og = O.canonicalize(n, u, v, w)
    g = S.sfg_laplacian(ctx, n, dev(u), dev(v), dev(w))
    k0 = O.kappa_dense(og, O.mst(og))
    target = k0 / 4.0
    om, otrace, orounds = O.sparsify_to_kappa(og, target, batch_frac=0.02, max_rounds=15, K=8,
                                              steps=10, seed=3)
    gm, ns, gtrace, grounds = S.sfg_sparsify_to_kappa(ctx, g, target, batch_frac=0.02, max_rounds=15,
                                                      kappa_steps=5000, K=8, steps=10, seed=3)
    print(f"\nTO_KAPPA {spec}: target {target:.4g}; oracle rounds {orounds} trace "
          f"{[round(x, 3) for x in otrace]}; gpu rounds {grounds} trace {[round(x, 3) for x in gtrace]}")
    assert abs(gtrace[0] - otrace[0]) <= 1e-7 * otrace[0]       # the spanning tree is bit-exact
    assert abs(grounds - orounds) <= 1
    assert gtrace[-1] <= target and ns == int(gm.sum().item())
    # same schedule: each round brings P to the same size
    assert ns - int(O.mst(og).sum()) == int(np.floor(grounds * 0.02 * n + 0.5))
    # the GPU's own kappa of its final P equals the dense oracle's
    assert abs(gtrace[-1] - O.kappa_dense(og, gm.cpu().numpy())) <= 1e-7 * gtrace[-1]
    # and each GPU round's kappa is within the 5% kappa bar of the oracle's at the same round
    for a, b in zip(gtrace, otrace):
        assert abs(a - b) <= 0.05 * b
