"""Pins of the oracle's learned-proposal restatement (CPU): its limiting cases reduce to the plain
flat method and to plain top-k selection, which are pinned elsewhere."""
import numpy as np

import oracle as O
from oracle import mlp as M
from paper_2008_07633_gb300 import inputs as gen


def test_learned_with_all_proposals_is_the_plain_method():
    # proposing every candidate makes the network irrelevant: the result is the plain flat method
    og = O.canonicalize(*gen.grid2d(20, 20, seed=2))
    theta = M.init_params(5)
    st = M.learned_stages(og, theta, K=8, steps=10, feat_steps=2, propose_frac=1.0, seed=3,
                          budget_frac=0.05)
    plain, _ = O.sparsify(og, K=8, steps=10, levels=0, seed=3, budget_frac=0.05, budget_unit=0)
    assert st["nprop"] == st["cand"].size
    assert np.array_equal(st["mask"], plain)


def test_learned_stage_invariants():
    og = O.canonicalize(*gen.knn3d(600, k=8, seed=4))
    theta = M.init_params(9)
    st = M.learned_stages(og, theta, K=8, steps=10, feat_steps=2, propose_frac=0.2, seed=7,
                          budget_frac=0.05)
    k, prop, pred, cand = st["k"], st["prop"], st["pred"], st["cand"]
    assert st["nprop"] == max(k, int(np.floor(0.2 * cand.size + 0.5)))
    # proposals: exactly the top-nprop predictions (score desc, id asc), ascending ids
    order = sorted(range(cand.size), key=lambda i: (-pred[i], cand[i]))
    assert np.array_equal(prop, np.sort(cand[order[:st["nprop"]]]))
    # selection: the top-k rescored proposals, all off-forest, joined to the forest
    order2 = sorted(range(prop.size), key=lambda i: (-st["scores"][i], prop[i]))
    assert np.array_equal(st["sel"], np.sort(prop[order2[:k]]))
    assert int(st["mask"].sum()) == int(st["forest"].sum()) + k
    assert np.all(st["forest"][st["sel"]] == 0)
    # the rescoring step is the plain scorer on the plain embeddings of G and P
    ref = O.score_edges(og, O.smooth(og, 8, 10, 0.7, 7),
                        O.smooth(og.subgraph(st["forest"]), 8, 10, 0.7, 7), prop)
    assert np.array_equal(st["scores"], ref)


def test_learned_minimum_proposals_is_the_budget():
    og = O.canonicalize(*gen.grid2d(16, 16, seed=5))
    st = M.learned_stages(og, M.init_params(1), K=8, steps=5, feat_steps=2, propose_frac=1e-6,
                          seed=2, budget_frac=0.05)
    assert st["nprop"] == st["k"]
    assert np.array_equal(np.sort(st["sel"]), st["prop"])   # every proposal is kept
