"""Pins of the MLP oracle (the learned edge-proposal scorer): central finite differences pin the
analytic gradients, the generator pins the initial weights, hand-made inputs pin the features."""
import numpy as np

import oracle.mlp as M


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = M.init_params(5) + 0.05 * rng.standard_normal(M.NPARAM)
    X = rng.standard_normal((40, M.F))
    X[:, 8:] = 0.0
    t = rng.standard_normal(40)
    g, L = M.grad(theta, X, t)
    assert abs(L - M.loss(theta, X, t)) < 1e-12
    h = 1e-6
    idx = np.concatenate([rng.choice(M.NPARAM, 300, replace=False), [M.NPARAM - 1]])
    for j in idx:
        e = np.zeros(M.NPARAM)
        e[j] = h
        fd = (M.loss(theta + e, X, t) - M.loss(theta - e, X, t)) / (2 * h)
        assert abs(fd - g[j]) <= 1e-7 + 1e-6 * abs(fd), (j, fd, g[j])


def test_init_is_kaiming_uniform_and_zero_bias():
    theta = M.init_params(123)
    p = M.unflatten(theta)
    assert M.NPARAM == 5313
    for name, fan in (("W1", 16), ("W2", 64), ("w3", 64)):
        b = np.sqrt(6.0 / fan)
        assert np.all(np.abs(p[name]) <= b)
        assert abs(np.std(p[name]) - b / np.sqrt(3)) < 0.1 * b
    for name in ("b1", "b2", "b3"):
        assert np.all(p[name] == 0)
    assert not np.array_equal(M.init_params(124), theta)


def test_features_definition_on_hand_inputs():
    X = M.features([2.0], [3.0], [5.0], [4], [7], [0.5], [8.0])
    e = np.e
    assert np.allclose(X[0, :8], [np.log(2), np.log(15), np.log(5 / 3), np.log(0.5), np.log(8.0),
                                  np.log(8.0) - np.log(0.5), np.log(28), np.log(8.5)])
    assert np.all(X[0, 8:] == 0)
    del e


def test_adam_moves_against_the_gradient_and_reduces_loss():
    rng = np.random.default_rng(1)
    theta = M.init_params(9)
    X = rng.standard_normal((256, M.F))
    X[:, 8:] = 0
    t = X[:, 0] - 0.5 * X[:, 3]
    m = np.zeros(M.NPARAM)
    v = np.zeros(M.NPARAM)
    L0 = M.loss(theta, X, t)
    for step in range(1, 201):
        g, _ = M.grad(theta, X, t)
        theta, m, v = M.adam_step(theta, m, v, g, step, lr=3e-3)
    assert M.loss(theta, X, t) < 0.2 * L0


def test_bf16_rounding_is_round_to_nearest_even():
    import numpy as np
    import oracle.mlp as M

    # exact BF16 numbers stay, halfway cases go to the even neighbour, others to the nearest
    one = 1.0
    ulp = 2.0 ** -7                      # BF16 spacing in [1, 2)
    xs = np.array([one, one + ulp / 2, one + 3 * ulp / 2, one + ulp / 4, -(one + 3 * ulp / 2), 0.0])
    ref = np.array([one, one, one + 2 * ulp, one, -(one + 2 * ulp), 0.0])
    assert np.array_equal(M.round_bf16(xs), ref)
    # the kernel-precision forward equals the exact forward when every rounded value is exact
    th = np.zeros(M.NPARAM)
    p = M.unflatten(th)
    p["W1"][0, 0], p["W2"][0, 0], p["w3"][0], p["b3"][0] = 2.0, 0.5, 3.0, 0.25
    th = M.flatten(p)
    X = np.zeros((3, 16))
    X[:, 0] = [1.0, -1.0, 4.0]
    assert np.allclose(M.forward_kernel_precision(th, X), M.forward(th, X)[0])
