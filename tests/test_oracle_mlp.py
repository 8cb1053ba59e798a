"""Pins for the degree-MLP reference: central finite differences,
special cases with a closed form, and one Adam step."""
import numpy as np

from oracle import mlp


def data(B=17, seed=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.standard_normal((B, mlp.N_FEAT))
    t = rng.uniform(0.1, 1.0, B)
    return x, t


def test_gradients_match_central_differences():
    p = mlp.init_params(1)
    for k in p:
        p[k] = p[k] + 0.1 * np.random.Generator(np.random.PCG64(2)).standard_normal(p[k].shape)
    x, t = data()
    _, g = mlp.loss_and_grads(p, x, t)
    h = 1e-6
    rng = np.random.Generator(np.random.PCG64(4))
    for k in p:
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in p[k].shape)
            p2 = {a: b.copy() for a, b in p.items()}
            p2[k][idx] += h
            lp, _ = mlp.loss_and_grads(p2, x, t)
            p2[k][idx] -= 2 * h
            lm, _ = mlp.loss_and_grads(p2, x, t)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[k][idx]) <= 1e-7 + 1e-5 * abs(fd), (k, idx)


def test_zero_output_layer_is_bias():
    p = mlp.init_params(2)
    p["W3"][:] = 0.0
    p["b3"][:] = 0.25
    x, t = data()
    y, _ = mlp.forward(p, x)
    assert np.allclose(y, 0.25)
    _, g = mlp.loss_and_grads(p, x, t)
    assert np.isclose(g["b3"][0], np.mean(0.25 - t))
    assert np.allclose(g["W1"], 0.0) and np.allclose(g["W2"], 0.0)


def test_first_adam_step_is_signed_lr():
    p = mlp.init_params(3)
    x, t = data()
    _, g = mlp.loss_and_grads(p, x, t)
    p0 = {k: v.copy() for k, v in p.items()}
    mlp.adam_step(p, g, {}, lr=1e-3)
    for k in p:
        big = np.abs(g[k]) > 1e-4
        assert np.allclose((p[k] - p0[k])[big], -1e-3 * np.sign(g[k][big]), rtol=1e-3)


def test_features_and_labels():
    x = mlp.features([-2.0, 0.5], [1e-4, 1e-2], 1.0, 2.0, -3.0, 7)
    assert np.allclose(x[0], [-1.5, -0.4, np.arccosh(1.5), -2.0, 0.7])
    assert x[1, 2] == 0.0
    # the step feature saturates at the tenth problem of a sequence
    assert mlp.features([-2.0], [1e-4], 1.0, 2.0, -3.0, 25)[0, 4] == 0.9
    # t = -2: acosh 2 = 1.316958; residual 1e-2 -> 1e-6 in 10 degrees gives
    # kappa = ln(1e4)/10 = 0.921034, ratio 0.699364
    y = mlp.decay_label([-3.0], [1e-2], [1e-6], [10], 1.0, 2.0)
    assert abs(y[0] - 0.921034037 / 1.316957897) < 1e-8
    assert mlp.decay_label([-3.0], [1e-2], [1e-2], [10], 1.0, 2.0)[0] == mlp.Y_LO
    # degree from the ratio: ln(1e-2/1e-10) / (1.316958 * 0.5) = 27.98 -> 28 + 2
    m = mlp.degrees_from_prediction([0.5], [-3.0], [1e-2], 1.0, 2.0, 1e-10, extra=2)
    assert m[0] == 30
    # a ratio of 1 reproduces the analytic rule (with the same margin)
    import oracle
    mr = oracle.degree_rule(np.array([-3.0]), np.array([1e-2]), 1.0, 2.0, 1e-10, 60, deg_extra=2)
    assert mlp.degrees_from_prediction([1.0], [-3.0], [1e-2], 1.0, 2.0, 1e-10, extra=2)[0] == mr[0]
    # inside the damped interval -> the cap; tiny residual -> the floor
    assert mlp.degrees_from_prediction([1.0], [2.0], [1e-2], 1.0, 2.0, 1e-10)[0] == mlp.DEG_HI
    assert mlp.degrees_from_prediction([1.0], [-3.0], [1e-12], 1.0, 2.0, 1e-10)[0] == mlp.DEG_LO
