"""Pins for the oracle's MLP cost model, Adam step and regret (CPU only)."""
import numpy as np

NP = 8705
H = 64
OFF_W1, OFF_B1 = 0, 256
OFF_W2, OFF_B2 = 320, 4416
OFF_W3, OFF_B3 = 4480, 8576
OFF_W4, OFF_B4 = 8640, 8704


def rand_params(seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, NP)


def test_layout_size():
    assert OFF_B4 + 1 == NP == 64 * 4 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 64 + 1


def test_forward_in_the_positive_regime_is_a_matrix_product(orc):
    # With non-negative weights, biases and inputs every ReLU is the identity,
    # so the network is the plain product W4 W3 W2 W1 x + (folded biases).
    rng = np.random.default_rng(1)
    p = rng.uniform(0.0, 0.2, NP)
    x = rng.uniform(0.0, 1.0, (7, 4))
    W1 = p[OFF_W1:OFF_B1].reshape(64, 4)
    W2 = p[OFF_W2:OFF_B2].reshape(64, 64)
    W3 = p[OFF_W3:OFF_B3].reshape(64, 64)
    W4 = p[OFF_W4:OFF_B4]
    h = x @ W1.T + p[OFF_B1:OFF_W2]
    h = h @ W2.T + p[OFF_B2:OFF_W3]
    h = h @ W3.T + p[OFF_B3:OFF_W4]
    y = h @ W4 + p[OFF_B4]
    assert np.allclose(orc.mlp_forward(p, x), y, rtol=1e-13, atol=0)


def test_loss_of_a_constant_network(orc):
    p = np.zeros(NP)
    p[OFF_B4] = 0.5
    x = np.random.default_rng(2).uniform(size=(10, 4))
    t = np.linspace(-1, 1, 10)
    loss, g = orc.mlp_loss_grad(p, x, t)
    assert abs(loss - np.mean((0.5 - t) ** 2)) < 1e-15
    assert abs(g[OFF_B4] - 2 * np.mean(0.5 - t)) < 1e-15
    assert np.count_nonzero(g[:OFF_B4]) == 0


def test_gradient_matches_central_differences(orc):
    rng = np.random.default_rng(3)
    p = rand_params(3)
    x = rng.uniform(0, 1, (16, 4))
    t = rng.uniform(-1, 1, 16)
    loss, g = orc.mlp_loss_grad(p, x, t)
    idx = np.concatenate([rng.choice(NP, 300, replace=False), np.arange(OFF_W4, NP)])
    h = 1e-6
    for i in idx:
        pp = p.copy()
        pp[i] += h
        lp, _ = orc.mlp_loss_grad(pp, x, t)
        pp[i] -= 2 * h
        lm, _ = orc.mlp_loss_grad(pp, x, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_first_adam_step_is_lr_times_sign(orc):
    # With m = v = 0 and bias correction, step 1 moves each parameter by
    # lr * g / (|g| + eps), i.e. lr * sign(g) up to eps.
    rng = np.random.default_rng(4)
    p = rand_params(4)
    g = rng.uniform(-1, 1, NP)
    m = np.zeros(NP)
    v = np.zeros(NP)
    p0 = p.copy()
    orc.adam_step(p, g, m, v, 1, lr=1e-3)
    assert np.allclose(p0 - p, 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=1e-15)
    assert np.all(np.sign(p0 - p) == np.sign(g))
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_regret_hand_table(orc):
    times = np.array([[1.0, 2.0, 3.0], [4.0, 2.0, 8.0], [5.0, 5.0, 6.0]])
    r = orc.regret(times, np.array([0, 2, 1]))
    assert np.array_equal(r, [0.0, 3.0, 0.0])
