"""Pins of the selector oracle (oracle/selector.py) against facts that do not
come from its own code: central finite differences of the loss, a network
whose output is a constant (closed-form loss and gradient), Adam's first step
(closed form: a step of lr against the sign of the gradient), and the FP16
rounding of the parameters."""
import numpy as np

from oracle import selector as S
from paper_2004_14229_gb300.workloads import selector_init


def _data(n=40, seed=0):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, (n, 4)), rng.uniform(-1, 1, (n, 2))


def test_parameter_count_and_layout():
    assert S.N_PARAMS == 8770
    th = np.arange(S.N_PARAMS, dtype=np.float64)
    (W1, b1), (W2, b2), (W3, b3), (W4, b4) = S.unpack(th)
    assert W1.shape == (64, 4) and W1[1, 0] == 4 and b1[0] == 256
    assert W2[0, 0] == 320 and b2[0] == 320 + 4096
    assert W4.shape == (2, 64) and b4[-1] == S.N_PARAMS - 1


def test_gradient_matches_finite_differences():
    x, t = _data()
    th = selector_init(3).astype(np.float64)
    th += np.random.default_rng(1).normal(0, 0.05, th.size)   # non-zero biases too
    _, g = S.loss_and_grad(th, x, t, fp16=False)
    rng = np.random.default_rng(2)
    idx = np.concatenate([rng.choice(S.N_PARAMS, 60, replace=False),
                          [0, 255, 256, 319, 320, 4415, 4416, 8639, 8640, 8767, 8768, 8769]])
    h = 1e-6
    for i in idx:
        e = np.zeros(S.N_PARAMS)
        e[i] = h
        fd = (S.loss_and_grad(th + e, x, t, fp16=False)[0] - S.loss_and_grad(th - e, x, t, fp16=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_constant_output_network_closed_form():
    x, t = _data(25, 4)
    th = selector_init(5).astype(np.float64)
    (_, _), (_, _), (_, _), (W4, b4) = S.unpack(th)
    W4[:] = 0.0
    b4[:] = [0.75, -0.5]        # exact in FP16
    y, acts = S.forward(th, x)
    assert np.all(y == b4)
    L, g = S.loss_and_grad(th, x, t)
    r = b4 - t
    assert np.isclose(L, 0.5 * np.mean(np.sum(r * r, axis=1)), rtol=1e-14)
    assert np.allclose(g[-2:], r.mean(axis=0), rtol=1e-13)
    gW4 = g[8640:8768].reshape(2, 64)
    assert np.allclose(gW4, r.T @ acts[2] / x.shape[0], rtol=1e-12)
    assert np.all(g[:8640] == 0.0)             # W4 = 0 blocks every earlier gradient


def test_adam_first_step_closed_form():
    x, t = _data(16, 6)
    th = selector_init(8).astype(np.float64)
    _, g = S.loss_and_grad(th, x, t)
    th1, losses = S.adam_train(th, x, t, epochs=1, lr=1e-2)
    assert np.allclose(th1, th - 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert losses.shape == (1,)


def test_fp16_rounding_of_parameters():
    x, _ = _data(10, 9)
    th = selector_init(10).astype(np.float64) * 1.2345
    y16, _ = S.forward(th, x, fp16=True)
    yr, _ = S.forward(th.astype(np.float16).astype(np.float64), x, fp16=False)
    assert np.array_equal(y16, yr)
    y64, _ = S.forward(th, x, fp16=False)
    assert not np.array_equal(y16, y64)


def test_training_decreases_loss():
    x, _ = _data(64, 11)
    t = np.stack([0.3 * x[:, 0] - 0.2 * x[:, 1] ** 2, np.tanh(x[:, 2] + x[:, 3])], axis=1)
    _, losses = S.adam_train(selector_init(12), x, t, epochs=60, lr=3e-3)
    assert losses[-1] < 0.3 * losses[0]
