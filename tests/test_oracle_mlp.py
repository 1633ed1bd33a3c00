"""Pins for the FP64 reference of the initial-guess network: the hand-written
backward pass must equal central finite differences of the loss."""
import numpy as np

from oracle import mlp


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    theta = mlp.init_params(3) + rng.normal(0, 0.05, mlp.N_PARAMS)
    x = rng.normal(size=(9, mlp.N_IN))
    t = rng.normal(size=9)
    L, g = mlp.loss_and_grad(theta, x, t)
    idx = rng.choice(mlp.N_PARAMS, 80, replace=False)
    idx = np.concatenate([idx, [0, 383, 384, 447, 448, 4543, 4544, 4607, 4608, 4671, 4672]])
    h = 1e-6
    for k in idx:
        e = np.zeros(mlp.N_PARAMS)
        e[k] = h
        Lp, _ = mlp.loss_and_grad(theta + e, x, t)
        Lm, _ = mlp.loss_and_grad(theta - e, x, t)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(fd)), (k, fd, g[k])


def test_forward_of_a_hand_built_network():
    # zero weights except a single path: y = w3 * tanh(w2 * tanh(w1 * x0))
    theta = np.zeros(mlp.N_PARAMS)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(theta)
    W1 = W1.copy(); W2 = W2.copy(); W3 = W3.copy(); b3 = b3.copy()
    W1[5, 0] = 0.7
    W2[2, 5] = -1.3
    W3[2] = 2.0
    b3[0] = 0.25
    th = mlp.pack([W1, b1, W2, b2, W3, b3])
    x = np.array([[0.4, 9, 9, 9, 9, 9]])
    y, _ = mlp.forward(th, x)
    assert abs(y[0] - (0.25 + 2.0 * np.tanh(-1.3 * np.tanh(0.7 * 0.4)))) < 1e-15


def test_parameter_count_matches_library_blob():
    # library blob = parameters + mean[6] + scale[6] + output scale and shift
    assert mlp.N_PARAMS + 6 + 6 + 2 == 4687
