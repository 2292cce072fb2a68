"""Pins of the FP64 CNN oracle of the learned closure (no GPU): the padding
convention against shifted copies, and the analytic gradient against central
finite differences."""
import numpy as np
import torch

from oracle import cnn_oracle as N


def test_parameter_count():
    assert N.N_PARAMS == 32 * 4 * 9 + 32 + 32 * 32 * 9 + 32 + 4 * 32 * 9 + 4 == 11588


def test_convolution_is_a_periodic_x_zero_y_cross_correlation():
    rng = np.random.default_rng(0)
    a = torch.tensor(rng.normal(size=(2, 5, 7)))
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            w = torch.zeros(2, 2, 3, 3, dtype=torch.float64)
            w[0, 0, dy + 1, dx + 1] = 1.0
            w[1, 1, dy + 1, dx + 1] = 2.0
            out = N.conv(a, w, torch.zeros(2, dtype=torch.float64))
            shifted = np.roll(a.numpy(), -dx, axis=2)          # value at x + dx (periodic)
            want = np.zeros_like(shifted)
            for y in range(5):
                if 0 <= y + dy < 5:
                    want[:, y] = shifted[:, y + dy]             # zero beyond the walls
            assert np.allclose(out.numpy(), want * np.array([1.0, 2.0])[:, None, None])


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(4)
    p = N.init_params(1)
    p[N.N_PARAMS - 4:] = rng.normal(0, 0.1, 4)            # non-zero output biases
    x = rng.normal(size=(4, 6, 8))
    t = rng.normal(size=(4, 6, 8))
    L, g = N.loss_and_grad(p, x, t)
    assert np.isclose(L, N.loss(p, x, t), rtol=1e-14)
    idx = np.concatenate([rng.choice(N.N_PARAMS, 60, replace=False), np.arange(N.N_PARAMS - 4, N.N_PARAMS)])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (N.loss(p + e, x, t) - N.loss(p - e, x, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) * max(abs(L), 1e-3), (i, fd, g[i])
