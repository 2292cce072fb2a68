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


def test_bf16_activation_forward_against_the_exact_network():
    # the BF16-activation network stays within the worst-case rounding bound of the
    # exact one, differs from it (the roundings happen), and a plausible mistake in
    # the middle layer (a dropped tap, transposed channels) moves most outputs by far
    # more than the 1e-5 the GPU comparison allows off the rounding-flip cases
    from tests.cnn_bound import bf16_activation_bound

    rng = np.random.default_rng(3)
    p = N.init_params(4)
    p[1152:1184] = rng.normal(0, 0.1, 32)
    for off, n in ((0, 1152), (1184, 9216), (10432, 1152)):
        p[off:off + n] = N.round_bf16(torch.tensor(p[off:off + n])).numpy()
    x = rng.normal(size=(4, 12, 20))
    ref, bound = bf16_activation_bound(p, x)
    emu = N.forward_bf16_activations(p, x)
    y = emu["y"].numpy()
    assert np.all(np.abs(y - ref) <= bound)
    assert np.max(np.abs(y - ref)) > 1e-3 * np.max(np.abs(ref))
    # rounding is idempotent: the stored activations are BF16 values
    assert torch.equal(N.round_bf16(emu["a1"]), emu["a1"])
    for mistake in ("dropped tap", "transposed"):
        q = p.copy()
        w = q[1184:1184 + 9216].reshape(32, 32, 3, 3)
        if mistake == "dropped tap":
            w[:, :, 0, 2] = 0.0
        else:
            w[:] = w.transpose(1, 0, 2, 3).copy()
        bad = N.forward_bf16_activations(q, x)["y"].numpy()
        assert np.mean(np.abs(bad - y) > 1e-5 * np.max(np.abs(y))) > 0.5, mistake


def test_bf16_unit_roundoff_of_the_bound():
    # the bound's unit roundoff covers every relative rounding error of round_bf16
    # and is not loose by a factor 2: 8 significant bits round to within 2^-8, and
    # values just below a tie come close to it
    from tests.cnn_bound import U_BF16

    v = np.random.default_rng(9).uniform(-300.0, 300.0, 200000)
    rel = np.abs(N.round_bf16(torch.tensor(v)).numpy() - v) / np.abs(v)
    assert rel.max() <= U_BF16
    assert rel.max() > 0.75 * U_BF16


def test_round_bf16_against_hand_values():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: to even (1); 1 + 3 * 2^-8 rounds up
    # to 1 + 2^-6 (even); 2^-7 spacing at 1; values already BF16 stay
    v = torch.tensor([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, -3.0, 0.0, 1.5 + 2.0 ** -7])
    want = [1.0, 1.0, 1.0 + 2.0 ** -6, 1.0, -3.0, 0.0, 1.5 + 2.0 ** -7]
    assert N.round_bf16(v).tolist() == want
