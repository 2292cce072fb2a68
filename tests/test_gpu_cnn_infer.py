"""Tensor-core inference of the closure CNN (BF16 activations, FP32 accumulation)
against the FP64 oracle, within the rounding bound of tests/cnn_bound.py."""
import numpy as np
import pytest

from oracle import cnn_oracle as N
from paper_2101_04847_gb300 import lbm
from tests.cnn_bound import bf16_activation_bound
from tests.test_gpu_closure import oracle_view

pytestmark = pytest.mark.gpu


def _params(seed):
    rng = np.random.default_rng(seed)
    p32 = N.init_params(seed).astype(np.float32)
    p32[1152:1184] = rng.normal(0, 0.1, 32)        # nonzero biases exercise the epilogue
    p32[10400:10432] = rng.normal(0, 0.1, 32)
    p32[-4:] = rng.normal(0, 0.1, 4)
    return p32


def _run(nx, ny, p32, x, mode="infer"):
    import torch

    cnn = lbm.Cnn(nx, ny)
    dp = torch.from_numpy(p32).cuda()
    dx = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    dy = torch.full_like(dx, float("nan"))
    getattr(cnn, mode)(dp, dx, dy)
    cnn.status()
    return dy.double().cpu().numpy()


def flip_effect(q):
    """Largest change of one output when one stored hidden activation a lands on the
    other BF16 neighbour of its exact value (a rounding decision that FP32 and FP64
    pre-rounding values take differently): one spacing 2^-7 |a| at most, carried to
    the output by at most sum_c2 (sum_t3 |w3|) (max_t2 |w2|) for a layer-1 value."""
    w1, _, w2, _, w3, _ = [t.numpy() for t in N.unpack(q)]
    g1 = np.max(np.einsum("ock,cd->od", np.abs(w3).reshape(4, 32, 9),
                          np.abs(w2).reshape(32, 32, 9).max(axis=2)))
    return g1, float(np.max(np.abs(w3)))


def check_against_oracle(got, q, x):
    """got: the tensor-core result.  Every output within the worst-case rounding
    bound of the exact network; against the oracle's BF16-activation network,
    at most 5 % of the outputs off by more than 1e-5 of the largest (rounding
    flips) and none by more than one flip's effect."""
    f = N.forward_bf16_activations(q, x)
    emu = f["y"].numpy()
    ref, bound = bf16_activation_bound(q, x)
    scale = np.max(np.abs(ref))
    assert np.all(np.isfinite(got))
    assert np.all(np.abs(got - ref) <= bound + 1e-7 * scale), float(np.max(np.abs(got - ref) - bound))
    d = np.abs(got - emu)
    g1, w3max = flip_effect(q)
    one_flip = 2.0 ** -7 * (float(f["a1"].abs().max()) * g1 + float(f["a2"].abs().max()) * w3max)
    assert np.mean(d > 1e-5 * scale) <= 0.05, float(np.mean(d > 1e-5 * scale))
    assert np.max(d) <= one_flip + 1e-5 * scale, (float(np.max(d)), one_flip)
    return d / scale


# single strips (nx < 128, exactly 128), several strips with a ragged last one,
# a one-column grid (x neighbours are the column itself) and one-row bands.
# Measured: median |got - emu| ~2e-8 of the largest output, at most 1.2 % of the
# outputs beyond 1e-5, the largest 6.4e-4 (a one-flip bound is ~1e-2).
@pytest.mark.parametrize("nx,ny", [(24, 40), (37, 19), (128, 9), (300, 70), (1, 12), (261, 3)])
def test_infer_matches_the_oracle(gpu, nx, ny):
    p32 = _params(nx + ny)
    x = np.random.default_rng(nx * ny).normal(size=(4, ny, nx)).astype(np.float32)
    got = _run(nx, ny, p32, x)
    rel = check_against_oracle(got, oracle_view(p32), x.astype(np.float64))
    assert np.median(rel) < 1e-6


def test_infer_is_deterministic_and_close_to_the_fp32_path(gpu):
    nx, ny = 300, 70
    p32 = _params(5)
    x = np.random.default_rng(6).normal(size=(4, ny, nx)).astype(np.float32)
    a = _run(nx, ny, p32, x)
    b = _run(nx, ny, p32, x)
    assert np.array_equal(a, b)
    f = _run(nx, ny, p32, x, mode="forward")
    ref, bound = bf16_activation_bound(oracle_view(p32), x.astype(np.float64))
    assert np.max(np.abs(f - ref)) <= 1e-5 * np.max(np.abs(ref))        # FP32 activations
    assert np.all(np.abs(a - f) <= bound + 1e-5 * np.max(np.abs(ref)))


def test_infer_full_size_sampled(gpu):
    # the closure's coarse grid of the 10000x5000 run: 5000 x 2500, in the launch
    # configuration the bench times; windows at the walls, the periodic seam and inside
    nx, ny = 5000, 2500
    p32 = _params(11)
    rng = np.random.default_rng(12)
    x = rng.normal(size=(4, ny, nx)).astype(np.float32)
    got = _run(nx, ny, p32, x)
    q = oracle_view(p32)
    w, halo = 24, 3                                 # outputs per window, receptive-field radius
    for (ya, xa) in [(0, 0), (0, nx - 20), (ny - w, 4990), (1250, 2500), (777, 127), (ny - w, 1000)]:
        rows = np.arange(ya - halo, ya + w + halo)
        cols = np.arange(xa - halo, xa + w + halo) % nx
        keep = (rows >= 0) & (rows < ny)            # beyond the walls: the oracle's zero padding
        crop = x[:, rows[keep]][:, :, cols].astype(np.float64)
        r0 = halo if ya - halo >= 0 else ya         # first output row of the window in the crop
        g = got[:, ya:ya + w][:, :, (np.arange(xa, xa + w) % nx)]
        # the oracle on the crop is exact away from the crop's own edges
        f = N.forward_bf16_activations(q, crop)
        emu = f["y"].numpy()[:, r0:r0 + w, halo:halo + w]
        ref, bound = bf16_activation_bound(q, crop)
        ref, bound = ref[:, r0:r0 + w, halo:halo + w], bound[:, r0:r0 + w, halo:halo + w]
        scale = np.max(np.abs(ref))
        g1, w3max = flip_effect(q)
        one_flip = 2.0 ** -7 * (float(f["a1"].abs().max()) * g1 + float(f["a2"].abs().max()) * w3max)
        assert np.all(np.abs(g - ref) <= bound + 1e-7 * scale), (ya, xa)
        assert np.mean(np.abs(g - emu) > 1e-5 * scale) <= 0.05, (ya, xa)
        assert np.max(np.abs(g - emu)) <= one_flip + 1e-5 * scale, (ya, xa)


def test_a_wait_that_gives_up_is_reported_and_the_context_stays_usable(gpu):
    # the kernels' copies are withheld: every wait gives up after a few thousand
    # polls, the status word is raised and read on the host; a normal call after it
    # runs and is correct
    import torch

    nx, ny = 300, 70
    p32 = _params(5)
    x = np.random.default_rng(6).normal(size=(4, ny, nx)).astype(np.float32)
    cnn = lbm.Cnn(nx, ny)
    dp = torch.from_numpy(p32).cuda()
    dx = torch.from_numpy(x).cuda()
    dy = torch.zeros_like(dx)
    cnn.infer_test_timeout(dp, dx, dy)
    with pytest.raises(lbm.LbmError) as err:
        cnn.status()
    assert err.value.status == lbm.LBM_ETIMEOUT
    cnn.infer(dp, dx, dy)
    cnn.status()
    check_against_oracle(dy.double().cpu().numpy(), oracle_view(p32), x.astype(np.float64))
