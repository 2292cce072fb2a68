"""Learned closure (GPU): the CNN kernels against the FP64 oracle, and what the
trained network gains over the coarse run without it."""
import ctypes as C

import numpy as np
import pytest

from oracle import closure_oracle as K
from oracle import cnn_oracle as N
from oracle import lbm_oracle as O
from paper_2101_04847_gb300 import lbm
from tests import inputs

pytestmark = pytest.mark.gpu


def bf16_round(a):
    """Round float32 values to bfloat16 (nearest even) and back."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32)


def oracle_view(p32):
    """The parameters the GPU convolutions use: weights in BF16, biases in FP32."""
    q = p32.astype(np.float64).copy()
    for off, n in ((0, 1152), (1184, 9216), (10432, 1152)):
        q[off:off + n] = bf16_round(p32[off:off + n])
    return q


def cnn_call(gpu, p32, x, t=None):
    import torch

    ny, nx = x.shape[1:]
    nbytes = C.c_size_t()
    assert gpu.lbm_cnn_workspace_bytes(nx, ny, C.byref(nbytes)) == 0
    ws = torch.empty(nbytes.value, dtype=torch.uint8, device="cuda")
    dp = torch.from_numpy(p32).cuda()
    dx = torch.from_numpy(x.astype(np.float32)).cuda()
    if t is None:
        dy = torch.empty_like(dx)
        assert gpu.lbm_cnn_forward(C.c_void_p(dp.data_ptr()), C.c_void_p(dx.data_ptr()), nx, ny,
                                   C.c_void_p(ws.data_ptr()), nbytes.value, None, C.c_void_p(dy.data_ptr())) == 0
        torch.cuda.synchronize()
        return dy.double().cpu().numpy()
    dt = torch.from_numpy(t.astype(np.float32)).cuda()
    g = torch.empty_like(dp)
    loss = C.c_double()
    assert gpu.lbm_cnn_loss_grad(C.c_void_p(dp.data_ptr()), C.c_void_p(dx.data_ptr()), C.c_void_p(dt.data_ptr()),
                                 nx, ny, C.c_void_p(ws.data_ptr()), nbytes.value, None, C.byref(loss),
                                 C.c_void_p(g.data_ptr())) == 0
    return loss.value, g.double().cpu().numpy()


@pytest.mark.parametrize("nx,ny", [(24, 40), (37, 19)])
def test_cnn_forward_matches_the_oracle(gpu, nx, ny):
    rng = np.random.default_rng(nx)
    p32 = N.init_params(3).astype(np.float32)
    p32[1152:1184] = rng.normal(0, 0.1, 32)
    x = rng.normal(size=(4, ny, nx)).astype(np.float32)
    got = cnn_call(gpu, p32, x)
    ref = N.forward(oracle_view(p32), x.astype(np.float64))["y"].numpy()
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("nx,ny", [(24, 40), (37, 19)])
def test_cnn_gradient_matches_the_oracle(gpu, nx, ny):
    rng = np.random.default_rng(nx + 1)
    p32 = N.init_params(5).astype(np.float32)
    p32[-4:] = rng.normal(0, 0.1, 4)
    x = rng.normal(size=(4, ny, nx)).astype(np.float32)
    t = rng.normal(size=(4, ny, nx)).astype(np.float32)
    loss, g = cnn_call(gpu, p32, x, t)
    rl, rg = N.loss_and_grad(oracle_view(p32), x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - rl) <= 1e-5 * rl
    # gradients (a sum over pixels of FP32 products) per block of parameters
    for off, n in ((0, 1152), (1152, 32), (1184, 9216), (10400, 32), (10432, 1152), (11584, 4)):
        scale = np.max(np.abs(rg[off:off + n]))
        assert np.max(np.abs(g[off:off + n] - rg[off:off + n])) <= 1e-4 * scale, off


# Equal pure densities: with the 1.0 / 0.9 pair the initial pressure imbalance
# launches an acoustic sloshing mode whose frequency differs on the coarse grid
# (diffusive scaling halves the sound speed), which a one-interval closure cannot
# learn; corrected runs then turn unstable (measured).
FINE = dict(inputs.C0, nx=128, ny=256, mass_B=1.0, g=3e-4, amp=4.0, crop_rows=10)


@pytest.fixture(scope="module")
def trained():
    fine = lbm.default_params(**FINE)
    c = lbm.Closure(fine, interval=10, seed=0)
    c.generate(n_runs=6, seed0=11, warmup=200, intervals=8)
    losses = [c.train(epochs=1, lr=2e-3, shuffle_seed=e) for e in range(25)]
    yield c, losses
    c.close()


def test_training_reduces_the_one_interval_error(gpu, trained):
    # the targets are normalised by their standard deviation: predicting no
    # correction gives a loss of about 1; the trained network must do clearly better
    c, losses = trained
    print("\\nclosure training loss per epoch:", [round(v, 4) for v in losses])
    assert losses[-1] < 0.5 * losses[0]
    assert losses[-1] < 0.6


def _errors(co, fi):
    """Relative errors of the coarse run against the fine run over the series (coarse
    cells are twice as large; energies per mass scale as (dx/dt)^2, i.e. by 4)."""
    out = {}
    for k, scale in (("h", 0.5), ("E_k", 4.0), ("E_p", 4.0), ("L_int", 0.5)):
        f = np.array([d[k] for d in fi]) * scale
        c = np.array([d[k] for d in co])
        out[k] = float(np.sqrt(np.mean((c - f) ** 2)) / max(np.sqrt(np.mean(f ** 2)), 1e-30))
    return out


def test_closure_against_the_coarse_run_without_it(gpu, trained):
    # held-out seed, 12 intervals (480 fine steps); the fine run is the reference
    c, _ = trained
    runs = {mode: c.evaluate(seed=101, warmup=200, intervals=12, use_net=mode) for mode in (0, 2, 3, 4)}
    e = {mode: _errors(*runs[mode]) for mode in runs}
    print("\nheld-out errors vs the fine run: without closure", e[0], " order parameter", e[2],
          " order parameter + velocity / 4", e[3], " on the interface only", e[4])
    # the fine run is identical in all evaluations
    assert [d["E_k"] for d in runs[0][1]] == [d["E_k"] for d in runs[4][1]]
    # the interface-only order-parameter correction with a quarter of the velocity
    # correction improves every measured quantity (measured: h 0.173 -> 0.080, E_k
    # 1.28 -> 0.77, E_p 0.034 -> 0.029, L_int 0.0074 -> 0.0065).  Applied everywhere
    # (modes 2 and 3) the order-parameter correction also moves the bulk compositions
    # and h, which sums c (1 - c) over every row, grows 25-fold (0.17 -> 4.6); E_p
    # and L_int still improve, and E_k with the velocity term.
    for k in ("h", "E_k", "E_p", "L_int"):
        assert e[4][k] < e[0][k], k
    for k in ("E_k", "E_p", "L_int"):
        assert e[3][k] < e[0][k], k
    for k in ("E_p", "L_int"):
        assert e[2][k] < e[0][k], k
    for mode in (2, 3, 4):
        co = runs[mode][0]
        for s in ("mass_A", "mass_B"):
            assert all(abs(d[s] - co[0][s]) <= 1e-5 * co[0][s] for d in co)   # corrections keep the masses
    with pytest.raises(lbm.LbmError):
        c.evaluate(seed=101, warmup=0, intervals=1, use_net=5)


def test_advance_runs_the_corrected_coarse_solver_alone(gpu, trained):
    # production use: the coarse run advanced in corrected intervals, no fine run
    c, _ = trained
    _, co = c.solvers()
    m0 = co.diagnostics()
    n0 = co.step_count
    c.advance(3, 4)
    m1 = co.diagnostics()
    assert co.step_count == n0 + 3 * 10, (n0, co.step_count)
    for s in ("mass_A", "mass_B"):
        assert abs(m1[s] - m0[s]) <= 1e-5 * m0[s], (s, m0[s], m1[s])
    c.advance(2, 0)
    assert co.step_count == n0 + 5 * 10
    fresh = lbm.Closure(lbm.default_params(**FINE), interval=10, seed=0)
    with pytest.raises(lbm.LbmError):
        fresh.advance(1, 4)                      # no trained or set parameters
    fresh.advance(1, 0)
    with pytest.raises(lbm.LbmError):
        fresh.advance(1, 5)
    with pytest.raises(lbm.LbmError):
        fresh.correct(4)                         # no trained or set parameters
    fresh.correct(0)
    with pytest.raises(lbm.LbmError):
        fresh.correct(5)
    fresh.close()


def coarse_oracle_params(c):
    d = lbm.params_dict(c.coarse)
    d = {k: v for k, v in d.items() if k in O.Params.__dataclass_fields__}
    if d["y0"] < 0:
        d["y0"] = None
    return O.Params(**d)


def seeded_correction_inputs(c):
    """Seeded inputs of one correction: the coarse state from the oracle (60 coarse
    steps of the coarsened workload, rounded to FP32), He-initialised parameters
    with a random output bias, and a normalisation from the state's statistics."""
    pc = coarse_oracle_params(c)
    f0 = inputs.as_float32(O.step(O.initial_populations(pc), pc, 60))
    rng = np.random.default_rng(23)
    p = N.init_params(23)
    p[-4:] = rng.normal(0.0, 0.3, 4)
    raw = K.network_input(f0, pc, np.zeros(4), np.ones(4))
    norm = (raw.mean(axis=(1, 2)).astype(np.float32), raw.std(axis=(1, 2)).astype(np.float32),
            np.array([3e-3, 3e-3, 4e-3, 4e-3], dtype=np.float32))
    return pc, f0, p.astype(np.float32), norm


@pytest.mark.parametrize("mode", [1, 2, 3, 4])
def test_one_correction_matches_the_oracle(gpu, mode):
    # the correction alone (lbm_closure_correct) on a state both sides hold exactly:
    # the network input in FP32 from the same populations differs from the oracle's
    # by rounding only, so BF16 rounding decisions agree (but for rare ties); the
    # oracle evaluates the network with BF16 activations, as the tensor cores do,
    # and applies the correction in FP64
    c = lbm.Closure(lbm.default_params(**FINE), interval=10, seed=0)
    try:
        pc, f0, p32, (in_mean, in_scale, out_scale) = seeded_correction_inputs(c)
        c.set_params(p32)
        c.set_normalisation(in_mean, in_scale, out_scale)
        _, co = c.solvers()
        co.set_populations(f0.astype(np.float32))
        c.correct(mode)
        f_gpu = co.populations()
    finally:
        c.close()
    x = K.network_input(f0, pc, in_mean.astype(np.float64), in_scale.astype(np.float64))
    y = N.forward_bf16_activations(oracle_view(p32), x)["y"].numpy()
    f_ref = K.correct(f0, y, out_scale.astype(np.float64), mode, pc)
    d_gpu, d_ref = f_gpu - f0, f_ref - f0
    big = np.max(np.abs(d_ref))
    err = np.abs(d_gpu - d_ref)
    off = float(np.mean(err > 1e-4 * big))
    print(f"\nmode {mode}: largest increment {big:.3e}; error max {err.max() / big:.2e}, "
          f"median {np.median(err) / big:.2e} of it; {off:.2%} of the values beyond 1e-4 of it")
    assert big > 1e-3
    # FP32 arithmetic on populations up to 0.58 (a few 1e-8 absolute) is ~2e-5 of
    # the largest increment, the mass-restoring offset an FP64 sum on both sides
    assert np.median(err) <= 1e-5 * big
    # where a stored input or activation rounds to the other BF16 neighbour in the two
    # evaluations (its FP32 and FP64 values straddle a rounding boundary), a 3 x 3 to
    # 5 x 5 patch of outputs moves, each by well under 1 % of the largest increment
    # (measured, modes 1-4: median 0.5-1.7e-7, 0.4-0.9 % of the values beyond 1e-4,
    # the largest 1.7-4.4e-3 of the largest increment)
    assert off <= 0.05
    assert err.max() <= 1e-2 * big
    m0 = O.densities(f0).sum(axis=(1, 2))
    m1 = O.densities(f_gpu).sum(axis=(1, 2))
    assert np.allclose(m1, m0, rtol=1e-6)


def test_advance_is_the_steps_then_the_correction(gpu):
    # lbm_closure_advance(1, 4) from a state equals lbm_step(interval) followed by
    # lbm_closure_correct(4), bit for bit; and against the oracle (its own 10 FP64
    # steps, then the correction) the advanced state agrees to the FP32 steps'
    # rounding plus the BF16 rounding decisions that this rounding moves
    c = lbm.Closure(lbm.default_params(**FINE), interval=10, seed=0)
    try:
        pc, f0, p32, (in_mean, in_scale, out_scale) = seeded_correction_inputs(c)
        c.set_params(p32)
        c.set_normalisation(in_mean, in_scale, out_scale)
        _, co = c.solvers()
        co.set_populations(f0.astype(np.float32))
        c.advance(1, 4)
        a = co.populations()
        co.set_populations(f0.astype(np.float32))
        c.advance(1, 0)
        plain = co.populations()
        c.correct(4)
        b = co.populations()
    finally:
        c.close()
    assert np.array_equal(a, b)
    f10 = O.step(f0, pc, 10)
    x = K.network_input(f10, pc, in_mean.astype(np.float64), in_scale.astype(np.float64))
    y = N.forward_bf16_activations(oracle_view(p32), x)["y"].numpy()
    f_ref = K.correct(f10, y, out_scale.astype(np.float64), 4, pc)
    d_gpu, d_ref = a - plain, f_ref - f10
    rms = np.sqrt(np.mean((d_gpu - d_ref) ** 2)) / np.sqrt(np.mean(d_ref ** 2))
    print(f"\nadvance: state error {np.max(np.abs(plain - f10)):.2e} before the correction, "
          f"{np.max(np.abs(a - f_ref)):.2e} after; relative RMS error of the correction {rms:.2e}")
    # (measured: 1.9e-7 before the correction, relative RMS 5.6e-4)
    assert np.max(np.abs(plain - f10)) <= 1e-5 * np.max(np.abs(f10))
    assert rms <= 1e-2


def test_in_place_correction_keeps_the_ghost_columns(gpu):
    # the correction rewrites the stored populations in place, periodic ghost
    # columns included; the staged step kernel reads those ghosts at the tile edges
    # (the 64-column coarse grid is one tile, so every step reads columns -2, -1, nx
    # and nx + 1).  Steps after the correction must equal steps from the same
    # populations loaded through set_populations, which writes the ghosts itself.
    c = lbm.Closure(lbm.default_params(**FINE), interval=10, seed=0)
    try:
        pc, f0, p32, (in_mean, in_scale, out_scale) = seeded_correction_inputs(c)
        c.set_params(p32)
        c.set_normalisation(in_mean, in_scale, out_scale)
        _, co = c.solvers()
        co.set_populations(f0.astype(np.float32))
        c.correct(4)
        corrected = co.populations(np.empty(f0.shape, dtype=np.float32))
        assert not np.array_equal(corrected, f0.astype(np.float32))
        co.step(5)
        after = co.populations()
        co.set_populations(corrected)
        co.step(5)
        again = co.populations()
    finally:
        c.close()
    assert np.array_equal(after, again)


def test_normalisation_can_be_set_and_is_checked(gpu):
    c = lbm.Closure(lbm.default_params(**FINE), interval=10, seed=0)
    try:
        c.set_normalisation([1, 2, 3, 4], [0.5, 0.25, 2, 4], [1e-3, 2e-3, 3e-3, 4e-3])
        assert np.array_equal(c.normalisation(),
                              np.array([1, 2, 3, 4, 0.5, 0.25, 2, 4, 1e-3, 2e-3, 3e-3, 4e-3], dtype=np.float32))
        for bad in (([0, 0, 0, np.nan], [1] * 4, [1] * 4), ([0] * 4, [1, 1, 0, 1], [1] * 4),
                    ([0] * 4, [1] * 4, [1, -1, 1, 1])):
            with pytest.raises(lbm.LbmError):
                c.set_normalisation(*bad)
        assert c.normalisation()[5] == np.float32(0.25)      # a refused call changes nothing
    finally:
        c.close()


def test_run_is_the_corrected_advance_then_the_diagnostics(gpu):
    # lbm_closure_run(3 intervals + 4 steps) = lbm_closure_advance(3, 4), four more
    # coarse steps and lbm_diagnostics of the coarse run, bit for bit
    c = lbm.Closure(lbm.default_params(**FINE), interval=10, seed=0)
    try:
        pc, f0, p32, norm = seeded_correction_inputs(c)
        c.set_params(p32)
        c.set_normalisation(*norm)
        _, co = c.solvers()
        co.set_populations(f0.astype(np.float32))
        d_run = c.run(34)
        a = co.populations()
        co.set_populations(f0.astype(np.float32))
        c.advance(3, 4)
        co.step(4)
        d_ref = co.diagnostics()
        b = co.populations()
        assert c.fallbacks == 0
        fresh = lbm.Closure(lbm.default_params(**FINE), interval=10, seed=0)
        with pytest.raises(lbm.LbmError):
            fresh.run(10)                        # no trained or set parameters
        fresh.close()
    finally:
        c.close()
    assert np.array_equal(a, b)
    for k in ("mass_A", "mass_B", "E_k", "E_p", "flux_pb", "flux_K", "flux_tau", "viscous", "h", "L_int"):
        assert d_run[k] == d_ref[k], k


def _prolong(fields):
    """Fine fields from coarse ones: bilinear in the cell centres, periodic in x, the
    wall rows held; velocities halved (fine lattice units)."""
    out = []
    for ch, a in enumerate(fields):
        ny, nx = a.shape
        xf = (np.arange(2 * nx) - 0.5) / 2.0
        yf = (np.arange(2 * ny) - 0.5) / 2.0
        x0 = np.floor(xf).astype(int)
        y0 = np.floor(yf).astype(int)
        tx, ty = xf - x0, yf - y0
        xa, xb = x0 % nx, (x0 + 1) % nx
        ya, yb = np.clip(y0, 0, ny - 1), np.clip(y0 + 1, 0, ny - 1)
        v = ((1 - ty)[:, None] * ((1 - tx)[None, :] * a[np.ix_(ya, xa)] + tx[None, :] * a[np.ix_(ya, xb)])
             + ty[:, None] * ((1 - tx)[None, :] * a[np.ix_(yb, xa)] + tx[None, :] * a[np.ix_(yb, xb)]))
        out.append(v if ch < 2 else 0.5 * v)
    return out


def test_run_falls_back_to_the_fine_solver(gpu):
    # velocity corrections ten thousand times too large drive the corrected coarse run
    # unstable; the call then re-runs its time on the fine plain solver from the saved
    # coarse fields and restarts the coarse run from the restriction of the result
    c = lbm.Closure(lbm.default_params(**FINE), interval=10, seed=0)
    try:
        pc, f0, p32, (mean, scale, oscale) = seeded_correction_inputs(c)
        c.set_params(p32)
        c.set_normalisation(mean, scale, np.array([3e-3, 3e-3, 40.0, 40.0], dtype=np.float32))
        _, co = c.solvers()
        co.set_populations(f0.astype(np.float32))
        start = co.fields()
        d = c.run(20)
        assert c.fallbacks == 1
        got = co.populations()
    finally:
        c.close()
    assert np.isfinite(d["E_k"]) and d["status"] == lbm.LBM_OK
    # the same fallback on the host side of the ABI: prolongation of the saved fields
    # (FP32, as saved), equilibrium fine populations, 80 steps of a plain fine solver,
    # 2 x 2 block means (densities averaged, velocity momentum-weighted, coarse units)
    fa, fb, fux, fuy = _prolong([start[k].astype(np.float32).astype(np.float64) for k in ("rhoA", "rhoB", "ux", "uy")])
    with lbm.Solver(lbm.default_params(**FINE)) as fine:
        fine.set_populations(np.stack([O.equilibrium(fa, fux, fuy), O.equilibrium(fb, fux, fuy)]))
        fine.step(80)
        ff = fine.fields()
    blk = lambda a: a.reshape(a.shape[0] // 2, 2, a.shape[1] // 2, 2).sum(axis=(1, 3))
    rho = ff["rhoA"] + ff["rhoB"]
    rA, rB = blk(ff["rhoA"]) / 4, blk(ff["rhoB"]) / 4
    ux = 2 * blk(rho * ff["ux"]) / blk(rho)
    uy = 2 * blk(rho * ff["uy"]) / blk(rho)
    ref = np.stack([O.equilibrium(rA, ux, uy), O.equilibrium(rB, ux, uy)])
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))
    # each component's mass survives the round trip (the restriction and the
    # prolongation keep it; the fine steps conserve it)
    for s, k in ((0, "rhoA"), (1, "rhoB")):
        assert abs(got[s].sum() - start[k].sum()) <= 1e-5 * start[k].sum()


def test_an_unstable_evaluation_does_not_spoil_the_next_one(gpu):
    # velocity corrections ten thousand times too large trip the coarse run's density
    # guard; the next evaluation starts a new coarse run and must give what a fresh
    # closure gives (the guard is cleared, not left raised)
    fresh = lbm.Closure(lbm.default_params(**FINE), interval=10, seed=0)
    try:
        want = fresh.evaluate(seed=101, warmup=50, intervals=3, use_net=0)
    finally:
        fresh.close()
    c = lbm.Closure(lbm.default_params(**FINE), interval=10, seed=0)
    try:
        _, _, p32, (mean, scale, _) = seeded_correction_inputs(c)
        c.set_params(p32)
        c.set_normalisation(mean, scale, np.array([3e-3, 3e-3, 40.0, 40.0], dtype=np.float32))
        with pytest.raises(lbm.LbmError) as err:
            c.evaluate(seed=101, warmup=50, intervals=2, use_net=4)
        assert err.value.status == lbm.LBM_EUNSTABLE
        got = c.evaluate(seed=101, warmup=50, intervals=3, use_net=0)
    finally:
        c.close()
    for run in (0, 1):   # coarse and fine series
        assert [d["E_k"] for d in got[run]] == [d["E_k"] for d in want[run]]
        assert [d["h"] for d in got[run]] == [d["h"] for d in want[run]]

