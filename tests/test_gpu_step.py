"""Parity of the CUDA time step with the FP64 oracle (GPU).

FP32 storage and arithmetic against FP64: one step from the same FP32-rounded
state agrees to ~1e-6 of the population scale; 1000 steps of the small
configuration agree to <= 1e-5 on each density (max |drho_s| / max |rho_s|).
"""
import numpy as np
import pytest

from oracle import lbm_oracle as O
from paper_2101_04847_gb300 import lbm
from tests import inputs

pytestmark = pytest.mark.gpu

KERNELS = ["fused", "two_pass", "staged", "warp", "pipe", "decoupled"]


def oracle_params(d):
    return O.Params(**{k: v for k, v in d.items() if k in O.Params.__dataclass_fields__})


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("kernel", KERNELS)
def test_initial_state_matches_the_oracle(gpu, kernel):
    d = inputs.params(inputs.C0, seed=3)
    with lbm.Solver(kernel=kernel, **d) as s:
        got = s.populations()
    ref = O.initial_populations(oracle_params(d))
    assert np.max(np.abs(got - ref)) <= 1e-7 * np.max(np.abs(ref))


CASES = [
    # nx, ny, tile_y: a tiny grid, ragged tails in x and y, tiles of 1 / 7 rows, one tile
    (4, 8, 0), (130, 37, 0), (300, 77, 7), (257, 64, 1), (128, 40, 64), (1000, 24, 5),
]


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("nx,ny,tile_y", CASES)
def test_one_step_from_random_populations(gpu, kernel, nx, ny, tile_y):
    d = inputs.params(inputs.C0, nx=nx, ny=ny, crop_rows=3)
    f = inputs.as_float32(inputs.random_populations(nx * 7 + ny, nx, ny))
    with lbm.Solver(kernel=kernel, tile_y=tile_y, **d) as s:
        s.set_populations(f)
        assert np.array_equal(s.populations(), f)   # set/get round trip is exact for FP32 values
        s.step(1)
        got = s.populations()
    ref = O.step(f, oracle_params(d), 1)
    assert rel_err(got, ref) < 2e-6


@pytest.mark.parametrize("kernel", ["staged", "decoupled"])
@pytest.mark.parametrize("tile_x", [128, 256])
@pytest.mark.parametrize("nx,ny,tile_y", CASES)
def test_block_tile_widths_one_step(gpu, kernel, tile_x, nx, ny, tile_y):
    # the block-staged kernels at each of their tile widths, whatever the default picks
    d = inputs.params(inputs.C0, nx=nx, ny=ny, crop_rows=3)
    f = inputs.as_float32(inputs.random_populations(nx * 7 + ny, nx, ny))
    with lbm.Solver(kernel=kernel, tile_x=tile_x, tile_y=tile_y, **d) as s:
        s.set_populations(f)
        s.step(1)
        got = s.populations()
        assert s.get_params().tile_x == tile_x
    ref = O.step(f, oracle_params(d), 1)
    assert rel_err(got, ref) < 2e-6


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_tile_widths_give_identical_states(gpu, storage):
    # per-site arithmetic and the stochastic rounding's random bits (site, component,
    # time step) do not depend on the tiling: both widths and the default agree bit
    # for bit over 25 steps, across three tiles of 256 columns with a ragged last one
    d = inputs.params(inputs.C0, nx=600, ny=90, crop_rows=3, g=1e-4)
    states = []
    for tx in (0, 128, 256):
        with lbm.Solver(kernel="staged", storage=storage, tile_x=tx, **d) as s:
            s.step(25)
            states.append(s.populations())
    assert np.array_equal(states[0], states[1]) and np.array_equal(states[1], states[2])


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("nx,ny,tile_y", [(600, 90, 0), (517, 64, 5), (255, 40, 1), (7, 16, 0)])
def test_paired_kernel_equals_the_staged_one(gpu, storage, nx, ny, tile_y):
    # two columns per thread (odd and ragged widths: a last column without its pair,
    # ghost columns on both edges) give the block-staged kernel's states bit for bit
    d = inputs.params(inputs.C0, nx=nx, ny=ny, crop_rows=3, g=1e-4, G_wall_B=0.1, wall_mode=1)
    states = []
    for kernel in ("staged", "paired"):
        with lbm.Solver(kernel=kernel, storage=storage, tile_x=256, tile_y=tile_y, **d) as s:
            s.step(25)
            states.append(s.populations())
    assert np.array_equal(states[0], states[1])


def test_paired_kernel_is_for_16bit_storage(gpu):
    with pytest.raises(lbm.LbmError):
        lbm.Solver(kernel="paired", storage="f32", **inputs.params(inputs.C0, nx=64, ny=32, crop_rows=3))


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("tile_x,tile_y", [(0, 0), (128, 7), (256, 1)])
def test_decoupled_kernel_equals_the_staged_one(gpu, storage, tile_x, tile_y):
    # the same pulls, collision and stores without the block barrier per row: bit for
    # bit the block-staged kernel's states, ragged tiles and halo rows included
    d = inputs.params(inputs.C0, nx=600, ny=90, crop_rows=3, g=1e-4, G_wall_A=0.1, wall_mode=1)
    states = []
    for kernel in ("staged", "decoupled"):
        with lbm.Solver(kernel=kernel, storage=storage, tile_x=tile_x, tile_y=tile_y, **d) as s:
            s.step(25)
            states.append(s.populations())
    assert np.array_equal(states[0], states[1])


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("extra", [
    dict(G_wall_A=0.3, G_wall_B=-0.2),                # fluid-boundary force on the wall rows
    dict(gravity_mode=1, g=3e-4, gx=2e-4),            # same-sign gravity and an x body force
    dict(tau_A=0.7, tau_B=1.3, G=0.9),                # unequal relaxation times
    dict(G=0.0, g=0.0),                               # no force at all
    dict(wall_mode=1),                                # pseudopotential mirrored across the walls
    dict(wall_mode=1, G_wall_A=0.3, G_wall_B=-0.2, tau_A=0.7, tau_B=1.3),
])
def test_one_step_force_variants(gpu, kernel, extra):
    nx, ny = 96, 40
    d = inputs.params(inputs.C0, nx=nx, ny=ny, crop_rows=3, **extra)
    f = inputs.as_float32(inputs.random_populations(5, nx, ny))
    with lbm.Solver(kernel=kernel, **d) as s:
        s.set_populations(f)
        s.step(1)
        got = s.populations()
    ref = O.step(f, oracle_params(d), 1)
    assert rel_err(got, ref) < 2e-6


@pytest.fixture(scope="module")
def c0_oracle_1000():
    d = inputs.params(inputs.C0, seed=1)
    p = oracle_params(d)
    f = O.step(O.initial_populations(p), p, 1000)
    return d, O.fields(f, p)


@pytest.mark.parametrize("kernel", KERNELS)
def test_small_configuration_1000_steps(gpu, kernel, c0_oracle_1000):
    # 128 x 256, tau 1, G 1.4, masses 1.0 / 0.9, g 1e-5, 8-mode interface: the FP32 path
    # stays within 1e-5 (max |drho_s| / max |rho_s|) of the FP64 oracle after 1000 steps
    d, ref = c0_oracle_1000
    with lbm.Solver(kernel=kernel, **d) as s:
        s.step(1000)
        got = s.fields()
    for k in ("rhoA", "rhoB"):
        assert rel_err(got[k], ref[k]) <= 1e-5, k
    # the velocity is small (~1e-3 of c): compare against its own scale
    for k in ("ux", "uy"):
        assert np.max(np.abs(got[k] - ref[k])) <= 1e-3 * np.max(np.abs(ref["ux"]) + np.abs(ref["uy"])), k


def test_mirror_walls_1000_steps(gpu):
    # wall_mode 1 (the pseudopotential of the wall rows mirrored across the walls) on
    # the small configuration: the same 1e-5 contract on each density after 1000 steps
    d = inputs.params(inputs.C0, seed=2, wall_mode=1)
    p = oracle_params(d)
    ref = O.fields(O.step(O.initial_populations(p), p, 1000), p)
    with lbm.Solver(kernel="staged", **d) as s:
        s.step(1000)
        got = s.fields()
    for k in ("rhoA", "rhoB"):
        assert rel_err(got[k], ref[k]) <= 1e-5, k


def test_miscible_variant_200_steps(gpu):
    # G = 0 with no minority component: rho_B is exactly 0 far above the interface
    d = inputs.params(inputs.C1_MISCIBLE, nx=128, ny=256)
    p = oracle_params(d)
    ref = O.fields(O.step(O.initial_populations(p), p, 200), p)
    with lbm.Solver(**d) as s:
        s.step(200)
        got = s.fields()
        s.sync()
    for k in ("rhoA", "rhoB"):
        assert rel_err(got[k], ref[k]) <= 1e-5, k


def test_graph_replay_equals_single_launches(gpu):
    d = inputs.params(inputs.C0, nx=256, ny=128)
    with lbm.Solver(**d) as a, lbm.Solver(**d) as b:
        a.step(123)                 # two 50-step graphs + 23 launches
        for _ in range(123):
            b.step(1)
        assert a.step_count == b.step_count == 123
        assert np.array_equal(a.populations(), b.populations())


@pytest.mark.parametrize("other", ["two_pass", "staged", "warp", "pipe", "decoupled"])
def test_kernels_agree(gpu, other):
    # same per-site arithmetic; only the compiler's contraction choices may differ
    d = inputs.params(inputs.C0, nx=200, ny=96)
    with lbm.Solver(kernel="fused", **d) as a, lbm.Solver(kernel=other, **d) as b:
        a.step(60)
        b.step(60)
        assert rel_err(a.populations(), b.populations()) < 1e-6


@pytest.mark.parametrize("kernel", ["fused", "staged", "warp", "pipe", "decoupled"])
@pytest.mark.parametrize("tile_y", [1, 5, 16, 64, 300])
def test_tile_shape_does_not_change_the_result(gpu, kernel, tile_y):
    d = inputs.params(inputs.C0, nx=140, ny=150)
    with lbm.Solver(tile_y=16, kernel=kernel, **d) as a, lbm.Solver(tile_y=tile_y, kernel=kernel, **d) as b:
        a.step(20)
        b.step(20)
        assert np.array_equal(a.populations(), b.populations())


@pytest.mark.parametrize("kernel,tile_x", [("fused", 0), ("staged", 0), ("staged", 256), ("warp", 0), ("pipe", 0),
                                           ("decoupled", 128), ("decoupled", 256)])
def test_bench_configuration_one_step_full_grid(gpu, kernel, tile_x):
    # 1024 x 2048 in the launch configurations the benchmark times (default tiles),
    # and the block-staged kernel's wide tile
    d = inputs.params(inputs.C1, seed=2)
    p = oracle_params(d)
    f = inputs.as_float32(O.step(O.initial_populations(p), p, 1))
    with lbm.Solver(kernel=kernel, tile_x=tile_x, **d) as s:
        s.set_populations(f)
        s.step(1)
        got = s.populations()
    ref = O.step(f, p, 1)
    assert rel_err(got, ref) < 2e-6


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_bench_configuration_one_step_full_grid_16bit(gpu, storage):
    # 1024 x 2048 with 16-bit storage in the launch configuration the benchmark times
    # (the paired tile, 4 x 152 tiles): one step from the stored (rounded) state
    # against the oracle, within one spacing of the stored shifted values
    d = inputs.params(inputs.C1, seed=2)
    p = oracle_params(d)
    with lbm.Solver(storage=storage, **d) as s:
        s.step(20)
        f = s.populations()
        s.step(1)
        got = s.populations()
    ref = O.step(f, p, 1)
    rho0 = np.array([d["mass_A"] * (1 + d["minority"]) / 2, d["mass_B"] * (1 + d["minority"]) / 2])
    h = ref - rho0[:, None, None, None] * O.W[None, :, None, None]
    bits = {"f16": 10, "bf16": 7}[storage]
    assert float(np.max(np.abs(got - ref))) <= 2.0 ** -bits * np.max(np.abs(h)) + 1e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("kernel", ["fused", "staged"])
def test_bench_configuration_mass_conservation(gpu, kernel):
    d = inputs.params(inputs.C1, seed=4)
    with lbm.Solver(kernel=kernel, **d) as s:
        m0 = s.diagnostics()
        s.step(500)
        m1 = s.diagnostics()
    for k in ("mass_A", "mass_B"):
        assert abs(m1[k] - m0[k]) <= 1e-6 * m0[k]


def test_full_size_grid_initial_rows_and_conservation(gpu):
    # 10000 x 5000 (5e7 sites): sampled rows of the initial densities against the oracle,
    # then conservation and finiteness over 100 steps
    d = inputs.params(inputs.C2, seed=5)
    p = oracle_params(d)
    rA, rB = O.initial_densities(p)
    rows = [0, 1, 2300, 2497, 2500, 2503, 4999]
    with lbm.Solver(kernel="staged", **d) as s:
        got = s.fields()
        for y in rows:
            assert np.max(np.abs(got["rhoA"][y] - rA[y])) <= 3e-7 * p.mass_A
            assert np.max(np.abs(got["rhoB"][y] - rB[y])) <= 3e-7 * p.mass_A
        del got
        m0 = s.diagnostics()
        s.step(100)
        m1 = s.diagnostics()
        s.sync()
    for k in ("mass_A", "mass_B"):
        assert abs(m1[k] - m0[k]) <= 1e-6 * m0[k]
    assert np.isfinite(m1["E_k"]) and m1["E_k"] > 0


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_full_size_one_step_on_sampled_rows(gpu, storage):
    # 10000 x 5000 in the launch configuration the benchmark times (FP32: the
    # 256-column tiles the grid's default picks; FP16: the paired tile), 30 steps in:
    # one more step on sampled rows against the oracle.  A row's update reads the
    # rows within two of it only, so the oracle steps the band of rows y - 2 .. y + 2
    # (cut to the grid at the walls); the band's own edges act as walls there, which
    # changes its outer rows but not row y
    d = inputs.params(inputs.C2, seed=6)
    p = oracle_params(d)
    rows = [0, 1, 2, 2470, 2500, 2531, 4997, 4999]
    shape = (2, 9, d["ny"], d["nx"])
    with lbm.Solver(storage=storage, **d) as s:
        s.step(30)
        f = s.populations(np.empty(shape, dtype=np.float32))
        bands = {y: f[:, :, max(0, y - 2):min(d["ny"], y + 3)].astype(np.float64) for y in rows}
        s.step(1)
        s.populations(f)
    got = {y: f[:, :, y].astype(np.float64) for y in rows}
    del f
    rho0 = np.array([d["mass_A"] * (1 + d["minority"]) / 2, d["mass_B"] * (1 + d["minority"]) / 2])
    for y in rows:
        lo = max(0, y - 2)
        band = bands[y]
        pb = O.Params(**{**p.__dict__, "ny": band.shape[2]})
        ref = O.step(band, pb, 1)[:, :, y - lo]
        err = float(np.max(np.abs(got[y] - ref)))
        if storage == "f32":
            assert err <= 2e-6 * np.max(np.abs(ref)), (y, err)
        else:   # one spacing of the stored shifted values (stochastic rounding), as in the one-step storage test
            h = ref - rho0[:, None, None] * O.W[None, :, None]
            assert err <= 2.0 ** -10 * np.max(np.abs(h)) + 1e-6 * np.max(np.abs(ref)), (y, err)
