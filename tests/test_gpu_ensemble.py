"""Ensemble launch and the tile tuner (GPU).

Every member of an ensemble advanced by the one-launch-per-step kernel must
match the FP64 oracle (FP32 members within the 1e-5 density contract, every
member within the one-step rounding bound of its storage), and the same
realisation advanced alone by the block-staged kernel (the same tile code,
compiled into another kernel, so equal up to FMA contraction); tuning must leave
states untouched.
"""
import numpy as np
import pytest

from oracle import lbm_oracle as O
from paper_2101_04847_gb300 import lbm
from tests import inputs

pytestmark = pytest.mark.gpu

MEMBERS = [
    dict(nx=256, ny=128, G=1.4, seed=1, storage="f32"),
    dict(nx=97, ny=200, G=0.0, minority=0.0, seed=2, storage="f32"),
    dict(nx=160, ny=64, G=1.2, seed=3, storage="f16"),
    dict(nx=300, ny=90, G=1.4, seed=4, storage="bf16"),
]


def member_params(m, tile_y=0, tile_x=0):
    d = inputs.params(inputs.C0, crop_rows=5, g=1e-4)
    d.update(m)
    return lbm.default_params(kernel="staged", tile_y=tile_y, tile_x=tile_x, **d)


# tile_y 16: one partial wave; tile_y 1 (and 3): more one-row tiles than GB300's
# resident blocks (700 at tile_x 0, 854 at 128 for 608 slots), two waves of mixed
# storage types; tile_x 0 runs the 16-bit members in paired 256-column tiles
@pytest.mark.parametrize("tile_y,tile_x", [(16, 0), (1, 0), (16, 128), (3, 128), (16, 256), (5, 256)])
def test_ensemble_members_equal_solo_runs(gpu, tile_y, tile_x):
    params = [member_params(m, tile_y=tile_y, tile_x=tile_x) for m in MEMBERS]
    with lbm.Ensemble(params) as ens:
        assert ens.tile_width == tile_x   # 0: paired tiles for the 16-bit members
        ens.step(73)                     # one 50-step graph + 23 single launches
        ens.sync()
        got = [m.populations() for m in ens.members]
        diags = ens.diagnostics()
    for m, p, g, d in zip(MEMBERS, params, got, diags):
        with lbm.Solver(member_params(m, tile_y=tile_y)) as s:
            s.step(73)
            want = s.populations()
        # one unit in the last place of the storage type
        tol = {"f32": 1e-6, "f16": 2e-3, "bf16": 1.6e-2}[m["storage"]]
        assert float(np.max(np.abs(g - want)) / np.max(np.abs(want))) < tol, m
        assert d["step"] == 73


def test_ensemble_member_cannot_be_stepped_alone(gpu):
    with lbm.Ensemble([member_params(MEMBERS[0])]) as ens:
        with pytest.raises(lbm.LbmError) as e:
            ens.members[0].step(1)
        assert e.value.status == lbm.LBM_ESTATE


def test_ensemble_tune_keeps_states(gpu):
    params = [member_params(m) for m in MEMBERS[:3]]
    with lbm.Ensemble(params) as ens:
        ens.step(10)
        before = [m.populations() for m in ens.members]
        ty, ms = ens.tune()
        assert 12 <= ty <= 256 and ms > 0
        assert ens.tile_width in (0, 128, 256)
        after = [m.populations() for m in ens.members]
        for a, b in zip(before, after):
            assert np.array_equal(a, b)
        ens.step(10)
        assert ens.diagnostics()[0]["step"] == 20


def test_tune_keeps_state_and_caches(gpu, tmp_path):
    d = inputs.params(inputs.C0, nx=300, ny=200)
    cache = tmp_path / "tune.txt"
    with lbm.Solver(kernel="staged", **d) as s, lbm.Solver(kernel="staged", **d) as ref:
        s.step(7)
        ref.step(7)
        f0 = s.populations()
        ty, ms = s.tune(cache)
        tx = s.get_params().tile_x
        assert tx in (128, 256) and ty >= 0 and ms > 0
        assert np.array_equal(s.populations(), f0)
        assert s.step_count == 7
        s.step(20)
        ref.step(20)
        assert np.array_equal(s.populations(), ref.populations())   # the tile shape does not change the result
    text = cache.read_text().split()
    assert (int(text[1]), int(text[2])) == (tx, ty)
    with lbm.Solver(kernel="staged", **d) as s2:
        ty2, ms2 = s2.tune(cache)                                      # found in the cache, not re-timed
        assert ty2 == ty and ms2 == pytest.approx(ms, rel=1e-3)   # stored with 6 decimals
        assert s2.get_params().tile_x == tx


def oracle_params(m):
    d = inputs.params(inputs.C0, crop_rows=5, g=1e-4)
    d.update(m)
    return O.Params(**{k: v for k, v in d.items() if k in O.Params.__dataclass_fields__})


# mixed grids, couplings and storage types; uneven grids with ragged tile tails
ORACLE_MEMBERS = [
    dict(nx=256, ny=128, G=1.4, seed=1, storage="f32"),
    dict(nx=97, ny=200, G=0.0, minority=0.0, seed=2, storage="f32"),
    dict(nx=150, ny=66, G=1.2, seed=5, storage="f32"),
    dict(nx=160, ny=64, G=1.2, seed=3, storage="f16"),
    dict(nx=300, ny=90, G=1.4, seed=4, storage="bf16"),
]


@pytest.mark.parametrize("tile_y", [16, 1])
def test_ensemble_fp32_members_match_the_oracle(gpu, tile_y):
    # every FP32 member, advanced from its initial state through one 50-step graph and
    # 23 single launches of the ensemble kernel, against the FP64 oracle's own run
    params = [member_params(m, tile_y=tile_y) for m in ORACLE_MEMBERS]
    with lbm.Ensemble(params) as ens:
        ens.step(73)
        ens.sync()
        got = [m.fields() for m in ens.members]
    for m, g in zip(ORACLE_MEMBERS, got):
        if m["storage"] != "f32":
            continue
        p = oracle_params(m)
        ref = O.fields(O.step(O.initial_populations(p), p, 73), p)
        for k in ("rhoA", "rhoB"):
            err = float(np.max(np.abs(g[k] - ref[k])) / np.max(np.abs(ref[k])))
            assert err <= 1e-5, (m, k, err)


@pytest.mark.parametrize("tile_y", [16, 1])
def test_ensemble_one_step_from_set_states_matches_the_oracle(gpu, tile_y):
    # each member set to seeded random populations (as its storage holds them), one
    # ensemble step, against one oracle step from the state read back: FP32 to the
    # arithmetic's rounding, 16-bit within one spacing of the stored mantissa
    # (stochastic rounding of the stores), as for the solo kernels
    params = [member_params(m, tile_y=tile_y) for m in ORACLE_MEMBERS]
    with lbm.Ensemble(params) as ens:
        start = []
        for k, mem in enumerate(ens.members):
            mem.set_populations(inputs.random_populations(40 + k, mem.nx, mem.ny, lo=0.02, hi=0.2))
            start.append(mem.populations())
        ens.step(1)
        ens.sync()
        got = [mem.populations() for mem in ens.members]
    for m, f, g in zip(ORACLE_MEMBERS, start, got):
        p = oracle_params(m)
        ref = O.step(f, p, 1)
        if m["storage"] == "f32":
            allowed = 2e-6 * np.max(np.abs(ref))
        else:
            rho0 = [p.mass_A * (1 + p.minority) / 2, p.mass_B * (1 + p.minority) / 2]
            h = ref - np.array(rho0)[:, None, None, None] * O.W[None, :, None, None]
            bits = {"f16": 10, "bf16": 7}[m["storage"]]
            allowed = 2.0 ** -bits * np.max(np.abs(h)) + 1e-6 * np.max(np.abs(ref))
        assert float(np.max(np.abs(g - ref))) <= allowed, m
