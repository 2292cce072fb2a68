"""Ensemble launch and the tile tuner (GPU).

Every member of an ensemble advanced by the one-launch-per-step kernel must
match the same realisation advanced alone by the block-staged kernel (the same
tile code, compiled into another kernel, so equal up to FMA contraction), and
tuning must leave states untouched.
"""
import numpy as np
import pytest

from paper_2101_04847_gb300 import lbm
from tests import inputs

pytestmark = pytest.mark.gpu

MEMBERS = [
    dict(nx=256, ny=128, G=1.4, seed=1, storage="f32"),
    dict(nx=97, ny=200, G=0.0, minority=0.0, seed=2, storage="f32"),
    dict(nx=160, ny=64, G=1.2, seed=3, storage="f16"),
    dict(nx=300, ny=90, G=1.4, seed=4, storage="bf16"),
]


def member_params(m, tile_y=0):
    d = inputs.params(inputs.C0, crop_rows=5, g=1e-4)
    d.update(m)
    return lbm.default_params(kernel="staged", tile_y=tile_y, **d)


# tile_y 16: 55 tiles in one partial wave; tile_y 1: 854 one-row tiles for the 608
# resident blocks of GB300, two waves of mixed storage types
@pytest.mark.parametrize("tile_y", [16, 1])
def test_ensemble_members_equal_solo_runs(gpu, tile_y):
    params = [member_params(m, tile_y=tile_y) for m in MEMBERS]
    with lbm.Ensemble(params) as ens:
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
