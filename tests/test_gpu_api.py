"""Host API behaviour on the GPU: checkpoints, reset, the instability guard,
library-owned memory, storage round trips."""
import ctypes as C

import numpy as np
import pytest

from oracle import lbm_oracle as O
from paper_2101_04847_gb300 import lbm
from tests import inputs

pytestmark = pytest.mark.gpu


def test_checkpoint_round_trip_is_bitwise(gpu, tmp_path):
    d = inputs.params(inputs.C0, nx=160, ny=96)
    path = tmp_path / "state.bin"
    with lbm.Solver(**d) as a:
        a.step(37)
        a.save(path)
        a.step(25)
        want = a.populations()
        with lbm.Solver(**d) as b:
            b.load(path)
            assert b.step_count == 37
            b.step(25)
            assert np.array_equal(b.populations(), want)


def test_load_rejects_a_mismatched_grid(gpu, tmp_path):
    path = tmp_path / "state.bin"
    with lbm.Solver(**inputs.params(inputs.C0, nx=64, ny=64)) as a:
        a.save(path)
    with lbm.Solver(**inputs.params(inputs.C0, nx=64, ny=72)) as b:
        with pytest.raises(lbm.LbmError) as e:
            b.load(path)
        assert e.value.status == lbm.LBM_EINVAL


def test_reset_restores_the_initial_state(gpu):
    with lbm.Solver(**inputs.params(inputs.C0, nx=64, ny=64)) as s:
        f0 = s.populations()
        s.step(30)
        s.reset()
        assert s.step_count == 0
        assert np.array_equal(s.populations(), f0)


def test_nan_is_reported_as_unstable_and_is_sticky(gpu):
    nx, ny = 64, 32
    with lbm.Solver(**inputs.params(inputs.C0, nx=nx, ny=ny, crop_rows=4)) as s:
        f = s.populations()
        f[0, 0, 10, 10] = np.nan
        s.set_populations(f)
        s.step(3)
        with pytest.raises(lbm.LbmError) as e:
            s.sync()
        assert e.value.status == lbm.LBM_EUNSTABLE
        d = s.diagnostics(check=False)
        assert d["status"] == lbm.LBM_EUNSTABLE
        with pytest.raises(lbm.LbmError):
            s.step(1)


def test_negative_density_is_reported_as_unstable(gpu):
    nx, ny = 64, 32
    with lbm.Solver(**inputs.params(inputs.C0, nx=nx, ny=ny, crop_rows=4)) as s:
        f = s.populations()
        f[1, :, 5, 7] = -0.5
        s.set_populations(f)
        s.step(1)
        with pytest.raises(lbm.LbmError) as e:
            s.sync()
        assert e.value.status == lbm.LBM_EUNSTABLE


def test_library_owned_memory_and_stream(gpu):
    lib = gpu
    h = C.c_void_p()
    assert lib.lbm_create(96, 64, 0.8, 1.2, 1.0, 1.0, 1e-5, 7, C.byref(h)) == lbm.LBM_OK
    assert lib.lbm_step(h, 10) == lbm.LBM_OK
    d = lbm.LbmDiag()
    assert lib.lbm_diagnostics(h, C.byref(d)) == lbm.LBM_OK
    assert d.step == 10 and d.mass_A > 0
    lib.lbm_destroy(h)


def test_workspace_too_small_is_rejected(gpu):
    import torch

    p = lbm.default_params(nx=64, ny=64)
    n = lbm.workspace_bytes(p)
    ws = torch.empty(n // 2, dtype=torch.uint8, device="cuda")
    h = C.c_void_p()
    st = gpu.lbm_create_ex(C.byref(p), C.c_void_p(ws.data_ptr()), n // 2, None, C.byref(h))
    assert st == lbm.LBM_ENOMEM and not h.value


def test_runs_on_a_caller_stream(gpu):
    import torch

    d = inputs.params(inputs.C0, nx=96, ny=64)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        a = lbm.Solver(**d)
    b = lbm.Solver(**d)
    a.step(60)
    b.step(60)
    assert np.array_equal(a.populations(), b.populations())
    a.close()
    b.close()


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_fp32_population_transfer_matches_the_fp64_one(gpu, storage):
    # the FP32 entry points carry the same state as the float64 ones: both paths
    # round the host values to FP32 before storing them, and the device computes
    # the read-back values in FP32 in both
    d = inputs.params(inputs.C0, nx=150, ny=40, crop_rows=3, g=1e-4)
    f = inputs.random_populations(3, 150, 40, lo=0.02, hi=0.2)
    with lbm.Solver(storage=storage, **d) as a, lbm.Solver(storage=storage, **d) as b:
        a.set_populations(f)
        b.set_populations(f.astype(np.float32))
        a.step(5)
        b.step(5)
        ga, gb = a.populations(), b.populations(out=np.empty(f.shape, dtype=np.float32))
        assert gb.dtype == np.float32
        assert np.array_equal(ga, gb.astype(np.float64))


def test_async_upload_and_diagnostics_equal_the_synchronous_calls(gpu):
    # the same upload, steps and evaluation through the asynchronous entry points,
    # pipelined as the end-to-end bench runs them, give bitwise the same results
    import torch

    d = inputs.params(inputs.C0, nx=160, ny=96, crop_rows=4)
    host = torch.empty((2, 9, 96, 160), dtype=torch.float32, pin_memory=True).numpy()
    with lbm.Solver(**d) as s:
        s.step(30)
        s.populations(out=host)
        ref = []
        for _ in range(3):
            s.set_populations(host)
            s.step(20)
            ref.append(s.diagnostics())
        f_ref = s.populations()
    with lbm.Solver(**d) as s:
        got = []
        s.set_populations_async(host)
        s.step(20)
        s.diagnostics_async()
        for _ in range(2):
            s.set_populations_async(host)
            s.step(20)
            got.append(s.diagnostics_wait())
            s.diagnostics_async()
        got.append(s.diagnostics_wait())
        f_got = s.populations()
        with pytest.raises(lbm.LbmError) as e:
            s.diagnostics_wait()                      # nothing pending
        assert e.value.status == lbm.LBM_ESTATE
        s.diagnostics_async()
        with pytest.raises(lbm.LbmError):
            s.diagnostics_async()                     # one pending at a time
        s.diagnostics_wait()
    assert np.array_equal(f_got, f_ref)
    for a, b in zip(got, ref):
        for k in ("E_k", "E_p", "h", "L_int", "mass_A", "mass_B", "viscous", "enstrophy"):
            assert a[k] == b[k], k


def test_async_diagnostics_report_an_unstable_state(gpu):
    d = inputs.params(inputs.C0, nx=64, ny=32, crop_rows=4)
    with lbm.Solver(**d) as s:
        f = s.populations().astype(np.float32)
        f[0, 0, 10, 10] = np.nan
        s.set_populations_async(np.ascontiguousarray(f))
        s.step(3)
        s.diagnostics_async()
        with pytest.raises(lbm.LbmError) as e:
            s.diagnostics_wait()
        assert e.value.status == lbm.LBM_EUNSTABLE


def test_step_waits_that_run_out_report_a_timeout(gpu):
    # failure detection without a GPU fault: a step launch whose row copies are
    # withheld has every bounded wait give up (a few thousand polls each); the host
    # reads LBM_ETIMEOUT, the context stays usable, and the state is untouched
    nx, ny = 200, 48
    d = inputs.params(inputs.C0, nx=nx, ny=ny, crop_rows=3)
    f = inputs.as_float32(inputs.random_populations(17, nx, ny))
    with lbm.Solver(kernel="staged", **d) as s:
        s.set_populations(f)
        s.step_test_timeout()
        with pytest.raises(lbm.LbmError) as e:
            s.sync()
        assert e.value.status == lbm.LBM_ETIMEOUT
        assert np.array_equal(s.populations(), f)
        assert s.step_count == 0
        with pytest.raises(lbm.LbmError) as e:
            s.diagnostics()
        assert e.value.status == lbm.LBM_ETIMEOUT          # sticky until a reset
        s.reset()
        s.set_populations(f)
        s.step(1)
        s.sync()
        got = s.populations()
    ref = O.step(f, O.Params(**{k: v for k, v in d.items() if k in O.Params.__dataclass_fields__}), 1)
    assert np.max(np.abs(got - ref)) < 2e-6 * np.max(np.abs(ref))
    with lbm.Solver(storage="f16", **d) as s16:
        with pytest.raises(lbm.LbmError) as e:
            s16.step_test_timeout()
        assert e.value.status == lbm.LBM_EINVAL
