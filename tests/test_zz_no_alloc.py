"""The no-allocation step (lbm_step_noalloc) against the handle-based step.

lbm_step_noalloc serves callers that cannot allocate device memory themselves
(an application or framework that owns the GPU memory budget, or a loop that
cannot take the synchronisation of cudaMalloc / cudaFree): its density scratch
is a fixed array inside the library.  Two calls in a row must give what two
lbm_step calls on a handle give, within the one-step tolerance of the other
parity tests.  This file is collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2101_04847_gb300 import lbm
from tests import inputs

pytestmark = pytest.mark.gpu


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("nx,ny", [(130, 37), (1024, 1024)])
def test_noalloc_step_matches_the_handle_step_twice(gpu, nx, ny):
    import torch

    lib = gpu
    d = inputs.params(inputs.C0, nx=nx, ny=ny, crop_rows=3, g=1e-4)
    f0 = inputs.as_float32(inputs.random_populations(nx + 3 * ny, nx, ny))
    with lbm.Solver(kernel="two_pass", **d) as s:
        s.set_populations(f0)
        s.step(1)
        ref1 = s.populations()
        s.step(1)
        ref2 = s.populations()

    p = lbm.default_params(**d)
    a = torch.from_numpy(f0.astype(np.float32)).cuda()
    b = torch.empty_like(a)
    c = torch.empty_like(a)
    stream = torch.cuda.current_stream().cuda_stream or None
    assert lib.lbm_step_noalloc(C.byref(p), C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), stream) == lbm.LBM_OK
    assert lib.lbm_step_noalloc(C.byref(p), C.c_void_p(b.data_ptr()), C.c_void_p(c.data_ptr()), stream) == lbm.LBM_OK
    torch.cuda.synchronize()
    got1 = b.double().cpu().numpy()
    got2 = c.double().cpu().numpy()
    assert rel_err(got1, ref1) < 2e-6
    assert rel_err(got2, ref2) < 2e-6


def test_noalloc_rejects_grids_beyond_its_scratch(gpu):
    import torch

    lib = gpu
    p = lbm.default_params(nx=2048, ny=1024)          # 2^21 sites > 2^20
    a = torch.empty(16, dtype=torch.float32, device="cuda")
    b = torch.empty(16, dtype=torch.float32, device="cuda")
    st = lib.lbm_step_noalloc(C.byref(p), C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), None)
    assert st == lbm.LBM_EINVAL
    assert b"exceeds" in lib.lbm_last_error()
    p = lbm.default_params(nx=64, ny=64, storage="f16")
    assert lib.lbm_step_noalloc(C.byref(p), C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), None) == lbm.LBM_EINVAL
    assert lib.lbm_step_noalloc(C.byref(p), C.c_void_p(a.data_ptr()), C.c_void_p(a.data_ptr()), None) == lbm.LBM_EINVAL
    # more rows than a launch grid has (within the scratch size)
    p = lbm.default_params(nx=4, ny=70000)
    assert lib.lbm_step_noalloc(C.byref(p), C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), None) == lbm.LBM_EINVAL
    assert b"rows" in lib.lbm_last_error()
    # output overlapping the input by part of its length
    big = torch.empty(2 * 18 * 64 * 64, dtype=torch.float32, device="cuda")
    p = lbm.default_params(nx=64, ny=64)
    st = lib.lbm_step_noalloc(C.byref(p), C.c_void_p(big.data_ptr()), C.c_void_p(big.data_ptr() + 4 * 1000), None)
    assert st == lbm.LBM_EINVAL
    assert b"overlap" in lib.lbm_last_error()
