"""Thin ctypes binding of liblbm.so (include/lbm.h).

Argument marshalling only: every step of the solver runs in the CUDA kernels of
the library.  PyTorch supplies device memory (the workspace) and the stream.
If the library has not been built, importing works but every call raises.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "liblbm.so"

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_ESTATE, LBM_EIO = range(8)
STORAGE = {"f32": 0, "f16": 1, "bf16": 2}
KERNEL = {"fused": 0, "two_pass": 1, "staged": 2, "warp": 3, "pipe": 4, "decoupled": 5, "paired": 6}


class LbmParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32),
        ("tau_A", C.c_double), ("tau_B", C.c_double),
        ("G", C.c_double), ("G_wall_A", C.c_double), ("G_wall_B", C.c_double),
        ("mass_A", C.c_double), ("mass_B", C.c_double),
        ("g", C.c_double), ("gravity_mode", C.c_int32), ("gx", C.c_double),
        ("seed", C.c_uint64), ("n_modes", C.c_int32),
        ("amp", C.c_double), ("width", C.c_double), ("minority", C.c_double), ("y0", C.c_double),
        ("crop_rows", C.c_int32), ("storage", C.c_int32), ("kernel", C.c_int32), ("tile_y", C.c_int32),
        ("shift_A", C.c_double), ("shift_B", C.c_double),
        ("tile_x", C.c_int32), ("wall_mode", C.c_int32), ("x_offset", C.c_int32), ("nx_total", C.c_int32),
    ]


class LbmDiag(C.Structure):
    _fields_ = [
        ("step", C.c_int64),
        ("mass_A", C.c_double), ("mass_B", C.c_double),
        ("E_k", C.c_double), ("E_p", C.c_double), ("buoyancy", C.c_double),
        ("flux_pb", C.c_double), ("flux_K", C.c_double), ("flux_tau", C.c_double),
        ("viscous", C.c_double), ("enstrophy", C.c_double), ("rho_bar", C.c_double),
        ("h", C.c_double), ("L_int", C.c_double),
        ("cc", C.c_int64 * 4), ("status", C.c_int32),
    ]


_P = C.POINTER
_dp = _P(C.c_double)
_h = C.c_void_p
_PROTOS = {
    "lbm_version": (C.c_char_p, []),
    "lbm_status_str": (C.c_char_p, [C.c_int]),
    "lbm_last_error": (C.c_char_p, []),
    "lbm_params_default": (C.c_int, [_P(LbmParams)]),
    "lbm_workspace_bytes": (C.c_int, [_P(LbmParams), _P(C.c_size_t)]),
    "lbm_create": (C.c_int, [C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double, C.c_double,
                             C.c_double, C.c_uint64, _P(_h)]),
    "lbm_create_ex": (C.c_int, [_P(LbmParams), C.c_void_p, C.c_size_t, C.c_void_p, _P(_h)]),
    "lbm_reset": (C.c_int, [_h]),
    "lbm_step": (C.c_int, [_h, C.c_int64]),
    "lbm_sync": (C.c_int, [_h]),
    "lbm_step_count": (C.c_int, [_h, _P(C.c_int64)]),
    "lbm_step_test_timeout": (C.c_int, [_h]),
    "lbm_halo_bytes": (C.c_int, [_h, _P(C.c_size_t)]),
    "lbm_halo_pack": (C.c_int, [_h, C.c_int32, C.c_void_p]),
    "lbm_halo_unpack": (C.c_int, [_h, C.c_int32, C.c_void_p]),
    "lbm_diagnostics": (C.c_int, [_h, _P(LbmDiag)]),
    "lbm_diagnostics_async": (C.c_int, [_h]),
    "lbm_diagnostics_wait": (C.c_int, [_h, _P(LbmDiag)]),
    "lbm_profile": (C.c_int, [_h, _dp]),
    "lbm_get_fields": (C.c_int, [_h, _dp, _dp, _dp, _dp]),
    "lbm_get_populations": (C.c_int, [_h, _dp]),
    "lbm_set_populations": (C.c_int, [_h, _dp]),
    "lbm_get_populations_f32": (C.c_int, [_h, C.c_void_p]),
    "lbm_set_populations_f32": (C.c_int, [_h, C.c_void_p]),
    "lbm_set_populations_f32_async": (C.c_int, [_h, C.c_void_p]),
    "lbm_save": (C.c_int, [_h, C.c_char_p]),
    "lbm_load": (C.c_int, [_h, C.c_char_p]),
    "lbm_destroy": (None, [_h]),
    "lbm_step_noalloc": (C.c_int, [_P(LbmParams), C.c_void_p, C.c_void_p, C.c_void_p]),
    "lbm_tune": (C.c_int, [_h, C.c_char_p, _P(C.c_int32), _P(C.c_double)]),
    "lbm_get_params": (C.c_int, [_h, _P(LbmParams)]),
    "lbm_ens_create": (C.c_int, [C.c_int32, _P(LbmParams), C.c_void_p, _P(C.c_void_p)]),
    "lbm_ens_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "lbm_ens_sync": (C.c_int, [C.c_void_p]),
    "lbm_ens_member": (C.c_int, [C.c_void_p, C.c_int32, _P(_h)]),
    "lbm_ens_diagnostics": (C.c_int, [C.c_void_p, _P(LbmDiag)]),
    "lbm_ens_tune": (C.c_int, [C.c_void_p, _P(C.c_int32), _P(C.c_double)]),
    "lbm_ens_tile_width": (C.c_int, [C.c_void_p, _P(C.c_int32)]),
    "lbm_ens_destroy": (None, [C.c_void_p]),
    "lbm_cnn_workspace_bytes": (C.c_int, [C.c_int32, C.c_int32, _P(C.c_size_t)]),
    "lbm_cnn_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_size_t,
                                  C.c_void_p, C.c_void_p]),
    "lbm_cnn_infer": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_size_t,
                                C.c_void_p, C.c_void_p]),
    "lbm_cnn_infer_status": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]),
    "lbm_cnn_infer_test_timeout": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_size_t,
                                             C.c_void_p, C.c_void_p]),
    "lbm_cnn_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                    C.c_size_t, C.c_void_p, _P(C.c_double), C.c_void_p]),
    "lbm_closure_coarse_params": (C.c_int, [_P(LbmParams), _P(LbmParams)]),
    "lbm_closure_create": (C.c_int, [_P(LbmParams), C.c_int32, C.c_uint64, C.c_void_p, _P(C.c_void_p)]),
    "lbm_closure_generate": (C.c_int, [C.c_void_p, C.c_int32, C.c_uint64, C.c_int32, C.c_int32]),
    "lbm_closure_train": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_uint64, _P(C.c_double)]),
    "lbm_closure_advance": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "lbm_closure_evaluate": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int32, C.c_int32, C.c_int32, _P(LbmDiag),
                                       _P(LbmDiag)]),
    "lbm_closure_params": (C.c_int, [C.c_void_p, _P(C.c_float), C.c_int32]),
    "lbm_closure_normalisation": (C.c_int, [C.c_void_p, _P(C.c_float)]),
    "lbm_closure_set_normalisation": (C.c_int, [C.c_void_p, _P(C.c_float)]),
    "lbm_closure_correct": (C.c_int, [C.c_void_p, C.c_int32]),
    "lbm_closure_run": (C.c_int, [C.c_void_p, C.c_int64, _P(LbmDiag)]),
    "lbm_closure_fallbacks": (C.c_int, [C.c_void_p, _P(C.c_int64)]),
    "lbm_closure_solvers": (C.c_int, [C.c_void_p, _P(_h), _P(_h)]),
    "lbm_closure_destroy": (None, [C.c_void_p]),
}

_lib = None


class LbmError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: status {status}: {message}")
        self.status = status


def load_library(path: str | Path | None = None) -> C.CDLL:
    """Load liblbm.so; raises if it is missing (there is no fallback)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = Path(path) if path is not None else _LIB_PATH
    if not p.exists():
        raise RuntimeError(f"liblbm.so not found at {p}: run __graft_entry__.build() "
                           "(python -c 'import __graft_entry__ as g; g.build()') first")
    lib = C.CDLL(str(p))
    for name, (res, args) in _PROTOS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(st: int, where: str) -> int:
    if st != LBM_OK:
        lib = load_library()
        raise LbmError(st, where, lib.lbm_last_error().decode() or lib.lbm_status_str(st).decode())
    return st


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def default_params(**overrides) -> LbmParams:
    p = LbmParams()
    _check(load_library().lbm_params_default(C.byref(p)), "lbm_params_default")
    for k, v in overrides.items():
        if k == "storage" and isinstance(v, str):
            v = STORAGE[v]
        if k == "kernel" and isinstance(v, str):
            v = KERNEL[v]
        if not hasattr(p, k):
            raise KeyError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def params_dict(p: LbmParams) -> dict:
    return {name: getattr(p, name) for name, _ in LbmParams._fields_}


def workspace_bytes(p: LbmParams) -> int:
    n = C.c_size_t()
    _check(load_library().lbm_workspace_bytes(C.byref(p), C.byref(n)), "lbm_workspace_bytes")
    return n.value


def diag_dict(d: LbmDiag) -> dict:
    out = {name: getattr(d, name) for name, _ in LbmDiag._fields_ if name != "cc"}
    out["cc"] = np.array(list(d.cc), dtype=np.int64)
    return out


class Solver:
    """One solver instance on the current CUDA device.

    The device workspace is a torch uint8 tensor owned by this object; work runs
    on the torch stream current at construction (or on a library stream when that
    is the legacy default stream).
    """

    def __init__(self, params: LbmParams | None = None, **overrides):
        import torch

        lib = load_library()
        self.lib = lib
        self.params = params if params is not None else default_params(**overrides)
        if params is not None and overrides:
            for k, v in overrides.items():
                setattr(self.params, k, v)
        self.nx, self.ny = self.params.nx, self.params.ny
        nbytes = workspace_bytes(self.params)
        if not torch.cuda.is_available():
            raise RuntimeError("Solver needs a CUDA device")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        stream = torch.cuda.current_stream()
        sp = stream.cuda_stream or None
        self._h = C.c_void_p()
        _check(lib.lbm_create_ex(C.byref(self.params), C.c_void_p(self.workspace.data_ptr()), nbytes,
                                 C.c_void_p(sp) if sp else None, C.byref(self._h)), "lbm_create_ex")

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.lbm_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- API -----------------------------------------------------------------
    def reset(self):
        _check(self.lib.lbm_reset(self._h), "lbm_reset")

    def step(self, n: int = 1):
        _check(self.lib.lbm_step(self._h, int(n)), "lbm_step")

    def sync(self):
        _check(self.lib.lbm_sync(self._h), "lbm_sync")

    def halo_bytes(self) -> int:
        n = C.c_size_t()
        _check(self.lib.lbm_halo_bytes(self._h, C.byref(n)), "lbm_halo_bytes")
        return n.value

    def halo_pack(self, side: int, dev_ptr: int):
        """Copy the two edge columns of side 0 (left) or 1 (right) to device memory."""
        _check(self.lib.lbm_halo_pack(self._h, int(side), C.c_void_p(dev_ptr)), "lbm_halo_pack")

    def halo_unpack(self, side: int, dev_ptr: int):
        """Copy device memory into the ghost columns of side 0 (left) or 1 (right)."""
        _check(self.lib.lbm_halo_unpack(self._h, int(side), C.c_void_p(dev_ptr)), "lbm_halo_unpack")

    def step_test_timeout(self):
        """One step launch whose row copies are withheld: its bounded waits give up
        (the timeout path's test; the state is left as it was)."""
        _check(self.lib.lbm_step_test_timeout(self._h), "lbm_step_test_timeout")

    @property
    def step_count(self) -> int:
        v = C.c_int64()
        _check(self.lib.lbm_step_count(self._h, C.byref(v)), "lbm_step_count")
        return v.value

    def diagnostics(self, check: bool = True) -> dict:
        d = LbmDiag()
        st = self.lib.lbm_diagnostics(self._h, C.byref(d))
        if check or st not in (LBM_OK, LBM_EUNSTABLE):
            _check(st, "lbm_diagnostics")
        return diag_dict(d)

    def diagnostics_async(self):
        """Queue a diagnostics evaluation; diagnostics_wait() collects it."""
        _check(self.lib.lbm_diagnostics_async(self._h), "lbm_diagnostics_async")

    def diagnostics_wait(self, check: bool = True) -> dict:
        d = LbmDiag()
        st = self.lib.lbm_diagnostics_wait(self._h, C.byref(d))
        if check or st not in (LBM_OK, LBM_EUNSTABLE):
            _check(st, "lbm_diagnostics_wait")
        return diag_dict(d)

    def set_populations_async(self, f: np.ndarray):
        """Replace the state from a float32 host array without waiting for the copy
        (pinned memory overlaps it with the work already queued); `f` must stay
        unchanged until sync() returns or a result queued after this call is read."""
        if f.dtype != np.float32 or not f.flags.c_contiguous or f.shape != (2, 9, self.ny, self.nx):
            raise ValueError(f"populations must be a C-contiguous float32 array of shape (2, 9, {self.ny}, {self.nx})")
        _check(self.lib.lbm_set_populations_f32_async(self._h, f.ctypes.data), "lbm_set_populations_f32_async")

    def profile(self) -> np.ndarray:
        rows = np.empty(self.ny - 2 * self.params.crop_rows)
        _check(self.lib.lbm_profile(self._h, _ptr(rows)), "lbm_profile")
        return rows

    def fields(self) -> dict:
        out = {k: np.empty((self.ny, self.nx)) for k in ("rhoA", "rhoB", "ux", "uy")}
        _check(self.lib.lbm_get_fields(self._h, *(_ptr(out[k]) for k in ("rhoA", "rhoB", "ux", "uy"))),
               "lbm_get_fields")
        return out

    def populations(self, out: np.ndarray | None = None) -> np.ndarray:
        """Post-streaming populations (2, 9, ny, nx); float64 unless `out` is float32."""
        if out is None:
            out = np.empty((2, 9, self.ny, self.nx))
        if out.shape != (2, 9, self.ny, self.nx) or not out.flags.c_contiguous:
            raise ValueError(f"out must be a C-contiguous array of shape (2, 9, {self.ny}, {self.nx})")
        if out.dtype == np.float32:
            _check(self.lib.lbm_get_populations_f32(self._h, out.ctypes.data), "lbm_get_populations_f32")
        elif out.dtype == np.float64:
            _check(self.lib.lbm_get_populations(self._h, _ptr(out)), "lbm_get_populations")
        else:
            raise ValueError("out must be float32 or float64")
        return out

    def set_populations(self, f: np.ndarray):
        """Replace the state; float32 arrays go through the FP32 entry point as they are."""
        if f.dtype == np.float32:
            f = np.ascontiguousarray(f)
        else:
            f = np.ascontiguousarray(f, dtype=np.float64)
        if f.shape != (2, 9, self.ny, self.nx):
            raise ValueError(f"populations must have shape (2, 9, {self.ny}, {self.nx})")
        if f.dtype == np.float32:
            _check(self.lib.lbm_set_populations_f32(self._h, f.ctypes.data), "lbm_set_populations_f32")
        else:
            _check(self.lib.lbm_set_populations(self._h, _ptr(f)), "lbm_set_populations")

    def save(self, path: str | Path):
        _check(self.lib.lbm_save(self._h, str(path).encode()), "lbm_save")

    def load(self, path: str | Path):
        _check(self.lib.lbm_load(self._h, str(path).encode()), "lbm_load")

    def tune(self, cache_path: str | Path | None = None) -> tuple[int, float]:
        ty, ms = C.c_int32(), C.c_double()
        _check(self.lib.lbm_tune(self._h, str(cache_path).encode() if cache_path else None,
                                 C.byref(ty), C.byref(ms)), "lbm_tune")
        self.params = self.get_params()
        return ty.value, ms.value

    def get_params(self) -> LbmParams:
        """The parameters as in use (tile_x / tile_y after tune())."""
        out = LbmParams()
        _check(self.lib.lbm_get_params(self._h, C.byref(out)), "lbm_get_params")
        return out


class _Member(Solver):
    """Borrowed view of an ensemble member (owned by the ensemble)."""

    def __init__(self, lib, handle, params):   # noqa: D401 - no Solver.__init__
        self.lib = lib
        self._h = handle
        self.params = params
        self.nx, self.ny = params.nx, params.ny

    def close(self):
        pass


class Ensemble:
    """Independent realisations advanced together by one launch per time step."""

    def __init__(self, members: list[LbmParams], stream=None):
        import torch

        lib = load_library()
        self.lib = lib
        self.params = list(members)
        arr = (LbmParams * len(members))(*members)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream or None
        self._e = C.c_void_p()
        _check(lib.lbm_ens_create(len(members), arr, C.c_void_p(stream) if stream else None, C.byref(self._e)),
               "lbm_ens_create")
        self.members = []
        for i, p in enumerate(self.params):
            h = C.c_void_p()
            _check(lib.lbm_ens_member(self._e, i, C.byref(h)), "lbm_ens_member")
            self.members.append(_Member(lib, h, p))

    def step(self, n: int = 1):
        _check(self.lib.lbm_ens_step(self._e, int(n)), "lbm_ens_step")

    def sync(self):
        _check(self.lib.lbm_ens_sync(self._e), "lbm_ens_sync")

    def diagnostics(self, check: bool = True) -> list[dict]:
        """Every member's diagnostics; with check=False an unstable member's status is
        reported in its dict instead of raising."""
        out = (LbmDiag * len(self.params))()
        st = self.lib.lbm_ens_diagnostics(self._e, out)
        if check or st not in (LBM_OK, LBM_EUNSTABLE):
            _check(st, "lbm_ens_diagnostics")
        return [diag_dict(d) for d in out]

    @property
    def tile_width(self) -> int:
        v = C.c_int32()
        _check(self.lib.lbm_ens_tile_width(self._e, C.byref(v)), "lbm_ens_tile_width")
        return v.value

    def tune(self) -> tuple[int, float]:
        ty, ms = C.c_int32(), C.c_double()
        _check(self.lib.lbm_ens_tune(self._e, C.byref(ty), C.byref(ms)), "lbm_ens_tune")
        return ty.value, ms.value

    def close(self):
        if getattr(self, "_e", None) and self._e.value:
            self.lib.lbm_ens_destroy(self._e)
            self._e = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


CNN_PARAMS = 11588


class Cnn:
    """The closure CNN on device tensors of one image size: `forward` (FP32
    activations, the training path) and `infer` (tensor cores, BF16 activations).
    Arguments are torch CUDA tensors: params [CNN_PARAMS] float32, x and y
    [4, ny, nx] float32.  Calls are asynchronous on `stream` (default: the
    current torch stream); `status()` synchronises and raises if a bounded wait
    inside the inference kernels gave up."""

    def __init__(self, nx: int, ny: int, stream=None):
        import torch

        self.lib = load_library()
        self.nx, self.ny = int(nx), int(ny)
        n = C.c_size_t()
        _check(self.lib.lbm_cnn_workspace_bytes(self.nx, self.ny, C.byref(n)), "lbm_cnn_workspace_bytes")
        self.ws = torch.empty(n.value, dtype=torch.uint8, device="cuda")
        self._stream = stream

    def _st(self):
        import torch

        s = self._stream if self._stream is not None else torch.cuda.current_stream()
        return C.c_void_p(s.cuda_stream)

    def _args(self, params, x, y):
        for t in (params, x, y):
            assert t.is_cuda and t.dtype.is_floating_point and t.is_contiguous()
        return (C.c_void_p(params.data_ptr()), C.c_void_p(x.data_ptr()), self.nx, self.ny,
                C.c_void_p(self.ws.data_ptr()), self.ws.numel(), self._st(), C.c_void_p(y.data_ptr()))

    def forward(self, params, x, y):
        _check(self.lib.lbm_cnn_forward(*self._args(params, x, y)), "lbm_cnn_forward")

    def infer(self, params, x, y):
        _check(self.lib.lbm_cnn_infer(*self._args(params, x, y)), "lbm_cnn_infer")

    def infer_test_timeout(self, params, x, y):
        """Tests of the timeout path: the inference kernels with their copies withheld."""
        _check(self.lib.lbm_cnn_infer_test_timeout(*self._args(params, x, y)), "lbm_cnn_infer_test_timeout")

    def status(self):
        _check(self.lib.lbm_cnn_infer_status(C.c_void_p(self.ws.data_ptr()), self.nx, self.ny, self._st()),
               "lbm_cnn_infer_status")


class Closure:
    """Learned closure of a 2x-coarsened run (fine solver, coarse solver, CNN)."""

    def __init__(self, fine: LbmParams, interval: int = 10, seed: int = 0, stream=None):
        import torch

        self.lib = load_library()
        self.fine = fine
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream or None
        self._c = C.c_void_p()
        _check(self.lib.lbm_closure_create(C.byref(fine), int(interval), int(seed), C.c_void_p(stream) if stream else None,
                                           C.byref(self._c)), "lbm_closure_create")
        self.coarse = LbmParams()
        _check(self.lib.lbm_closure_coarse_params(C.byref(fine), C.byref(self.coarse)), "lbm_closure_coarse_params")

    def generate(self, n_runs: int, seed0: int, warmup: int, intervals: int):
        _check(self.lib.lbm_closure_generate(self._c, n_runs, seed0, warmup, intervals), "lbm_closure_generate")

    def train(self, epochs: int, lr: float = 1e-3, shuffle_seed: int = 0) -> float:
        loss = C.c_double()
        _check(self.lib.lbm_closure_train(self._c, epochs, lr, shuffle_seed, C.byref(loss)), "lbm_closure_train")
        return loss.value

    def evaluate(self, seed: int, warmup: int, intervals: int, use_net: int) -> tuple[list[dict], list[dict]]:
        """use_net: 0 no correction, 1 densities and velocity, 2 order parameter only,
        3 order parameter and a quarter of the velocity correction, 4 as 3 with the
        order parameter corrected on the interface only (weight 4 c (1 - c) of the
        normalised mass fraction)."""
        co = (LbmDiag * (intervals + 1))()
        fi = (LbmDiag * (intervals + 1))()
        _check(self.lib.lbm_closure_evaluate(self._c, seed, warmup, intervals, int(use_net), co, fi),
               "lbm_closure_evaluate")
        return [diag_dict(d) for d in co], [diag_dict(d) for d in fi]

    def advance(self, intervals: int, use_net: int):
        """Advance the coarse run by `intervals` corrected intervals (no fine run)."""
        _check(self.lib.lbm_closure_advance(self._c, int(intervals), int(use_net)), "lbm_closure_advance")

    def correct(self, use_net: int):
        """One correction of the coarse run's current state (no time steps)."""
        _check(self.lib.lbm_closure_correct(self._c, int(use_net)), "lbm_closure_correct")

    def run(self, coarse_steps: int) -> dict:
        """Production advance (mode 4 corrections, the fine solver as fallback); the
        coarse run's diagnostics afterwards."""
        d = LbmDiag()
        _check(self.lib.lbm_closure_run(self._c, int(coarse_steps), C.byref(d)), "lbm_closure_run")
        return diag_dict(d)

    @property
    def fallbacks(self) -> int:
        n = C.c_int64()
        _check(self.lib.lbm_closure_fallbacks(self._c, C.byref(n)), "lbm_closure_fallbacks")
        return n.value

    def params(self) -> np.ndarray:
        out = np.empty(CNN_PARAMS, dtype=np.float32)
        _check(self.lib.lbm_closure_params(self._c, out.ctypes.data_as(_P(C.c_float)), 0), "lbm_closure_params")
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(self.lib.lbm_closure_params(self._c, p.ctypes.data_as(_P(C.c_float)), 1), "lbm_closure_params")

    def solvers(self) -> tuple["Solver", "Solver"]:
        """Borrowed views of the fine and coarse solvers (owned by the closure)."""
        f, c = C.c_void_p(), C.c_void_p()
        _check(self.lib.lbm_closure_solvers(self._c, C.byref(f), C.byref(c)), "lbm_closure_solvers")
        return _Member(self.lib, f, self.fine), _Member(self.lib, c, self.coarse)

    def normalisation(self) -> np.ndarray:
        out = np.empty(12, dtype=np.float32)
        _check(self.lib.lbm_closure_normalisation(self._c, out.ctypes.data_as(_P(C.c_float))), "lbm_closure_normalisation")
        return out

    def set_normalisation(self, in_mean, in_scale, out_scale):
        v = np.ascontiguousarray(np.concatenate([in_mean, in_scale, out_scale]), dtype=np.float32)
        if v.size != 12:
            raise ValueError("normalisation: 4 input means, 4 input scales, 4 output scales")
        _check(self.lib.lbm_closure_set_normalisation(self._c, v.ctypes.data_as(_P(C.c_float))),
               "lbm_closure_set_normalisation")

    def close(self):
        if getattr(self, "_c", None) and self._c.value:
            self.lib.lbm_closure_destroy(self._c)
            self._c = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
