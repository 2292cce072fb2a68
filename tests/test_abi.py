"""The C-ABI library builds, loads and exports every symbol include/lbm.h
declares; host-side parameter handling (no GPU needed, no compute calls)."""
import ctypes as C
import re
from pathlib import Path

import pytest

from paper_2101_04847_gb300 import lbm

HEADERS = sorted((Path(__file__).resolve().parents[1] / "include").glob("*.h"))


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        names |= set(re.findall(r"\b(lbm\w*)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "lbm_step" in names and "lbm_diagnostics" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_status_strings(lib):
    for st in range(8):
        assert lib.lbm_status_str(st)
    assert lib.lbm_status_str(99) == b"unknown status"


def test_defaults(lib):
    p = lbm.default_params()
    assert (p.nx, p.ny) == (128, 256)
    assert (p.tau_A, p.tau_B, p.G, p.mass_A, p.mass_B, p.g) == (1.0, 1.0, 1.4, 1.0, 0.9, 1e-5)
    assert (p.n_modes, p.amp, p.width, p.crop_rows, p.storage, p.kernel) == (8, 2.0, 1.5, 10, 0, lbm.KERNEL["staged"])


def test_workspace_grows_with_the_grid(lib):
    small = lbm.workspace_bytes(lbm.default_params(nx=128, ny=256))
    big = lbm.workspace_bytes(lbm.default_params(nx=1024, ny=2048))
    assert small > 128 * 256 * 144
    assert 20 < big / small < 70
    half = lbm.workspace_bytes(lbm.default_params(nx=1024, ny=2048, storage="f16"))
    assert half < big


@pytest.mark.parametrize("field,value", [
    ("nx", 3), ("ny", 7), ("tau_A", 0.5), ("tau_B", 0.4), ("mass_A", 0.0), ("mass_B", -1.0),
    ("width", 0.0), ("minority", 1.0), ("n_modes", 65), ("crop_rows", 2), ("storage", 3),
    ("kernel", 6), ("kernel", -1), ("tile_y", -1), ("gravity_mode", 2), ("G", float("nan")), ("g", float("inf")),
    ("tile_x", 64), ("tile_x", -1), ("wall_mode", 2), ("wall_mode", -1), ("x_offset", 5), ("x_offset", -1),
    ("nx_total", -3), ("nx_total", 100),
])
def test_invalid_parameters_are_rejected(lib, field, value):
    p = lbm.default_params()
    setattr(p, field, value)
    n = C.c_size_t()
    assert lib.lbm_workspace_bytes(C.byref(p), C.byref(n)) == lbm.LBM_EINVAL
    assert lib.lbm_last_error()
    h = C.c_void_p()
    assert lib.lbm_create_ex(C.byref(p), None, 0, None, C.byref(h)) == lbm.LBM_EINVAL
    assert not h.value


def test_crop_must_leave_rows(lib):
    p = lbm.default_params(ny=24, crop_rows=12)
    n = C.c_size_t()
    assert lib.lbm_workspace_bytes(C.byref(p), C.byref(n)) == lbm.LBM_EINVAL


def test_null_arguments(lib):
    assert lib.lbm_params_default(None) == lbm.LBM_EINVAL
    assert lib.lbm_create_ex(None, None, 0, None, None) == lbm.LBM_EINVAL
    assert lib.lbm_step(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm_diagnostics(None, None) == lbm.LBM_EINVAL
    lib.lbm_destroy(None)


def test_ctypes_layout_matches_the_header_order():
    # the binding's structures list the header's fields in order
    hdr = (Path(__file__).resolve().parents[1] / "include" / "lbm.h").read_text()
    body = hdr[hdr.index("typedef struct {"):hdr.index("} lbm_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        m = re.match(r"\s*(?:typedef struct \{)?\s*(?:int32_t|double|uint64_t)\s+(.*)", decl, flags=re.S)
        if m:
            fields += [n.strip() for n in m.group(1).split(",")]
    assert fields == [name for name, _ in lbm.LbmParams._fields_]
