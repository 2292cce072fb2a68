"""Parity of the CUDA diagnostics and field extraction with the oracle (GPU).

Both sides evaluate the per-site terms from the same FP32-rounded populations:
the oracle in FP64, the GPU in double-float arithmetic (pairs of FP32 values,
about 44 significant bits) with FP64 block sums; the terms agree to ~1e-9 of
their scale and the crossing counts exactly.
"""
import numpy as np
import pytest

from oracle import lbm_oracle as O
from paper_2101_04847_gb300 import lbm
from tests import inputs

pytestmark = pytest.mark.gpu

TERMS = ["E_k", "E_p", "buoyancy", "flux_pb", "flux_K", "flux_tau", "viscous", "enstrophy", "rho_bar", "h"]


def oracle_params(d):
    return O.Params(**{k: v for k, v in d.items() if k in O.Params.__dataclass_fields__})


def evolved_state(d, steps):
    p = oracle_params(d)
    return inputs.as_float32(O.step(O.initial_populations(p), p, steps)), p


def check_diag(got, ref, rtol=1e-9):
    for k in ("mass_A", "mass_B"):
        assert abs(got[k] - ref[k]) <= 1e-12 * abs(ref[k]), k
    # scale of the budget terms: the largest of them (they can cross zero individually)
    flux_scale = max(abs(ref[k]) for k in ("flux_pb", "flux_K", "flux_tau", "viscous", "buoyancy"))
    for k in TERMS:
        scale = flux_scale if k in ("flux_pb", "flux_K", "flux_tau", "viscous", "buoyancy") else abs(ref[k])
        assert abs(got[k] - ref[k]) <= rtol * scale + 1e-300, (k, got[k], ref[k])
    assert got["cc"].tolist() == ref["cc"].tolist()
    assert abs(got["L_int"] - ref["L_int"]) <= 1e-12 * ref["L_int"]


@pytest.mark.parametrize("nx,ny,G,steps,wall_mode", [(96, 80, 1.4, 300, 0), (100, 70, 0.0, 150, 0), (33, 64, 1.4, 40, 0),
                                                  (96, 80, 1.4, 300, 1)])
def test_diagnostics_match_the_oracle(gpu, nx, ny, G, steps, wall_mode):
    d = inputs.params(inputs.C0, nx=nx, ny=ny, G=G, g=1e-4, amp=4.0,
                      minority=0.0 if G == 0.0 else 0.08, crop_rows=6, wall_mode=wall_mode)
    f, p = evolved_state(d, steps)
    ref = O.diagnostics(f, p)
    with lbm.Solver(**d) as s:
        s.set_populations(f)
        got = s.diagnostics()
        rows = s.profile()
    check_diag(got, ref)
    assert np.max(np.abs(rows - ref["phi_rows"])) <= 1e-12


@pytest.mark.parametrize("wall_mode", [0, 1])
def test_fields_match_the_oracle(gpu, wall_mode):
    d = inputs.params(inputs.C0, nx=70, ny=50, g=1e-4, G_wall_A=0.2, crop_rows=5, wall_mode=wall_mode)
    f, p = evolved_state(d, 100)
    ref = O.fields(f, p)
    with lbm.Solver(**d) as s:
        s.set_populations(f)
        got = s.fields()
    for k in ("rhoA", "rhoB", "ux", "uy"):
        assert np.max(np.abs(got[k] - ref[k])) <= 1e-13, k


def test_diagnostics_bench_configuration(gpu):
    # 1024 x 2048 (the measured workload) one oracle step after the initial state
    d = inputs.params(inputs.C1, seed=6)
    f, p = evolved_state(d, 1)
    ref = O.diagnostics(f, p)
    with lbm.Solver(**d) as s:
        s.set_populations(f)
        got = s.diagnostics()
    check_diag(got, ref, rtol=1e-8)
