"""Physics at the paper's parameters through the CUDA path (GPU).

The Laplace law of static droplets at the paper's coupling (Section 2: tau = 0.53,
G_AB = 0.1381, pure densities 1.10) against the surface tension of the oracle's
flat interface (its normal-minus-tangential stress excess, pinned in
tests/test_oracle_stress.py).  At tau = 0.53 the sound waves of the droplet box
are barely damped, so the pressure jump is averaged over the second half of a
long run.
"""
import numpy as np
import pytest

from oracle import lbm_oracle as O
from paper_2101_04847_gb300 import lbm
from tests.test_oracle_stress import PAPER, paper_flat_interface

pytestmark = pytest.mark.gpu
CS2 = 1.0 / 3.0


def droplet_tension(R, n, maj=1.10, mino=0.075, chunks=40, chunk=10000):
    G, tau = PAPER["G_immiscible"], PAPER["tau"]
    p = lbm.default_params(nx=n, ny=n, tau_A=tau, tau_B=tau, G=G, g=0.0, mass_A=maj, mass_B=maj, n_modes=0,
                           minority=0.0, crop_rows=3)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    r = np.hypot(x - n / 2 + 0.5, y - n / 2 + 0.5)
    H = 0.5 * (1 - np.tanh((r - R) / 2.0))
    rA, rB = mino + (maj - mino) * H, mino + (maj - mino) * (1 - H)
    z = np.zeros_like(rA)
    series = []
    with lbm.Solver(p) as s:
        s.set_populations(np.stack([O.equilibrium(rA, z, z), O.equilibrium(rB, z, z)]))
        for k in range(chunks):
            s.step(chunk)
            if k < chunks // 2:
                continue
            f = s.fields()
            a, b = f["rhoA"], f["rhoB"]
            pb = CS2 * (a + b) + G * CS2 * a * b
            Reff = np.sqrt(np.sum(a - b > 0) / np.pi)
            inside = pb[r < 0.5 * Reff].mean()
            outside = pb[(r > Reff + 10) & (y > 12) & (y < n - 13)].mean()
            series.append((inside - outside) * Reff)
    return float(np.mean(series))


def test_laplace_law_at_the_paper_coupling(gpu):
    bond, spurious = paper_flat_interface()
    sigma_flat = bond + spurious
    got = [droplet_tension(32, 256), droplet_tension(48, 256)]
    print(f"\nLaplace sigma at the paper's coupling: droplets {got}, flat interface {sigma_flat:.5f}, "
          f"paper {PAPER['surface_tension']}")
    # (measured: droplets 0.00453 / 0.00451, flat interface 0.0046)
    for v in got:
        assert abs(v - sigma_flat) < 0.1 * sigma_flat


# The paper's parameter set (Section 2) on the small grid: tau = 0.53 (nu = 0.01),
# G_AB = 0.1381 (immiscible) with the coexistence minority of 6.8 %, pure densities
# 1.10, g = 9e-6; an interface of 8 modes (wavelengths of 16 cells and more) and
# amplitude 4.  (64 modes on 128 columns make wavelengths of 2 cells, steeper than
# the interface is wide: the oracle's densities then go negative in the first steps.)
PAPER_SMALL = dict(nx=128, ny=256, tau_A=0.53, tau_B=0.53, G=0.1381, mass_A=1.1, mass_B=1.1, g=9e-6,
                   n_modes=8, amp=4.0, width=1.5, minority=0.068, crop_rows=10, seed=3)


@pytest.fixture(scope="module")
def paper_small_oracle():
    p = O.Params(**PAPER_SMALL)
    f = O.step(O.initial_populations(p), p, 1000)
    return O.fields(f, p), O.diagnostics(f, p)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_paper_parameters_1000_steps(gpu, storage, paper_small_oracle):
    # low tau is the stiffest case for the FP32 repair and for 16-bit storage: FP32
    # keeps the 1e-5 density contract; FP16 stays within its bound of the default
    # workload (0.02 on the densities) and conserves mass
    ref, rdiag = paper_small_oracle
    with lbm.Solver(storage=storage, **PAPER_SMALL) as s:
        s.step(1000)
        got = s.fields()
        d = s.diagnostics()
    err = max(float(np.max(np.abs(got[k] - ref[k])) / np.max(np.abs(ref[k]))) for k in ("rhoA", "rhoB"))
    print(f"\npaper parameters, {storage}: density error {err:.2e}, mass error "
          f"{abs(d['mass_A'] - rdiag['mass_A']) / rdiag['mass_A']:.1e}")
    assert err <= {"f32": 1e-5, "f16": 0.02}[storage]
    assert abs(d["mass_A"] - rdiag["mass_A"]) <= {"f32": 1e-6, "f16": 1e-4}[storage] * rdiag["mass_A"]
    assert d["status"] == lbm.LBM_OK
