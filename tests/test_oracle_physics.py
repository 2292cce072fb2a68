"""Physics pins of the oracle (no GPU): conservation, closed forms and the
numbers the paper prints for its parameter set (Section 2)."""
import json
import math
from pathlib import Path

import numpy as np
import pytest

from oracle import lbm_oracle as O

PAPER = json.loads((Path(__file__).resolve().parent / "golden" / "paper_values.json").read_text())
CS2 = 1.0 / 3.0


def state_from_densities(rhoA, rhoB):
    z = np.zeros_like(rhoA)
    return np.stack([O.equilibrium(rhoA, z, z), O.equilibrium(rhoB, z, z)])


def test_mass_of_each_component_is_conserved():
    p = O.Params(nx=48, ny=64, G=1.4, g=1e-4, seed=9, amp=4.0)
    f = O.initial_populations(p)
    m0 = O.densities(f).sum(axis=(1, 2))
    f = O.step(f, p, 400)
    m1 = O.densities(f).sum(axis=(1, 2))
    assert np.all(np.abs(m1 - m0) <= 1e-12 * m0)


def test_paper_viscosity_value():
    # Section 2: tau = 0.53 gives nu = cs^2 (tau - 1/2) = 0.01
    assert math.isclose(CS2 * (PAPER["tau"] - 0.5), PAPER["nu"], rel_tol=1e-12)


def _channel(tau, ny, steps, gx=1e-6):
    p = O.Params(nx=4, ny=ny, G=0.0, g=0.0, gx=gx, n_modes=0, minority=0.5,
                 mass_A=1.0, mass_B=1.0, tau_A=tau, tau_B=tau)
    f = O.step(O.initial_populations(p), p, steps)
    ux, uy = O.physical_velocity(f, p)
    return ux[:, 0], uy


def test_poiseuille_parabola_at_the_exact_bounce_back_tau():
    # Body-forced channel with half-way bounce-back walls at y = -1/2 and ny - 1/2: the BGK
    # solution is the exact parabola gx (y + 1/2)(ny - 1/2 - y) / (2 nu) when
    # tau = 1/2 + sqrt(3/16) (textbook result for half-way bounce-back).
    tau, ny, gx = 0.5 + math.sqrt(3.0 / 16.0), 16, 1e-6
    u, uy = _channel(tau, ny, 6000, gx)
    nu = CS2 * (tau - 0.5)
    y = np.arange(ny)
    exact = gx * (y + 0.5) * (ny - 0.5 - y) / (2.0 * nu)
    assert np.max(np.abs(u - exact)) < 1e-8 * exact.max()
    assert np.abs(uy).max() < 1e-13   # rounding level


@pytest.mark.parametrize("tau", [0.6, 1.0])
def test_poiseuille_curvature_is_minus_force_over_viscosity(tau):
    ny, gx = 16, 1e-6
    nu = CS2 * (tau - 0.5)
    steps = int(30 * ny * ny / (math.pi ** 2 * nu))
    u, _ = _channel(tau, ny, steps, gx)
    d2 = u[2:] - 2 * u[1:-1] + u[:-2]
    assert np.max(np.abs(d2 + gx / nu)) < 1e-7 * gx / nu
    assert np.max(np.abs(u - u[::-1])) < 1e-9 * u.max()


def _flat_interface(G, tau, mass, eps, ny, steps):
    p = O.Params(nx=2, ny=ny, G=G, g=0.0, tau_A=tau, tau_B=tau, mass_A=mass, mass_B=mass,
                 n_modes=0, minority=eps, y0=ny / 2.0)
    f = O.step(O.initial_populations(p), p, steps)
    return p, f


def _gradient_width(phi_col):
    span = phi_col.max() - phi_col.min()
    return span / np.max(np.abs(np.diff(phi_col)))


def test_flat_interface_at_rest_has_equal_bulk_pressures():
    p, f = _flat_interface(1.4, 1.0, 1.0, 0.08, 48, 24000)
    ux, uy = O.physical_velocity(f, p)
    assert np.max(np.hypot(ux, uy)) < 1e-8
    r = O.densities(f)
    rho, rAB = r[0] + r[1], r[0] * r[1]
    pb = CS2 * rho + p.G * CS2 * rAB
    col = pb[:, 0]
    # bulk B at y = 12 and bulk A at y = 36: 12 rows from the interface and from the
    # walls (the wall rows, where the pseudopotential outside is 0, perturb ~8 rows)
    assert abs(col[12] - col[36]) < 1e-7 * col[12]
    assert 2.0 < _gradient_width((r[0] - r[1])[:, 0]) < 4.5


def test_paper_parameters_minority_fraction_and_interface_width():
    # Section 2: with tau 0.53, G_AB 0.1381 and pure densities 1.10 each phase holds
    # about 9 % of the other component and the interface is about 3 nodes wide.
    p, f = _flat_interface(PAPER["G_immiscible"], PAPER["tau"], PAPER["pure_density"], 0.02, 24, 40000)
    r = O.densities(f)
    # the B-rich bulk (bottom, away from the wall row) and the A-rich bulk (top)
    minority_bottom = r[0, 5, 0] / r[1, 5, 0]
    minority_top = r[1, 18, 0] / r[0, 18, 0]
    for frac in (minority_bottom, minority_top):
        assert abs(frac - PAPER["minority_fraction"]) < 0.3 * PAPER["minority_fraction"], frac
    w = _gradient_width((r[0] - r[1])[:, 0])
    assert abs(w - PAPER["interface_width_nodes"]) < 1.0, w


def _diffusion_coefficient(G, tau, rho_tot, nx, ny, steps, a=0.01):
    """Decay rate of a small sinusoidal order-parameter mode along x, divided by k^2,
    measured on the middle row of a tall channel (away from the walls)."""
    p = O.Params(nx=nx, ny=ny, G=G, g=0.0, tau_A=tau, tau_B=tau, n_modes=0)
    k = 2.0 * math.pi / nx
    s = np.sin(k * np.arange(nx))[None, :] * np.ones((ny, 1))
    f = state_from_densities(0.5 * rho_tot * (1 + a * s), 0.5 * rho_tot * (1 - a * s))
    ts, amps = [], []
    chunk = steps // 10
    for t in range(11):
        if t:
            f = O.step(f, p, chunk)
        r = O.densities(f)
        amps.append(np.sum((r[0] - r[1])[ny // 2] * s[0]) * 2.0 / nx)
        ts.append(t * chunk)
    rate = -np.polyfit(ts[3:], np.log(np.abs(amps[3:])), 1)[0]
    return rate / (k * k), amps


@pytest.mark.parametrize("tau", [1.0, 0.7])
def test_pure_diffusion_at_zero_coupling(tau):
    # G = 0: the order parameter diffuses with D = cs^2 (tau - 1/2)
    D, _ = _diffusion_coefficient(0.0, tau, 1.0, nx=32, ny=96, steps=1500 if tau == 1.0 else 3000)
    assert abs(D - CS2 * (tau - 0.5)) < 0.01 * CS2 * (tau - 0.5)


@pytest.mark.parametrize("G,tau", [(0.5, 1.0), (0.3, 0.7)])
def test_diffusion_reduced_by_coupling_as_in_the_paper_estimate(G, tau):
    # Section 2: D ~ cs^2 [(tau - 1/2) - rho tau G / 2]; a long wave (k = 2 pi / 32) keeps
    # the lattice correction of the neighbour sum (sin k / k) below 1 %
    D, _ = _diffusion_coefficient(G, tau, 1.0, nx=32, ny=96, steps=3000)
    est = CS2 * ((tau - 0.5) - 1.0 * tau * G / 2.0)
    assert abs(D - est) < 0.03 * est


def test_paper_miscible_diffusion_estimate():
    # Section 2: for G_AB = 0.0805, tau = 0.53, rho = 1.1 the rough estimate is D = 0.002
    G, tau, rho = PAPER["G_miscible"], PAPER["tau"], PAPER["pure_density"]
    D, _ = _diffusion_coefficient(G, tau, rho, nx=16, ny=64, steps=8000)
    est = CS2 * ((tau - 0.5) - rho * tau * G / 2.0)
    assert abs(est - PAPER["diffusion_estimate"]) < 0.1 * PAPER["diffusion_estimate"]
    assert abs(D - est) < 0.25 * est


def test_spinodal_threshold_of_the_estimate():
    # the estimate changes sign at G_c = 2 (tau - 1/2) / (rho tau) = 1 for tau = 1, rho = 1:
    # below it a small mode decays, above it the mode grows (phase separation)
    _, below = _diffusion_coefficient(0.9, 1.0, 1.0, nx=16, ny=48, steps=2000)
    _, above = _diffusion_coefficient(1.1, 1.0, 1.0, nx=16, ny=48, steps=2000)
    assert abs(below[-1]) < 0.5 * abs(below[0])
    assert abs(above[-1]) > 2.0 * abs(above[0])


def _droplet_pressure_jump(R, n=64, steps=3000):
    p = O.Params(nx=n, ny=n, G=1.4, g=0.0, n_modes=0, mass_A=1.0, mass_B=1.0)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    r = np.hypot(x - n / 2 + 0.5, y - n / 2 + 0.5)
    H = 0.5 * (1 - np.tanh((r - R) / 1.5))
    eps = 0.07
    f = state_from_densities(eps + (1 - eps) * H, eps + (1 - eps) * (1 - H))
    f = O.step(f, p, steps)
    rs = O.densities(f)
    pb = CS2 * (rs[0] + rs[1]) + p.G * CS2 * rs[0] * rs[1]
    inside = pb[r < R / 2].mean()
    outside = pb[(r > R + 6) & (y > 5) & (y < n - 6)].mean()
    return inside - outside


def test_laplace_law_for_droplets():
    # 2D Laplace law: dp = sigma / R, the same sigma for every radius
    Rs = np.array([8.0, 12.0, 16.0])
    dps = np.array([_droplet_pressure_jump(R) for R in Rs])
    A = np.vstack([1.0 / Rs, np.ones_like(Rs)]).T
    (sigma, icpt), *_ = np.linalg.lstsq(A, dps, rcond=None)
    pred = A @ np.array([sigma, icpt])
    r2 = 1 - np.sum((dps - pred) ** 2) / np.sum((dps - dps.mean()) ** 2)
    assert r2 > 0.995
    assert sigma > 0
    assert abs(icpt) < 0.1 * dps.min()
    assert np.ptp(dps * Rs) < 0.05 * np.mean(dps * Rs)


# ---------------------------------------------------------------------------
# Small-amplitude Rayleigh-Taylor growth with viscosity and surface tension.
#
# The Boussinesq pair of Section 2 (A on top pushed down by -rho_A g, B below
# pushed up by +rho_B g, equal bulk densities rho0 and equal nu = cs2 (tau - 1/2))
# is the symmetric two-layer problem, whose linear normal modes follow from the
# Stokes-type equations gamma u = -grad p / rho0 + nu lap u on either side of a
# sharp interface: with w = A e^{-k|z|} + B e^{-m|z|}, m^2 = k^2 + gamma / nu,
# continuity of u and w forces k A + m B = 0, and the normal-stress jump
# (buoyancy jump Delta_f eta minus surface tension sigma k^2 eta) gives
#     gamma^2 = k (Delta_f - sigma k^2) / (2 rho0) * (1 - k / m),
# Delta_f = g [(rho_A - rho_B)_top + (rho_B - rho_A)_bottom].
# Limits: nu -> 0 gives the inviscid gamma^2 = k (Delta_f - sigma k^2) / (2 rho0);
# gamma << nu k^2 gives the Stokes rate (Delta_f - sigma k^2) / (4 rho0 nu k).
# ---------------------------------------------------------------------------
def _rt_rate_viscous(k, df, sigma, rho0, nu):
    drive = k * (df - sigma * k * k) / (2.0 * rho0)
    lo, hi = 0.0, math.sqrt(max(drive, 0.0)) + 1e-30
    for _ in range(200):   # bisection: the right-hand side grows slower than gamma^2
        mid = 0.5 * (lo + hi)
        if mid * mid - drive * (1.0 - k / math.sqrt(k * k + mid / nu)) > 0.0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def test_viscous_rt_dispersion_relation_limits():
    k, df, sigma, rho0 = 0.05, 5e-4, 0.05, 1.0
    inviscid = math.sqrt(k * (df - sigma * k * k) / (2 * rho0))
    assert _rt_rate_viscous(k, df, sigma, rho0, 1e-9) == pytest.approx(inviscid, rel=1e-3)
    nu = 50.0
    assert _rt_rate_viscous(k, df, sigma, rho0, nu) == pytest.approx((df - sigma * k * k) / (4 * rho0 * nu * k), rel=1e-3)
    # below the capillary cut-off k_c = sqrt(Delta_f / sigma) nothing grows
    assert _rt_rate_viscous(0.2, df, sigma, rho0, 0.1) < 1e-12


def _rt_single_mode(nx, ny, g, amp, steps, every, eps=0.08, width=1.5):
    p = O.Params(nx=nx, ny=ny, G=1.4, g=g, n_modes=0, mass_A=1.0, mass_B=1.0)
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    H = 0.5 * (1 + np.tanh((y - ny / 2 - amp * np.cos(2 * np.pi * x / nx)) / width))
    f = state_from_densities(eps + (1 - eps) * H, eps + (1 - eps) * (1 - H))
    ts, amps = [], []
    for n in range(0, steps + 1, every):
        if n:
            f = O.step(f, p, every)
        r = O.densities(f)
        # the first x-Fourier mode of the column sums of phi is proportional to eta_1
        amps.append(abs(np.fft.rfft((r[0] - r[1]).sum(axis=0))[1]))
        ts.append(n)
    return np.array(ts, dtype=float), np.array(amps), O.densities(f)


@pytest.mark.parametrize("nx", [128, 96])
def test_small_amplitude_viscous_rt_growth_rate(nx):
    # sigma from the Laplace law of static droplets, then the growth rate of one
    # interface mode (amplitude 0.25 -> ~2.5 cells, k eta <= 0.15) against the
    # viscous dispersion relation of a sharp interface: at most 8 % below it (the
    # tanh interface of half-width ~1.5 lowers the rate by O(k W) <= 0.1), while the
    # inviscid rate is >= 25 % above it.
    sigma = np.mean([_droplet_pressure_jump(R) * R for R in (12.0, 16.0)])
    g, ny = 3e-4, 192
    ts, amps, r = _rt_single_mode(nx, ny, g, 0.25, 1200, 50)
    window = ts >= 600
    rate = np.polyfit(ts[window], np.log(amps[window]), 1)[0]
    top = r[:, ny - 40:ny - 20].mean(axis=(1, 2))
    bot = r[:, 20:40].mean(axis=(1, 2))
    df = g * ((top[0] - top[1]) + (bot[1] - bot[0]))
    rho0 = 0.5 * (top.sum() + bot.sum())
    k = 2 * np.pi / nx
    viscous = _rt_rate_viscous(k, df, sigma, rho0, CS2 * 0.5)
    inviscid = math.sqrt(k * (df - sigma * k * k) / (2 * rho0))
    assert 0.0 < 1.0 - rate / viscous < 0.08, (rate, viscous)
    assert inviscid / viscous > 1.25
