"""Pins of the pressure-tensor parts behind the budget diagnostics (Section 3, Eq.
"Three parts of the pressure tensor": bulk pressure p_b, Korteweg stress P^K and the
spurious tau-dependent stress K^(tau)) and of the surface tension the paper quotes
for its parameters (Section 2).  No GPU.

What pins them:
  * the Laplace law of static droplets (pressure jump times radius) against the
    normal-minus-tangential stress integrated across a flat interface of the same
    fluids: the interaction part of that integral is the mechanical (virial) stress
    of the pairwise Shan-Chen force, the kinetic part is K^(tau);
  * the paper's sigma = 0.0059 at tau = 0.53, G_AB = 0.1381, pure densities 1.10;
  * smooth analytic fields for which <u . grad p_b> and <u . div K^(tau)> follow
    from symbolic differentiation, approached at second order by the oracle's
    centred differences.
"""
import json
from pathlib import Path

import numpy as np
import pytest

from oracle import lbm_oracle as O

PAPER = json.loads((Path(__file__).resolve().parent / "golden" / "paper_values.json").read_text())
CS2 = 1.0 / 3.0


def _flat_interface(G, tau, mass, eps, ny, steps):
    """A flat A-over-B interface in a one-column periodic channel, relaxed for `steps`."""
    p = O.Params(nx=1, ny=ny, G=G, g=0.0, tau_A=tau, tau_B=tau, mass_A=mass, mass_B=mass,
                 n_modes=0, minority=eps, y0=ny / 2.0, crop_rows=3)
    r = O.densities(O.step(O.initial_populations(p), p, steps))
    return p, r[0], r[1]


def _bond_tension(G, rA, rB, lo, hi):
    """Integral of (P_yy - P_xx) across a flat interface from the pairwise force alone.

    The Shan-Chen force (Section 2, Eq. "Shan-Chen forcing term") is a sum of pair
    repulsions: sites x and x + c_i push each other apart along c_i with strength
    G w_i [rho_A(x) rho_B(x + c_i) + rho_B(x) rho_A(x + c_i)].  The virial of a pair
    contributes (strength) c_i^a c_i^b to the stress, shared half by each end; on a
    profile that depends on y only the tangential and normal parts differ by
    (c_iy^2 - c_ix^2), and in a uniform bulk the per-site sum vanishes (isotropy)."""
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    c = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    total = 0.0
    for y in range(lo, hi):
        for i in range(1, 9):
            cx, cy = c[i]
            pair = G * w[i] * (rA[y] * rB[y + cy] + rB[y] * rA[y + cy])
            total += 0.5 * pair * (cy * cy - cx * cx)
    return float(total)


def _stress_excess(T, name_yy, name_xx, lo, hi):
    return float(np.sum((T[name_yy] - T[name_xx])[lo:hi, 0]))


def _droplet_tension(G, tau, mass, eps, radii, n=64, steps=3000):
    """Laplace law in 2D: the bulk-pressure jump times the radius of a static droplet."""
    p = O.Params(nx=n, ny=n, G=G, g=0.0, tau_A=tau, tau_B=tau, n_modes=0, mass_A=mass, mass_B=mass)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    r = np.hypot(x - n / 2 + 0.5, y - n / 2 + 0.5)
    out = []
    for R in radii:
        H = 0.5 * (1 - np.tanh((r - R) / 1.5))
        rhoA, rhoB = mass * (eps + (1 - eps) * H), mass * (eps + (1 - eps) * (1 - H))
        z = np.zeros_like(rhoA)
        f = O.step(np.stack([O.equilibrium(rhoA, z, z), O.equilibrium(rhoB, z, z)]), p, steps)
        rs = O.densities(f)
        # bulk pressure: the ideal part plus the mean-field repulsion of the two components
        pb = CS2 * (rs[0] + rs[1]) + G * CS2 * rs[0] * rs[1]
        inside = pb[r < R / 2].mean()
        outside = pb[(r > R + 6) & (y > 5) & (y < n - 6)].mean()
        out.append((inside - outside) * R)
    return float(np.mean(out))


@pytest.fixture(scope="module")
def strong_coupling():
    """G = 1.4, tau = 1, equal masses: the droplets of the Laplace pin and a flat interface."""
    sigma_laplace = _droplet_tension(1.4, 1.0, 1.0, 0.07, (12.0, 16.0))
    p, rA, rB = _flat_interface(1.4, 1.0, 1.0, 0.07, 48, 8000)
    return sigma_laplace, p, rA[:, 0], rB[:, 0], O.stress_tensors(rA, rB, p)


def _tension_parts(p, rA, rB, T):
    ny = rA.shape[0]
    lo, hi = 4, ny - 4
    bond = _bond_tension(p.G, rA, rB, lo, hi)
    korteweg = _stress_excess(T, "PKyy", "PKxx", lo, hi)
    spurious = _stress_excess(T, "Kyy", "Kxx", lo, hi)
    return bond, korteweg, spurious


def test_droplet_tension_equals_the_stress_excess_of_a_flat_interface(strong_coupling):
    # Section 3: P = p_b I + P^K + K^(tau).  Across a flat interface the normal-minus-
    # tangential excess of P is the surface tension that the Laplace law measures on
    # droplets.  p_b is isotropic and drops out; the interaction stress is the virial of
    # the pair force (P^K is its gradient expansion) and K^(tau) is the kinetic stress the
    # forcing scheme adds, large at tau = 1 where (tau - 1/2)^2 = 1/4.
    sigma_l, p, rA, rB, T = strong_coupling
    bond, korteweg, spurious = _tension_parts(p, rA, rB, T)
    assert abs(bond + spurious - sigma_l) < 0.10 * sigma_l, (bond, spurious, sigma_l)
    assert spurious > 0.3 * sigma_l
    # the Korteweg tensor of the diagnostics (centred differences) follows the bond stress
    assert abs(korteweg - bond) < 0.15 * bond, (korteweg, bond)


def test_a_spurious_stress_linear_in_tau_minus_half_is_caught(strong_coupling, monkeypatch):
    # planted mistake: (tau - 1/2) instead of (tau - 1/2)^2 in K^(tau) doubles its share
    sigma_l, p, rA, rB, _ = strong_coupling
    monkeypatch.setattr(O, "spurious_coefficient", lambda tau: CS2 * CS2 * (tau - 0.5))
    T = O.stress_tensors(rA[:, None], rB[:, None], p)
    bond, _, spurious = _tension_parts(p, rA, rB, T)
    assert abs(bond + spurious - sigma_l) > 0.10 * sigma_l


def test_normal_stress_is_uniform_across_a_flat_interface(strong_coupling):
    # mechanical equilibrium of a flat interface: P_yy = p_b + P^K_yy + K_yy is the same
    # on every row, while p_b alone dips through the interface
    _, p, rA, rB, T = strong_coupling
    R = slice(4, rA.shape[0] - 4)
    pyy = (T["pb"] + T["PKyy"] + T["Kyy"])[R, 0]
    pb = T["pb"][R, 0]
    assert np.ptp(pyy) < 0.4 * np.ptp(pb), (np.ptp(pyy), np.ptp(pb))
    no_tau = (T["pb"] + T["PKyy"])[R, 0]
    assert np.ptp(pyy) < 0.75 * np.ptp(no_tau)


def paper_flat_interface(eps=0.068):
    """The paper's coupling (Section 2): tau = 0.53, G_AB = 0.1381, pure densities 1.10,
    read as the density of each component in its own phase, which holds the coexistence
    fraction of the other one (about 6.8 % of it; the relaxed profile must keep it)."""
    p, rA, rB = _flat_interface(PAPER["G_immiscible"], PAPER["tau"], PAPER["pure_density"], eps, 32, 30000)
    minority = float(rA[8, 0] / rB[8, 0])
    assert abs(minority - eps) < 0.01, minority
    T = O.stress_tensors(rA, rB, p)
    bond, _, spurious = _tension_parts(p, rA[:, 0], rB[:, 0], T)
    return bond, spurious


def test_surface_tension_at_the_paper_parameters():
    # Section 2 quotes sigma = 0.0059 from the pressure in large bubbles.  The flat
    # interface's stress excess (the pin above) gives 0.0046 under this reading, 22 %
    # below the quoted value (reading 1.10 as the total density gives 0.0035, and the
    # 9 % minority); droplets of radius 32 and 48 run by the CUDA path give the same
    # value through the Laplace law (tests/test_gpu_physics.py).  The paper gives no
    # error for sigma and calls its diffusion estimate rough; the bound is 30 %.
    bond, spurious = paper_flat_interface()
    sigma = bond + spurious
    assert abs(sigma - PAPER["surface_tension"]) < 0.3 * PAPER["surface_tension"], sigma
    # near tau = 1/2 the spurious stress is a small correction
    assert spurious < 0.05 * sigma


# ---------------------------------------------------------------- closed forms
def _analytic_fields(n_per_wave):
    """Smooth periodic-in-x fields, symbolic and on an nx x ny grid with n_per_wave
    cells per wavelength: rho_A, rho_B positive, u an arbitrary smooth vector."""
    sp = pytest.importorskip("sympy")
    X, Y = sp.symbols("x y", real=True)
    kx = 2 * sp.pi / n_per_wave
    ky = 2 * sp.pi / (sp.Rational(5, 4) * n_per_wave)
    rA = 0.6 + 0.25 * sp.sin(kx * X + 0.4) * sp.cos(ky * Y) + 0.1 * sp.cos(2 * kx * X - ky * Y)
    rB = 0.5 - 0.2 * sp.cos(kx * X) * sp.sin(ky * Y + 0.3)
    ux = 1e-2 * sp.cos(kx * X) * sp.sin(2 * ky * Y + 0.1)
    uy = 1e-2 * sp.sin(kx * X + 0.7) * sp.cos(ky * Y)
    return sp, X, Y, rA, rB, ux, uy


def _symbolic_fluxes(G, tau, n_per_wave):
    sp, X, Y, rA, rB, ux, uy = _analytic_fields(n_per_wave)
    rho, phi = rA + rB, rA - rB
    pb = sp.Rational(1, 3) * rho + G * sp.Rational(1, 3) / 4 * (rho ** 2 - phi ** 2)
    # K^(tau) = cs^4 (tau - 1/2)^2 (rho_A rho_B / rho) v (x) v, v = grad ln rho_A - grad ln rho_B
    vx = sp.diff(rA, X) / rA - sp.diff(rB, X) / rB
    vy = sp.diff(rA, Y) / rA - sp.diff(rB, Y) / rB
    c = sp.Rational(1, 9) * (tau - sp.Rational(1, 2)) ** 2 * rA * rB / rho
    Kxx, Kxy, Kyy = c * vx * vx, c * vx * vy, c * vy * vy
    fpb = ux * sp.diff(pb, X) + uy * sp.diff(pb, Y)
    ftau = ux * (sp.diff(Kxx, X) + sp.diff(Kxy, Y)) + uy * (sp.diff(Kxy, X) + sp.diff(Kyy, Y))
    names = (rA, rB, ux, uy, fpb, ftau)
    return [sp.lambdify((X, Y), e, "numpy") for e in names]


def _flux_errors(n_per_wave):
    G, tau = 1.2, 0.9
    nx, ny = n_per_wave, int(round(2.5 * n_per_wave))
    fA, fB, fux, fuy, fpb, ftau = _symbolic_fluxes(G, tau, n_per_wave)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    ev = lambda fn: np.broadcast_to(fn(x, y), (ny, nx)).astype(float)
    p = O.Params(nx=nx, ny=ny, G=G, tau_A=tau, tau_B=tau, crop_rows=max(3, ny // 10))
    out = O.field_diagnostics(ev(fA), ev(fB), ev(fux), ev(fuy), p)
    R = slice(p.crop_rows, ny - p.crop_rows)
    exact_pb = float(np.mean(ev(fpb)[R]))
    exact_tau = float(np.mean(ev(ftau)[R]))
    return (out["flux_pb"] - exact_pb) / abs(exact_pb), (out["flux_tau"] - exact_tau) / abs(exact_tau)


def test_bulk_pressure_and_spurious_fluxes_converge_to_the_closed_forms():
    # centred differences are second order: doubling the resolution divides the error by ~4
    e1 = np.abs(_flux_errors(32))
    e2 = np.abs(_flux_errors(64))
    assert np.all(e2 < 0.02), e2
    ratio = e1 / e2
    assert np.all((ratio > 3.0) & (ratio < 5.5)), ratio


# ---------------------------------------------------------------- interface energy
def test_korteweg_flux_follows_the_interface_energy(strong_coupling):
    # Section 3, Eq. "Korteweg stress and total length": <(div P^K) . u> ~ (1/D) d(gamma L)/dt,
    # L the Cauchy-Crofton length.  Integrated over the nonlinear growth of a
    # Rayleigh-Taylor interface (L grows from 140 to 750 cells), the Korteweg flux
    # equals the change of gamma L / D within 15 % (measured 0.90); gamma is the
    # Korteweg part of the flat interface's tension, the part P^K carries (the whole
    # Laplace tension, twice as large at tau = 1, misses by a factor of two).
    _, p1, rA, rB, T = strong_coupling
    lo, hi = 4, rA.shape[0] - 4
    gamma_k = float(np.sum((T["PKyy"] - T["PKxx"])[lo:hi, 0]))
    p = O.Params(nx=128, ny=256, G=1.4, g=3e-4, seed=3, amp=4.0, n_modes=2, mass_A=1.0, mass_B=1.0,
                 minority=0.07, crop_rows=10)
    f = O.step(O.initial_populations(p), p, 1000)
    D = p.nx * (p.ny - 2 * p.crop_rows)
    every = 50
    ts, flux, L = [], [], []
    for n in range(1000, 3001, every):
        if n > 1000:
            f = O.step(f, p, every)
        d = O.diagnostics(f, p)
        ts.append(n)
        flux.append(d["flux_K"])
        L.append(d["L_int"])
    assert L[-1] > 4 * L[0]
    work = float(np.trapezoid(flux, ts))
    energy = gamma_k * (L[-1] - L[0]) / D
    assert 0.85 < work / energy < 1.15, (work, energy)
