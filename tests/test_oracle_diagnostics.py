"""Pins of the oracle's diagnostics (Section 3) against identities, closed forms
and the dynamics of the solver itself (no GPU)."""
import math

import numpy as np
import pytest

from oracle import lbm_oracle as O


def fields_params(nx, ny, **kw):
    d = dict(nx=nx, ny=ny, G=1.4, tau_A=1.0, tau_B=1.0, g=1e-5, crop_rows=10)
    d.update(kw)
    return O.Params(**d)


# ---------------------------------------------------------------- interface length
def test_cauchy_crofton_counts_of_a_horizontal_interface():
    nx, ny = 40, 30
    phi = np.where(np.arange(ny)[:, None] >= 15, 1.0, -1.0) * np.ones((1, nx))
    cc = O.cauchy_crofton_counts(phi, 5, 25)
    assert cc.tolist() == [0, nx, nx, nx]
    assert math.isclose(O.cauchy_crofton_length(cc), math.pi / 8 * (1 + math.sqrt(2)) * nx, rel_tol=1e-15)


def test_cauchy_crofton_counts_of_a_vertical_strip():
    nx, ny, r0, r1 = 40, 30, 5, 25
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    phi = np.where((x >= 10) & (x < 22), 1.0, -1.0)
    cc = O.cauchy_crofton_counts(phi, r0, r1)
    rows = r1 - r0
    assert cc.tolist() == [2 * rows, 0, 2 * (rows - 1), 2 * (rows - 1)]


@pytest.mark.parametrize("R", [50.0, 80.0])
def test_cauchy_crofton_length_of_a_disk(R):
    n = 256
    y, x = np.mgrid[0:n, 0:n].astype(float)
    phi = R - np.hypot(x - 127.3, y - 128.6)
    L = O.cauchy_crofton_length(O.cauchy_crofton_counts(phi, 0, n))
    assert abs(L / (2 * math.pi * R) - 1.0) < 0.02


# ---------------------------------------------------------------- mixing width
def _width_of_profile(c, p):
    top, bot = O.bulk_mass_fraction(p)
    return O.mixing_width(bot + c * (top - bot), p)


def test_mixing_width_of_a_tanh_profile_is_three_half_widths():
    # 6 * integral of c (1 - c) for c = (1 + tanh(y / W)) / 2 equals 3 W
    p = fields_params(8, 400)
    for W in (2.0, 7.5, 20.0):
        y = np.arange(380) - 190.3
        c = 0.5 * (1 + np.tanh(y / W))
        # (the lattice sum differs from the integral by ~exp(-pi^2 W) terms)
        assert abs(_width_of_profile(c, p) - 3 * W) < 1e-6 * W


def test_mixing_width_of_a_linear_ramp():
    # c = (k + 1/2) / w on w rows: 6 sum c (1 - c) = w + 1 / (2 w)
    p = fields_params(8, 400)
    for w in (5, 40):
        c = np.concatenate([np.zeros(30), (np.arange(w) + 0.5) / w, np.ones(30)])
        assert abs(_width_of_profile(c, p) - (w + 0.5 / w)) < 1e-12 * w


def test_mixing_width_ignores_a_compression_of_the_bulks():
    # gravity compresses a tall column: both densities grow with depth by the same
    # factor, which shifts the bulk rho_A - rho_B but not the mass fraction
    p = fields_params(16, 400)
    y = np.arange(400, dtype=float)[:, None] * np.ones((1, 16))
    H = 0.5 * (1 + np.tanh((y - 200.3) / 3.0))
    eps = p.minority
    rhoA = p.mass_A * (eps + (1 - eps) * H)
    rhoB = p.mass_B * (eps + (1 - eps) * (1 - H))
    z = np.zeros_like(rhoA)
    flat = O.field_diagnostics(rhoA, rhoB, z, z, p)["h"]
    squeeze = 1.0 + 0.06 * (1.0 - y / 400.0)
    pressed = O.field_diagnostics(rhoA * squeeze, rhoB * squeeze, z, z, p)["h"]
    assert abs(pressed - flat) < 1e-9 * flat
    assert abs(flat - 9.0) < 0.5          # about 3 half-widths of the tanh (W = 3)


# ---------------------------------------------------------------- stress identities
def test_korteweg_flux_matches_minus_kappa_phi_grad_laplacian_phi():
    # Section 3, Eq. "Curvature and stress tensor": div P^K = -kappa phi grad(lap phi);
    # this holds only with |grad phi|^2 in the isotropic part of P^K.
    nx, ny = 128, 160
    p = fields_params(nx, ny, G=1.2)
    kappa = p.G / 36.0
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    kx, ky = 2 * math.pi / 64, 2 * math.pi / 80
    A, U = 0.4, 1e-3
    phi = A * np.cos(kx * x + 0.3) * np.sin(ky * y + 0.2)
    # analytic: lap phi = -(kx^2 + ky^2) phi, so -kappa phi grad lap phi = kappa K^2 phi grad phi
    K2 = kx * kx + ky * ky
    dphx = -A * kx * np.sin(kx * x + 0.3) * np.sin(ky * y + 0.2)
    dphy = A * ky * np.cos(kx * x + 0.3) * np.cos(ky * y + 0.2)
    # a smooth velocity along phi grad phi, so that the average does not vanish
    ux = U * phi * dphx / (A * A * kx)
    uy = U * phi * dphy / (A * A * ky)
    out = O.field_diagnostics(1.0 + phi / 2, 1.0 - phi / 2, ux, uy, p)
    R = slice(p.crop_rows, ny - p.crop_rows)
    exact = float(np.mean((kappa * K2 * phi * (ux * dphx + uy * dphy))[R]))
    assert abs(out["flux_K"] - exact) < 0.03 * abs(exact)


def test_viscous_term_equals_minus_two_eta_enstrophy_for_a_divergence_free_field():
    # Section 3, Eq. "Dissipation function": <u . div(eta grad u + eta grad u^T)> = -2 eta Omega / D.
    # For u = discrete curl of a stream function supported inside the averaged rows the
    # centred-difference identity is exact (summation by parts, div u = 0 exactly).
    nx, ny = 64, 96
    p = fields_params(nx, ny, tau_A=0.8, tau_B=0.8)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    ya, yb = 25.0, 70.0
    inside = (y > ya) & (y < yb)
    psi = np.where(inside, np.sin(2 * math.pi * x / nx) * np.sin(math.pi * (y - ya) / (yb - ya)) ** 4, 0.0) * 1e-3
    ux = O.ddy(psi)
    uy = -O.ddx(psi)
    ux[0], ux[-1] = 0.0, 0.0
    rho = np.ones((ny, nx))
    out = O.field_diagnostics(0.5 * rho, 0.5 * rho, ux, uy, p)
    Dn = nx * (ny - 2 * p.crop_rows)
    target = -2.0 * out["eta"] * out["enstrophy"] / Dn
    assert abs(out["viscous"] - target) < 1e-10 * abs(target)
    assert math.isclose(out["eta"], 1.0 * (0.8 - 0.5) / 3.0, rel_tol=1e-14)


# ---------------------------------------------------------------- budget against the dynamics
@pytest.mark.parametrize("G,eps", [(0.0, 0.0), (1.4, 0.08)])
def test_kinetic_energy_budget_closes_along_a_run(G, eps):
    # Section 3, Eq. "Kinetic energy balance": dE_k/dt = -<u . div P> + <u . div(eta ...)> - <u phi g e_y>
    # with <u . div P> split into bulk-pressure, Korteweg and tau parts (Eq. "Three parts of
    # the pressure tensor"); the time derivative is a centred difference over 2 steps.
    p = O.Params(nx=64, ny=128, G=G, g=1e-4, seed=3, amp=4.0, minority=eps,
                 mass_A=1.0, mass_B=1.0, crop_rows=10)
    f = O.step(O.initial_populations(p), p, 300)
    dt = 2
    D = []
    for k in range(25):
        if k:
            f = O.step(f, p, dt)
        D.append(O.diagnostics(f, p))
    Ek = np.array([d["E_k"] for d in D])
    for i in range(1, 24, 2):
        d = D[i]
        terms = np.array([-d["flux_pb"], -d["flux_K"], -d["flux_tau"], d["viscous"], -d["buoyancy"]])
        dEk = (Ek[i + 1] - Ek[i - 1]) / (2 * dt)
        assert abs(dEk - terms.sum()) < 0.08 * np.max(np.abs(terms)), (i, dEk, terms)


def test_energies_of_a_uniform_flow_and_flat_profile():
    nx, ny = 16, 60
    p = fields_params(nx, ny, g=2e-5)
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    phi = np.tanh((y - 30.0) / 3.0)
    rhoA, rhoB = 0.5 + phi / 2, 0.5 - phi / 2
    ux = np.full((ny, nx), 3e-3)
    uy = np.full((ny, nx), -2e-3)
    out = O.field_diagnostics(rhoA, rhoB, ux, uy, p)
    R = slice(10, 50)
    assert math.isclose(out["E_k"], 0.5 * 1.0 * (9e-6 + 4e-6), rel_tol=1e-12)
    assert math.isclose(out["E_p"], 2e-5 * float(np.mean((y * phi)[R])), rel_tol=1e-12)
    assert math.isclose(out["buoyancy"], 2e-5 * (-2e-3) * float(np.mean(phi[R])), rel_tol=1e-12, abs_tol=1e-20)
    assert out["enstrophy"] == 0.0
    assert abs(out["viscous"]) < 1e-20
