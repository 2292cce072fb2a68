"""FP64 CPU oracle for the two-component D2Q9 Shan-Chen lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this module:
only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code, table or
constant generator with the CUDA library; it is written directly from the
paper (Tavares, Biferale, Sbragaglia, Mailybaev, arXiv 2101.04847, Section 2
"Lattice Boltzmann model" and Section 3 "Results and discussion") in plain
numpy, float64 throughout, whole-array operations in the paper's order.

State convention: ``f`` has shape (2, 9, ny, nx), component index 0 = A (the
heavy fluid, on top) and 1 = B; direction index as in ``C`` below; row y = 0 is
the bottom wall row, y = ny-1 the top wall row; x is periodic.  ``f`` always
holds the *post-streaming* populations f_i^s(x, t) of the kinetic equation
(Section 2, "Kinetic equation"), i.e. the quantities whose sums are the
densities of Eq. (1).

One time step (Section 2, "Kinetic equation" and "Equilibrium distribution"):
  1. rho_s = sum_i f_i^s, u = sum_{s,i} f_i^s c_i / tau_s / sum_s rho_s / tau_s
  2. F_s = F_s^ff + F_s^fb + F_s^ext (Shan-Chen, fluid-boundary, buoyancy)
  3. u'_s = u + tau_s F_s / rho_s,  f*_i = f_i - (f_i - f_i^eq(rho_s, u'_s)) / tau_s
  4. push-stream f*_i to x + c_i; a population that would cross the top or
     bottom wall comes back at its own node as the opposite direction
     (half-way bounce-back, walls at y = -1/2 and y = ny - 1/2).

Readings of points the paper leaves open:
  * bounce-back variant: half-way (the paper only says "bounce-back");
  * the pseudopotential of a wall node is 0 (no fluid in the solid), and the
    wall indicator S is 1 on the virtual rows y = -1 and y = ny; wall_mode = 1
    instead mirrors the pseudopotential across the wall (the virtual row y = -1
    holds row 0's values, y = ny row ny - 1's), a neutral wall that exerts no
    Shan-Chen force on a uniform fluid;
  * weights are the textbook solution 4/9, 1/9, 1/36 of the isotropy
    conditions printed after the equilibrium distribution (pinned by a test);
  * diagnostic velocity: u_phys = (sum_{s,i} f c + F/2) / rho;
  * the garbled |grad phi^2| in the Korteweg tensor is read as |grad phi|^2;
  * eta = rho_bar * c_s^2 (tau - 1/2), rho_bar = mean density of the sub-domain;
  * mixing-layer width h = 6 sum_y cbar (1 - cbar) on the normalised row mean of
    the mass fraction rho_A / (rho_A + rho_B) (the definition lives in a companion
    paper we do not have);
  * interface length: 4-direction Cauchy-Crofton estimate, phi > 0 is "A".

Pins: tests/test_oracle_*.py check this module against closed forms,
invariants and the numbers the paper prints; none of them re-types a formula
of this file.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np

# --- D2Q9 lattice (Section 2: velocities (0,0), (+-c,0), (0,+-c), (+-c,+-c), c = 1)
C = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1],
              [1, 1], [-1, 1], [-1, -1], [1, -1]], dtype=np.int64)
# weights: the solution of the second- and fourth-order isotropy conditions
# sum_i w c^a c^b = cs^2 delta, sum_i w c^a c^b c^c c^d = cs^4 (ddd) with cs^2 = 1/3
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=np.float64)
OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6], dtype=np.int64)
CS2 = 1.0 / 3.0


@dataclass(frozen=True)
class Params:
    """Physical and run parameters (lattice units, dx = dt = 1)."""
    nx: int = 128
    ny: int = 256
    tau_A: float = 1.0
    tau_B: float = 1.0
    G: float = 1.4            # G_AB, Shan-Chen coupling (Section 2, Shan-Chen forcing term)
    G_wall_A: float = 0.0     # G_Ab (fluid-boundary force); the paper uses 0 (neutral wetting)
    G_wall_B: float = 0.0     # G_Bb
    mass_A: float = 1.0       # bulk density of pure A (top)
    mass_B: float = 0.9       # bulk density of pure B (bottom)
    g: float = 1e-5           # g~ of Eq. (3_Fex)
    gravity_mode: int = 0     # 0: Boussinesq pair -rho_A g e_y / +rho_B g e_y; 1: -rho_s g e_y for both
    gx: float = 0.0           # uniform body acceleration along x (tests only)
    seed: int = 1
    n_modes: int = 8
    amp: float = 2.0          # interface perturbation amplitude (cells)
    width: float = 1.5        # tanh half-width W of the initial interface
    minority: float = 0.08    # epsilon: fraction of the other component in each bulk
    y0: float | None = None   # mean interface height (default ny / 2)
    crop_rows: int = 10       # rows cut at top and bottom for averages (Section 3)
    wall_mode: int = 0        # pseudopotential beyond a wall: 0 = none (psi = 0), 1 = mirror of the wall row

    def with_(self, **kw) -> "Params":
        return replace(self, **kw)


# --------------------------------------------------------------------------
# splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
# generators", OOPSLA 2014): state += golden gamma; output = mix64 of state.
# --------------------------------------------------------------------------
_MASK = (1 << 64) - 1


def splitmix64_stream(seed: int, n: int) -> list[int]:
    state = seed & _MASK
    out = []
    for _ in range(n):
        state = (state + 0x9E3779B97F4A7C15) & _MASK
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        out.append(z ^ (z >> 31))
    return out


def uniform01(u64: int) -> float:
    """Top 53 bits of a 64-bit draw as a double in [0, 1)."""
    return (u64 >> 11) * (1.0 / 9007199254740992.0)


def interface_modes(seed: int, n_modes: int) -> tuple[np.ndarray, np.ndarray]:
    """Amplitudes a_m in [0,1) and phases theta_m in [0, 2 pi), drawn in the order a_1, theta_1, a_2, ..."""
    draws = splitmix64_stream(seed, 2 * n_modes)
    a = np.array([uniform01(draws[2 * m]) for m in range(n_modes)])
    th = np.array([2.0 * math.pi * uniform01(draws[2 * m + 1]) for m in range(n_modes)])
    return a, th


def interface_height(p: Params) -> np.ndarray:
    """y0(x) = ny/2 + amp * eta(x) / max|eta|, eta = sum_m a_m sin(2 pi m x / nx + theta_m)."""
    a, th = interface_modes(p.seed, p.n_modes)
    x = np.arange(p.nx, dtype=np.float64)
    eta = np.zeros(p.nx)
    for m in range(p.n_modes):
        eta += a[m] * np.sin(2.0 * math.pi * (m + 1) * x / p.nx + th[m])
    peak = np.max(np.abs(eta)) if p.n_modes > 0 else 0.0
    base = p.ny / 2.0 if p.y0 is None else p.y0
    if peak > 0.0:
        return base + p.amp * eta / peak
    return np.full(p.nx, base)


def initial_densities(p: Params) -> tuple[np.ndarray, np.ndarray]:
    """Tanh interface between pure A (top) and pure B (bottom), each bulk holding a
    fraction `minority` of the other component (Section 2, last paragraph: the run
    starts from an equilibrium immiscible configuration plus an interface deformation)."""
    y = np.arange(p.ny, dtype=np.float64)[:, None]
    H = 0.5 * (1.0 + np.tanh((y - interface_height(p)[None, :]) / p.width))
    eps = p.minority
    rhoA = p.mass_A * (eps + (1.0 - eps) * H)
    rhoB = p.mass_B * (eps + (1.0 - eps) * (1.0 - H))
    return rhoA, rhoB


def equilibrium(rho_s: np.ndarray, ux: np.ndarray, uy: np.ndarray) -> np.ndarray:
    """f_i^eq(rho, u') = rho w_i (1 + 3 c.u' + 9/2 (c.u')^2 - 3/2 u'.u')  (Eq. "Equilibrium distribution", c = 1)."""
    feq = np.empty((9,) + rho_s.shape)
    usq = ux * ux + uy * uy
    for i in range(9):
        cu = C[i, 0] * ux + C[i, 1] * uy
        feq[i] = rho_s * W[i] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq)
    return feq


def initial_populations(p: Params) -> np.ndarray:
    """f_i^s = f_i^eq(rho_s, 0) for the initial densities (fluid at rest)."""
    rhoA, rhoB = initial_densities(p)
    z = np.zeros_like(rhoA)
    return np.stack([equilibrium(rhoA, z, z), equilibrium(rhoB, z, z)])


# --------------------------------------------------------------------------
# moments and forces
# --------------------------------------------------------------------------
def densities(f: np.ndarray) -> np.ndarray:
    """rho_s = sum_i f_i^s  (Eq. 1).  Returns shape (2, ny, nx)."""
    return f.sum(axis=1)


def momenta(f: np.ndarray) -> np.ndarray:
    """j_s = sum_i f_i^s c_i.  Returns shape (2 components, 2 axes, ny, nx)."""
    jx = np.einsum('sixy,i->sxy', f, C[:, 0].astype(np.float64))
    jy = np.einsum('sixy,i->sxy', f, C[:, 1].astype(np.float64))
    return np.stack([jx, jy], axis=1)


def common_velocity(f: np.ndarray, p: Params) -> tuple[np.ndarray, np.ndarray]:
    """u = sum_{s,i} f_i^s c_i / tau_s  /  sum_s rho_s / tau_s  (Eq. 1)."""
    rho = densities(f)
    j = momenta(f)
    taus = (p.tau_A, p.tau_B)
    num_x = j[0, 0] / taus[0] + j[1, 0] / taus[1]
    num_y = j[0, 1] / taus[0] + j[1, 1] / taus[1]
    den = rho[0] / taus[0] + rho[1] / taus[1]
    return num_x / den, num_y / den


def neighbour_sum(field: np.ndarray, ghost: float | None) -> tuple[np.ndarray, np.ndarray]:
    """sum_i w_i field(x + c_i) c_i (both components of the vector), with x periodic
    and `ghost` as the value on the virtual wall rows y = -1 and y = ny (None: the
    wall rows' own values, mirrored across the walls)."""
    ny, nx = field.shape
    padded = np.empty((ny + 2, nx), dtype=np.float64)
    padded[1:-1] = field
    if ghost is None:
        padded[0], padded[-1] = field[0], field[-1]
    else:
        padded[0], padded[-1] = ghost, ghost
    sx = np.zeros((ny, nx))
    sy = np.zeros((ny, nx))
    for i in range(1, 9):
        cx, cy = int(C[i, 0]), int(C[i, 1])
        shifted = np.roll(padded, -cx, axis=1)[1 + cy:1 + cy + ny]   # value at (x + cx, y + cy)
        sx += W[i] * cx * shifted
        sy += W[i] * cy * shifted
    return sx, sy


def forces(f: np.ndarray, p: Params) -> np.ndarray:
    """F_s = F_s^ff + F_s^fb + F_s^ext, shape (2 components, 2 axes, ny, nx).

    F_s^ff = -G rho_s sum_i w_i rho_s'(x + c_i) c_i  (Eq. "Shan-Chen forcing term", psi = rho,
             no self-interaction; the pseudopotential of a wall node is 0, or with
             wall_mode = 1 that of the fluid node it mirrors)
    F_s^fb = -G_sb rho_s sum_i w_i S(x + c_i) c_i   (fluid-boundary force, S = 1 on wall nodes)
    F_A^ext = -rho_A g e_y, F_B^ext = +rho_B g e_y  (Eq. 3_Fex; gravity_mode = 1 gives both -rho_s g e_y)
    plus rho_s gx e_x (a test-only body force).
    """
    rho = densities(f)
    ny, nx = rho.shape[1:]
    wall_x, wall_y = neighbour_sum(np.zeros((ny, nx)), ghost=1.0)
    gwall = (p.G_wall_A, p.G_wall_B)
    if p.gravity_mode == 0:
        gsign = (-1.0, 1.0)
    else:
        gsign = (-1.0, -1.0)
    F = np.zeros((2, 2, ny, nx))
    for s in range(2):
        other_x, other_y = neighbour_sum(rho[1 - s], ghost=None if p.wall_mode == 1 else 0.0)
        F[s, 0] = -p.G * rho[s] * other_x - gwall[s] * rho[s] * wall_x + rho[s] * p.gx
        F[s, 1] = -p.G * rho[s] * other_y - gwall[s] * rho[s] * wall_y + gsign[s] * rho[s] * p.g
    return F


# --------------------------------------------------------------------------
# collision, streaming, step
# --------------------------------------------------------------------------
def collide(f: np.ndarray, p: Params) -> np.ndarray:
    """Forced BGK relaxation (Eq. "Kinetic equation" right-hand side):
    f* = f - (f - f^eq(rho_s, u + tau_s F_s / rho_s)) / tau_s."""
    rho = densities(f)
    ux, uy = common_velocity(f, p)
    F = forces(f, p)
    out = np.empty_like(f)
    for s, tau in enumerate((p.tau_A, p.tau_B)):
        # where rho_s = 0 the equilibrium is 0 whatever u' is; avoid the 0/0
        ax = np.divide(F[s, 0], rho[s], out=np.zeros_like(rho[s]), where=rho[s] != 0.0)
        ay = np.divide(F[s, 1], rho[s], out=np.zeros_like(rho[s]), where=rho[s] != 0.0)
        upx = ux + tau * ax
        upy = uy + tau * ay
        feq = equilibrium(rho[s], upx, upy)
        out[s] = f[s] - (f[s] - feq) / tau
    return out


def stream(fstar: np.ndarray) -> np.ndarray:
    """Push f*_i(x) to x + c_i (left-hand side of the kinetic equation); x periodic;
    a population leaving through the bottom or top wall returns to its own node in
    the opposite direction (half-way bounce-back)."""
    ny = fstar.shape[2]
    new = np.zeros_like(fstar)
    for i in range(9):
        cx, cy = int(C[i, 0]), int(C[i, 1])
        moved = np.roll(fstar[:, i], cx, axis=2)          # moved[..., x] = f*(x - cx)
        if cy == 0:
            new[:, i] += moved
        elif cy == 1:
            new[:, i, 1:, :] += moved[:, :-1, :]
            new[:, OPP[i], ny - 1, :] += fstar[:, i, ny - 1, :]
        else:  # cy == -1
            new[:, i, :-1, :] += moved[:, 1:, :]
            new[:, OPP[i], 0, :] += fstar[:, i, 0, :]
    return new


def step(f: np.ndarray, p: Params, nsteps: int = 1) -> np.ndarray:
    for _ in range(nsteps):
        f = stream(collide(f, p))
    return f


# --------------------------------------------------------------------------
# diagnostics (Section 3: energies, energy budget, stress split, interface
# length, enstrophy), on the sub-domain without `crop_rows` rows at each wall.
# --------------------------------------------------------------------------
def ddx(a: np.ndarray) -> np.ndarray:
    """Centred difference along the periodic x axis."""
    return 0.5 * (np.roll(a, -1, axis=-1) - np.roll(a, 1, axis=-1))


def ddy(a: np.ndarray) -> np.ndarray:
    """Centred difference along y; NaN on the two wall rows (never used: crop >= 3)."""
    out = np.full_like(a, np.nan)
    out[..., 1:-1, :] = 0.5 * (a[..., 2:, :] - a[..., :-2, :])
    return out


def laplacian(a: np.ndarray) -> np.ndarray:
    """Five-point centred Laplacian; NaN on the wall rows."""
    out = np.full_like(a, np.nan)
    out[1:-1] = (np.roll(a, -1, axis=1) + np.roll(a, 1, axis=1))[1:-1] + a[2:] + a[:-2] - 4.0 * a[1:-1]
    return out


def physical_velocity(f: np.ndarray, p: Params) -> tuple[np.ndarray, np.ndarray]:
    """u = (sum_{s,i} f_i^s c_i + (F_A + F_B) / 2) / rho."""
    rho = densities(f).sum(axis=0)
    j = momenta(f).sum(axis=0)
    F = forces(f, p).sum(axis=0)
    return (j[0] + 0.5 * F[0]) / rho, (j[1] + 0.5 * F[1]) / rho


def bulk_order_parameter(p: Params) -> tuple[float, float]:
    """phi = rho_A - rho_B in the pure top (A) and pure bottom (B) bulk of the initial state."""
    eps = p.minority
    return p.mass_A - eps * p.mass_B, eps * p.mass_A - p.mass_B


def bulk_mass_fraction(p: Params) -> tuple[float, float]:
    """c = rho_A / (rho_A + rho_B) in the pure top (A) and pure bottom (B) bulk of the initial state."""
    eps = p.minority
    return p.mass_A / (p.mass_A + eps * p.mass_B), eps * p.mass_A / (eps * p.mass_A + p.mass_B)


def mixing_width(c_rows: np.ndarray, p: Params) -> float:
    """h = 6 sum_y ct (1 - ct), ct = (cbar - c_bot) / (c_top - c_bot) clamped to [0, 1], cbar the row
    means of the mass fraction c = rho_A / (rho_A + rho_B).  The mass fraction, unlike rho_A - rho_B,
    keeps its bulk values when gravity compresses a tall column."""
    top, bot = bulk_mass_fraction(p)
    c = np.clip((c_rows - bot) / (top - bot), 0.0, 1.0)
    return float(6.0 * np.sum(c * (1.0 - c)))


def cauchy_crofton_counts(phi: np.ndarray, r0: int, r1: int) -> np.ndarray:
    """Sign changes of the indicator (phi > 0) between lattice neighbours along
    0, 90, 45 and 135 degrees, for pairs with both ends in rows [r0, r1); x periodic."""
    b = (phi > 0.0)
    rows = b[r0:r1]
    n0 = np.count_nonzero(rows != np.roll(rows, -1, axis=1))
    lo, hi = b[r0:r1 - 1], b[r0 + 1:r1]
    n90 = np.count_nonzero(lo != hi)
    n45 = np.count_nonzero(lo != np.roll(hi, -1, axis=1))    # (x, y) - (x+1, y+1)
    n135 = np.count_nonzero(lo != np.roll(hi, 1, axis=1))    # (x, y) - (x-1, y+1)
    return np.array([n0, n90, n45, n135], dtype=np.int64)


def cauchy_crofton_length(counts: np.ndarray) -> float:
    """L = (1/2) sum_theta d(theta) N(theta) dtheta with 4 directions (dtheta = pi/4,
    line spacing 1 on the axes and 1/sqrt 2 on the diagonals)."""
    n0, n90, n45, n135 = (float(v) for v in counts)
    return (math.pi / 8.0) * (n0 + n90 + (n45 + n135) / math.sqrt(2.0))


def diagnostics(f: np.ndarray, p: Params) -> dict:
    """All instantaneous diagnostic terms of Section 3 for the state f: the masses
    of the whole grid plus field_diagnostics of the densities and the physical
    velocity."""
    rho_s = densities(f)
    ux, uy = physical_velocity(f, p)
    out = field_diagnostics(rho_s[0], rho_s[1], ux, uy, p)
    out["mass_A"] = float(rho_s[0].sum())
    out["mass_B"] = float(rho_s[1].sum())
    return out


def spurious_coefficient(tau: float) -> float:
    """cs^4 (tau - 1/2)^2, the prefactor of the spurious stress K^(tau) (Section 3, Eq. "Three
    parts of the pressure tensor")."""
    return CS2 * CS2 * (tau - 0.5) ** 2


def stress_tensors(rhoA: np.ndarray, rhoB: np.ndarray, p: Params) -> dict:
    """The three parts of the pressure tensor of Section 3 (Eq. "Three parts of the pressure
    tensor") on the grid, derivatives by centred differences (NaN on the wall rows):
      p_b  = cs^2 rho + G cs^2 (rho^2 - phi^2) / 4                       (bulk pressure)
      P^K  = [-k phi lap phi - k/2 |grad phi|^2] I + k grad phi (x) grad phi, k = cs^4 G / 4
      K^tau = cs^4 (tau - 1/2)^2 rho_A rho_B / rho  v (x) v,  v = grad rho_A / rho_A - grad rho_B / rho_B
    K^tau is evaluated as (rho_B grad rho_A - rho_A grad rho_B) (x) (...) / (rho_A rho_B rho) with
    rho_A rho_B clamped at 1e-12; tau is the mean of the two relaxation times."""
    rho = rhoA + rhoB
    phi = rhoA - rhoB
    tau = 0.5 * (p.tau_A + p.tau_B)
    kappa = CS2 * CS2 * p.G / 4.0
    pb = CS2 * rho + p.G * CS2 / 4.0 * (rho * rho - phi * phi)
    phx, phy = ddx(phi), ddy(phi)
    iso = -kappa * phi * laplacian(phi) - 0.5 * kappa * (phx * phx + phy * phy)
    prod = np.maximum(rhoA * rhoB, 1e-12)
    vx = rhoB * ddx(rhoA) - rhoA * ddx(rhoB)
    vy = rhoB * ddy(rhoA) - rhoA * ddy(rhoB)
    coef = spurious_coefficient(tau) / (prod * rho)
    return dict(pb=pb,
                PKxx=iso + kappa * phx * phx, PKxy=kappa * phx * phy, PKyy=iso + kappa * phy * phy,
                Kxx=coef * vx * vx, Kxy=coef * vx * vy, Kyy=coef * vy * vy)


def field_diagnostics(rhoA: np.ndarray, rhoB: np.ndarray, ux: np.ndarray, uy: np.ndarray, p: Params) -> dict:
    """Diagnostic terms of Section 3 from the density and velocity fields.

    Averages <.> are means over the sub-domain rows [crop, ny - crop) and all x;
    derivatives are centred differences (Section 3).
      E_k = <rho |u|^2 / 2>, E_p = g <y phi>            (Eq. "Kinetic energy balance", first line)
      buoyancy = g <u_y phi>                             (contribution of the buoyancy term)
      flux_pb = <u . grad p_b>, p_b = cs^2 rho + G cs^2 (rho^2 - phi^2) / 4
      flux_K = <u . div P^K>, P^K = [-k phi lap phi - k/2 |grad phi|^2] I + k grad phi (x) grad phi, k = cs^4 G / 4
      flux_tau = <u . div K^tau>, K^tau = cs^4 rho_A rho_B / rho (tau-1/2)^2 v (x) v, v = grad rho_A / rho_A - grad rho_B / rho_B
      viscous = <u . div(eta grad u + eta grad u^T)>, eta = rho_bar cs^2 (tau - 1/2)
      enstrophy = 1/2 sum omega^2, omega = d_x u_y - d_y u_x  (Section 3, "Viscous dissipation and enstrophy")
      h: mixing-layer width (6 sum c(1-c)) of the normalised row means of the mass fraction
         c = rho_A / (rho_A + rho_B); L_int: Cauchy-Crofton length of {phi = 0}.
    """
    rho = rhoA + rhoB
    phi = rhoA - rhoB
    ny, nx = rho.shape
    r0, r1 = p.crop_rows, ny - p.crop_rows
    R = slice(r0, r1)

    def mean(a):
        return float(np.mean(a[R]))

    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    tau = 0.5 * (p.tau_A + p.tau_B)

    T = stress_tensors(rhoA, rhoB, p)
    pb = T["pb"]
    flux_pb = mean(ux * ddx(pb) + uy * ddy(pb))
    flux_K = mean(ux * (ddx(T["PKxx"]) + ddy(T["PKxy"])) + uy * (ddx(T["PKxy"]) + ddy(T["PKyy"])))
    flux_tau = mean(ux * (ddx(T["Kxx"]) + ddy(T["Kxy"])) + uy * (ddx(T["Kxy"]) + ddy(T["Kyy"])))

    # viscous term
    rho_bar = mean(rho)
    eta = rho_bar * CS2 * (tau - 0.5)
    dxux, dyux, dxuy, dyuy = ddx(ux), ddy(ux), ddx(uy), ddy(uy)
    Sxx, Sxy, Syy = 2.0 * dxux, dxuy + dyux, 2.0 * dyuy
    viscous = eta * mean(ux * (ddx(Sxx) + ddy(Sxy)) + uy * (ddx(Sxy) + ddy(Syy)))
    omega = dxuy - dyux
    enstrophy = float(0.5 * np.sum(omega[R] ** 2))

    counts = cauchy_crofton_counts(phi, r0, r1)
    phi_rows = phi[R].mean(axis=1)
    c = np.divide(rhoA, rho, out=np.zeros_like(rho), where=rho > 0.0)
    c_rows = c[R].mean(axis=1)
    return dict(
        E_k=mean(0.5 * rho * (ux * ux + uy * uy)),
        E_p=p.g * mean(y * phi),
        buoyancy=p.g * mean(uy * phi),
        flux_pb=flux_pb, flux_K=flux_K, flux_tau=flux_tau,
        viscous=viscous, enstrophy=enstrophy, rho_bar=rho_bar, eta=eta,
        h=mixing_width(c_rows, p), L_int=cauchy_crofton_length(counts),
        cc=counts, phi_rows=phi_rows, c_rows=c_rows,
    )


def fields(f: np.ndarray, p: Params) -> dict:
    """rho_A, rho_B and the physical velocity on the whole grid."""
    rho_s = densities(f)
    ux, uy = physical_velocity(f, p)
    return dict(rhoA=rho_s[0], rhoB=rho_s[1], ux=ux, uy=uy)
