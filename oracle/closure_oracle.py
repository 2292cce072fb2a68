"""FP64 CPU oracle of one correction of the learned closure: the network input
taken from the coarse run's populations, and the re-equilibration that applies the
network's output to them.

TEST INFRASTRUCTURE ONLY (tests, smoke and the CPU legs of bench.py).  The learned
closure is an extension built on the solver; the paper has no such step.  This
module follows the definition that include/lbm.h gives for lbm_closure_advance,
written from that definition in plain numpy (float64), whole-array operations in
the order the definition states, and shares no code with the CUDA library.  The
lattice, the forces and the equilibrium come from ``lbm_oracle`` (Section 2); the
network itself from ``cnn_oracle``.

State convention as in ``lbm_oracle``: f has shape (2, 9, ny, nx) and holds the
post-streaming populations.  The network output y has shape (4, ny, nx) in
normalised units: channel 0, 1 the density corrections of A and B, channel 2, 3
the velocity correction; y * out_scale is the correction in lattice units.

Pins: tests/test_oracle_closure.py (the identity for a zero output, exact density
and momentum moments of the corrected state, mass conservation, bulk sites left
alone by the interface weight, the limiter, planted mistakes).
"""
from __future__ import annotations

import numpy as np

from oracle import lbm_oracle as O

# velocity fraction of each mode: 1 the full correction, 2 none, 3 and 4 a quarter
VELOCITY_FRACTION = {1: 1.0, 2: 0.0, 3: 0.25, 4: 0.25}


def network_input(f: np.ndarray, p: O.Params, mean, scale) -> np.ndarray:
    """x[c] = (v_c - mean[c]) / scale[c] for v = (rho_A, rho_B, u_x, u_y), u the
    physical velocity (sum_{s,i} f c_i + F / 2) / rho."""
    rho = O.densities(f)
    ux, uy = O.physical_velocity(f, p)
    v = np.stack([rho[0], rho[1], ux, uy])
    return (v - np.asarray(mean, dtype=np.float64)[:, None, None]) / np.asarray(scale, dtype=np.float64)[:, None, None]


def interface_weight(rho: np.ndarray, p: O.Params) -> np.ndarray:
    """w = 4 c (1 - c), c the mass fraction rho_A / (rho_A + rho_B) normalised by its
    two bulk values and clamped to [0, 1]: 0 in either bulk, 1 where c is halfway."""
    top, bot = O.bulk_mass_fraction(p)
    c = np.clip((rho[0] / (rho[0] + rho[1]) - bot) / (top - bot), 0.0, 1.0)
    return 4.0 * c * (1.0 - c)


def density_corrections(rho: np.ndarray, dy: np.ndarray, mode: int, p: O.Params) -> np.ndarray:
    """The corrections d_s of rho_s (shape (2, ny, nx)) from the network's density
    outputs dy = (dA, dB) in lattice units.

    mode 1: d_s = max(dy_s, -rho_s / 2) minus its grid mean.
    modes 2, 3: h = (dA - dB) / 2 limited to [-rho_A / 2, rho_B / 2]; d_A = h - mean(h),
      d_B = -d_A.
    mode 4: h = w (dA - dB) / 2 limited the same way, w the interface weight;
      d_A = h - w sum(h) / sum(w), d_B = -d_A (the offset that restores the masses is
      itself weighted, so the bulk is not moved)."""
    if mode == 1:
        d = np.maximum(dy, -0.5 * rho)
        return d - d.mean(axis=(1, 2), keepdims=True)
    w = interface_weight(rho, p) if mode == 4 else np.ones_like(rho[0])
    h = np.clip(0.5 * w * (dy[0] - dy[1]), -0.5 * rho[0], 0.5 * rho[1])
    if mode == 4:
        sw = w.sum()
        dA = h - w * (h.sum() / sw if sw > 0 else 0.0)
    else:
        dA = h - h.mean()
    return np.stack([dA, -dA])


def correct(f: np.ndarray, y: np.ndarray, out_scale, mode: int, p: O.Params) -> np.ndarray:
    """The corrected populations: with rho_s = sum_i f_i^s, u_b = sum_{s,i} f c_i / rho
    (rho = rho_A + rho_B), rho'_s = max(rho_s + d_s, 0) (d from density_corrections)
    and u' = u_b + a du (a from VELOCITY_FRACTION, du = y[2:4] * out_scale[2:4]),
        f_i^s <- f_i^eq(rho'_s, u') + (rho'_s / rho_s) (f_i^s - f_i^eq(rho_s, u_b)).
    Mode 0 returns f unchanged."""
    if mode == 0:
        return f.copy()
    os = np.asarray(out_scale, dtype=np.float64)
    yp = np.asarray(y, dtype=np.float64) * os[:, None, None]
    rho = O.densities(f)
    j = O.momenta(f).sum(axis=0)
    rt = rho.sum(axis=0)
    ux, uy = j[0] / rt, j[1] / rt
    a = VELOCITY_FRACTION[mode]
    vx, vy = ux + a * yp[2], uy + a * yp[3]
    d = density_corrections(rho, yp[:2], mode, p)
    out = np.empty_like(f)
    for s in range(2):
        r1 = np.maximum(rho[s] + d[s], 0.0)
        out[s] = O.equilibrium(r1, vx, vy) + (r1 / rho[s]) * (f[s] - O.equilibrium(rho[s], ux, uy))
    return out
