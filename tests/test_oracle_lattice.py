"""Pins of the oracle's lattice, generator, equilibrium and streaming against
what the paper and the mathematics fix (no GPU)."""
import itertools
import json
import math
from pathlib import Path

import numpy as np
import pytest

from oracle import lbm_oracle as O

GOLDEN = Path(__file__).resolve().parent / "golden"


def test_velocity_set_is_d2q9():
    # Section 2: (0,0), (+-c,0), (0,+-c), (+-c,+-c) with c = 1
    vecs = {tuple(v) for v in O.C.tolist()}
    assert vecs == {(a, b) for a in (-1, 0, 1) for b in (-1, 0, 1)}
    for i in range(9):
        assert tuple(O.C[O.OPP[i]]) == tuple(-O.C[i])


def test_weights_satisfy_isotropy_conditions():
    # Section 2: sum_i w c^a c^b = cs^2 delta_ab and the fourth-order condition, cs^2 = 1/3
    cs2 = 1.0 / 3.0
    assert math.isclose(O.W.sum(), 1.0, rel_tol=0, abs_tol=1e-15)
    for a, b in itertools.product(range(2), repeat=2):
        lhs = sum(O.W[i] * O.C[i, a] * O.C[i, b] for i in range(9))
        assert math.isclose(lhs, cs2 * (a == b), abs_tol=1e-15)
    for a, b, c, d in itertools.product(range(2), repeat=4):
        lhs = sum(O.W[i] * O.C[i, a] * O.C[i, b] * O.C[i, c] * O.C[i, d] for i in range(9))
        rhs = cs2 * cs2 * ((a == b) * (c == d) + (a == d) * (b == c) + (a == c) * (b == d))
        assert math.isclose(lhs, rhs, abs_tol=1e-15)
    # odd moments vanish
    for a, b, c in itertools.product(range(2), repeat=3):
        assert abs(sum(O.W[i] * O.C[i, a] * O.C[i, b] * O.C[i, c] for i in range(9))) < 1e-15


def test_splitmix64_reference_vectors():
    g = json.loads((GOLDEN / "splitmix64.json").read_text())
    for v in g["vectors"]:
        if "outputs_hex" in v:
            want = [int(h, 16) for h in v["outputs_hex"]]
        else:
            want = [int(d) for d in v["outputs_dec"]]
        assert O.splitmix64_stream(v["seed"], len(want)) == want


def test_equilibrium_moments_closed_form():
    # textbook moments of the second-order equilibrium: rho, rho u, rho (cs^2 I + u u)
    rng = np.random.default_rng(3)
    rho = rng.uniform(0.1, 2.0, 50)
    ux = rng.uniform(-0.1, 0.1, 50)
    uy = rng.uniform(-0.1, 0.1, 50)
    feq = O.equilibrium(rho, ux, uy)
    c = O.C.astype(float)
    assert np.allclose(feq.sum(0), rho, rtol=1e-14)
    assert np.allclose((feq * c[:, 0:1]).sum(0), rho * ux, atol=1e-15)
    assert np.allclose((feq * c[:, 1:2]).sum(0), rho * uy, atol=1e-15)
    pxx = (feq * (c[:, 0:1] ** 2)).sum(0)
    pxy = (feq * (c[:, 0:1] * c[:, 1:2])).sum(0)
    assert np.allclose(pxx, rho / 3 + rho * ux * ux, rtol=1e-13)
    assert np.allclose(pxy, rho * ux * uy, atol=1e-15)


def test_streaming_moves_each_population_along_its_velocity():
    nx, ny = 7, 9
    for i in range(9):
        for (x, y) in [(3, 4), (0, 0), (6, ny - 1), (2, 0), (5, ny - 1)]:
            f = np.zeros((2, 9, ny, nx))
            f[1, i, y, x] = 1.0
            g = O.stream(f)
            assert g.sum() == 1.0
            (s, j, yy, xx), = np.argwhere(g == 1.0)
            ty = y + O.C[i, 1]
            if 0 <= ty < ny:
                assert (s, j, yy, xx) == (1, i, ty, (x + O.C[i, 0]) % nx)
            else:  # half-way bounce-back: back at its own node, opposite direction
                assert (s, j, yy, xx) == (1, O.OPP[i], y, x)


def test_interface_height_amplitude_and_mean_level():
    p = O.Params(nx=128, ny=256, seed=5, amp=2.0)
    y0 = O.interface_height(p)
    assert math.isclose(np.max(np.abs(y0 - 128.0)), 2.0, rel_tol=1e-12)
    # a sum of full-period sines has zero mean over the period
    assert abs(np.mean(y0) - 128.0) < 1e-12


def test_initial_state_is_at_rest_with_the_bulk_densities():
    p = O.Params(nx=32, ny=64, seed=2, minority=0.08, mass_A=1.0, mass_B=0.9)
    f = O.initial_populations(p)
    r = O.densities(f)
    j = O.momenta(f)
    assert np.abs(j).max() < 1e-16
    # far from the interface the bulks hold the stated majority / minority densities
    assert math.isclose(r[0, -1].mean(), 1.0, rel_tol=1e-6)
    assert math.isclose(r[1, -1].mean(), 0.08 * 0.9, rel_tol=1e-4)
    assert math.isclose(r[1, 0].mean(), 0.9, rel_tol=1e-6)
    assert math.isclose(r[0, 0].mean(), 0.08, rel_tol=1e-4)


@pytest.mark.parametrize("tau", [0.7, 1.0, 1.6])
def test_collision_keeps_each_component_mass_and_adds_the_force_impulse(tau):
    # BGK with the shifted-velocity equilibrium keeps rho_s and gives the total
    # momentum change sum_s F_s per step (the forcing acts as an impulse F dt)
    rng = np.random.default_rng(11)
    # unequal relaxation times: the 1/tau_s weighting of the common velocity (Eq. 1)
    # is what makes the total momentum change equal to the total force
    p = O.Params(nx=16, ny=12, tau_A=tau, tau_B=tau + 0.35, G=1.1, g=3e-4, gx=2e-4)
    f = rng.uniform(0.02, 0.2, (2, 9, p.ny, p.nx))
    fs = O.collide(f, p)
    assert np.allclose(O.densities(fs), O.densities(f), rtol=1e-14)
    dj = (O.momenta(fs) - O.momenta(f)).sum(axis=0)
    F = O.forces(f, p).sum(axis=0)
    assert np.allclose(dj, F, atol=1e-15)
