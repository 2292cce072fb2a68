"""Pins of the oracle's wall treatment of the Shan-Chen pseudopotential (Section 2,
the fluid-boundary force and the solid indicator S): the default reading puts no
fluid beyond the walls (psi = 0 on the virtual rows y = -1 and y = ny); wall_mode 1
mirrors the wall rows' pseudopotential across the walls.  No GPU."""
import numpy as np
import pytest

from oracle import lbm_oracle as O


def state_from_densities(rhoA, rhoB):
    z = np.zeros_like(rhoA)
    return np.stack([O.equilibrium(rhoA, z, z), O.equilibrium(rhoB, z, z)])


@pytest.mark.parametrize("G", [0.1381, 1.4])
def test_a_uniform_fluid_is_at_rest_between_mirror_walls(G):
    # with the pseudopotential mirrored, every site of a uniform fluid sees the same
    # neighbours on both sides: no force, and the rest state is a fixed point of the
    # step (streaming plus bounce-back keep a uniform equilibrium)
    ny, nx = 16, 8
    f = state_from_densities(np.full((ny, nx), 0.9), np.full((ny, nx), 0.15))
    mirror = O.step(f, O.Params(nx=nx, ny=ny, G=G, g=0.0, n_modes=0, wall_mode=1), 50)
    assert np.max(np.abs(mirror - f)) < 1e-15
    # with psi = 0 beyond the walls the same fluid forms a layer at each wall
    empty = O.step(f, O.Params(nx=nx, ny=ny, G=G, g=0.0, n_modes=0, wall_mode=0), 50)
    assert np.max(np.abs(empty - f)) > 1e-4


def test_mirror_wall_forces_are_those_of_the_reflected_domain():
    # the mirror reading means that the virtual row beyond each wall is the reflection
    # of the wall row: the forces on the fluid rows equal those of a stack of copies of
    # the domain reflected about y = -1/2 and y = ny - 1/2, evaluated away from the
    # stack's own walls by the psi = 0 reading
    rng = np.random.default_rng(4)
    ny, nx = 12, 10
    rhoA = rng.uniform(0.1, 1.0, (ny, nx))
    rhoB = rng.uniform(0.1, 1.0, (ny, nx))
    p = O.Params(nx=nx, ny=ny, G=1.3, G_wall_A=0.0, G_wall_B=0.0, g=2e-4, n_modes=0, wall_mode=1)
    got = O.forces(state_from_densities(rhoA, rhoB), p)
    stack = lambda a: np.concatenate([a[::-1], a, a[::-1]])      # rows -ny .. 2 ny - 1
    big = O.forces(state_from_densities(stack(rhoA), stack(rhoB)), p.with_(ny=3 * ny, wall_mode=0))
    assert np.array_equal(got, big[:, :, ny:2 * ny])


def _vertical_interfaces(wall_mode, steps):
    nx, ny = 64, 32
    p = O.Params(nx=nx, ny=ny, G=1.4, g=0.0, n_modes=0, mass_A=1.0, mass_B=1.0, wall_mode=wall_mode, crop_rows=3)
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    H = 0.5 * (1 + np.tanh((x - nx / 4) / 1.5)) - 0.5 * (1 + np.tanh((x - 3 * nx / 4) / 1.5))
    eps = 0.07
    f = O.step(state_from_densities(eps + (1 - eps) * H, eps + (1 - eps) * (1 - H)), p, steps)
    r = O.densities(f)
    ux, uy = O.physical_velocity(f, p)
    return r[0] - r[1], np.hypot(ux, uy)


def _crossing(phi_row):
    i = int(np.where((phi_row[:-1] < 0) & (phi_row[1:] >= 0))[0][0])
    return i + phi_row[i] / (phi_row[i] - phi_row[i + 1])


def test_interfaces_meet_mirror_walls_at_right_angles():
    # two vertical interfaces between equal-mass fluids touching both walls: with the
    # mirror the walls are neutral (contact angle 90 degrees, G_sb = 0) and the
    # interfaces stay straight and at rest up to the wall rows; with psi = 0 beyond
    # the walls the wall layers drive a circulation along them
    phi, speed = _vertical_interfaces(1, 3000)
    ny = phi.shape[0]
    for row in (0, ny - 1):
        assert abs(_crossing(phi[row]) - _crossing(phi[ny // 2])) < 1e-6
    assert speed.max() < 1e-6
    _, speed0 = _vertical_interfaces(0, 3000)
    assert speed0.max() > 1e-4
