"""Pins of the closure-correction oracle (CPU): what the definition of the
re-equilibration fixes independently of how the oracle writes it (the moments of
the corrected state, conservation, the limiter, where the interface weight is
zero), plus planted mistakes that one of the pins must catch."""
import numpy as np
import pytest

from oracle import closure_oracle as K
from oracle import lbm_oracle as O

NX, NY = 16, 12
P = O.Params(nx=NX, ny=NY, G=0.0, g=0.0)


def equilibrium_state(seed, rhoA=None, rhoB=None):
    """f_s = f^eq(rho_s, u) with one velocity field u shared by both components."""
    rng = np.random.default_rng(seed)
    rA = rng.uniform(0.3, 1.0, (NY, NX)) if rhoA is None else rhoA
    rB = rng.uniform(0.3, 1.0, (NY, NX)) if rhoB is None else rhoB
    ux, uy = rng.uniform(-0.05, 0.05, (2, NY, NX))
    return np.stack([O.equilibrium(rA, ux, uy), O.equilibrium(rB, ux, uy)]), (rA, rB, ux, uy)


def pattern():
    """A field with zero mean on every row (a full period of a sine along x)."""
    return np.broadcast_to(np.sin(2 * np.pi * (np.arange(NX) + 0.5) / NX), (NY, NX)).copy()


def moments(f):
    rho = O.densities(f)
    j = O.momenta(f).sum(axis=0)
    return rho, j


def output(dA=0.0, dB=0.0, dux=0.0, duy=0.0):
    return np.stack([np.broadcast_to(np.asarray(v, dtype=np.float64), (NY, NX)) for v in (dA, dB, dux, duy)])


ONES = np.ones(4)


@pytest.mark.parametrize("mode", [0, 1, 2, 3, 4])
def test_zero_output_leaves_any_state_unchanged(mode):
    rng = np.random.default_rng(3)
    f = rng.uniform(0.01, 0.2, (2, 9, NY, NX))
    assert np.allclose(K.correct(f, output(), ONES, mode, P), f, rtol=0, atol=1e-15)


@pytest.mark.parametrize("mode,a", [(2, 0.0), (3, 0.25)])
def test_order_parameter_modes_move_the_densities_by_half_the_difference(mode, a):
    # equilibrium in, equilibrium out: rho_A + s/2, rho_B - s/2 for a zero-mean
    # difference s = dA - dB; u + a du (mode 2 keeps the velocity, mode 3 moves a
    # quarter of the way)
    f, (rA, rB, ux, uy) = equilibrium_state(1)
    s = 0.01 * pattern()
    du = (0.004, -0.002)
    g = K.correct(f, output(dA=0.7 * s, dB=-0.3 * s, dux=du[0], duy=du[1]), ONES, mode, P)
    rho, j = moments(g)
    assert np.allclose(rho[0], rA + 0.5 * s, atol=1e-14)
    assert np.allclose(rho[1], rB - 0.5 * s, atol=1e-14)
    r = rA + rB
    assert np.allclose(j[0], r * (ux + a * du[0]), atol=1e-14)
    assert np.allclose(j[1], r * (uy + a * du[1]), atol=1e-14)


def test_mode_1_moves_each_density_by_its_output_minus_the_mean():
    f, (rA, rB, ux, uy) = equilibrium_state(2)
    s = 0.01 * pattern()
    g = K.correct(f, output(dA=s + 0.003, dB=-2 * s - 0.001, dux=0.002, duy=0.001), ONES, 1, P)
    rho, j = moments(g)
    assert np.allclose(rho[0], rA + s, atol=1e-14)        # the constant 0.003 is the mean: removed
    assert np.allclose(rho[1], rB - 2 * s, atol=1e-14)
    r = rho.sum(axis=0)
    assert np.allclose(j[0], r * (ux + 0.002), atol=1e-14)
    assert np.allclose(j[1], r * (uy + 0.001), atol=1e-14)


@pytest.mark.parametrize("mode", [1, 2, 3, 4])
def test_corrections_keep_each_components_mass(mode):
    rng = np.random.default_rng(4)
    f = rng.uniform(0.02, 0.2, (2, 9, NY, NX))
    y = rng.normal(0.0, 0.02, (4, NY, NX))
    g = K.correct(f, y, ONES, mode, P)
    m0, m1 = O.densities(f).sum(axis=(1, 2)), O.densities(g).sum(axis=(1, 2))
    assert np.allclose(m1, m0, rtol=1e-13)
    assert not np.allclose(g, f)


def test_interface_weight_confines_mode_4_to_the_interface():
    # rows 0-3: the bottom bulk mass fraction (w = 0); row 6: halfway between the
    # bulk values (w = 1); row 7: a quarter of the way from the bottom (w = 3/4);
    # the rest the top bulk (w = 0).  An output dA = s + k (s zero mean on each row)
    # moves rho_A by w s / 2 on the interface rows: the constant k, which would
    # change the mass, is taken out again where it was put in.
    top, bot = O.bulk_mass_fraction(P)
    c = np.full(NY, top)
    c[:4] = bot
    c[6] = 0.5 * (top + bot)
    c[7] = bot + 0.25 * (top - bot)
    rho = np.full((NY, NX), 0.9)
    rA, rB = rho * c[:, None], rho * (1.0 - c[:, None])
    f, (_, _, ux, uy) = equilibrium_state(5, rA, rB)
    s = 0.02 * pattern()
    g = K.correct(f, output(dA=s + 0.01, dB=0.0), ONES, 4, P)
    r = O.densities(g)
    w = np.zeros(NY)
    w[6], w[7] = 1.0, 0.75
    assert np.allclose(r[0], rA + w[:, None] * s / 2, atol=1e-14)
    assert np.allclose(r[1], rB - w[:, None] * s / 2, atol=1e-14)


def test_limiter_stops_a_density_at_half_its_value():
    # one site asks for a huge transfer from B to A: h stops at rho_B / 2 there; the
    # mean of h (mode 2) is then taken from every site, the site included
    f, (rA, rB, _, _) = equilibrium_state(6)
    dA = np.zeros((NY, NX))
    dA[5, 7] = 1e3
    g = K.correct(f, output(dA=dA), ONES, 2, P)
    r = O.densities(g)
    n = NX * NY
    h = 0.5 * rB[5, 7]
    expect_B = rB + h / n
    expect_B[5, 7] -= h
    assert np.allclose(r[1], expect_B, atol=1e-14)
    assert np.allclose(r[0], rA + rB - expect_B, atol=1e-14)


def test_non_equilibrium_part_is_kept_in_proportion_to_the_density():
    # f = f^eq + k q with q carrying no density and no momentum: the correction is
    # affine in k and leaves the corrected moments alone; the slope is q scaled by
    # the ratio of the corrected to the old density of each component
    f, _ = equilibrium_state(7)
    q = np.zeros_like(f)
    q[:, 0] = -4.0          # rest
    q[:, 1:5] = 1.0         # axis directions
    q *= 1e-3
    y = np.stack([0.02 * pattern(), -0.01 * pattern(), np.full((NY, NX), 0.003), np.zeros((NY, NX))])
    c0, c1, c2 = (K.correct(f + k * q, y, ONES, 4, P) for k in (0.0, 1.0, 2.0))
    assert np.allclose(c2 - c1, c1 - c0, atol=1e-15)
    ratio = O.densities(c0) / O.densities(f)
    assert np.allclose(c1 - c0, ratio[:, None] * q, atol=1e-15)
    for a, b in zip(moments(c1), moments(c0)):
        assert np.allclose(a, b, atol=1e-14)


def test_output_scale_multiplies_the_network_output():
    f, _ = equilibrium_state(8)
    y = np.stack([0.02 * pattern(), -0.01 * pattern(), 0.3 * pattern(), np.full((NY, NX), 0.1)])
    os = np.array([0.5, 2.0, 0.01, 0.02])
    assert np.allclose(K.correct(f, y, os, 3, P), K.correct(f, y * os[:, None, None], ONES, 3, P), atol=1e-15)


def test_network_input_of_a_uniform_state_at_rest():
    # no Shan-Chen, wall or gravity force, a body acceleration gx along x: the
    # physical velocity is gx / 2 (half a step of the force), the densities as given
    p = P.with_(gx=2e-4)
    rA, rB = np.full((NY, NX), 0.8), np.full((NY, NX), 0.3)
    z = np.zeros((NY, NX))
    f = np.stack([O.equilibrium(rA, z, z), O.equilibrium(rB, z, z)])
    x = K.network_input(f, p, mean=(0.5, 0.5, 0.0, 0.0), scale=(0.5, 0.25, 1e-4, 1e-4))
    assert np.allclose(x[0], 0.6, atol=1e-14)
    assert np.allclose(x[1], -0.8, atol=1e-14)
    assert np.allclose(x[2], 1.0, atol=1e-10)
    assert np.allclose(x[3], 0.0, atol=1e-10)


def test_planted_mistakes_are_caught(monkeypatch):
    # each mistake must break one of the pins above
    f, (rA, rB, ux, uy) = equilibrium_state(1)
    s = 0.01 * pattern()

    def order_parameter_pin():
        g = K.correct(f, output(dA=0.7 * s, dB=-0.3 * s, dux=0.004), ONES, 3, P)
        rho, j = moments(g)
        return (np.allclose(rho[0], rA + 0.5 * s, atol=1e-14)
                and np.allclose(j[0], (rA + rB) * (ux + 0.001), atol=1e-14))

    assert order_parameter_pin()
    with monkeypatch.context() as m:
        m.setitem(K.VELOCITY_FRACTION, 3, 1.0)                 # the full velocity correction
        assert not order_parameter_pin()
    with monkeypatch.context() as m:                           # d_B = +d_A
        orig = K.density_corrections
        m.setattr(K, "density_corrections", lambda *a: np.stack([orig(*a)[0]] * 2))
        assert not order_parameter_pin()
    with monkeypatch.context() as m:                           # the weight without the factor 4
        orig_w = K.interface_weight
        m.setattr(K, "interface_weight", lambda rho, p: 0.25 * orig_w(rho, p))
        top, bot = O.bulk_mass_fraction(P)
        c = np.full(NY, top)
        c[6] = 0.5 * (top + bot)
        rA2 = 0.9 * c[:, None] * np.ones((NY, NX))
        rB2 = 0.9 - rA2
        f2, _ = equilibrium_state(5, rA2, rB2)
        r = O.densities(K.correct(f2, output(dA=0.02 * pattern()), ONES, 4, P))
        assert not np.allclose(r[0, 6], rA2[6] + 0.01 * pattern()[6], atol=1e-14)
