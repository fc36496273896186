"""Pins of the FP64 oracle against facts fixed independently of it.

Each test checks the oracle against something other than its own formulas:
the velocity table and weights as printed in the paper (Eq. 4 and the text
after Eq. 5, transcribed in tests/golden/d3q19_eq4.txt), the lattice
isotropy identities, exact conservation laws, library shifts (numpy.roll),
closed-form flows (shear-wave decay, force-driven Poiseuille flow between
halfway walls) and mirror symmetry of the cavity.
"""

import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1309_1983_gb300 import workloads as W


def _golden_eq4(golden_dir):
    rows = {}
    with open(os.path.join(golden_dir, "d3q19_eq4.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            rows[key] = vals
    e = np.array([[int(v) for v in rows[k]] for k in ("ex", "ey", "ez")]).T
    w = np.array([float(Fraction(v)) for v in rows["w"]])
    cs2 = float(Fraction(rows["cs2"][0]))
    return e, w, cs2


@pytest.fixture(scope="module")
def eq4(golden_dir):
    return _golden_eq4(golden_dir)


# --------------------------------------------------------------- constants

def test_velocity_set_is_eq4(eq4):
    e, _, _ = eq4
    assert e.shape == (19, 3)
    np.testing.assert_array_equal(O.velocity_set(), e)


def test_weights_are_the_printed_ones(eq4):
    _, w, _ = eq4
    np.testing.assert_allclose(O.weights(), w, rtol=0, atol=1e-17)


def test_lattice_isotropy(eq4):
    """Sum w = 1, odd moments vanish, sum w e_a e_b = c_s^2 delta,
    sum w e_a e_b e_c e_d = c_s^4 (dd + dd + dd): the conditions under which
    the expansion in Sec. 3 recovers Navier-Stokes."""
    e = O.velocity_set().astype(float)
    w = O.weights()
    _, _, cs2 = eq4
    d = np.eye(3)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(np.einsum("i,ia->a", w, e), 0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, e, e), cs2 * d, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic->abc", w, e, e, e), 0, atol=1e-16)
    four = cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                       + np.einsum("ad,bc->abcd", d, d))
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e), four, atol=1e-16)


def test_opposites():
    e = O.velocity_set()
    opp = O.opposites()
    for i in range(19):
        np.testing.assert_array_equal(e[opp[i]], -e[i])
    assert opp[0] == 0


# --------------------------------------------------------------- equilibrium / collision

def _moments_np(f, e):
    rho = f.sum(axis=0)
    m = np.einsum("ia,i...->a...", e.astype(float), f)
    return rho, m


def test_equilibrium_moments(eq4):
    """Eq. 5 reproduces rho, rho u and the Maxwellian second moment
    rho (u u + c_s^2 I) exactly (Eqs. 6-7)."""
    e, _, cs2 = eq4
    L = O.Lattice(4, 3, 2, 0.7)
    rho = 1.0 + W.noise(L.shape, 11, 0.05)
    u = W.noise((3,) + L.shape, 12, 0.08)
    f = O.init_equilibrium(L, rho, u)
    r, m = _moments_np(f, e)
    np.testing.assert_allclose(r, rho, rtol=1e-14)
    np.testing.assert_allclose(m, rho * u, atol=1e-15)
    P = np.einsum("ia,ib,i...->ab...", e.astype(float), e.astype(float), f)
    Pex = rho * (np.einsum("a...,b...->ab...", u, u) + cs2 * np.eye(3)[:, :, None, None, None])
    np.testing.assert_allclose(P, Pex, atol=1e-15)


def _random_nonequilibrium(L, seed):
    rho = 1.0 + W.noise(L.shape, seed, 0.05)
    u = W.noise((3,) + L.shape, seed + 1, 0.05)
    f = O.init_equilibrium(L, rho, u)
    return f * (1.0 + W.noise(f.shape, seed + 2, 0.2))


def test_collision_conserves_mass_and_momentum(eq4):
    e, _, _ = eq4
    L = O.Lattice(5, 4, 3, 0.63)
    g = _random_nonequilibrium(L, 100)
    fs = O.collide(L, g)
    r0, m0 = _moments_np(g, e)
    r1, m1 = _moments_np(fs, e)
    np.testing.assert_allclose(r1, r0, rtol=1e-13)
    np.testing.assert_allclose(m1, m0, rtol=0, atol=1e-13)


def test_collision_with_force_adds_force_to_momentum(eq4):
    """Guo forcing: the collision adds exactly F to the momentum and nothing
    to the mass."""
    e, _, _ = eq4
    L = O.Lattice(5, 4, 3, 0.9)
    g = _random_nonequilibrium(L, 200)
    F = W.noise((3,) + L.shape, 203, 1e-3)
    fs = O.collide(L, g, F)
    r0, m0 = _moments_np(g, e)
    r1, m1 = _moments_np(fs, e)
    np.testing.assert_allclose(r1, r0, rtol=1e-13)
    np.testing.assert_allclose(m1, m0 + F, rtol=0, atol=1e-13)


def test_equilibrium_is_fixed_point():
    L = O.Lattice(3, 4, 5, 0.57)
    rho = 1.0 + W.noise(L.shape, 7, 0.05)
    u = W.noise((3,) + L.shape, 8, 0.08)
    f = O.init_equilibrium(L, rho, u)
    np.testing.assert_allclose(O.collide(L, f), f, rtol=0, atol=1e-15)


@pytest.mark.parametrize("tau", [0.51, 0.8, 1.0, 1.7])
def test_bgk_relaxes_nonequilibrium_by_one_over_tau(eq4, tau):
    """Eq. 3 with F = 0: f* - f^eq = (1 - 1/tau)(g - f^eq), f^eq taken at the
    moments of g (rebuilt here from the golden table and Eq. 5 via the
    oracle's initialiser)."""
    e, _, _ = eq4
    L = O.Lattice(4, 2, 3, tau)
    g = _random_nonequilibrium(L, 300)
    r, m = _moments_np(g, e)
    feq = O.init_equilibrium(L, r, m / r)
    fs = O.collide(L, g)
    np.testing.assert_allclose(fs - feq, (1.0 - 1.0 / tau) * (g - feq), rtol=0, atol=1e-15)


# --------------------------------------------------------------- streaming / boundaries

def test_periodic_streaming_is_a_roll(eq4):
    """Pull streaming on a periodic lattice: g_i = f_i shifted by e_i,
    compared with numpy.roll (non-cubic box so that axis mix-ups show)."""
    e, _, _ = eq4
    L = O.Lattice(5, 4, 3, 0.7)
    f = W.noise((19,) + L.shape, 1, 1.0)
    g = O.stream(L, f)
    for i in range(19):
        ex, ey, ez = e[i]
        exp = np.roll(f[i], shift=(ez, ey, ex), axis=(0, 1, 2))
        np.testing.assert_array_equal(g[i], exp)


def test_single_population_moves_by_e(eq4):
    e, _, _ = eq4
    L = O.Lattice(6, 5, 4, 0.7)
    for i in range(19):
        f = np.zeros((19,) + L.shape)
        f[i, 2, 2, 3] = 1.0
        g = O.stream(L, f)
        assert g.sum() == 1.0
        ex, ey, ez = e[i]
        assert g[i, 2 + ez, 2 + ey, 3 + ex] == 1.0


def test_bounce_back_single_cell_box():
    """A one-cell box walled on all axes returns every population as its
    opposite (halfway bounce-back)."""
    L = O.Lattice(1, 1, 1, 0.7, walls=(True, True, True))
    f = W.noise((19, 1, 1, 1), 5, 1.0)
    g = O.stream(L, f)
    opp = O.opposites()
    for i in range(1, 19):
        assert g[i, 0, 0, 0] == f[opp[i], 0, 0, 0]
    assert g[0, 0, 0, 0] == f[0, 0, 0, 0]


@pytest.mark.parametrize("walls", [(True, True, True), (False, True, False), (True, False, True)])
def test_stationary_walls_make_streaming_a_permutation(walls):
    """With stationary walls every value is moved, never created or lost:
    the stream pass is a permutation of the values, each value staying in its
    direction or moving to the opposite one."""
    L = O.Lattice(4, 5, 3, 0.7, walls=walls)
    f = W.noise((19,) + L.shape, 9, 1.0)
    g = O.stream(L, f)
    np.testing.assert_array_equal(np.sort(g.ravel()), np.sort(f.ravel()))
    opp = O.opposites()
    for i in range(19):
        allowed = set(f[i].ravel()) | set(f[opp[i]].ravel())
        assert set(g[i].ravel()) <= allowed


def test_lid_injects_momentum_not_mass(eq4):
    """At rest (f = w_i) the moving plane z = nz adds, per top cell, zero mass
    and momentum 2 rho_w sum_{i in} w_i (e_i . u_w) e_i / c_s^2 = U/3 along x
    for u_w = (U, 0, 0) (the two incoming diagonals i with e_x = +-1)."""
    e, w, cs2 = eq4
    U = 0.05
    L = O.Lattice(4, 3, 5, 0.7, walls=(True, True, True), lid=True, lid_u=(U, 0, 0))
    f = O.init_equilibrium(L)
    g = O.stream(L, f)
    r, m = _moments_np(g, e)
    np.testing.assert_allclose(r, 1.0, rtol=1e-15)
    np.testing.assert_allclose(m[0, -1], U / 3.0, rtol=1e-13)
    np.testing.assert_allclose(m[0, :-1], 0.0, atol=1e-16)
    np.testing.assert_allclose(m[1:], 0.0, atol=1e-16)
    # the same figure from the weights and velocities printed in the paper
    inc = [i for i in range(19) if e[i, 2] == -1]
    exp = sum(2.0 * w[i] * (e[i, 0] * U) * e[i, 0] / cs2 for i in inc)
    assert abs(exp - U / 3.0) < 1e-16


# --------------------------------------------------------------- closed-form flows

def _shear_decay_rate(N, tau, steps=2000, every=100):
    L = O.Lattice(1, 1, N, tau)
    f = O.init_equilibrium(L, None, W.shear_wave(1, 1, N, 0.01))
    s = np.sin(2 * np.pi * np.arange(N) / N)
    t, A = [], []
    for k in range(steps // every + 1):
        _, u = O.moments(L, f)
        t.append(k * every)
        A.append(2.0 / N * (u[0, :, 0, 0] * s).sum())
        if k < steps // every:
            f = O.run(L, f, every)
    rate = -np.polyfit(np.array(t), np.log(np.array(A)), 1)[0]
    nu = (tau - 0.5) / 3.0
    k = 2 * np.pi / N
    return rate / (nu * k * k) - 1.0


@pytest.mark.parametrize("tau", [0.6, 0.8])
def test_shear_wave_decays_at_nu_k2(tau):
    """A periodic shear wave u_x = 0.01 sin(2 pi z/N) decays as
    exp(-nu k^2 t), nu = (tau - 1/2)/3, within 1% over 2000 steps; the
    deviation shrinks as k^2 (second-order lattice)."""
    e32 = _shear_decay_rate(32, tau)
    e64 = _shear_decay_rate(64, tau)
    assert abs(e32) < 1e-2 and abs(e64) < 1e-2
    assert 3.0 < e32 / e64 < 5.0


def _poiseuille(n, tau, F, nsteps):
    L = O.Lattice(1, n, 1, tau, walls=(False, True, False))
    force = W.uniform_force(1, n, 1, (F, 0.0, 0.0))
    f = O.run(L, O.init_equilibrium(L), nsteps, force)
    _, u = O.moments(L, f, force)
    nu = (tau - 0.5) / 3.0
    y = np.arange(n)
    exact = F / (2.0 * nu) * (y + 0.5) * (n - 0.5 - y)
    return u[0, 0, :, 0], exact


def test_poiseuille_exact_at_magic_tau():
    """Force-driven Poiseuille flow between halfway walls at y = -1/2 and
    n - 1/2: for BGK with (tau - 1/2)^2 = 3/16 the lattice solution is the
    parabola u = F/(2 rho nu) (y + 1/2)(n - 1/2 - y) to round-off."""
    tau = 0.5 + np.sqrt(3.0 / 16.0)
    for n in (8, 12):
        nu = (tau - 0.5) / 3.0
        u, exact = _poiseuille(n, tau, 1e-5 * (8.0 / n) ** 2, int(20 * n * n / nu))
        assert np.abs(u - exact).max() / exact.max() < 1e-10


def test_poiseuille_second_order():
    tau = 0.8
    errs = []
    for n in (8, 16, 32):
        nu = (tau - 0.5) / 3.0
        u, exact = _poiseuille(n, tau, 1e-5 * (8.0 / n) ** 2, int(20 * n * n / nu))
        errs.append(np.abs(u - exact).max() / exact.max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (orders >= 1.9).all(), (errs, orders)


def test_cavity_conserves_mass_and_is_mirror_symmetric():
    """Lid-driven cavity (lid along +x): total mass constant to round-off
    (the lid's two incoming diagonals cancel), and the flow is symmetric
    under y -> ny-1-y (u_y odd, rho, u_x, u_z even)."""
    L = O.Lattice(8, 8, 8, 0.6, walls=(True, True, True), lid=True, lid_u=(0.05, 0, 0))
    f = O.run(L, O.init_equilibrium(L), 200)
    rho, u = O.moments(L, f)
    assert abs(rho.sum() / L.ncells - 1.0) < 1e-13
    flip = lambda a: a[:, ::-1, :]
    np.testing.assert_allclose(rho, flip(rho), rtol=0, atol=1e-14)
    np.testing.assert_allclose(u[0], flip(u[0]), rtol=0, atol=1e-14)
    np.testing.assert_allclose(u[1], -flip(u[1]), rtol=0, atol=1e-14)
    np.testing.assert_allclose(u[2], flip(u[2]), rtol=0, atol=1e-14)
    assert np.abs(u).max() > 1e-3  # the lid actually drives a flow


def test_moments_of_stored_state_equal_collision_moments(eq4):
    """rho and u reported from a post-collision state (velocity with -F/2)
    equal those the collision used (velocity with +F/2)."""
    e, _, _ = eq4
    L = O.Lattice(3, 4, 5, 0.75)
    g = _random_nonequilibrium(L, 400)
    F = W.noise((3,) + L.shape, 404, 1e-3)
    r_g, m_g = _moments_np(g, e)
    fs = O.collide(L, g, F)
    r, u = O.moments(L, fs, F)
    np.testing.assert_allclose(r, r_g, rtol=1e-14)
    np.testing.assert_allclose(u, (m_g + 0.5 * F) / r_g, rtol=0, atol=1e-15)
