"""Pins of the oracle's on-site velocity walls (Hecht & Harting's D3Q19
on-site conditions, the boundary scheme the paper's cavity used, Sec. 5).

The oracle states the rule as constraints and solves them generically (a
3x3 system per boundary node). These tests check it against things fixed
independently of that solve:
* the closed-form face formulas of the scheme (non-equilibrium bounce-back
  along the normal, transverse momentum correction N_t = 1/2 sum_{e.n=0}
  e_t g - j_t/3), restated here from the velocity table of Eq. 4;
* the prescribed velocity reproduced exactly on faces, edges and corners,
  the known populations left as plain pulls, and the edge/corner density
  taken from the inner diagonal neighbour (the reading this library uses);
* exact closed-form flows: plane Couette flow and force-driven Poiseuille
  flow between on-site walls are reproduced to round-off at any tau;
* the rest state is a fixed point; the cavity is mirror symmetric.
"""

import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1309_1983_gb300 import workloads as W


@pytest.fixture(scope="module")
def table(golden_dir):
    rows = {}
    with open(os.path.join(golden_dir, "d3q19_eq4.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                key, *vals = line.split()
                rows[key] = vals
    e = np.array([[int(v) for v in rows[k]] for k in ("ex", "ey", "ez")]).T
    w = np.array([float(Fraction(v)) for v in rows["w"]])
    return e, w


def _index(e, v):
    return int(np.flatnonzero((e == np.asarray(v)).all(axis=1))[0])


def _random_state(L, seed, amp=0.1):
    rho = 1.0 + W.noise(L.shape, seed, 0.02)
    u = W.noise((3,) + L.shape, seed + 1, 0.05)
    f = O.init_equilibrium(L, rho, u)
    return f * (1.0 + W.noise(f.shape, seed + 2, amp))


def _pull(f, e, x, y, z):
    """Plain periodic pulls g_i = f_i(x - e_i) at one node."""
    nz, ny, nx = f.shape[1:]
    return np.array([f[i, (z - e[i, 2]) % nz, (y - e[i, 1]) % ny, (x - e[i, 0]) % nx]
                     for i in range(19)])


def _velocity(g, e, F):
    rho = g.sum()
    return rho, (e.T @ g + 0.5 * F) / rho


def test_face_nodes_follow_the_closed_form_rule(table):
    """A channel walled (on-site) in z with a lid on z = nz-1 whose
    velocity has a normal component too; random state and body force. On
    every node of both walls the rebuilt populations equal the closed-form
    rule written out here per face."""
    e, w = table
    lid = (0.03, -0.02, 0.01)
    L = O.Lattice(5, 4, 6, 0.8, walls=(False, False, True), lid=True, lid_u=lid, onsite=True)
    f = _random_state(L, 7)
    F = W.noise((3,) + L.shape, 9, 1e-3)
    g = O.stream(L, f, F)
    for z, nvec, uw in ((0, (0, 0, 1), (0.0, 0.0, 0.0)), (L.nz - 1, (0, 0, -1), lid)):
        n = np.array(nvec)
        tang = [np.array(t) for t in ((1, 0, 0), (0, 1, 0))]
        for y in range(L.ny):
            for x in range(L.nx):
                p = _pull(f, e, x, y, z)
                Fc = F[:, z, y, x]
                en = e @ n
                known = en <= 0
                # the known populations are plain pulls from inside the lattice
                np.testing.assert_allclose(g[known, z, y, x], p[known], rtol=0, atol=1e-15)
                s0 = p[en == 0].sum()
                sm = p[en == -1].sum()
                un = float(np.dot(uw, n))
                rho = (s0 + 2.0 * sm - 0.5 * float(np.dot(Fc, n))) / (1.0 - un)
                j = rho * np.asarray(uw) - 0.5 * Fc
                want = {}
                want[_index(e, n)] = p[_index(e, -n)] + float(np.dot(j, n)) / 3.0
                for t in tang:
                    Nt = 0.5 * float(((e @ t) * p)[en == 0].sum()) - float(np.dot(j, t)) / 3.0
                    for sgn in (1, -1):
                        i = _index(e, n + sgn * t)
                        want[i] = (p[_index(e, -(n + sgn * t))]
                                   + (float(np.dot(j, n)) + sgn * float(np.dot(j, t))) / 6.0
                                   - sgn * Nt)
                for i, v in want.items():
                    assert abs(g[i, z, y, x] - v) < 1e-14, (z, y, x, i)
                # normal non-equilibrium bounce-back in its plain form (F = 0
                # part): g_n - g_-n = f^eq_n - f^eq_-n at (rho, u_w) + F-term
                i, ib = _index(e, n), _index(e, -n)
                eq_diff = 6.0 * w[i] * rho * float(np.dot(uw, n))
                assert abs((g[i, z, y, x] - g[ib, z, y, x]) - eq_diff
                           + float(np.dot(Fc, n)) / 6.0) < 1e-14


@pytest.mark.parametrize("walls", [(True, True, True), (True, False, True), (False, True, True)])
def test_boundary_nodes_take_the_prescribed_velocity(table, walls):
    """Faces, edges and corners: after streaming, (sum e g + F/2)/rho is
    exactly the wall velocity (the lid velocity on the top face's interior
    nodes, zero elsewhere, top edges included); edge and corner densities
    equal the inner diagonal neighbour's density in the stored state;
    buried pairs are equal; interior nodes are plain pulls."""
    e, _ = table
    lid = (0.05, 0.02, 0.0)
    L = O.Lattice(5, 4, 6, 0.7, walls=walls, lid=True, lid_u=lid, onsite=True)
    f = _random_state(L, 3)
    F = W.noise((3,) + L.shape, 5, 1e-3)
    g = O.stream(L, f, F)
    dims = (L.nx, L.ny, L.nz)
    for z in range(L.nz):
        for y in range(L.ny):
            for x in range(L.nx):
                p = (x, y, z)
                s = np.array([(1 if p[a] == 0 else -1 if p[a] == dims[a] - 1 else 0)
                              if walls[a] else 0 for a in range(3)])
                faces = int(np.count_nonzero(s))
                gc = g[:, z, y, x]
                if faces == 0:
                    np.testing.assert_allclose(gc, _pull(f, e, x, y, z), rtol=0, atol=1e-15)
                    continue
                uw = np.asarray(lid) if (faces == 1 and z == L.nz - 1) else np.zeros(3)
                rho, u = _velocity(gc, e, F[:, z, y, x])
                np.testing.assert_allclose(u, uw, rtol=0, atol=1e-14, err_msg=str(p))
                if faces > 1:
                    nb = f[:, z + s[2], y + s[1], x + s[0]].sum()
                    assert abs(rho - nb) < 1e-14, p
                    unknown = (e @ s > 0) | ((e * s) > 0).any(axis=1)
                    for i in range(19):
                        ib = _index(e, -e[i])
                        if unknown[i] and unknown[ib]:
                            assert abs(gc[i] - gc[ib]) < 1e-15, (p, i)


@pytest.mark.parametrize("tau", [0.6, 0.9, 1.5])
def test_couette_flow_is_exact(tau):
    """Plane Couette flow between an on-site wall at rest (z = 0) and the
    lid (z = nz-1) moving along x: the steady lattice solution is the
    linear profile u_x = U z / (nz - 1) to round-off, at any tau."""
    nz, U = 9, 0.04
    L = O.Lattice(1, 1, nz, tau, walls=(False, False, True), lid=True, lid_u=(U, 0, 0),
                  onsite=True)
    f = O.run(L, O.init_equilibrium(L), 40000)
    _, u = O.moments(L, f)
    z = np.arange(nz)
    assert np.abs(u[0, :, 0, 0] - U * z / (nz - 1)).max() < 1e-13
    assert np.abs(u[1:]).max() < 1e-13


@pytest.mark.parametrize("tau", [0.6, 1.0, 1.7])
def test_poiseuille_flow_is_exact(tau):
    """Force-driven Poiseuille flow between on-site walls at z = 0 and
    z = H = nz-1: u_x = F / (2 rho nu) z (H - z), nu = (tau - 1/2)/3, to
    round-off at any tau (halfway bounce-back is exact only at one tau)."""
    nz, Fx = 9, 1e-5
    L = O.Lattice(1, 1, nz, tau, walls=(False, False, True), onsite=True)
    F = W.uniform_force(1, 1, nz, (Fx, 0.0, 0.0))
    f = O.run(L, O.init_equilibrium(L), 60000, F)
    rho, u = O.moments(L, f, F)
    nu = (tau - 0.5) / 3.0
    z = np.arange(nz)
    exact = Fx / (2.0 * nu) * z * (nz - 1 - z)
    assert np.abs(rho - 1.0).max() < 1e-11
    assert np.abs(u[0, :, 0, 0] - exact).max() / exact.max() < 1e-10


def test_rest_is_a_fixed_point_and_lid_cavity_is_symmetric():
    L = O.Lattice(6, 5, 7, 0.7, walls=(True, True, True), onsite=True)
    f = O.init_equilibrium(L)
    assert np.abs(O.run(L, f, 5) - f).max() < 1e-15
    L = O.Lattice(7, 7, 7, 0.6, walls=(True, True, True), lid=True, lid_u=(0.05, 0, 0),
                  onsite=True)
    f = O.run(L, O.init_equilibrium(L), 150)
    rho, u = O.moments(L, f)
    np.testing.assert_allclose(rho, rho[:, ::-1, :], rtol=0, atol=1e-14)
    np.testing.assert_allclose(u[0], u[0][:, ::-1, :], rtol=0, atol=1e-14)
    np.testing.assert_allclose(u[2], u[2][:, ::-1, :], rtol=0, atol=1e-14)
    np.testing.assert_allclose(u[1], -u[1][:, ::-1, :], rtol=0, atol=1e-14)
    # the top face's interior nodes move with the lid, every other wall node rests
    np.testing.assert_allclose(u[0, -1, 1:-1, 1:-1], 0.05, rtol=0, atol=1e-14)
    np.testing.assert_allclose(u[:, 0], 0.0, rtol=0, atol=1e-14)


def test_onsite_walls_need_three_nodes():
    L = O.Lattice(4, 2, 5, 0.7, walls=(False, True, False), onsite=True)
    with pytest.raises(Exception):
        O.init_equilibrium(L)
