"""Pins of the oracle's force density (Eqs. PD_EOM_Dynamic, PD_Force_Function)
against properties the mathematics fixes, and of its explicit integrator."""
import dataclasses
import math

import numpy as np

import pd_workloads as W
from oracle import core


def _tiny(notch=False):
    g = W.Grid(7, 6, 5, 1e-3, 3.01, 1 if notch else 0, 7, 6)
    mat = W.Material(E=30e9, law=W.LAW_BILINEAR, s0=1.0, s_ratio=10.0)  # s0 huge: no damage
    bc = W.BC(W.BC_BAR_TENSION, u_max=0.0, n_ramp=1, grip_planes=0)
    return W.Workload("t", g, mat, bc, 1)


def _coords(g):
    n = np.arange(g.n_nodes)
    return np.stack([(n % g.nx + 0.5) * g.dx, ((n // g.nx) % g.ny + 0.5) * g.dx,
                     (n // (g.nx * g.ny) + 0.5) * g.dx], 1)


def _energy(m, u):
    """E = 1/2 sum_i sum_j (1/2) c s^2 |xi| V_i V_j, written independently of the oracle."""
    g = m.w.grid
    x = _coords(g)
    V = g.dx ** 3
    i = np.repeat(np.arange(m.n), np.diff(m.row))
    j = m.col
    xi = x[j] - x[i]
    y = xi + u[j] - u[i]
    L0 = np.linalg.norm(xi, axis=1)
    s = np.linalg.norm(y, axis=1) / L0 - 1.0
    return 0.5 * np.sum(0.5 * m.c * s * s * L0) * V * V


def test_force_is_energy_gradient():
    w = _tiny(notch=True)
    m = core.Model(w)
    rng = np.random.default_rng(3)
    u = rng.standard_normal((m.n, 3)) * 2e-8
    F, _, _ = m.force(u, np.zeros(m.nb))
    V = w.grid.dx ** 3
    h = 1e-11
    for k in rng.choice(m.n * 3, 25, replace=False):
        e = np.zeros(m.n * 3)
        e[k] = h
        dE = (_energy(m, u + e.reshape(-1, 3)) - _energy(m, u - e.reshape(-1, 3))) / (2 * h)
        assert abs(-dE / V - F.reshape(-1)[k]) <= 1e-5 * np.abs(F).max()


def test_rigid_translation_zero():
    w = _tiny()
    m = core.Model(w)
    u = np.tile([3e-4, -1e-4, 2e-4], (m.n, 1))
    F, _, sm = m.force(u, np.zeros(m.nb))
    assert np.all(F == 0.0) and sm == 0.0


def test_rigid_rotation_zero():
    w = _tiny()
    m = core.Model(w)
    th = 1e-3
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    a = 0.7
    R = R @ np.array([[1, 0, 0], [0, math.cos(a), -math.sin(a)], [0, math.sin(a), math.cos(a)]])
    x = _coords(w.grid)
    u = x @ R.T - x
    F, _, sm = m.force(u, np.zeros(m.nb))
    V = w.grid.dx ** 3
    scale = m.c * V * 1e-4 * 122  # a node's force at stretch 1e-4
    assert np.abs(F).max() <= 1e-9 * scale
    assert abs(sm) < 1e-12


def test_net_internal_force_zero():
    w = _tiny(notch=True)
    m = core.Model(w)
    u = np.random.default_rng(5).standard_normal((m.n, 3)) * 1e-7
    F, _, _ = m.force(u, np.zeros(m.nb))
    assert np.abs(F.sum(0)).max() <= 1e-12 * np.abs(F).sum()


def test_uniform_stretch_interior_force_zero():
    g = W.Grid(9, 9, 9, 1e-3, 3.01)
    w = dataclasses.replace(_tiny(), grid=g)
    m = core.Model(w)
    eps = 1e-4
    u = eps * _coords(g)
    F, _, sm = m.force(u, np.zeros(m.nb))
    assert abs(sm - eps) <= 1e-12
    centre = 4 + 9 * (4 + 9 * 4)
    scale = m.c * g.dx ** 3 * eps * 122
    assert np.abs(F[centre]).max() <= 1e-10 * scale
    assert np.abs(F).max() > 1e-3 * scale  # free surfaces carry the unbalanced bonds
    # interior strain energy density of the lattice vs the continuum value
    # pi c eps^2 delta^4 / 4 that defines the micromodulus (lattice excess 10.6%)
    x = _coords(g)
    js = m.col[m.row[centre]:m.row[centre + 1]]
    W_lat = 0.25 * m.c * eps ** 2 * np.linalg.norm(x[js] - x[centre], axis=1).sum() * g.dx ** 3
    W_cont = math.pi * m.c * eps ** 2 * (3.01 * g.dx) ** 4 / 4
    assert abs(W_lat / W_cont - 285.2204 / (math.pi * 3.01 ** 4)) < 1e-3
    assert 1.0 < W_lat / W_cont < 1.12


def test_two_node_leapfrog_recurrence():
    """Two nodes, one bond: the relative displacement follows the damped
    leapfrog recurrence (1 + z/2) r+ - 2 r + (1 - z/2) r- = -w^2 dt^2 r."""
    g = W.Grid(2, 1, 1, 1e-3, 1.01)
    for zeta in (0.0, 3e5):
        mat = W.Material(E=30e9, law=W.LAW_BILINEAR, s0=1.0, s_ratio=10.0, zeta=zeta)
        bc = W.BC(W.BC_BAR_TENSION, u_max=0.0, n_ramp=1, grip_planes=0)
        w = W.Workload("pair", g, mat, bc, 1)
        m = core.Model(w)
        a0 = 1e-12
        u0 = np.array([[-a0, 0, 0], [a0, 0, 0]])
        steps = 400
        out = m.run(steps, state=(u0, np.zeros((2, 3)), np.zeros(m.nb)))
        V = g.dx ** 3
        w2 = 2 * m.c * V / (mat.rho * g.dx)
        dt = m.dt
        z = zeta * dt
        r_prev, r = 2 * a0, 2 * a0          # v^{-1/2} = 0
        for _ in range(steps):
            r_next = (2 * r - (1 - z / 2) * r_prev - w2 * dt * dt * r) / (1 + z / 2)
            r_prev, r = r, r_next
        rel = out["u"][1, 0] - out["u"][0, 0]
        assert abs(rel - r) <= 1e-6 * 2 * a0
        assert abs(out["u"][0, 0] + out["u"][1, 0]) <= 1e-20  # centre of mass at rest


def test_stable_dt_closed_form():
    """dt = safety sqrt(2 rho / (c V sum_j 1/|xi_j|)) for the full 122-point stencil."""
    g = W.Grid(9, 9, 9, 1e-3, 3.01)
    w = dataclasses.replace(_tiny(), grid=g)
    m = core.Model(w)
    inv = sum(1.0 / math.sqrt(a * a + b * b + c * c) for a in range(-3, 4) for b in range(-3, 4)
              for c in range(-3, 4) if 0 < a * a + b * b + c * c <= 9) / g.dx
    expect = 0.5 * math.sqrt(2 * w.mat.rho / (m.c * g.dx ** 3 * inv))
    assert abs(m.dt - expect) <= 1e-13 * expect


def test_broken_bond_at_zero_length_carries_no_force():
    """A fully damaged bond contributes nothing, even when it has collapsed to
    zero length (its direction is undefined there): the forces stay finite and
    equal those of the same configuration with the broken bond a hair apart."""
    w = _tiny()
    m = core.Model(w)
    x = _coords(w.grid)
    i = 2 + w.grid.nx * (2 + w.grid.ny * 2)     # interior node
    j = i + 1                                   # its +x neighbour
    d = np.zeros(m.nb)
    for a, b in ((i, j), (j, i)):
        q = m.row[a] + int(np.nonzero(m.col[m.row[a]:m.row[a + 1]] == b)[0][0])
        d[q] = 1.0
    u = np.zeros((m.n, 3))
    u[j] = x[i] - x[j]                          # node j sits on node i
    F, _, _ = m.force(u, d)
    assert np.all(np.isfinite(F))
    u2 = u.copy()
    u2[j, 1] += 1e-9 * w.grid.dx                # the broken bond a hair apart
    F2, _, _ = m.force(u2, d)
    assert np.abs(F - F2).max() <= 1e-6 * np.abs(F2).max()
