"""Pins of the plane (two-dimensional) model, the paper's own dimensionality:
the 28-neighbour horizon at m = pi and the bond counts of the paper's five
mesh levels (Table discretisation); the plane-stress and plane-strain
micromoduli of Eq. bond_stiffness_constant against linear elasticity for a
uniform biaxial stretch; the two-dimensional fracture-energy calibration
(Eq. exp_sc_2D) against numerical integration of the law and the geometry."""
import dataclasses
import math

import numpy as np
import pytest
from scipy import integrate

import pd_workloads as W
from oracle import core

# nodes of the paper's levels (175 x 50 mm at dx = 5 ... 0.3125 mm) and their
# directed bond counts at delta = pi dx, unnotched
LEVELS = [(35, 10, 8_216), (70, 20, 35_996), (140, 40, 150_356), (280, 80, 614_276), (560, 160, 2_482_916)]


def test_plane_horizon_has_28_neighbours():
    g = W.Grid(21, 21, 1, 1e-3, math.pi)
    row, col = core.neighbours(g)
    c = 10 + 21 * 10
    js = col[row[c]:row[c + 1]]
    off = np.stack([js % 21 - 10, js // 21 - 10], 1)
    assert len(js) == 28 and np.all((off ** 2).sum(1) <= 9) and not np.any((off == 0).all(1))


@pytest.mark.parametrize("nx,ny,nb", LEVELS)
def test_plane_level_bond_counts(nx, ny, nb):
    g = W.Grid(nx, ny, 1, 5e-3 * 35 / nx, math.pi)
    row, col = core.neighbours(g)
    assert int(row[-1]) == nb
    if nx <= 70:
        rb, cb = core.neighbours(g, brute=True)
        assert np.array_equal(rb, row) and np.array_equal(cb, col)


@pytest.mark.parametrize("model,nu,modulus", [(W.MODEL_PLANE_STRESS, 1.0 / 3.0, lambda E, nu: E / (1.0 - nu)),
                                              (W.MODEL_PLANE_STRAIN, 0.25,
                                               lambda E, nu: E / ((1.0 + nu) * (1.0 - 2.0 * nu)))])
def test_plane_micromodulus_against_elasticity(model, nu, modulus):
    """Uniform biaxial stretch eps: interior force zero; the continuum strain energy
    density (c eps^2 / 4) int_H |xi| t dA = pi c t delta^3 eps^2 / 6 equals the
    plane elasticity value modulus(E, nu) eps^2 (the Poisson ratio of a bond-based
    plane model); the lattice sum exceeds it by its lattice factor."""
    E, dx, t, eps = 30e9, 1e-3, 0.05, 1e-4
    g = W.Grid(15, 15, 1, dx, math.pi)
    mat = W.Material(E=E, law=W.LAW_BILINEAR, s0=1.0, model=model, thickness=t)
    w = W.Workload("plate", g, mat, W.BC(W.BC_BAR_TENSION, u_max=0.0, n_ramp=1, grip_planes=0), 1)
    m = core.Model(w)
    i = np.arange(g.n_nodes)
    x = np.stack([(i % 15 + 0.5) * dx, (i // 15 + 0.5) * dx, np.full(g.n_nodes, 0.5 * dx)], 1)
    u = eps * x
    u[:, 2] = 0.0
    F, _, _ = m.force(u, np.zeros(m.nb))
    centre = 7 + 15 * 7
    assert np.abs(F[centre]).max() <= 1e-10 * m.c * dx * dx * t * eps * 28
    delta = math.pi * dx
    W_cont = math.pi * m.c * t * delta ** 3 * eps ** 2 / 6.0
    assert W_cont == pytest.approx(modulus(E, nu) * eps ** 2, rel=1e-12)
    js = m.col[m.row[centre]:m.row[centre + 1]]
    W_lat = 0.25 * m.c * eps ** 2 * np.linalg.norm(x[js] - x[centre], axis=1).sum() * dx * dx * t
    lattice = sum(math.hypot(a, b) for a in range(-3, 4) for b in range(-3, 4) if 0 < a * a + b * b <= 9)
    assert W_lat / W_cont == pytest.approx(lattice / (2.0 * math.pi * math.pi ** 3 / 3.0), rel=1e-12)


@pytest.mark.parametrize("law", [W.LAW_EXPLINEAR, W.LAW_BILINEAR])
def test_plane_calibrated_critical_stretch(law):
    """G_F = 2h int_0^delta int_z^delta int_0^acos(z/xi) w xi dphi dxi dz (Eq.
    exp_fracture_energy_2D) with w from the law itself recovers G_F."""
    E, dx, t, s0, G_F = 30e9, 2.5e-3, 0.05, 1e-4, 30.0
    delta = math.pi * dx
    for model in (W.MODEL_PLANE_STRESS, W.MODEL_PLANE_STRAIN):
        c = core.micromodulus_2d(E, delta, t, model == W.MODEL_PLANE_STRAIN)
        A = core.gf_coefficient_2d(law, c, delta, t, G_F)
        sc = s0 + A / s0
        kw, _ = integrate.quad(lambda s: c * (1.0 - core.damage_law(law, s, s0, sc, 25.0, 0.25)) * s, s0, sc,
                               epsabs=0, epsrel=1e-13, limit=400)
        geo, _ = integrate.dblquad(lambda xi, z: 2.0 * t * xi * xi * math.acos(z / xi), 0.0, delta,
                                   lambda z: z, lambda z: delta, epsabs=0, epsrel=1e-11)
        assert kw * geo == pytest.approx(G_F, rel=1e-7)


def test_plane_beam_reaches_a_peak():
    """A notched plane-stress beam under three-point bending softens past its peak."""
    g = W.Grid(28, 8, 1, 2.5e-3, math.pi, 1, 28, 3)
    mat = W.Material(E=30e9, law=W.LAW_EXPLINEAR, s0=1e-4, zeta=5e4, G_F=30.0,
                     model=W.MODEL_PLANE_STRESS, thickness=0.05)
    bc = W.BC(W.BC_BEAM_3PT, u_max=3e-5, n_ramp=1500, support_x2=(3, 53), load_x2=28)
    m = core.Model(W.Workload("plane_beam", g, mat, bc, 1500))
    r = m.run(1500, use_stop=True)
    assert r["peak"] > 0 and r["peak_step"] < r["n_done"] - 100
    assert r["d"].max() == 1.0
