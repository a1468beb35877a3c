"""Pins of the oracle's reaction force R_n (the peak-load quantity, Sections 4
and 6.2) by static equilibrium, independent of how the oracle sums it.

The oracle reports R_n = -sum over prescribed DOFs of F sign V. Once a damped
run has settled (every free node's force is zero to rounding), statics fixes
that number in two other ways, both computed here from the CSR and the final
displacements with this file's own pair forces (c s (xi+eta)/|xi+eta|,
c = 12 E / (pi delta^4), Eq. bond_stiffness_constant):

* bar in tension: the load carried by the moving grip equals the axial force
  that the bonds crossing any interior cross-section transmit,
  sum over bonds (i left, j right) of f_x V_i V_j;
* notched beam in three-point bending: the load equals the sum of the two
  support reactions, and by mirror symmetry each support carries half.

A flipped sign, a dropped or doubled node volume, or a wrong micromodulus in
the oracle's reaction fails these checks. The elastic bar stiffness is also
checked against E A / L: the bond-based lattice is 10.6 % stiffer than the
continuum in the interior and softer near free surfaces, and this thin bar
(6 x 6 nodes across, horizon 3 cells) sits inside 0.6 .. 1.2 of it.
"""
import dataclasses

import numpy as np

import pd_workloads as W
from oracle import core


def _pair_forces(w, m, u):
    """Per directed bond (i, j): pair force density f_ij (N/m^6) of an undamaged state."""
    g = w.grid
    n = g.n_nodes
    i = np.repeat(np.arange(n), np.diff(m.row))
    j = m.col.astype(np.int64)
    idx = np.arange(n)
    X = np.stack([idx % g.nx, (idx // g.nx) % g.ny, idx // (g.nx * g.ny)], 1) * g.dx
    xi = X[j] - X[i]
    y = xi + (u[j] - u[i])
    L0 = np.linalg.norm(xi, axis=1)
    L = np.linalg.norm(y, axis=1)
    c = 12.0 * w.mat.E / (np.pi * (g.m_ratio * g.dx) ** 4)
    return i, j, (c * (L - L0) / L0)[:, None] * y / L[:, None]


def _settled(w, steps):
    m = core.Model(w)
    r = m.run(steps)
    return m, r


def test_bar_reaction_equals_section_force():
    U = 2e-7
    base = W.bar()
    w = dataclasses.replace(base, grid=W.Grid(20, 6, 6, 1e-3, 3.01),
                            mat=dataclasses.replace(base.mat, s0=1.0, zeta=5e5),
                            bc=dataclasses.replace(base.bc, u_max=U, n_ramp=100))
    m, r = _settled(w, 3000)
    R = r["reaction"][-1]
    assert R > 0.0, "tension: the grip is pulled back by the bar"
    assert abs(r["reaction"][-2] - R) <= 1e-12 * R, "settled"
    g = w.grid
    i, j, f = _pair_forces(w, m, r["u"])
    V = g.dx ** 3
    for xs in (5, 9, 13):  # interior sections between node planes xs and xs + 1
        cross = (i % g.nx <= xs) & (j % g.nx > xs)
        S = (f[cross, 0] * V * V).sum()
        assert abs(R - S) <= 1e-9 * abs(S), (xs, R, S)
    EAL = w.mat.E * (g.ny * g.nz * g.dx ** 2) * U / ((g.nx - 5) * g.dx)
    assert 0.6 <= R / EAL <= 1.2, R / EAL


def test_beam_load_equals_support_reactions():
    base = W.tiny_beam(16, 6, 4, notch=True)
    w = dataclasses.replace(base, mat=dataclasses.replace(base.mat, s0=1.0, zeta=5e5),
                            bc=dataclasses.replace(base.bc, u_max=1e-7, n_ramp=100))
    m, r = _settled(w, 3000)
    R = r["reaction"][-1]
    assert R > 0.0, "the load pushes down; the reaction is positive"
    g = w.grid
    n = g.n_nodes
    i, j, f = _pair_forces(w, m, r["u"])
    V = g.dx ** 3
    F = np.zeros((n, 3))
    np.add.at(F, i, f * V)
    free = m.codes == 0
    assert np.abs(F[free]).max() <= 1e-8 * np.abs(F).max(), "settled"
    sup = m.codes[:, 1] == 1
    ix = np.arange(n) % g.nx
    left = -(F[sup & (ix < g.nx // 2), 1] * V).sum()
    right = -(F[sup & (ix >= g.nx // 2), 1] * V).sum()
    assert abs(R - (left + right)) <= 1e-9 * R, (R, left, right)
    assert abs(left - 0.5 * R) <= 1e-9 * R and abs(right - 0.5 * R) <= 1e-9 * R
