"""Pins of the oracle's neighbour list (Eq. PD_Horizon) and boundary sets."""
from fractions import Fraction
from itertools import product

import numpy as np
import pytest

import pd_workloads as W
from oracle import core


def _fraction_list(g):
    """Independent brute force with exact rationals and real positions."""
    n = g.nx * g.ny * g.nz
    dx = Fraction(1)
    delta2 = Fraction(g.m_ratio).limit_denominator(10**9) ** 2
    pos = []
    for i in range(n):
        ix, iy, iz = i % g.nx, (i // g.nx) % g.ny, i // (g.nx * g.ny)
        pos.append((Fraction(2 * ix + 1, 2), Fraction(2 * iy + 1, 2), Fraction(2 * iz + 1, 2)))
    xn = Fraction(g.notch_x2, 2)
    yd = Fraction(g.notch_y2, 2)
    rows = []
    for i in range(n):
        r = []
        for j in range(n):
            if i == j:
                continue
            d2 = sum((pos[j][c] - pos[i][c]) ** 2 for c in range(3))
            if d2 > delta2 * dx * dx:
                continue
            if g.notch:
                xi_, xj = pos[i][0], pos[j][0]
                if (xi_ - xn) * (xj - xn) < 0:
                    t = (xn - xi_) / (xj - xi_)
                    yc = pos[i][1] + t * (pos[j][1] - pos[i][1])
                    if yc < yd:
                        continue
            r.append(j)
        rows.append(r)
    return rows


@pytest.mark.parametrize("g", [
    W.Grid(5, 4, 3, 1e-3, 3.01),
    W.Grid(8, 5, 2, 2.5e-3, 3.01, 1, 8, 4),     # notch on a cell face
    W.Grid(7, 5, 2, 2.5e-3, 3.01, 1, 7, 3),     # notch plane through node centres
    W.Grid(6, 6, 1, 1e-3, 1.5, 1, 6, 2),
    W.Grid(4, 4, 4, 1e-3, 3.0),                  # horizon exactly on lattice points
])
def test_bruteforce_matches_exact_rationals(g):
    row, col = core.neighbours(g, brute=True)
    rows = _fraction_list(g)
    assert row[-1] == sum(len(r) for r in rows)
    for i, r in enumerate(rows):
        assert list(col[row[i]:row[i + 1]]) == r


@pytest.mark.parametrize("g", [
    W.Grid(9, 7, 5, 1e-3, 3.01),
    W.Grid(12, 6, 4, 2.5e-3, 3.01, 1, 12, 4),
    W.Grid(11, 6, 4, 2.5e-3, np.pi, 1, 11, 5),
])
def test_window_equals_bruteforce(g):
    a = core.neighbours(g, brute=True)
    b = core.neighbours(g, brute=False)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_interior_stencil_122():
    """m = 3.01, pi and 3.14 give the same 122-point interior stencil (|k|^2 <= 9)."""
    for m in (3.01, np.pi, 3.14):
        g = W.Grid(9, 9, 9, 1e-3, m)
        row, col = core.neighbours(g)
        centre = 4 + 9 * (4 + 9 * 4)
        assert row[centre + 1] - row[centre] == 122
    # direct count of integer offsets with 0 < |k|^2 <= 9
    assert sum(1 for k in product(range(-3, 4), repeat=3) if 0 < sum(x * x for x in k) <= 9) == 122


def test_symmetric_list():
    g = W.Grid(10, 6, 4, 2.5e-3, 3.01, 1, 10, 4)
    row, col = core.neighbours(g)
    pairs = set()
    for i in range(g.n_nodes):
        for j in col[row[i]:row[i + 1]]:
            pairs.add((i, int(j)))
    assert all((j, i) in pairs for (i, j) in pairs)


@pytest.mark.parametrize("w,expected", [
    (W.bar(), 370728),
    (W.beam(5.0), 322444),
    (W.beam(2.5), 2975344),
])
def test_workload_bond_counts(w, expected):
    row, col = core.neighbours(w.grid)
    assert row[-1] == expected


def test_bc_sets():
    w = W.beam(2.5)
    c = core.bc_codes(w.grid, w.bc)
    g = w.grid
    idx = np.arange(g.n_nodes)
    ix, iy = idx % g.nx, (idx // g.nx) % g.ny
    # supports at x = 25 and 150 mm fall on cell faces: two columns each, bottom layer, y held
    sup = (c[:, 1] == 1)
    assert set(ix[sup]) == {9, 10, 59, 60} and set(iy[sup]) == {0}
    assert sup.sum() == 4 * g.nz
    load = (c[:, 1] == 3)
    assert set(ix[load]) == {34, 35} and set(iy[load]) == {g.ny - 1}
    assert (c[:, 0] == 0).all() and (c[:, 2] == 0).all()
    wb = W.bar()
    cb = core.bc_codes(wb.grid, wb.bc)
    ixb = np.arange(wb.grid.n_nodes) % wb.grid.nx
    assert (cb[ixb < 3] == 1).all()
    assert (cb[ixb >= 37, 0] == 2).all() and (cb[ixb >= 37, 1:] == 1).all()
    assert (cb[(ixb >= 3) & (ixb < 37)] == 0).all()
