"""Pins of the oracle's random-field sampler (Section 5) and Philox generator."""
import math
import os

import numpy as np
import pytest

import pd_workloads as W
from oracle import field

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        out = field.philox4x32_10(np.array([v[:4]], np.uint32), np.array([v[4:6]], np.uint32))[0]
        assert [int(x) for x in out] == v[6:]


def test_xi_standard_normal_and_coupling():
    xi = field.draw_xi(12345, 1, np.arange(4000), 64)
    assert xi.shape == (4000, 64)
    z = xi.reshape(-1)
    assert abs(z.mean()) < 4 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 4 * math.sqrt(2 / z.size)
    # the same (seed, level, sample) gives the same xi; another level or sample does not
    a = field.draw_xi(12345, 1, [7], 64)
    assert np.array_equal(a[0], xi[7])
    assert not np.array_equal(field.draw_xi(12345, 2, [7], 64)[0], a[0])
    # odd K is a prefix of the next even K
    assert np.array_equal(field.draw_xi(9, 0, [3], 7)[0], field.draw_xi(9, 0, [3], 8)[0][:7])


def test_separable_equals_dense_kl():
    """Kronecker-product modes are eigenvectors of the dense 3D covariance."""
    g = W.Grid(6, 5, 4, 2.5e-3, 3.01)
    l = 6e-3
    Phi, lam = field.kl_separable(g, l, 10)
    C = field.dense_cov(g, l, 0)
    for k in range(10):
        assert np.abs(C @ Phi[:, k] - lam[k] * Phi[:, k]).max() <= 1e-10 * lam[0]
    assert np.abs(Phi.T @ Phi - np.eye(10)).max() < 1e-12
    lam_dense = np.sort(np.linalg.eigvalsh(C))[::-1][:10]
    assert np.abs(lam - lam_dense).max() <= 1e-10 * lam[0]


def test_truncated_covariance_converges():
    g = W.Grid(4, 3, 3, 2.5e-3, 3.01)
    C = field.dense_cov(g, 5e-3, 0)
    errs = []
    for K in (4, 12, 36):
        Phi, lam = field.kl_separable(g, 5e-3, K)
        errs.append(np.abs(Phi @ np.diag(lam) @ Phi.T - C).max())
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-12
    # dense exponential kernel (the paper's): full expansion reproduces C
    Ce = field.dense_cov(g, 5e-3, 1)
    Phi, lam = field.kl_dense(g, 5e-3, g.n_nodes, 1)
    assert np.abs(Phi @ np.diag(lam) @ Phi.T - Ce).max() < 1e-12


def test_mode_order_rule():
    lx = np.array([3.0, 1.0])
    ly = np.array([2.0, 0.5])
    lz = np.array([2.0, 0.5])
    sel = field.select_modes(lx, ly, lz, 8)
    assert sel[:2] == [(0, 0, 0), (1, 0, 0)]      # products 12, 4
    # (0,0,1) and (0,1,0) tie exactly at 3: ascending (a,b,c)
    assert sel[2:4] == [(0, 0, 1), (0, 1, 0)]


def test_lognormal_and_weibull_moments():
    g = np.random.default_rng(0).standard_normal(400000)
    s = field.lognormal(g, 1e-4, 0.1)
    assert abs(s.mean() / 1e-4 - 1) < 2e-3 and abs(s.std() / s.mean() - 0.1) < 3e-3
    wb = field.weibull(g, 1e-4, 3.0)
    assert abs(wb.mean() / 1e-4 - 1) < 3e-3
    cov_w = math.sqrt(math.gamma(1 + 2 / 3) / math.gamma(1 + 1 / 3) ** 2 - 1)
    assert abs(wb.std() / wb.mean() - cov_w) < 5e-3


def test_restriction_is_child_mean():
    g = W.Grid(4, 4, 2, 1e-3, 3.01)
    f = np.arange(32, dtype=np.float64)[None, :] ** 1.5
    c = field.restrict(f, g)
    fine = f.reshape(2, 4, 4)  # (z, y, x)
    expect = []
    for Z in range(1):
        for Y in range(2):
            for X in range(2):
                expect.append(fine[2 * Z:2 * Z + 2, 2 * Y:2 * Y + 2, 2 * X:2 * X + 2].sum() / 8)
    assert c.shape == (1, 4)
    assert np.allclose(c[0], expect, rtol=1e-15, atol=0)


def test_plane_restriction_is_in_plane_child_mean():
    """A plane hierarchy keeps one layer: the coarse node is the mean of its 2x2 children."""
    g = W.Grid(6, 4, 1, 1e-3, 3.01)
    f = np.arange(24, dtype=np.float64)[None, :] ** 1.5
    c = field.restrict(f, g)
    fine = f.reshape(4, 6)  # (y, x)
    expect = [fine[2 * Y:2 * Y + 2, 2 * X:2 * X + 2].sum() / 4 for Y in range(2) for X in range(3)]
    assert c.shape == (1, 6)
    assert np.allclose(c[0], expect, rtol=1e-15, atol=0)
