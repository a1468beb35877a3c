"""Pins of the oracle's bond laws (Appendix A) and micromodulus."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import core

S0, K, ALPHA = 1e-4, 25.0, 0.25


@pytest.mark.parametrize("law,sc", [(0, 10 * S0), (1, 25 * S0)])
def test_endpoints_and_monotone(law, sc):
    assert core.damage_law(law, S0, S0, sc, K, ALPHA) == 0.0
    assert core.damage_law(law, 0.5 * S0, S0, sc, K, ALPHA) == 0.0
    assert core.damage_law(law, sc, S0, sc, K, ALPHA) == 1.0
    assert core.damage_law(law, 2 * sc, S0, sc, K, ALPHA) == 1.0
    # continuity at both ends
    assert core.damage_law(law, S0 * (1 + 1e-9), S0, sc, K, ALPHA) < 1e-7
    assert core.damage_law(law, sc * (1 - 1e-9), S0, sc, K, ALPHA) > 1 - 1e-6
    s = np.linspace(S0, sc, 2001)
    d = np.array([core.damage_law(law, x, S0, sc, K, ALPHA) for x in s])
    assert np.all(np.diff(d) >= 0)


def test_explinear_bond_energy_closed_form():
    """w = int_{s0}^{sc} f xi ds with f = c (1-d) s (Eq. exp_bond_energy)."""
    c, xi, sc = 3.3e19, 2.5e-3, 25 * S0
    f = lambda s: c * (1 - core.damage_law(1, s, S0, sc, K, ALPHA)) * s * xi
    w_num, _ = quad(f, S0, sc, epsabs=0, epsrel=1e-13, limit=200)
    ek = math.exp(K)
    w_paper = c * S0 * xi * (S0 - sc) * (2 * K - 2 * ek + ALPHA * K - ALPHA * K * ek + 2) / (
        2 * K * (ek - 1) * (1 + ALPHA))
    assert abs(w_num - w_paper) <= 1e-10 * abs(w_paper)


def test_bilinear_bond_energy_triangle():
    c, xi, sf = 3.3e19, 2.5e-3, 10 * S0
    f = lambda s: c * (1 - core.damage_law(0, s, S0, sf)) * s * xi
    w_num, _ = quad(f, S0, sf, epsabs=0, epsrel=1e-13)
    assert abs(w_num - 0.5 * c * S0 * xi * (sf - S0)) <= 1e-10 * w_num


def test_explinear_force_shape():
    """Force starts at c s0, falls exponentially then linearly to zero at sc."""
    sc = 25 * S0
    f = lambda s: (1 - core.damage_law(1, s, S0, sc, K, ALPHA)) * s
    assert abs(f(S0) - S0) < 1e-18
    assert f(sc) == 0.0
    # just before sc the decay is linear with slope -alpha s0 / ((1+alpha)(sc-s0)) (the linear term)
    h = 1e-3 * (sc - S0)
    slope = (f(sc - h) - f(sc - 2 * h)) / h
    expect = -S0 * (ALPHA + K * math.exp(-K) / (1 - math.exp(-K))) / ((1 + ALPHA) * (sc - S0))
    assert abs(slope - expect) < 1e-3 * abs(expect)


def test_micromodulus_continuum_energy():
    """c = 12E/(pi delta^4): the continuum strain energy of a uniform dilatation
    eps is int_H (1/2)(c eps^2 |xi|/2) dV = pi c eps^2 delta^4 / 4, which equals
    the classical 9 K eps^2 / 2 with K = E / (3 (1 - 2 nu)), nu = 1/4."""
    E, delta = 30e9, 7.525e-3
    c = core.micromodulus(E, delta)
    Kb = E / (3 * (1 - 2 * 0.25))
    W_cont = math.pi * c * delta ** 4 / 4
    assert abs(W_cont - 4.5 * Kb) <= 1e-12 * W_cont
