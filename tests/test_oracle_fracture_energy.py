"""Pins of the fracture-energy calibration of the critical stretch (Appendix
A, three-dimensional case): the bond energy integrated numerically from the
law itself, then over the bonds that cross a unit area of a plane, gives back
G_F; the printed Eq. exp_sc differs from the form that satisfies Eq.
exp_fracture_energy by exactly alpha s0; the adjoint with per-bond critical
stretches matches central differences."""
import dataclasses
import math

import numpy as np
import pytest
from scipy import integrate

import pd_workloads as W
from oracle import core, field

E, DX, M = 30e9, 2.5e-3, 3.01
DELTA = M * DX


def _plane_factor(delta):
    """int_0^delta int_0^2pi int_z^delta int_0^acos(z/xi) xi^3 sin(phi) dphi dxi dtheta dz,
    done numerically over (xi, z) after the elementary phi and theta integrals."""
    val, _ = integrate.dblquad(lambda xi, z: 2.0 * math.pi * xi ** 3 * (1.0 - z / xi), 0.0, delta,
                               lambda z: z, lambda z: delta, epsabs=0, epsrel=1e-12)
    return val


@pytest.mark.parametrize("law,k,alpha", [(W.LAW_EXPLINEAR, 25.0, 0.25), (W.LAW_EXPLINEAR, 10.0, 0.5),
                                         (W.LAW_BILINEAR, 25.0, 0.25)])
@pytest.mark.parametrize("s0", [8e-5, 1e-4, 1.3e-4])
def test_calibrated_critical_stretch_reproduces_the_fracture_energy(law, k, alpha, s0):
    c = core.micromodulus(E, DELTA)
    G_F = 40.0
    A = core.gf_coefficient(law, c, DELTA, G_F, k, alpha)
    sc = s0 + A / s0
    assert sc > s0
    # energy per unit bond length absorbed while softening, from the law: int c (1 - d(s)) s ds
    kw, _ = integrate.quad(lambda s: c * (1.0 - core.damage_law(law, s, s0, sc, k, alpha)) * s, s0, sc,
                           epsabs=0, epsrel=1e-13, limit=400)
    G_num = kw * _plane_factor(DELTA)
    assert G_num == pytest.approx(G_F, rel=1e-8)
    assert core.fracture_energy(law, c, DELTA, s0, sc, k, alpha) == pytest.approx(G_F, rel=1e-12)


def test_printed_critical_stretch_reading():
    """The printed Eq. exp_sc gives (1 + alpha) s0 - (...) where Eq. exp_fracture_energy
    gives s0 - (...); only the latter reproduces G_F."""
    c, s0, G_F, k, a = core.micromodulus(E, DELTA), 1e-4, 40.0, 25.0, 0.25
    d5 = DELTA ** 5
    P = 2 * k - 2 * math.exp(k) + a * k - a * k * math.exp(k) + 2
    printed = (10 * k * (1 - math.exp(k)) * (1 + a) * (G_F - math.pi * c * d5 * s0 ** 2 * P / (10 * k * (math.exp(k) - 1)))
               / (c * d5 * s0 * math.pi * P))
    sc = s0 + core.gf_coefficient(W.LAW_EXPLINEAR, c, DELTA, G_F, k, a) / s0
    assert printed - sc == pytest.approx(a * s0, rel=1e-9)
    assert core.fracture_energy(W.LAW_EXPLINEAR, c, DELTA, s0, sc, k, a) == pytest.approx(G_F, rel=1e-12)
    assert abs(core.fracture_energy(W.LAW_EXPLINEAR, c, DELTA, s0, printed, k, a) - G_F) > 1e-3 * G_F


@pytest.mark.parametrize("law,G_F", [(W.LAW_BILINEAR, 6.0), (W.LAW_EXPLINEAR, 2.0)])
def test_adjoint_with_calibrated_critical_stretch(law, G_F):
    """s_crit = s0 + A/s0 adds dA-terms to dD/ds0; central differences with
    h = 1e-6 relative (the calibrated softening windows are narrow, so larger
    steps move bonds across the onset of softening)."""
    w = W.tiny_beam(16, 6, 4, n_steps=1500)
    w = dataclasses.replace(w, bc=dataclasses.replace(w.bc, u_max=2.5e-5),
                            mat=dataclasses.replace(w.mat, law=law, G_F=G_F))
    Phi, lam = field.kl_separable(w.grid, w.field.length, w.field.n_modes)
    s0 = field.sample_field(w, Phi, lam, w.seed, 0, [0])[0]
    m = core.Model(w, s0=s0)
    T = 320
    obs, wts = [T - 1, T // 2], [1.0, 0.5]
    gs, _ = m.adjoint(T, obs, wts)
    assert np.abs(gs).max() > 0

    def J(v):
        r = core.Model(w, s0=v, dt=m.dt).run(T)["reaction"]
        return sum(wt * r[o] for o, wt in zip(obs, wts))
    for i in list(np.argsort(-np.abs(gs))[:3]) + list(np.flatnonzero(gs)[:2]):
        h = 1e-6 * abs(s0[i])
        p, q = s0.copy(), s0.copy()
        p[i] += h
        q[i] -= h
        fd = (J(p) - J(q)) / (2 * h)
        print(f"law {law} s0[{i}]: adjoint {gs[i]:.9e} fd {fd:.9e}")
        assert abs(gs[i] - fd) <= 1e-4 * abs(fd) + 1e-12 * abs(J(s0)) / h
