"""Pins of the oracle's discrete adjoint (reverse-mode derivative of a
weighted sum of reactions with respect to the node fields s0 and kappa):
central finite differences of the oracle's own forward run, before and
during softening, for both bond laws; s0 has no influence before any bond
softens; the gradient is linear in the observation weights."""
import dataclasses

import numpy as np
import pytest

import pd_workloads as W
from oracle import core, field


def _case(law=W.LAW_BILINEAR):
    w = W.tiny_beam(16, 6, 4, n_steps=1500)
    ratio = 10.0 if law == W.LAW_BILINEAR else 25.0
    w = dataclasses.replace(w, bc=dataclasses.replace(w.bc, u_max=2.5e-5),
                            mat=dataclasses.replace(w.mat, law=law, s_ratio=ratio))
    Phi, lam = field.kl_separable(w.grid, w.field.length, w.field.n_modes)
    s0 = field.sample_field(w, Phi, lam, w.seed, 0, [0])[0]
    kap = np.exp(0.1 * np.random.default_rng(1).standard_normal(w.grid.n_nodes))
    return w, s0, kap


def _J(w, dt, s0, kap, T, obs, wts):
    r = core.Model(w, s0=s0, kappa=kap, dt=dt).run(T)["reaction"]
    return sum(wt * r[o] for o, wt in zip(obs, wts))


def _fd(w, dt, s0, kap, T, obs, wts, which, i, rel=1e-3):
    base = s0 if which == "s0" else kap
    h = rel * abs(base[i])
    p, q = base.copy(), base.copy()
    p[i] += h
    q[i] -= h
    if which == "s0":
        return (_J(w, dt, p, kap, T, obs, wts) - _J(w, dt, q, kap, T, obs, wts)) / (2 * h)
    return (_J(w, dt, s0, p, T, obs, wts) - _J(w, dt, s0, q, T, obs, wts)) / (2 * h)


def test_no_strength_sensitivity_before_softening():
    w, s0, kap = _case()
    m = core.Model(w, s0=s0, kappa=kap)
    r = m.run(150)
    assert r["smax"].max() < s0.min()  # no bond has left the elastic range
    gs, gk = m.adjoint(150, [149, 75], [1.0, 0.5])
    assert np.all(gs == 0.0)
    assert np.abs(gk).max() > 0.0


@pytest.mark.parametrize("law,T", [(W.LAW_BILINEAR, 150), (W.LAW_BILINEAR, 300), (W.LAW_EXPLINEAR, 330)])
def test_adjoint_against_central_differences(law, T):
    w, s0, kap = _case(law)
    m = core.Model(w, s0=s0, kappa=kap)
    obs, wts = [T - 1, T // 2, T - 40], [1.0, 0.5, -0.3]
    gs, gk = m.adjoint(T, obs, wts)
    checks = [("k", int(i)) for i in np.argsort(-np.abs(gk))[:2]] + [("k", 5), ("k", 100)]
    if np.abs(gs).max() > 0:
        checks += [("s0", int(i)) for i in np.argsort(-np.abs(gs))[:3]]
        checks += [("s0", int(i)) for i in np.flatnonzero(gs)[:2]]
    # Before softening the response is smooth: h = 1e-3 relative (truncation
    # ~1e-7). Once bonds soften, a larger step moves some bond across the
    # onset of softening inside +-h; h = 1e-5 relative keeps every bond on its
    # branch (FD rounding is then ~1e-5 of these gradients).
    softening = np.abs(gs).max() > 0
    for which, i in checks:
        g = (gs if which == "s0" else gk)[i]
        rel, tol = (1e-5, 1e-4) if softening else (1e-3, 1e-5)
        fd = _fd(w, m.dt, s0, kap, T, obs, wts, which, i, rel)
        print(f"law {law} T={T} {which}[{i}]: adjoint {g:.9e} fd {fd:.9e}")
        assert abs(g - fd) <= tol * abs(fd), (which, i, g, fd)


def test_adjoint_is_linear_in_the_weights():
    w, s0, kap = _case()
    m = core.Model(w, s0=s0, kappa=kap)
    T = 260
    g1s, g1k = m.adjoint(T, [T - 1], [1.0])
    g2s, g2k = m.adjoint(T, [T // 3], [1.0])
    gs, gk = m.adjoint(T, [T - 1, T // 3], [2.0, -0.5])
    assert np.allclose(gs, 2.0 * g1s - 0.5 * g2s, rtol=1e-10, atol=1e-10 * np.abs(gs).max())
    assert np.allclose(gk, 2.0 * g1k - 0.5 * g2k, rtol=1e-10, atol=1e-10 * np.abs(gk).max())


def _chain_case(marginal=W.MARG_LOGNORMAL):
    w, _, _ = _case()
    fs = dataclasses.replace(w.field, marginal=marginal, weibull_m=3.0)
    fk = W.FieldCfg(W.COV_SQEXP, w.field.length, 8, W.MARG_LOGNORMAL, 1.0, 0.1)
    Phi, lam = field.kl_separable(w.grid, fs.length, fs.n_modes)
    Pk, lk = field.kl_separable(w.grid, fk.length, fk.n_modes)
    xs = field.draw_xi(w.seed, 0, [0], fs.n_modes)
    xk = field.draw_xi(w.seed + 1, 0, [0], fk.n_modes)

    def fields(xs_, xk_):
        gs = field.gaussian(Phi, lam, xs_)
        s0 = field.lognormal(gs, fs.mean, fs.cov) if marginal == W.MARG_LOGNORMAL else \
            field.weibull(gs, fs.mean, 3.0)
        return s0[0], field.lognormal(field.gaussian(Pk, lk, xk_), 1.0, 0.1)[0]
    return w, fs, fk, (Phi, lam), (Pk, lk), xs, xk, fields


@pytest.mark.parametrize("marginal,T", [(W.MARG_LOGNORMAL, 150), (W.MARG_LOGNORMAL, 300), (W.MARG_WEIBULL, 300)])
def test_coefficient_gradient_against_central_differences(marginal, T):
    """dJ/dxi for the strength and stiffness KL coefficients: adjoint + chain
    rule against central differences of xi -> fields -> run -> J."""
    w, fs, fk, (Phi, lam), (Pk, lk), xs, xk, fields = _chain_case(marginal)
    s0, kap = fields(xs, xk)
    m = core.Model(w, s0=s0, kappa=kap)
    obs, wts = [T - 1, T // 2], [1.0, -0.4]
    gs, gk = m.adjoint(T, obs, wts)
    gxs = field.grad_xi(fs, Phi, lam, xs, gs[None, :])[0]
    gxk = field.grad_xi(fk, Pk, lk, xk, gk[None, :])[0]
    softening = np.abs(gs).max() > 0
    h = 1e-5 if softening else 1e-3
    # rounding of J (FP64 over T steps, ~1e-13 relative) divided by 2h bounds the FD noise
    noise = 1e-12 * abs(_J(w, m.dt, s0, kap, T, obs, wts)) / h
    for which, k in [("k", 0), ("k", 3), ("k", 7), ("s", 0), ("s", 5), ("s", 15)]:
        g = (gxs if which == "s" else gxk)[k]
        p_s, q_s, p_k, q_k = xs.copy(), xs.copy(), xk.copy(), xk.copy()
        if which == "s":
            p_s[0, k] += h
            q_s[0, k] -= h
        else:
            p_k[0, k] += h
            q_k[0, k] -= h
        fd = (_J(w, m.dt, *fields(p_s, p_k), T, obs, wts) - _J(w, m.dt, *fields(q_s, q_k), T, obs, wts)) / (2 * h)
        print(f"marginal {marginal} T={T} xi_{which}[{k}]: adjoint {g:.9e} fd {fd:.9e}")
        if which == "s" and not softening:
            assert g == 0.0 and fd == 0.0
        else:
            assert abs(g - fd) <= (1e-4 if softening else 1e-5) * abs(fd) + noise
