"""Pins of the oracle's explicit run: linear regime, damage history, stop rule."""
import dataclasses

import numpy as np

import pd_workloads as W
from oracle import core


def _small_bar(u_max, s0=1e-4, steps=300):
    w = W.bar()
    g = W.Grid(16, 5, 5, 1e-3, 3.01)
    bc = dataclasses.replace(w.bc, u_max=u_max, n_ramp=steps)
    mat = dataclasses.replace(w.mat, s0=s0)
    return dataclasses.replace(w, grid=g, bc=bc, mat=mat, n_steps=steps)


def test_linear_regime_scales():
    """Without damage the response is linear to first order in U: R(2U) = 2 R(U)."""
    r1 = core.Model(_small_bar(1e-7, s0=1.0)).run(200)["reaction"]
    r2 = core.Model(_small_bar(2e-7, s0=1.0)).run(200)["reaction"]
    assert np.abs(r2 - 2 * r1).max() <= 1e-4 * np.abs(r2).max()
    assert np.abs(r2).max() > 0


def test_damage_monotone_and_stop_rule():
    w = _small_bar(2e-5, steps=600)
    m = core.Model(w)
    state = None
    d_prev = np.zeros(m.nb)
    peak, ps = -np.inf, -1
    done_total = 0
    for chunk in range(6):
        r = m.run(100, state=state, step0=100 * chunk, use_stop=True, peak=peak, peak_step=ps)
        assert np.all(r["d"] >= d_prev)
        assert np.all((r["d"] >= 0) & (r["d"] <= 1))
        d_prev = r["d"]
        state = (r["u"], r["v"], r["d"])
        peak, ps = r["peak"], r["peak_step"]
        done_total += r["n_done"]
        if r["n_done"] < 100:
            # stopped: R < Q/2 at least 100 steps after the peak
            assert r["reaction"][-1] < 0.5 * peak
            assert 100 * chunk + r["n_done"] - 1 - ps >= 100
            break
    assert (d_prev >= 1).any(), "the bar should break"
    # one continuous run gives the same peak as the chunked one
    full = m.run(600, use_stop=True)
    assert full["peak"] == peak and full["peak_step"] == ps and full["n_done"] == done_total


def test_prescribed_and_fixed_dofs():
    w = _small_bar(3e-6, steps=50)
    m = core.Model(w)
    r = m.run(50)
    g = w.grid
    ix = np.arange(g.n_nodes) % g.nx
    assert np.all(r["u"][ix < 3] == 0.0)
    assert np.allclose(r["u"][ix >= g.nx - 3, 0], 3e-6, rtol=0, atol=1e-20)
    assert np.all(r["u"][ix >= g.nx - 3, 1:] == 0.0)
