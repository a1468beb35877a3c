"""Parity at the benchmark's full sizes and launch configurations: the
28,000-node beam stepped in the one-sample schedule the benchmark times, the
same beam with 32 samples per launch (the batched schedule, two samples
checked), and the 448,000-node beam of the size-effect sweep (D = 200 mm,
every node's force; the sweep's largest member runs the same schedule, and
the oracle's neighbour search alone takes about a minute there). Random displacements large enough that bonds soften exercise the
law; the oracle computes every checked value from the same inputs."""
import numpy as np
import pytest
import torch

import pd_workloads as W
from oracle import core

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd(built_lib):
    import paper_2212_04415_gb300 as pd
    return pd


def _dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def test_bench_beam_steps_one_sample(pd):
    w = W.beam(2.5)
    g = w.grid
    orow, ocol = core.neighbours(g)
    s0 = W.lognormal_like_field(g.n_nodes, 1, 41)
    u, v = W.random_state(g.n_nodes, 1, 42, u_scale=1.5e-7)
    i_idx = np.repeat(np.arange(g.n_nodes), np.diff(orow))
    d = W.pair_damage(i_idx, ocol, 43, 1, frac=0.05)
    row, col = pd.build_neighbours(g)
    st = pd.State(g, row, col, w.mat, w.bc, batch=1)  # the benchmark's one-sample schedule
    st.reset(_dev(s0, torch.float32))
    st.load(_dev(u), _dev(v), _dev(d), step=100)
    R = st.step(20).cpu().numpy()[0]
    ug, _, dg = [x.cpu().numpy()[0] for x in st.store()]
    r = core.Model(w, orow, ocol, s0=s0[0].astype(np.float64), dt=st.dt).run(
        20, state=(u[0], v[0], d[0]), step0=100)
    changed = int((r["d"] > d[0]).sum())
    print(f"bonds whose damage grew: {changed}; R err {np.abs(R - r['reaction']).max() / np.abs(r['reaction']).max():.2e}")
    assert changed > 1000
    assert np.abs(R - r["reaction"]).max() <= 1e-5 * np.abs(r["reaction"]).max()
    assert np.abs(ug - r["u"]).max() <= 1e-5 * np.abs(r["u"]).max()
    assert np.abs(dg - r["d"]).max() <= 1e-5
    st.close()


def test_bench_beam_batched_force(pd):
    w = W.beam(2.5)
    g = w.grid
    B = 32
    orow, ocol = core.neighbours(g)
    s0 = W.lognormal_like_field(g.n_nodes, B, 51)
    u, _ = W.random_state(g.n_nodes, B, 52, u_scale=1.5e-7)
    row, col = pd.build_neighbours(g)
    st = pd.State(g, row, col, w.mat, w.bc, batch=B)  # the batched schedule
    st.reset(_dev(s0, torch.float32))
    st.load(_dev(u), _dev(np.zeros_like(u)), None, step=0)
    F = st.force().cpu().numpy()
    for b in (0, B - 1):
        m = core.Model(w, orow, ocol, s0=s0[b].astype(np.float64), dt=st.dt)
        Fo, do, _ = m.force(u[b], np.zeros(m.nb))
        assert (do > 0).sum() > 1000
        assert np.abs(F[b] - Fo).max() <= 1e-5 * np.abs(Fo).max()
    st.close()


def test_sweep_beam_force(pd):
    """D = 200 mm: 448,000 nodes, 50,527,480 bonds."""
    w = W.sweep(200.0)
    g = w.grid
    orow, ocol = core.neighbours(g)
    assert int(orow[-1]) == 50_527_480
    s0 = W.lognormal_like_field(g.n_nodes, 1, 61)
    u, _ = W.random_state(g.n_nodes, 1, 62, u_scale=1.5e-7)
    row, col = pd.build_neighbours(g)
    st = pd.State(g, row, col, w.mat, w.bc, batch=1, schedule=(4, 4, 1))  # the sweep's brick and warp split
    st.reset(_dev(s0, torch.float32))
    st.load(_dev(u), _dev(np.zeros_like(u)), None, step=0)
    F = st.force().cpu().numpy()[0]
    m = core.Model(w, orow, ocol, s0=s0[0].astype(np.float64), dt=st.dt)
    Fo, do, _ = m.force(u[0], np.zeros(m.nb))
    print(f"softened bonds {(do > 0).sum()}, force err {np.abs(F - Fo).max() / np.abs(Fo).max():.2e}")
    assert (do > 0).sum() > 10000
    assert np.abs(F - Fo).max() <= 1e-5 * np.abs(Fo).max()
    st.close()
