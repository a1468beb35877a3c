"""Degenerate and edge inputs on the GPU: a call of zero steps, a run to the
peak with no steps allowed, a grid thinner than the horizon and than one
brick (every node on the boundary), and MLMC levels of a single sample."""
import numpy as np
import pytest
import torch

import pd_workloads as W
from oracle import core
from oracle import mlmc as omlmc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd(built_lib):
    import paper_2212_04415_gb300 as pd
    return pd


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def test_zero_steps_change_nothing(pd):
    w = W.tiny_beam(13, 7, 5)
    g = w.grid
    row, col = pd.build_neighbours(g)
    st = pd.State(g, row, col, w.mat, w.bc, batch=2)
    st.reset(torch.full((2, g.n_nodes), 1e-4, device="cuda"))
    st.step(10)
    before = [x.clone() for x in st.store()]
    R = st.step(0)
    assert tuple(R.shape) == (2, 0)
    pk, ps, nd = st.run_to_peak(0)  # no step allowed: the state stays at step 10
    assert nd.tolist() == [10, 10]
    for x, y in zip(before, st.store()):
        assert torch.equal(x, y)
    st.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_grid_thinner_than_the_horizon_and_a_brick(pd, prec):
    """8 x 2 x 2 nodes: every node is on the boundary and the staged box is
    mostly halo; steps from a random state against the oracle."""
    w = W.tiny_beam(8, 2, 2, notch=False, n_steps=60)
    g = w.grid
    orow, ocol = core.neighbours(g)
    n = g.n_nodes
    s0 = W.lognormal_like_field(n, 2, 11)
    u, v = W.random_state(n, 2, 12, u_scale=2e-7)
    d = W.pair_damage(np.repeat(np.arange(n), np.diff(orow)), ocol, 13, 2)
    row, col = pd.build_neighbours(g)
    assert np.array_equal(row.cpu().numpy(), orow) and np.array_equal(col.cpu().numpy(), ocol)
    st = pd.State(g, row, col, w.mat, w.bc, batch=2, precision=prec)
    st.reset(_dev(s0))
    st.load(_dev(u), _dev(v), _dev(d), step=3)
    R = st.step(20).cpu().numpy()
    ug, _, dg = [x.cpu().numpy() for x in st.store()]
    tol = 1e-10 if prec == 0 else 1e-5
    for b in range(2):
        m = core.Model(w, orow, ocol, s0=s0[b].astype(np.float64))
        r = m.run(20, state=(u[b], v[b], d[b]), step0=3)
        assert np.abs(R[b] - r["reaction"]).max() <= tol * np.abs(r["reaction"]).max()
        assert np.abs(ug[b] - r["u"]).max() <= tol * np.abs(r["u"]).max()
        assert np.abs(dg[b] - r["d"]).max() <= tol
    st.close()


def test_mlmc_levels_of_one_sample(pd):
    levels = W.small_beam_levels()
    res = pd.mlmc_estimate(grids=[w.grid for w in levels], bcs=[w.bc for w in levels],
                           max_steps=[w.n_steps for w in levels], n_samples=[1, 1], mat=levels[0].mat,
                           field=levels[0].field, seed=levels[0].seed, batch=1, return_samples=True)
    for lv in res["levels"]:  # one sample: the biased variance is zero up to rounding
        assert lv["n"] == 1 and abs(lv["var"]) <= 1e-12 * lv["mean"] ** 2
    assert abs(res["var_ml"]) <= 1e-12 * sum(lv["mean"] ** 2 for lv in res["levels"])
    assert res["q_ml"] == pytest.approx(sum(lv["mean"] for lv in res["levels"]), rel=1e-14)
    y = res["q_fine"] - res["q_coarse"]
    assert res["levels"][1]["mean"] == pytest.approx(y[1], rel=1e-14)
    mean, var_b, _ = omlmc.level_stats(np.array([y[1]]))
    assert var_b == 0.0 and mean == pytest.approx(y[1], rel=1e-14)


def test_run_to_peak_after_an_odd_number_of_steps(pd):
    """A run to the peak that starts after three plain steps (odd step
    parity, so the captured chunks start from the other record buffer) gives
    the same peak, peak step, step count and final state as the
    uninterrupted run; so does a second state loaded at an odd step."""
    w = W.tiny_beam(16, 6, 4, n_steps=400)
    g = w.grid
    row, col = pd.build_neighbours(g)
    s0 = _dev(W.lognormal_like_field(g.n_nodes, 2, 17))

    def run(pre):
        st = pd.State(g, row, col, w.mat, w.bc, batch=2)
        st.reset(s0)
        if pre:
            st.step(pre)
        out = [x.clone() for x in st.run_to_peak(w.n_steps)]
        state = st.store()
        st.close()
        return out, state

    (pk0, ps0, nd0), (u0, v0, d0) = run(0)
    (pk3, ps3, nd3), (u3, v3, d3) = run(3)
    assert torch.equal(pk0, pk3) and torch.equal(ps0, ps3) and torch.equal(nd0, nd3)
    assert torch.equal(u0, u3) and torch.equal(v0, v3) and torch.equal(d0, d3)
    assert int(nd0.max()) > 64  # several captured chunks

    # a state loaded at step 7 from the 7-step state of the same run continues it bit for bit
    st = pd.State(g, row, col, w.mat, w.bc, batch=2)
    st.reset(s0)
    st.step(7)
    u7, v7, d7 = st.store()
    st.close()
    st2 = pd.State(g, row, col, w.mat, w.bc, batch=2)
    st2.reset(s0)
    st2.load(u7, v7, d7, step=7)
    R_a = st2.step(40)
    ua = st2.store()[0]
    st2.close()
    st = pd.State(g, row, col, w.mat, w.bc, batch=2)
    st.reset(s0)
    st.step(7)
    R_b = st.step(40)
    ub = st.store()[0]
    st.close()
    assert torch.equal(R_a, R_b) and torch.equal(ua, ub)
