"""Launch schedules and the autotuner: every schedule regroups the same
arithmetic, so trajectories agree to rounding; the autotuner returns one of
its candidates, caches it, and MLMC with tuned schedules matches the built-in
choice to rounding."""
import numpy as np
import pytest
import torch

import pd_workloads as W
from oracle import field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd(built_lib):
    import paper_2212_04415_gb300 as pd
    return pd


SCHEDULES = [(2, 2, 1), (2, 2, 4), (4, 2, 1), (4, 2, 2), (4, 4, 1), (8, 2, 1), (2, 8, 2), (6, 2, 1),
             (4, 2, 1, 1), (4, 4, 2, 2)]


def _run(pd, w, row, col, s0, sched, n=120):
    st = pd.State(w.grid, row, col, w.mat, w.bc, batch=s0.shape[0], schedule=sched)
    st.reset(s0)
    R = st.step(n)
    u = st.store()[0]
    st.close()
    return R, u


def test_every_schedule_gives_the_same_trajectory(pd):
    levels = W.small_beam_levels()
    w = levels[1]
    row, col = pd.build_neighbours(w.grid)
    Phi, lam = field.kl_separable(w.grid, w.field.length, w.field.n_modes)
    s0 = field.sample_field(w, Phi, lam, w.seed, 1, [0, 1, 2])
    s0 = torch.tensor(np.ascontiguousarray(s0, np.float32), device="cuda")
    R0, u0 = _run(pd, w, row, col, s0, None)
    for sch in SCHEDULES:
        R, u = _run(pd, w, row, col, s0, sch)
        er = ((R - R0).abs().max() / R0.abs().max()).item()
        eu = ((u - u0).abs().max() / u0.abs().max()).item()
        print(f"schedule {sch}: reaction {er:.1e}, displacement {eu:.1e}")
        assert er <= 1e-6 and eu <= 1e-6


def test_bad_schedules_are_rejected(pd):
    w = W.small_beam_levels()[0]
    row, col = pd.build_neighbours(w.grid)
    for sch in [(0, 2, 1), (17, 1, 1), (2, 2, 3), (4, 2, 1, 3)]:
        with pytest.raises(pd.PdError):
            pd.State(w.grid, row, col, w.mat, w.bc, schedule=sch)


def test_autotune_picks_a_candidate_and_caches(pd):
    w = W.beam(5.0)
    row, col = pd.build_neighbours(w.grid)
    import time
    t0 = time.perf_counter()
    sch, us = pd.autotune(w.grid, row, col, w.mat, w.bc, batch=64, trial_steps=10)
    t1 = time.perf_counter()
    sch2, us2 = pd.autotune(w.grid, row, col, w.mat, w.bc, batch=64, trial_steps=10)
    t2 = time.perf_counter()
    print(f"tuned {sch} at {us:.1f} us/step in {t1 - t0:.2f} s; cached call {1e3 * (t2 - t1):.3f} ms")
    assert sch == sch2 and us == us2 and us > 0
    by, bz, q, ns = sch
    assert (by * bz) % 2 == 0 and by * bz <= 32 and q in (1, 2, 4) and ns in (1, 2)
    assert t2 - t1 < 0.05
    st = pd.State(w.grid, row, col, w.mat, w.bc, batch=64, schedule=sch)
    st.step(2)
    st.close()


def test_mlmc_with_tuned_schedules(pd):
    levels = W.small_beam_levels()
    a = dict(grids=[w.grid for w in levels], bcs=[w.bc for w in levels], max_steps=[w.n_steps for w in levels],
             n_samples=[4, 2], mat=levels[0].mat, field=levels[0].field, seed=levels[0].seed, batch=4)
    base = pd.mlmc_estimate(return_samples=True, **a)
    tuned = pd.mlmc_estimate(return_samples=True, tune_steps=5, **a)
    for key in ("q_fine", "q_coarse"):
        d = np.abs(tuned[key] - base[key]).max() / np.abs(base[key]).max()
        print(key, d)
        assert d <= 1e-5


def _fields(w, n, seed_level=1):
    Phi, lam = field.kl_separable(w.grid, w.field.length, w.field.n_modes)
    s0 = field.sample_field(w, Phi, lam, w.seed, seed_level, list(range(n)))
    return torch.tensor(np.ascontiguousarray(s0, np.float32), device="cuda")


def _full_run(pd, w, row, col, s0, sched, kappa=None, n=0):
    """n > 0: n steps with reactions; n == 0: run to the peak with the stop rule."""
    st = pd.State(w.grid, row, col, w.mat, w.bc, batch=s0.shape[0], schedule=sched)
    st.reset(s0, kappa)
    out = st.step(n) if n else st.run_to_peak(w.n_steps)
    u, v, d = st.store()
    st.close()
    return out, u, v, d


@pytest.mark.parametrize("law", [0, 1])
def test_paired_samples_match_single_samples_bit_for_bit(pd, law):
    """Two samples per block (paired FP32 instructions) give every sample the
    same bits as one sample per block: trajectories, damage, an odd batch (the
    last pair has one real member) and a stiffness field."""
    import dataclasses
    w = W.small_beam_levels()[1]
    w = dataclasses.replace(w, mat=dataclasses.replace(w.mat, law=law, s_ratio=10.0 if law == 0 else 25.0))
    row, col = pd.build_neighbours(w.grid)
    s0 = _fields(w, 3)
    kap = (1.0 + 0.1 * torch.rand(s0.shape, generator=torch.Generator().manual_seed(5))).to("cuda")
    for kappa in (None, kap):
        for q in (1, 2, 4):
            a = _full_run(pd, w, row, col, s0, (4, 2, q, 1), kappa, n=400)
            b = _full_run(pd, w, row, col, s0, (4, 2, q, 2), kappa, n=400)
            for x, y in zip(a, b):
                assert torch.equal(x, y), (law, kappa is not None, q)
            assert (a[3] > 0).any() or law == 1  # softening reached (bilinear)


def test_paired_run_to_peak_with_samples_finishing_apart(pd):
    """run_to_peak with pairs whose members stop at different steps: peaks,
    peak steps, step counts and final states equal the one-sample kernel's."""
    w = W.small_beam_levels()[1]
    row, col = pd.build_neighbours(w.grid)
    s0 = _fields(w, 5)
    s0[1] *= 0.8  # an earlier peak for one member of the first pair
    (pk1, ps1, nd1), u1, v1, d1 = _full_run(pd, w, row, col, s0, (4, 2, 1, 1))
    (pk2, ps2, nd2), u2, v2, d2 = _full_run(pd, w, row, col, s0, (4, 2, 1, 2))
    print("steps", nd1.tolist(), "peaks", pk1.tolist())
    assert len(set(nd1.tolist())) > 1
    assert torch.equal(pk1, pk2) and torch.equal(ps1, ps2) and torch.equal(nd1, nd2)
    assert torch.equal(u1, u2) and torch.equal(v1, v2) and torch.equal(d1, d2)


def test_paired_plane_samples_match_single_samples(pd):
    w = W.small_plane_levels()[1]
    row, col = pd.build_neighbours(w.grid)
    s0 = _fields(w, 4)
    a = _full_run(pd, w, row, col, s0, (4, 1, 1, 1), n=300)
    b = _full_run(pd, w, row, col, s0, (4, 1, 1, 2), n=300)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_deferred_reaction_matches_reduction_in_the_launch(pd):
    """Each step's reaction reduced in its own launch (reduce = 1) or by the
    next launch (reduce = 2): the same per-step reactions, peaks, peak steps,
    step counts and final states, bit for bit, including samples that stop at
    different steps and a call that ends mid-run."""
    w = W.small_beam_levels()[1]
    row, col = pd.build_neighbours(w.grid)
    s0 = _fields(w, 3)
    s0[1] *= 0.8
    for ns in (1, 2):
        a = _full_run(pd, w, row, col, s0, (4, 2, 2, ns, 1), n=300)
        b = _full_run(pd, w, row, col, s0, (4, 2, 2, ns, 2), n=300)
        for x, y in zip(a, b):
            assert torch.equal(x, y)
        (pk1, ps1, nd1), u1, v1, d1 = _full_run(pd, w, row, col, s0, (4, 2, 2, ns, 1))
        (pk2, ps2, nd2), u2, v2, d2 = _full_run(pd, w, row, col, s0, (4, 2, 2, ns, 2))
        assert len(set(nd1.tolist())) > 1
        assert torch.equal(pk1, pk2) and torch.equal(ps1, ps2) and torch.equal(nd1, nd2)
        assert torch.equal(u1, u2) and torch.equal(v1, v2) and torch.equal(d1, d2)
    # steps split over several calls (each call's last launch reduces its own
    # reaction) equal one call
    st = pd.State(w.grid, row, col, w.mat, w.bc, batch=3, schedule=(4, 2, 2, 1, 2))
    st.reset(s0)
    R = torch.cat([st.step(k) for k in (1, 7, 64, 28)], dim=1)
    st.close()
    R1, _, _, _ = _full_run(pd, w, row, col, s0, (4, 2, 2, 1, 2), n=100)
    assert torch.equal(R, R1)
