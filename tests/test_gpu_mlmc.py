"""MLMC estimator on the GPU against the oracle (Section 4): per-sample peak
loads of the coupled fine / coarse pairs, the FP64 level sums, the estimator,
and a two-shard run merged back to the single-run totals bit for bit."""
import numpy as np
import pytest

import pd_workloads as W
from oracle import core, field
from oracle import mlmc as omlmc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd(built_lib):
    import paper_2212_04415_gb300 as pd
    return pd


def _args(levels, n_samples=None):
    return dict(grids=[w.grid for w in levels], bcs=[w.bc for w in levels],
                max_steps=[w.n_steps for w in levels],
                n_samples=n_samples if n_samples is not None else [w.batch for w in levels],
                mat=levels[0].mat, field=levels[0].field, seed=levels[0].seed)


def _oracle_pairs(levels, l, ids):
    """Q of the fine member (level l) and coarse member (level l-1) of each pair:
    one Gaussian field on the finest grid from xi(seed, l, id), restricted down."""
    f = levels[0].field
    L = len(levels)
    Phi, lam = field.kl_separable(levels[-1].grid, f.length, f.n_modes)
    g = field.gaussian(Phi, lam, field.draw_xi(levels[0].seed, l, ids, f.n_modes))
    for k in range(L - 1, l, -1):
        g = field.restrict(g, levels[k].grid)
    qf = core.run_batch(core.Model(levels[l]), field.lognormal(g, f.mean, f.cov), levels[l].n_steps)["peak"]
    if l == 0:
        return qf, np.zeros_like(qf)
    gc = field.restrict(g, levels[l].grid)
    qc = core.run_batch(core.Model(levels[l - 1]), field.lognormal(gc, f.mean, f.cov),
                        levels[l - 1].n_steps)["peak"]
    return qf, qc


def test_mlmc_estimate_against_oracle(pd):
    levels = W.small_beam_levels()
    a = _args(levels)
    res = pd.mlmc_estimate(batch=4, return_samples=True, **a)  # level 0: batches of 4 and 2
    off = 0
    Yh, V = [], []
    for l, n in enumerate(a["n_samples"]):
        qf, qc = res["q_fine"][off:off + n], res["q_coarse"][off:off + n]
        off += n
        of, oc = _oracle_pairs(levels, l, list(range(n)))
        scale = np.abs(of).max()
        print(f"level {l}: Qf {qf} vs {of}; Qc {qc} vs {oc}")
        assert np.all(np.abs(qf - of) <= 1e-3 * np.abs(of))
        assert np.all(np.abs(qc - oc) <= 1e-3 * np.maximum(np.abs(oc), 1e-30))
        lv = res["levels"][l]
        y = qf - qc
        assert lv["n"] == n
        # the GPU's FP64 level sums of its own samples (summation order differs: 1e-12)
        assert lv["sum_y"] == pytest.approx(y.sum(), rel=1e-12, abs=1e-12 * scale * n)
        assert lv["sum_y2"] == pytest.approx((y * y).sum(), rel=1e-12)
        mean, var_b, _ = omlmc.level_stats(of - oc)
        # the level's own mean (a correction level's |Y_hat| is well below the
        # peak load), floored at 1 % of the peak scale for a vanishing correction
        print(f"level {l}: Y_hat {lv['mean']:.9g} vs {mean:.9g}")
        assert abs(lv["mean"] - mean) <= 1e-3 * max(abs(mean), 1e-2 * scale)
        Yh.append(mean)
        V.append(var_b)
        assert lv["steps"] > 0 and lv["bond_updates"] > 0
    q, _ = omlmc.mlmc_estimate(Yh, V, a["n_samples"])
    assert abs(res["q_ml"] - q) <= 1e-3 * abs(q)
    # the estimator is the sum of the level means; its variance sum_l V_l / N_l
    assert res["q_ml"] == pytest.approx(sum(lv["mean"] for lv in res["levels"]), rel=1e-14)
    assert res["var_ml"] == pytest.approx(sum(lv["var"] / lv["n"] for lv in res["levels"]), rel=1e-14)


def test_mlmc_two_shards_merge_to_the_single_run(pd):
    from paper_2212_04415_gb300 import shard
    levels = W.small_beam_levels()
    a = _args(levels, n_samples=[5, 3])
    batch = 2
    one = pd.mlmc_estimate(batch=batch, return_samples=True, **a)
    parts = []
    for r in range(2):
        first, count = shard.split(a["n_samples"], batch, 2, r)
        b = dict(a, n_samples=count)
        parts.append((first, count, pd.mlmc_estimate(batch=batch, first_sample=first, return_samples=True, **b)))
    merged = shard.merge([p[2]["batch_sums"] for p in parts])
    for l in range(2):
        for key in ("n", "sum_y", "sum_y2", "mean", "var"):
            assert merged["levels"][l][key] == one["levels"][l][key]
    assert merged["q_ml"] == one["q_ml"] and merged["var_ml"] == one["var_ml"]
    # per-sample results do not depend on which process ran them
    off_one = 0
    offs = [0, 0]
    for l, n in enumerate(a["n_samples"]):
        got = []
        for r, (first, count, res) in enumerate(parts):
            got.append(res["q_fine"][offs[r]:offs[r] + count[l]])
            offs[r] += count[l]
        assert np.array_equal(np.concatenate(got), one["q_fine"][off_one:off_one + n])
        off_one += n


def test_mlmc_rejects_unnested_grids(pd):
    levels = W.small_beam_levels()
    a = _args(levels)
    a["grids"] = [levels[0].grid, levels[0].grid]
    with pytest.raises(pd.PdError, match="refinement"):
        pd.mlmc_estimate(batch=4, **a)


def test_states_of_two_meshes_coexist(pd):
    """A state created after another (smaller bricks) must not break the first
    one's launches, captured or not (the fine and coarse members of a pair)."""
    import torch
    fine, coarse = W.beam(2.5), W.beam(5.0)
    rf, cf = pd.build_neighbours(fine.grid)
    rc, cc = pd.build_neighbours(coarse.grid)
    big = pd.State(fine.grid, rf, cf, fine.mat, fine.bc, batch=16)    # 8x4x4 bricks
    small = pd.State(coarse.grid, rc, cc, coarse.mat, coarse.bc, batch=1)
    R = big.step(3)
    pk, _, nd = big.run_to_peak(70)
    small.step(3)
    torch.cuda.synchronize()
    assert torch.isfinite(R).all() and (nd == 70).all()
    big.close()
    small.close()


def test_adaptive_mlmc_against_oracle(pd):
    """Algorithm MLMC on the two-level small beam with a fixed cost model: the
    GPU run and the oracle's adaptive run (on the oracle's own coupled-pair
    physics, same sample ids) take the same decisions (last level, samples per
    level within one), and every sample's peak loads agree within 1e-3."""
    levels = W.small_beam_levels()
    a = _args(levels)
    del a["n_samples"]
    cost = [1.0, 8.0]
    settings = dict(eps_s=1.5, eps_b=10.0, m_dof=8.0, alpha=1.0, n_star=8)
    res = pd.mlmc_adaptive(batch=16, cost_model=cost, cap=4096, **settings, **a)
    print("GPU adaptive: L", res["L"], "N", [lv["n"] for lv in res["levels"]], "bias", res["bias"],
          "Q", res["q_ml"])

    taken = [0, 0]

    def sampler(l, n):
        ids = list(range(taken[l], taken[l] + n))
        taken[l] += n
        qf, qc = _oracle_pairs(levels, l, ids)
        return qf - qc, cost[l]
    ora = omlmc.adaptive(sampler, settings["eps_s"], settings["eps_b"], settings["m_dof"], settings["alpha"],
                         n_star=settings["n_star"], L_max=len(levels) - 1)
    print("oracle adaptive: L", ora["L"], "N", ora["N"], "bias", ora["bias"], "Q", ora["Q"])
    assert res["L"] == ora["L"] == 1  # the bias test added the second level and then passed
    for l in range(res["L"] + 1):
        assert abs(res["levels"][l]["n"] - ora["N"][l]) <= 1
        assert res["levels"][l]["n"] >= settings["n_star"]
        # every sample of the GPU run against the oracle's run of the same id
        qf, qc = res["samples"][l]
        of, oc = _oracle_pairs(levels, l, list(range(len(qf))))
        assert np.all(np.abs(qf - of) <= 1e-3 * np.abs(of))
        if l > 0:
            assert np.all(np.abs(qc - oc) <= 1e-3 * np.abs(oc))
    assert abs(res["q_ml"] - ora["Q"]) <= 2e-3 * abs(ora["Q"])
    # the same samples through the fixed-allocation estimator give the same level sums
    fixed = pd.mlmc_estimate(n_samples=[lv["n"] for lv in res["levels"]], batch=16, **a)
    for l in range(2):
        assert fixed["levels"][l]["sum_y"] == pytest.approx(res["levels"][l]["sum_y"], rel=1e-12)


def test_multi_state_run_equals_separate_runs(pd):
    """The fine and coarse members run together in one chunk graph give the
    same peaks, steps and final states as two separate runs, bit for bit."""
    import torch
    levels = W.small_beam_levels()
    fw, cw = levels[1], levels[0]
    rf, cf = pd.build_neighbours(fw.grid)
    rc, cc = pd.build_neighbours(cw.grid)
    fld = pd.Field(fw.grid, 2, fw.field)
    xi = pd.draw_xi(fw.seed, 1, torch.arange(3, dtype=torch.int64, device="cuda"), fw.field.n_modes)
    ff, fc = fld.sample(1, xi, coarse=True)
    sf = pd.State(fw.grid, rf, cf, fw.mat, fw.bc, batch=3)
    sc = pd.State(cw.grid, rc, cc, cw.mat, cw.bc, batch=3)
    sf.reset(ff)
    sc.reset(fc)
    sep = [sf.run_to_peak(fw.n_steps), sc.run_to_peak(cw.n_steps)]
    u_sep = [sf.store()[0], sc.store()[0]]
    sf.reset(ff)
    sc.reset(fc)
    multi = pd.run_to_peak_multi([sf, sc], [fw.n_steps, cw.n_steps])
    u_multi = [sf.store()[0], sc.store()[0]]
    for a, b in zip(sep, multi):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    for a, b in zip(u_sep, u_multi):
        assert torch.equal(a, b)
    sf.close()
    sc.close()
    fld.close()


@pytest.mark.parametrize("level", [1, 2])
def test_paired_launch_of_a_level_equals_separate_runs(pd, level):
    """The benchmark hierarchy's coupled pairs (level 1: 28,000 + 3,500 nodes;
    level 2: 224,000 + 28,000 nodes), two samples, both members in the same
    launch shape: one launch per step covering both meshes gives the peaks,
    steps and final states of two separate runs, bit for bit."""
    import time

    import torch
    levels = W.beam_levels()
    fw, cw = levels[level], levels[level - 1]
    rf, cf = pd.build_neighbours(fw.grid)
    rc, cc = pd.build_neighbours(cw.grid)
    fld = pd.Field(fw.grid, 2, fw.field)
    xi = pd.draw_xi(fw.seed, 1, torch.arange(2, dtype=torch.int64, device="cuda"), fw.field.n_modes)
    ff, fc = fld.sample(1, xi, coarse=True)
    shape = (4, 4, 1, 1, 0)
    sf = pd.State(fw.grid, rf, cf, fw.mat, fw.bc, batch=2, schedule=shape)
    sc = pd.State(cw.grid, rc, cc, cw.mat, cw.bc, batch=2, schedule=shape)
    sf.reset(ff)
    sc.reset(fc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sep = [sf.run_to_peak(fw.n_steps), sc.run_to_peak(cw.n_steps)]
    torch.cuda.synchronize()
    t_sep = time.perf_counter() - t0
    u_sep = [sf.store()[0], sc.store()[0]]
    sf.reset(ff)
    sc.reset(fc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    multi = pd.run_to_peak_multi([sf, sc], [fw.n_steps, cw.n_steps])
    torch.cuda.synchronize()
    t_multi = time.perf_counter() - t0
    u_multi = [sf.store()[0], sc.store()[0]]
    print(f"level {level}: separate {t_sep:.3f} s, one launch per step {t_multi:.3f} s "
          f"(peaks {multi[0][0].tolist()}, {multi[1][0].tolist()})")
    for a, b in zip(sep, multi):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    for a, b in zip(u_sep, u_multi):
        assert torch.equal(a, b)
    sf.close()
    sc.close()
    fld.close()


def test_plane_mlmc_against_oracle(pd):
    """A two-level plane-stress hierarchy (one-layer grids, the field restricted
    over 2 x 2 in-plane children): per-sample pairs and the estimator."""
    levels = W.small_plane_levels()
    a = _args(levels)
    res = pd.mlmc_estimate(batch=4, return_samples=True, **a)
    off = 0
    Yh, V = [], []
    for l, n in enumerate(a["n_samples"]):
        qf, qc = res["q_fine"][off:off + n], res["q_coarse"][off:off + n]
        off += n
        of, oc = _oracle_pairs(levels, l, list(range(n)))
        print(f"plane level {l}: Qf {qf} vs {of}; Qc {qc} vs {oc}")
        assert np.all(np.abs(qf - of) <= 1e-3 * np.abs(of))
        assert np.all(np.abs(qc - oc) <= 1e-3 * np.maximum(np.abs(oc), 1e-30))
        mean, var_b, _ = omlmc.level_stats(of - oc)
        print(f"plane level {l}: Y_hat {res['levels'][l]['mean']:.9g} vs {mean:.9g}")
        assert abs(res["levels"][l]["mean"] - mean) <= 1e-3 * max(abs(mean), 1e-2 * np.abs(of).max())
        Yh.append(mean)
        V.append(var_b)
    q, _ = omlmc.mlmc_estimate(Yh, V, a["n_samples"])
    assert abs(res["q_ml"] - q) <= 1e-3 * abs(q)
