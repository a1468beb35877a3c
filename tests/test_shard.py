"""Host logic of the sharded MLMC estimator: whole-batch splits and a merge
that reproduces the single-process level sums bit for bit (CPU; the
two-process case runs on gloo)."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import mlmc as omlmc
from paper_2212_04415_gb300 import shard


@pytest.fixture(autouse=True, scope="module")
def _library(built_lib):
    """shard.merge calls the library's host-only mlmc_merge (no GPU involved)."""
    return built_lib


def _batch_sums(Y, first, count, batch):
    """(n, sum Y, sum Y^2) per batch of ``batch`` consecutive samples, added in sample order."""
    rows = []
    for s in range(first, first + count, batch):
        e = min(first + count, s + batch)
        a = b = 0.0
        for y in Y[s:e]:
            a += float(y)
            b += float(y) * float(y)
        rows.append((e - s, a, b))
    return np.array(rows, np.float64).reshape(-1, 3)


def _level_Y(n_samples, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(n) * 10.0 ** (-l) + 3.0 for l, n in enumerate(n_samples)]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
@pytest.mark.parametrize("batch", [1, 2, 5, 64])
def test_split_deals_whole_batches(world, batch):
    n_samples = [0, 1, 7, 64, 129, 1000]
    parts = [shard.split(n_samples, batch, world, r) for r in range(world)]
    for l, n in enumerate(n_samples):
        pos = 0
        for first, count in parts:
            assert first[l] == pos  # contiguous, in rank order
            assert first[l] % batch == 0 or count[l] == 0
            end = first[l] + count[l]
            assert count[l] % batch == 0 or end == n  # only the level's last batch may be short
            pos = end
        assert pos == n
        nb = -(-n // batch)
        sizes = [-(-c[l] // batch) for _, c in parts]
        assert max(sizes) - min(sizes) <= 1 and sum(sizes) == nb


def test_split_rejects_bad_arguments():
    with pytest.raises(ValueError):
        shard.split([4], 2, 2, 2)
    with pytest.raises(ValueError):
        shard.split([4], 0, 1, 0)
    with pytest.raises(ValueError):
        shard.split([-1], 2, 1, 0)


@pytest.mark.parametrize("world", [2, 3, 5])
def test_merge_is_bit_identical_to_one_process(world):
    n_samples, batch = [37, 12, 5], 4
    Y = _level_Y(n_samples, 11)
    one = shard.merge([[_batch_sums(Y[l], 0, n, batch) for l, n in enumerate(n_samples)]])
    by_rank = []
    for r in range(world):
        first, count = shard.split(n_samples, batch, world, r)
        by_rank.append([_batch_sums(Y[l], first[l], count[l], batch) for l in range(len(n_samples))])
    many = shard.merge(by_rank)
    for a, b in zip(one["levels"], many["levels"]):
        assert a == b
    assert one["q_ml"] == many["q_ml"] and one["var_ml"] == many["var_ml"]


def test_merge_follows_the_estimator():
    """Merged totals against the oracle's sample variance and estimator (Eqs.
    sample_variance, MLMC_estimator, MLMC_error)."""
    n_samples, batch = [50, 20, 8], 3
    Y = _level_Y(n_samples, 5)
    m = shard.merge([[_batch_sums(Y[l], 0, n, batch) for l, n in enumerate(n_samples)]])
    Yh, V = [], []
    for l, lv in enumerate(m["levels"]):
        mean, var_b, var_u = omlmc.level_stats(Y[l])
        assert lv["n"] == n_samples[l]
        assert lv["mean"] == pytest.approx(mean, rel=1e-13)
        assert lv["var"] == pytest.approx(var_b, rel=1e-9)
        assert lv["var_unbiased"] == pytest.approx(var_u, rel=1e-9)
        Yh.append(mean)
        V.append(var_b)
    q, v = omlmc.mlmc_estimate(Yh, V, n_samples)
    assert m["q_ml"] == pytest.approx(q, rel=1e-13)
    assert m["var_ml"] == pytest.approx(v, rel=1e-9)


def test_merge_with_an_empty_shard():
    n_samples, batch = [3, 1], 4
    Y = _level_Y(n_samples, 2)
    parts = []
    for r in range(3):
        first, count = shard.split(n_samples, batch, 3, r)
        parts.append([_batch_sums(Y[l], first[l], count[l], batch) for l in range(2)])
    assert parts[1][0].shape == (0, 3) and parts[2][1].shape == (0, 3)
    one = shard.merge([[_batch_sums(Y[l], 0, n, batch) for l, n in enumerate(n_samples)]])
    assert shard.merge(parts)["levels"] == one["levels"]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n_samples, batch, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        Y = _level_Y(n_samples, 23)
        first, count = shard.split(n_samples, batch, world, rank)
        local = [_batch_sums(Y[l], first[l], count[l], batch) for l in range(len(n_samples))]
        merged = shard.merge(shard.allgather(local))
        np.save(f"{out_path}.{rank}.npy",
                np.array([[lv["n"], lv["sum_y"], lv["sum_y2"]] for lv in merged["levels"]] +
                         [[0, merged["q_ml"], merged["var_ml"]]], np.float64))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_merge(tmp_path):
    n_samples, batch, world = [21, 9, 2], 4, 2
    out = str(tmp_path / "merged")
    mp.start_processes(_rank_main, args=(world, _free_port(), n_samples, batch, out), nprocs=world,
                       join=True, start_method="spawn")
    Y = _level_Y(n_samples, 23)
    one = shard.merge([[_batch_sums(Y[l], 0, n, batch) for l, n in enumerate(n_samples)]])
    want = np.array([[lv["n"], lv["sum_y"], lv["sum_y2"]] for lv in one["levels"]] +
                    [[0, one["q_ml"], one["var_ml"]]], np.float64)
    for r in range(world):
        got = np.load(f"{out}.{r}.npy")
        assert np.array_equal(got, want)  # every rank holds the single-process totals, bit for bit
