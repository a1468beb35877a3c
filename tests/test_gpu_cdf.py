"""Multilevel inverse CDF and CDF (Section 7) on the GPU against the oracle,
bit for bit: exact rank ordering with ties, the ceil(N u) order statistic at
and between the 1/N boundaries, and the level sum taken in level order."""
import numpy as np
import pytest
import torch

from oracle import mlmc as omlmc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd(built_lib):
    import paper_2212_04415_gb300 as pd
    return pd


def _levels(seed, sizes=(1000, 50, 7)):
    rng = np.random.default_rng(seed)
    q0 = np.round(rng.normal(2800.0, 150.0, sizes[0]), 1)  # rounded: ties
    out = [q0]
    for l, n in enumerate(sizes[1:], 1):
        c = np.round(rng.normal(2800.0, 150.0, n), 1)
        out.append((c + rng.normal(-500.0 / l, 40.0 / l, n), c))
    return out


def _dev(levels):
    return [torch.tensor(levels[0], device="cuda")] + [
        (torch.tensor(f, device="cuda"), torch.tensor(c, device="cuda")) for f, c in levels[1:]]


@pytest.mark.parametrize("sizes", [(1000,), (1000, 50), (1000, 50, 7), (3, 2, 1)])
def test_inverse_cdf_bit_exact(pd, sizes):
    lv = _levels(1, sizes)
    N = np.array(sizes, np.float64)
    # u on a grid, at every exact k / N_0 boundary of the first 40, and at the ends
    u = np.concatenate([np.linspace(0.0, 1.0, 257), np.arange(1, 41) / N[0], [1e-12, 1.0 - 1e-12]])
    got = pd.ml_inverse_cdf(_dev(lv), torch.tensor(u, device="cuda")).cpu().numpy()
    want = np.array([omlmc.ml_inverse_cdf(lv, x) for x in u])
    assert np.array_equal(got, want)


def test_cdf_bit_exact(pd):
    lv = _levels(3)
    x = np.linspace(2000.0, 2800.0, 41)
    got = pd.ml_cdf(_dev(lv), torch.tensor(x, device="cuda"), n_u=1000).cpu().numpy()
    want = omlmc.ml_cdf(lv, x, n_u=1000)
    assert np.array_equal(got, want)
    assert np.all(np.diff(got) >= 0) and got[0] >= 0 and got[-1] <= 1


def test_rank_sort_of_a_large_level(pd):
    """The finest MLMC level counts of the tolerance run (tens of thousands)."""
    rng = np.random.default_rng(5)
    q0 = np.round(rng.normal(0.0, 1.0, 23_322), 3)
    u = torch.tensor(np.linspace(0.0, 1.0, 1001), device="cuda")
    got = pd.ml_inverse_cdf([torch.tensor(q0, device="cuda")], u).cpu().numpy()
    s = np.sort(q0)
    idx = np.clip(np.ceil(q0.size * np.linspace(0.0, 1.0, 1001)).astype(np.int64), 1, q0.size) - 1
    assert np.array_equal(got, s[idx])
