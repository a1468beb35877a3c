"""KL field sampling on the tensor cores (Section 3) against the oracle:
several 128-node tiles with a ragged tail, several sample tiles, mode counts
that are not a multiple of the 32-mode chunk, both marginals, and the
coarse member of a level pair."""
import dataclasses

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


CASES = [
    # (nx, ny, nz), K, B, marginal
    ((20, 10, 7), 40, 300, W.MARG_LOGNORMAL),   # 1,400 nodes = 10 tiles + 120; 2 sample tiles of 256
    ((13, 9, 5), 64, 3, W.MARG_WEIBULL),        # 585 nodes; one 32-column sample tile
    ((8, 8, 8), 16, 33, W.MARG_LOGNORMAL),      # one chunk, padded from 16 modes
    ((24, 12, 6), 100, 130, W.MARG_WEIBULL),    # 4 chunks (100 -> 128 modes), sample tiles of 256
    ((70, 20, 20), 64, 1, W.MARG_LOGNORMAL),    # the 28,000-node beam, one sample
]


@pytest.mark.parametrize("dims,K,B,marg", CASES)
def test_tensor_core_field_against_oracle(pd, dims, K, B, marg):
    g = W.Grid(*dims, 2.5e-3, 3.01)
    cfg = W.FieldCfg(W.COV_SQEXP, 7.5e-3, K, marg, 1e-4, 0.1, 3.0)
    fld = pd.Field(g, 1, cfg)
    ids = np.arange(B, dtype=np.int64) * 7 + 3
    xi = pd.draw_xi(11, 0, torch.tensor(ids, device="cuda"), K)
    s0 = fld.sample(0, xi).cpu().numpy()
    Phi, lam = field.kl_separable(g, cfg.length, K)
    gg = field.gaussian(Phi, lam, field.draw_xi(11, 0, ids.tolist(), K))
    so = field.lognormal(gg, cfg.mean, cfg.cov) if marg == W.MARG_LOGNORMAL else field.weibull(gg, cfg.mean, 3.0)
    err = np.abs(s0 - so) / np.abs(so).max()
    print(f"{dims} K={K} B={B}: max rel err {err.max():.2e}")
    assert np.isfinite(s0).all()
    assert err.max() <= 1e-5
    fld.close()


def test_coarse_member_is_the_coarse_level_field(pd):
    """pd_sample_field(level, coarse) gives the level-(l-1) field of the same xi, bit for bit."""
    w = W.small_beam_levels()[1]
    fld = pd.Field(w.grid, 2, w.field)
    xi = pd.draw_xi(w.seed, 1, torch.arange(5, dtype=torch.int64, device="cuda"), w.field.n_modes)
    f1, f0 = fld.sample(1, xi, coarse=True)
    assert torch.equal(f0, fld.sample(0, xi))
    assert torch.equal(f1, fld.sample(1, xi))
    fld.close()


def test_sample_is_independent_of_the_batch(pd):
    """A sample's field does not depend on which other samples share the launch."""
    g = W.Grid(20, 10, 7, 2.5e-3, 3.01)
    cfg = W.FieldCfg(W.COV_SQEXP, 7.5e-3, 40, W.MARG_LOGNORMAL, 1e-4, 0.1)
    fld = pd.Field(g, 1, cfg)
    ids = torch.arange(300, dtype=torch.int64, device="cuda")
    xi = pd.draw_xi(5, 0, ids, 40)
    full = fld.sample(0, xi)
    for lo, hi in ((0, 1), (17, 50), (256, 300)):
        assert torch.equal(fld.sample(0, xi[lo:hi].contiguous()), full[lo:hi])
    fld.close()


def test_full_size_field_on_sampled_nodes(pd):
    """The finest grid of the MLMC hierarchy (140 x 40 x 40 = 224,000 nodes, 64
    modes) with 256 samples in one launch, checked against the oracle on 2,000
    sampled nodes (every sample)."""
    w = W.beam(1.25)
    g, cfg = w.grid, w.field
    B = 256
    fld = pd.Field(g, 1, cfg)
    ids = list(range(1000, 1000 + B))
    xi = pd.draw_xi(w.seed, 2, torch.tensor(ids, dtype=torch.int64, device="cuda"), cfg.n_modes)
    s0 = fld.sample(0, xi)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    nodes = np.sort(rng.choice(g.n_nodes, 2000, replace=False))
    got = s0[:, torch.tensor(nodes, device="cuda")].cpu().numpy()
    Phi, lam = field.kl_separable(g, cfg.length, cfg.n_modes)
    gg = field.gaussian(Phi[nodes], lam, field.draw_xi(w.seed, 2, ids, cfg.n_modes))
    so = field.lognormal(gg, cfg.mean, cfg.cov)
    err = np.abs(got - so) / np.abs(so).max()
    print(f"224k nodes x 256 samples: max rel err {err.max():.2e} on 2,000 nodes")
    assert err.max() <= 1e-5
    fld.close()
