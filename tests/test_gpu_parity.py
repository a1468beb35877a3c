"""GPU-vs-oracle parity of the hot path, through the C ABI.

Tolerances (stated per quantity; derivations in the design notes):
* neighbour lists, boundary sets, the KL coefficient stream: bit-exact / 1e-14;
* FP64 path: forces and displacements within 1e-10 relative (rounding order only);
* mixed path (FP32 bond arithmetic, compensated / FP64 sums): forces within
  1e-5 of max |F|, displacements within 1e-5 relative (the pre-damage target),
  damage within 1e-5 absolute, reaction within 1e-5 relative;
* peak load within 1e-3 relative.
"""
import dataclasses

import numpy as np
import pytest
import torch

import pd_workloads as W
from oracle import core, field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd(built_lib):
    assert torch.cuda.is_available()
    return built_lib


def _dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


@pytest.mark.parametrize("g", [
    W.tiny_beam().grid,
    W.Grid(7, 5, 3, 2.5e-3, 3.01, 1, 7, 3),
    W.Grid(33, 3, 2, 1e-3, np.pi),
    W.Grid(1, 1, 1, 1e-3, 3.01),
    W.bar().grid,
    W.beam(5.0).grid,
    W.beam(2.5).grid,
])
def test_neighbours_bit_exact(pd, g):
    row, col = pd.build_neighbours(g)
    orow, ocol = core.neighbours(g, brute=g.n_nodes <= 4000)
    assert np.array_equal(row.cpu().numpy(), orow)
    assert np.array_equal(col.cpu().numpy(), ocol)


def test_neighbours_capacity_error(pd):
    import ctypes
    g = W.tiny_beam().grid
    G = pd.grid_struct(g)
    row = torch.empty(g.n_nodes + 1, dtype=torch.int32, device="cuda")
    col = torch.full((10,), -7, dtype=torch.int32, device="cuda")
    nb = ctypes.c_int64(0)
    rc = pd.lib().pd_build_neighbours(ctypes.byref(G), pd._ptr(row), pd._ptr(col), 10, ctypes.byref(nb), None)
    assert rc == pd.PD_ERR_CAP and nb.value == core.neighbours(g)[0][-1]
    assert (col.cpu() == -7).all()


@pytest.mark.parametrize("w", [W.tiny_beam(), W.bar(), W.beam(2.5)])
def test_bc_codes_bit_exact(pd, w):
    assert np.array_equal(pd.bc_codes(w.grid, w.bc).cpu().numpy(), core.bc_codes(w.grid, w.bc))


def _random_case(w, B, seed, u_scale=2e-7):
    g = w.grid
    orow, ocol = core.neighbours(g)
    n = g.n_nodes
    s0 = W.lognormal_like_field(n, B, seed)
    u, v = W.random_state(n, B, seed + 1, u_scale=u_scale)
    i_idx = np.repeat(np.arange(n), np.diff(orow))
    d = W.pair_damage(i_idx, ocol, seed + 2, B)
    return orow, ocol, s0, u, v, d


CASES = [(pd_prec, law) for pd_prec in (0, 1) for law in (W.LAW_BILINEAR, W.LAW_EXPLINEAR)]


@pytest.mark.parametrize("prec,law", CASES)
@pytest.mark.parametrize("shape", [(16, 6, 4), (13, 7, 5), (40, 10, 10)])
def test_force_and_damage_parity(pd, prec, law, shape):
    w = W.tiny_beam(*shape)
    mat = dataclasses.replace(w.mat, law=law, s_ratio=10.0 if law == 0 else 25.0)
    w = dataclasses.replace(w, mat=mat)
    orow, ocol, s0, u, v, d = _random_case(w, 2, 21)
    row, col = pd.build_neighbours(w.grid)
    st = pd.State(w.grid, row, col, w.mat, w.bc, batch=2, precision=prec)
    st.reset(_dev(s0))
    st.load(_dev(u), _dev(v), _dev(d), step=0)
    F = st.force().cpu().numpy()
    _, _, dg = st.store()
    dg = dg.cpu().numpy()
    ftol, dtol = (1e-10, 1e-10) if prec == 0 else (1e-5, 1e-5)
    for b in range(2):
        m = core.Model(w, orow, ocol, s0=s0[b].astype(np.float64))
        assert abs(m.dt - st.dt) <= 1e-13 * m.dt
        Fo, do, _ = m.force(u[b], d[b])
        assert np.abs(F[b] - Fo).max() <= ftol * np.abs(Fo).max()
        assert np.abs(dg[b] - do).max() <= dtol
        assert (do > d[b]).sum() > 10  # the case exercises the law
    st.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_broken_bond_collapsed_to_zero_length(pd, prec):
    """A broken bond (d = 1) squeezed to zero length carries no force on the
    GPU either: the forces and damage stay finite and match the oracle's
    (node j is placed on node i, as under a crushing load)."""
    w = W.tiny_beam(16, 6, 4)
    orow, ocol, s0, u, v, d = _random_case(w, 1, 41)
    g = w.grid
    i = 3 + g.nx * (2 + g.ny * 1)
    j = i + 1
    u[0][j] = u[0][i] - np.array([g.dx, 0.0, 0.0])
    for a, b in ((i, j), (j, i)):
        q = orow[a] + int(np.nonzero(ocol[orow[a]:orow[a + 1]] == b)[0][0])
        d[0][q] = 1.0
    row, col = pd.build_neighbours(g)
    st = pd.State(g, row, col, w.mat, w.bc, batch=1, precision=prec)
    st.reset(_dev(s0))
    st.load(_dev(u), _dev(v), _dev(d), step=0)
    F = st.force().cpu().numpy()[0]
    dg = st.store()[2].cpu().numpy()[0]
    st.close()
    m = core.Model(w, orow, ocol, s0=s0[0].astype(np.float64))
    Fo, do, _ = m.force(u[0], d[0])
    assert np.all(np.isfinite(F)) and np.all(np.isfinite(Fo))
    tol = 1e-10 if prec == 0 else 1e-5
    assert np.abs(F - Fo).max() <= tol * np.abs(Fo).max()
    assert np.abs(dg - do).max() <= tol


@pytest.mark.parametrize("prec", [0, 1])
def test_steps_from_random_state(pd, prec):
    w = W.tiny_beam(13, 7, 5)
    orow, ocol, s0, u, v, d = _random_case(w, 3, 33)
    row, col = pd.build_neighbours(w.grid)
    st = pd.State(w.grid, row, col, w.mat, w.bc, batch=3, precision=prec)
    st.reset(_dev(s0))
    st.load(_dev(u), _dev(v), _dev(d), step=5)
    R = st.step(25).cpu().numpy()
    ug, vg, dg = [x.cpu().numpy() for x in st.store()]
    tol = 1e-10 if prec == 0 else 1e-5
    for b in range(3):
        m = core.Model(w, orow, ocol, s0=s0[b].astype(np.float64))
        r = m.run(25, state=(u[b], v[b], d[b]), step0=5)
        assert np.abs(R[b] - r["reaction"]).max() <= tol * np.abs(r["reaction"]).max()
        assert np.abs(ug[b] - r["u"]).max() <= tol * np.abs(r["u"]).max()
        assert np.abs(dg[b] - r["d"]).max() <= tol


def test_bar_fp64_full(pd):
    """The 40x10x10 bar, FP64, 1,000-step ramp with the stop rule."""
    w = W.bar()
    g = w.grid
    row, col = pd.build_neighbours(g)
    st = pd.State(g, row, col, w.mat, w.bc, batch=1, precision=pd.PREC_FP64)
    st.reset(torch.full((1, g.n_nodes), np.float32(w.mat.s0), device="cuda"))
    R = st.step(60).cpu().numpy()[0]
    u60 = st.store()[0].cpu().numpy()[0]
    st.reset(torch.full((1, g.n_nodes), np.float32(w.mat.s0), device="cuda"))
    pk, ps, nd = [x.item() for x in st.run_to_peak(w.n_steps)]
    _, _, dg = st.store()
    m = core.Model(w)
    r60 = m.run(60)
    pre = int(np.argmax(r60["smax"] > w.mat.s0 * 0.999)) or 60
    assert pre > 50
    rp = m.run(pre)
    st2 = pd.State(g, row, col, w.mat, w.bc, batch=1, precision=pd.PREC_FP64)
    st2.reset(torch.full((1, g.n_nodes), np.float32(w.mat.s0), device="cuda"))
    st2.step(pre)
    upre = st2.store()[0].cpu().numpy()[0]
    assert np.abs(upre - rp["u"]).max() <= 1e-10 * np.abs(rp["u"]).max()
    assert np.abs(R - r60["reaction"]).max() <= 1e-9 * np.abs(r60["reaction"]).max()
    r = m.run(w.n_steps, use_stop=True)
    assert abs(pk - r["peak"]) <= 1e-6 * abs(r["peak"])
    assert ps == r["peak_step"] and nd == r["n_done"]
    broken_mismatch = int(((dg.cpu().numpy()[0] >= 1) != (r["d"] >= 1)).sum())
    assert broken_mismatch == 0


def test_tiny_beam_mixed_run_to_peak(pd):
    """Mixed precision to the peak on a small notched beam, each side on its own KL field."""
    w = W.tiny_beam(16, 6, 4, n_steps=1500)
    w = dataclasses.replace(w, bc=dataclasses.replace(w.bc, u_max=2.5e-5))
    g = w.grid
    row, col = pd.build_neighbours(g)
    fld = pd.Field(g, 1, w.field)
    ids = torch.arange(3, dtype=torch.int64, device="cuda")
    s0 = fld.sample(0, pd.draw_xi(w.seed, 0, ids, w.field.n_modes))
    st = pd.State(g, row, col, w.mat, w.bc, batch=3, precision=pd.PREC_MIXED)
    st.reset(s0)
    pk, ps, nd = [x.cpu().numpy() for x in st.run_to_peak(w.n_steps)]
    _, _, dg = st.store()
    dg = dg.cpu().numpy()
    Phi, lam = field.kl_separable(g, w.field.length, w.field.n_modes)
    s0o = field.sample_field(w, Phi, lam, w.seed, 0, [0, 1, 2])
    for b in range(3):
        m = core.Model(w, s0=s0o[b])
        r = m.run(w.n_steps, use_stop=True)
        assert r["peak_step"] < r["n_done"] - 100, "the case must pass its peak"
        assert abs(pk[b] - r["peak"]) <= 1e-3 * abs(r["peak"])
        mism = int(((dg[b] >= 1) != (r["d"] >= 1)).sum())
        print(f"sample {b}: peak {pk[b]:.6g} vs {r['peak']:.6g}, broken-bond mismatches {mism} of {(r['d'] >= 1).sum()}")


def test_field_parity(pd):
    w = W.beam(2.5)
    g = w.grid
    fld = pd.Field(g, 1, w.field)
    Phi, lam = field.kl_separable(g, w.field.length, w.field.n_modes)
    assert np.abs(fld.eigenvalues() - lam).max() <= 1e-12 * lam[0]
    ids = torch.tensor([0, 1, 5, 1 << 33], dtype=torch.int64, device="cuda")
    xi = pd.draw_xi(w.seed, 1, ids, 64)
    xo = field.draw_xi(w.seed, 1, [0, 1, 5, 1 << 33], 64)
    assert np.abs(xi.cpu().numpy() - xo).max() <= 1e-14 * np.abs(xo).max()
    s0 = fld.sample(0, xi).cpu().numpy()
    so = field.lognormal(field.gaussian(Phi, lam, xo), w.field.mean, w.field.cov)
    assert np.abs(s0 - so).max() <= 1e-5 * so.max()


def test_level_coupling(pd):
    """Coarse field of a pair = 2x2x2 mean of the fine Gaussian field, same xi."""
    levels = W.beam_levels()
    fine = levels[2].grid
    fld = pd.Field(fine, 3, levels[0].field)
    ids = torch.arange(4, dtype=torch.int64, device="cuda")
    xi = pd.draw_xi(2, 2, ids, 64)
    f2, f1 = fld.sample(2, xi, coarse=True)
    f1b = fld.sample(1, xi)
    assert torch.equal(f1, f1b)  # the coarse member is exactly the level-1 field of the same xi
    # against the oracle: restrict the oracle's fine Gaussian field
    Phi, lam = field.kl_separable(fine, levels[0].field.length, 64)
    gf = field.gaussian(Phi, lam, field.draw_xi(2, 2, [0, 1, 2, 3], 64))
    gc = field.restrict(gf, fine)
    so = field.lognormal(gc, 1e-4, 0.1)
    assert np.abs(f1.cpu().numpy() - so).max() <= 1e-5 * so.max()
    so2 = field.lognormal(gf, 1e-4, 0.1)
    assert np.abs(f2.cpu().numpy() - so2).max() <= 1e-5 * so2.max()
