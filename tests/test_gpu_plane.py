"""Plane (two-dimensional) model on the GPU against the oracle: the
calibration constant, forces of a random state, and notched plane beams run
to the peak in both precisions and both plane models."""
import math

import numpy as np
import pytest
import torch

import pd_workloads as W
from oracle import core, field

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd(built_lib):
    import paper_2212_04415_gb300 as pd
    return pd


def _plane_beam(model, law=W.LAW_EXPLINEAR, nx=56, ny=16, dx=1.25e-3):
    g = W.Grid(nx, ny, 1, dx, math.pi, 1, nx, round(0.2 * ny * 2))
    mat = W.Material(E=30e9, law=law, s0=1e-4, zeta=5e4, G_F=30.0, model=model, thickness=0.05)
    span = 2.5 * ny
    bc = W.BC(W.BC_BEAM_3PT, u_max=3e-5, n_ramp=2000,
              support_x2=(round(nx - span), round(nx + span)), load_x2=nx)
    fld = W.FieldCfg(W.COV_SQEXP, 4 * dx, 16, W.MARG_LOGNORMAL, 1e-4, 0.1)
    return W.Workload(f"plane_beam_{nx}x{ny}", g, mat, bc, 2000, fld, 9)


@pytest.mark.parametrize("model", [W.MODEL_PLANE_STRESS, W.MODEL_PLANE_STRAIN])
def test_plane_calibration_constant(pd, model):
    delta, t = math.pi * 1.25e-3, 0.05
    c = core.micromodulus_2d(30e9, delta, t, model == W.MODEL_PLANE_STRAIN)
    for law in (W.LAW_BILINEAR, W.LAW_EXPLINEAR):
        got = pd.gf_coefficient_plane(law, model, 30e9, delta, t, 30.0)
        assert got == pytest.approx(core.gf_coefficient_2d(law, c, delta, t, 30.0), rel=1e-13)


@pytest.mark.parametrize("prec,model", [("fp64", W.MODEL_PLANE_STRESS), ("mixed", W.MODEL_PLANE_STRESS),
                                        ("mixed", W.MODEL_PLANE_STRAIN)])
def test_plane_beam_to_the_peak(pd, prec, model):
    w = _plane_beam(model)
    g = w.grid
    Phi, lam = field.kl_separable(g, w.field.length, w.field.n_modes)
    s0 = np.ascontiguousarray(field.sample_field(w, Phi, lam, w.seed, 0, [0, 1, 2]), np.float32)
    row, col = pd.build_neighbours(g)
    st = pd.State(g, row, col, w.mat, w.bc, batch=3, precision=pd.PREC_FP64 if prec == "fp64" else pd.PREC_MIXED)
    st.reset(torch.tensor(s0, device="cuda"))
    pk, ps, nd = [x.cpu().numpy() for x in st.run_to_peak(w.n_steps)]
    m = core.Model(w, dt=st.dt)
    assert st.dt == pytest.approx(m.dt, rel=1e-12)
    for b in range(3):
        m.set_field(s0[b].astype(np.float64))
        r = m.run(w.n_steps, use_stop=True)
        assert r["peak_step"] < r["n_done"] - 100, "the case must pass its peak"
        print(f"{prec} model {model} sample {b}: peak {pk[b]:.6g} (step {ps[b]}) vs {r['peak']:.6g} "
              f"(step {r['peak_step']})")
        if prec == "fp64":
            assert abs(pk[b] - r["peak"]) <= 1e-9 * abs(r["peak"]) and ps[b] == r["peak_step"]
        else:
            assert abs(pk[b] - r["peak"]) <= 1e-3 * abs(r["peak"])
    st.close()


def test_plane_model_rejects_a_thick_grid(pd):
    w = _plane_beam(W.MODEL_PLANE_STRESS)
    g = W.Grid(16, 8, 2, 1.25e-3, math.pi)
    row, col = pd.build_neighbours(g)
    with pytest.raises(pd.PdError, match="one-layer"):
        pd.State(g, row, col, w.mat, w.bc)
