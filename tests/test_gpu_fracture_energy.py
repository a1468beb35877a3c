"""Critical stretch calibrated from the fracture energy (Appendix A) on the
GPU: the calibration constant, runs to the peak of an unnotched beam in both
precisions, and the adjoint, each against the oracle."""
import dataclasses

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


@pytest.mark.parametrize("law", [W.LAW_BILINEAR, W.LAW_EXPLINEAR])
def test_calibration_constant(pd, law):
    delta = 3.01 * 2.5e-3
    for G_F in (2.0, 20.0, 120.0):
        got = pd.gf_coefficient(law, 30e9, delta, G_F)
        want = core.gf_coefficient(law, core.micromodulus(30e9, delta), delta, G_F)
        assert got == pytest.approx(want, rel=1e-13)


def _small_type1(law, G_F):
    w = W.tiny_beam(16, 6, 4, notch=False, n_steps=1500)
    return dataclasses.replace(w, bc=dataclasses.replace(w.bc, u_max=3.0e-5),
                               mat=dataclasses.replace(w.mat, law=law, G_F=G_F, s_ratio=99.0))


@pytest.mark.parametrize("prec,law,G_F", [("fp64", W.LAW_EXPLINEAR, 2.0), ("mixed", W.LAW_EXPLINEAR, 2.0),
                                          ("mixed", W.LAW_BILINEAR, 6.0)])
def test_unnotched_beam_to_the_peak(pd, prec, law, G_F):
    w = _small_type1(law, G_F)
    g = w.grid
    Phi, lam = field.kl_separable(g, w.field.length, w.field.n_modes)
    s0 = np.ascontiguousarray(field.sample_field(w, Phi, lam, w.seed, 0, [0, 1]), np.float32)
    row, col = pd.build_neighbours(g)
    st = pd.State(g, row, col, w.mat, w.bc, batch=2,
                  precision=pd.PREC_FP64 if prec == "fp64" else pd.PREC_MIXED)
    st.reset(torch.tensor(s0, device="cuda"))
    pk, ps, nd = [x.cpu().numpy() for x in st.run_to_peak(w.n_steps)]
    for b in range(2):
        r = core.Model(w, s0=s0[b].astype(np.float64), dt=st.dt).run(w.n_steps, use_stop=True)
        assert r["peak_step"] < r["n_done"] - 100, "the case must pass its peak"
        print(f"{prec} law {law} sample {b}: peak {pk[b]:.6g} (step {ps[b]}) vs {r['peak']:.6g} (step {r['peak_step']})")
        if prec == "fp64":
            assert abs(pk[b] - r["peak"]) <= 1e-9 * abs(r["peak"])
            assert ps[b] == r["peak_step"] and nd[b] == r["n_done"]
        else:
            assert abs(pk[b] - r["peak"]) <= 1e-3 * abs(r["peak"])
    st.close()


def test_adjoint_in_calibrated_mode(pd):
    w = _small_type1(W.LAW_EXPLINEAR, 2.0)
    g = w.grid
    Phi, lam = field.kl_separable(g, w.field.length, w.field.n_modes)
    s0 = np.ascontiguousarray(field.sample_field(w, Phi, lam, w.seed, 0, [3]), np.float32)
    row, col = pd.build_neighbours(g)
    st = pd.State(g, row, col, w.mat, w.bc, batch=1, precision=pd.PREC_FP64)
    s0d = torch.tensor(s0, device="cuda")
    T = 340
    obs, wts = [T - 1, T // 2], np.array([[1.0, 0.5]])
    st.reset(s0d)
    gs, _, _ = st.adjoint(T, obs, torch.tensor(wts, device="cuda"), s0d, None, ckpt_every=50, grad_kappa=False)
    ogs, _ = core.Model(w, s0=s0[0].astype(np.float64), dt=st.dt).adjoint(T, obs, wts[0])
    assert np.abs(ogs).max() > 0
    err = np.abs(gs.cpu().numpy()[0] - ogs).max() / np.abs(ogs).max()
    print(f"calibrated-mode adjoint: max rel err {err:.2e}")
    assert err <= 1e-8
    st.close()
