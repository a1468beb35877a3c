"""Parity of the benchmarked workload itself: the notched three-point-bending
beam 175 x 50 x 50 mm at dx = 2.5 mm (28,000 nodes, 2,975,344 directed bonds),
sample 0 of seed 1, mixed precision, one sample per launch, run to the peak
with the stop rule (at most 5,000 steps) through pd_run_to_peak, exactly as
the benchmark times it.

Against the FP64 oracle on its own KL field of the same coefficients:
* displacements within 1e-5 relative (max-norm) at the last 100-step mark
  before the oracle's first bond passes its elastic limit;
* peak load within 1e-3 relative (Sections 4 and 6.2: the quantity of
  interest);
* peak step, steps executed and the broken-bond (d = 1) mismatch count are
  printed; the mismatch count is bounded loosely (5 % of the oracle's broken
  bonds), since the crack's last bonds break within a step or two of each
  other.
"""
import numpy as np
import pytest
import torch

import pd_workloads as W
from oracle import core, field

pytestmark = pytest.mark.gpu


def test_bench_beam_run_to_peak_parity(built_lib):
    pd = built_lib
    w = W.beam()
    g = w.grid
    K = w.field.n_modes
    # oracle: pre-damage mark, then on to the peak
    Phi, lam = field.kl_separable(g, w.field.length, K)
    s0o = field.sample_field(w, Phi, lam, w.seed, 0, [0])[0]
    m = core.Model(w, s0=s0o)
    state, n_pre, u_pre = None, 0, None
    Q, qs = -np.inf, -1
    n = 0
    while True:
        r = m.run(100, state=state, step0=n, peak=Q, peak_step=qs)
        if (r["d"] > 0).any():
            break
        state, n = (r["u"], r["v"], r["d"]), n + 100
        Q, qs = r["peak"], r["peak_step"]
        n_pre, u_pre = n, r["u"]
    assert n_pre >= 500, "the case has an elastic window"
    ro = m.run(w.n_steps - n_pre, state=state, step0=n_pre, use_stop=True, peak=Q, peak_step=qs)
    n_done_o = n_pre + ro["n_done"]
    assert ro["peak_step"] < n_done_o - 100, "the case must pass its peak"

    # GPU, the benchmark's path
    row, col = pd.build_neighbours(g)
    fld = pd.Field(g, 1, w.field)
    xi = pd.draw_xi(w.seed, 0, torch.zeros(1, dtype=torch.int64, device="cuda"), K)
    s0 = fld.sample(0, xi)
    st = pd.State(g, row, col, w.mat, w.bc, batch=1, precision=pd.PREC_MIXED)
    st.reset(s0)
    st.run_to_peak(n_pre)
    ug = st.store()[0].cpu().numpy()[0]
    err_u = np.abs(ug - u_pre).max() / np.abs(u_pre).max()
    st.reset(s0)
    pk, ps, nd = [x.item() for x in st.run_to_peak(w.n_steps)]
    dg = st.store()[2].cpu().numpy()[0]
    err_pk = abs(pk - ro["peak"]) / abs(ro["peak"])
    broken_o = int((ro["d"] >= 1).sum())
    mism = int(((dg >= 1) != (ro["d"] >= 1)).sum())
    print(f"\npre-damage mark {n_pre}: u rel err {err_u:.2e}; peak {pk:.6g} vs {ro['peak']:.6g} (rel {err_pk:.2e}), "
          f"peak step {ps} vs {ro['peak_step']}, steps {nd} vs {n_done_o}, "
          f"broken-bond mismatches {mism} of {broken_o}")
    st.close()
    assert err_u <= 1e-5
    assert err_pk <= 1e-3
    assert mism <= 0.05 * broken_o
