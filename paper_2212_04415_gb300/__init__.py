"""GB300-native probabilistic bond-based peridynamics (arXiv 2212.04415).

Thin Python binding of ``libpd_gb300.so`` (the C ABI declared in
``include/pd.h``): argument marshalling only. Every step of the hot path runs
in the library's sm_103a kernels; PyTorch provides device memory and streams.
There is no CPU fallback: if the library is not built, or no GPU is present,
the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB as _LIB_PATH

PD_OK, PD_ERR_ARG, PD_ERR_CUDA, PD_ERR_OOM, PD_ERR_TIMEOUT, PD_ERR_NAN, PD_ERR_CAP = 0, -1, -2, -3, -4, -5, -6
PREC_FP64, PREC_MIXED = 0, 1
MAX_LEVELS = 8


class PdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pd error {code}: {msg}")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("dx", C.c_double),
                ("m_ratio", C.c_double), ("notch", C.c_int32), ("notch_x2", C.c_int32),
                ("notch_y2", C.c_int32)]


class Material(C.Structure):
    _fields_ = [("E", C.c_double), ("rho", C.c_double), ("law", C.c_int32), ("s_ratio", C.c_double),
                ("k", C.c_double), ("alpha", C.c_double), ("dt", C.c_double), ("dt_safety", C.c_double),
                ("zeta", C.c_double), ("precision", C.c_int32), ("G_F", C.c_double),
                ("model", C.c_int32), ("thickness", C.c_double)]


class BC(C.Structure):
    _fields_ = [("type", C.c_int32), ("grip_planes", C.c_int32), ("support_x2", C.c_int32 * 2),
                ("load_x2", C.c_int32), ("u_max", C.c_double), ("n_ramp", C.c_int32)]


class FieldCfg(C.Structure):
    _fields_ = [("kernel", C.c_int32), ("length", C.c_double), ("n_modes", C.c_int32),
                ("marginal", C.c_int32), ("mean", C.c_double), ("cov", C.c_double),
                ("weibull_m", C.c_double)]


class MlmcCfg(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("grid", C.POINTER(Grid)), ("bc", C.POINTER(BC)),
                ("max_steps", C.POINTER(C.c_int32)), ("n_samples", C.POINTER(C.c_int64)),
                ("mat", Material), ("field", FieldCfg), ("seed", C.c_uint64), ("batch", C.c_int32),
                ("first_sample", C.POINTER(C.c_int64)), ("tune_steps", C.c_int32)]


class AdaptiveCfg(C.Structure):
    _fields_ = [("eps_s", C.c_double), ("eps_b", C.c_double), ("m_dof", C.c_double), ("alpha", C.c_double),
                ("n_star", C.c_int32), ("cost_model", C.POINTER(C.c_double))]


class Schedule(C.Structure):
    _fields_ = [("by", C.c_int32), ("bz", C.c_int32), ("q", C.c_int32), ("ns", C.c_int32), ("reduce", C.c_int32)]


class MlmcLevel(C.Structure):
    _fields_ = [("n", C.c_int64), ("sum_y", C.c_double), ("sum_y2", C.c_double), ("mean", C.c_double),
                ("var", C.c_double), ("var_unbiased", C.c_double), ("cost_s", C.c_double),
                ("steps", C.c_int64), ("bond_updates", C.c_int64)]


class MlmcResult(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("level", MlmcLevel * MAX_LEVELS), ("q_ml", C.c_double),
                ("var_ml", C.c_double)]


_VP = C.c_void_p
_SIGS = {
    "pd_last_error": (C.c_int, [C.c_char_p, C.c_size_t]),
    "pd_version": (C.c_char_p, []),
    "pd_build_neighbours": (C.c_int, [C.POINTER(Grid), _VP, _VP, C.c_int64, C.POINTER(C.c_int64), _VP]),
    "pd_build_neighbours_noalloc": (C.c_int, [C.POINTER(Grid), _VP, _VP, C.c_int64, C.POINTER(C.c_int64), _VP]),
    "pd_bc_codes": (C.c_int, [C.POINTER(Grid), C.POINTER(BC), _VP, _VP]),
    "pd_state_create": (C.c_int, [C.POINTER(Grid), _VP, _VP, C.c_int64, C.POINTER(Material), C.POINTER(BC),
                                  C.c_int32, C.POINTER(_VP)]),
    "pd_state_destroy": (C.c_int, [_VP]),
    "pd_state_create_sched": (C.c_int, [C.POINTER(Grid), _VP, _VP, C.c_int64, C.POINTER(Material), C.POINTER(BC),
                                        C.c_int32, C.POINTER(Schedule), C.POINTER(_VP)]),
    "pd_autotune": (C.c_int, [C.POINTER(Grid), _VP, _VP, C.c_int64, C.POINTER(Material), C.POINTER(BC), C.c_int32,
                              C.c_int32, C.POINTER(Schedule), C.POINTER(C.c_double)]),
    "pd_state_info": (C.c_int, [_VP, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                C.POINTER(C.c_int64)]),
    "pd_state_reset": (C.c_int, [_VP, _VP, _VP, _VP]),
    "pd_state_reset_f64": (C.c_int, [_VP, _VP, _VP, _VP]),
    "pd_state_load": (C.c_int, [_VP, _VP, _VP, _VP, C.c_int32, _VP]),
    "pd_state_store": (C.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "pd_force": (C.c_int, [_VP, _VP, _VP]),
    "pd_step": (C.c_int, [_VP, C.c_int32, _VP, _VP]),
    "pd_run_to_peak": (C.c_int, [_VP, C.c_int32, _VP, _VP, _VP, _VP]),
    "pd_run_to_peak_multi": (C.c_int, [_VP, C.c_int32, _VP, _VP, _VP, _VP, _VP]),
    "pd_draw_xi": (C.c_int, [C.c_uint64, C.c_int32, _VP, C.c_int32, C.c_int32, _VP, _VP]),
    "pd_field_create": (C.c_int, [C.POINTER(Grid), C.c_int32, C.POINTER(FieldCfg), C.POINTER(_VP)]),
    "pd_field_destroy": (C.c_int, [_VP]),
    "pd_field_info": (C.c_int, [_VP, C.POINTER(C.c_int32), _VP]),
    "pd_sample_field": (C.c_int, [_VP, C.c_int32, _VP, C.c_int32, _VP, _VP, _VP]),
    "mlmc_estimate": (C.c_int, [C.POINTER(MlmcCfg), C.POINTER(MlmcResult), _VP, _VP, _VP, _VP]),
    "pd_gf_coefficient": (C.c_int, [C.c_int32, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                    C.POINTER(C.c_double)]),
    "pd_gf_coefficient_plane": (C.c_int, [C.c_int32, C.c_int32] + [C.c_double] * 6 + [C.POINTER(C.c_double)]),
    "pd_ml_inverse_cdf": (C.c_int, [C.c_int32, _VP, _VP, _VP, C.c_int32, _VP, _VP, _VP]),
    "pd_ml_cdf": (C.c_int, [C.c_int32, _VP, _VP, _VP, C.c_int32, C.c_int32, _VP, _VP, _VP]),
    "mlmc_adaptive": (C.c_int, [C.POINTER(MlmcCfg), C.POINTER(AdaptiveCfg), C.POINTER(MlmcResult),
                                C.POINTER(C.c_int32), C.POINTER(C.c_double), _VP, _VP, C.c_int64, _VP]),
    "pd_adjoint": (C.c_int, [_VP, C.c_int32, C.c_int32, C.c_int32, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "pd_field_adjoint": (C.c_int, [_VP, C.c_int32, _VP, C.c_int32, _VP, _VP, _VP]),
    "pd_mlmc_allocation": (C.c_int, [C.c_int32, _VP, _VP, C.c_double, _VP]),
    "mlmc_merge": (C.c_int, [C.c_int32, _VP, _VP, C.POINTER(MlmcResult)]),
}

_lib = None


def lib_path() -> str:
    return _LIB_PATH


def lib():
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != PD_OK:
        buf = C.create_string_buffer(512)
        lib().pd_last_error(buf, 512)
        raise PdError(rc, buf.value.decode())


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be CUDA and contiguous"
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ------------------------------------------------------------ conversions

def grid_struct(g) -> Grid:
    return Grid(g.nx, g.ny, g.nz, g.dx, g.m_ratio, g.notch, g.notch_x2, g.notch_y2)


def material_struct(m, precision: int, dt: float = 0.0) -> Material:
    return Material(m.E, m.rho, m.law, m.s_ratio, m.k, m.alpha, dt, m.dt_safety, m.zeta, precision,
                    getattr(m, "G_F", 0.0), getattr(m, "model", 0), getattr(m, "thickness", 0.0))


def bc_struct(b) -> BC:
    return BC(b.type, b.grip_planes, (C.c_int32 * 2)(*b.support_x2), b.load_x2, b.u_max, b.n_ramp)


def field_struct(f) -> FieldCfg:
    return FieldCfg(f.kernel, f.length, f.n_modes, f.marginal, f.mean, f.cov, f.weibull_m)


# ------------------------------------------------------------------ calls

def build_neighbours(g, stream=None):
    """CSR (row_ptr int32[N+1], col int32[nb]) as CUDA tensors (Eq. PD_Horizon)."""
    import torch
    G = grid_struct(g)
    n = g.nx * g.ny * g.nz
    row = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    nb = C.c_int64(0)
    _check(lib().pd_build_neighbours(C.byref(G), _ptr(row), None, 0, C.byref(nb), _stream(stream)))
    col = torch.empty(max(nb.value, 1), dtype=torch.int32, device="cuda")
    _check(lib().pd_build_neighbours(C.byref(G), _ptr(row), _ptr(col), nb.value, C.byref(nb), _stream(stream)))
    return row, col[: nb.value]


def bc_codes(g, b, stream=None):
    import torch
    G, Bc = grid_struct(g), bc_struct(b)
    out = torch.empty((g.nx * g.ny * g.nz, 3), dtype=torch.uint8, device="cuda")
    _check(lib().pd_bc_codes(C.byref(G), C.byref(Bc), _ptr(out), _stream(stream)))
    return out


class State:
    """B independent samples of the explicit peridynamic dynamics on one mesh."""

    def __init__(self, g, row, col, mat, bc, batch=1, precision=PREC_MIXED, dt=0.0, schedule=None):
        """schedule: None (built-in choice) or (by, bz, q[, ns[, reduce]]), e.g.
        from ``autotune`` (ns: samples per block; reduce: 1 = each step's
        reaction in its own launch, 2 = in the next launch; 0 = built-in)."""
        import torch
        torch.cuda.synchronize()
        self.grid = g
        self.B = batch
        self._G, self._M, self._BC = grid_struct(g), material_struct(mat, precision, dt), bc_struct(bc)
        h = C.c_void_p()
        sch = Schedule(*schedule) if schedule is not None else None
        _check(lib().pd_state_create_sched(C.byref(self._G), _ptr(row), _ptr(col), int(col.numel()),
                                           C.byref(self._M), C.byref(self._BC), batch,
                                           C.byref(sch) if sch is not None else None, C.byref(h)))
        self.h = h
        dtv, cv, nn, nb = C.c_double(), C.c_double(), C.c_int64(), C.c_int64()
        _check(lib().pd_state_info(h, C.byref(dtv), C.byref(cv), C.byref(nn), C.byref(nb)))
        self.dt, self.c, self.N, self.nb = dtv.value, cv.value, nn.value, nb.value

    def close(self):
        if getattr(self, "h", None):
            lib().pd_state_destroy(self.h)
            self.h = None

    __del__ = close

    def reset(self, s0, kappa=None, stream=None):
        _check(lib().pd_state_reset(self.h, _ptr(s0), _ptr(kappa), _stream(stream)))

    def reset_f64(self, s0, kappa=None, stream=None):
        """reset with the strength field s0 in FP64 (pd_state_reset_f64)."""
        _check(lib().pd_state_reset_f64(self.h, _ptr(s0), _ptr(kappa), _stream(stream)))

    def load(self, u, v, d=None, step=0, stream=None):
        _check(lib().pd_state_load(self.h, _ptr(u), _ptr(v), _ptr(d), step, _stream(stream)))

    def store(self, stream=None):
        import torch
        u = torch.empty((self.B, self.N, 3), dtype=torch.float64, device="cuda")
        v = torch.empty_like(u)
        d = torch.empty((self.B, self.nb), dtype=torch.float64, device="cuda")
        _check(lib().pd_state_store(self.h, _ptr(u), _ptr(v), _ptr(d), _stream(stream)))
        return u, v, d

    def force(self, stream=None):
        import torch
        F = torch.empty((self.B, self.N, 3), dtype=torch.float64, device="cuda")
        _check(lib().pd_force(self.h, _ptr(F), _stream(stream)))
        return F

    def step(self, n_steps, reaction=True, stream=None):
        import torch
        R = torch.empty((self.B, n_steps), dtype=torch.float64, device="cuda") if reaction else None
        _check(lib().pd_step(self.h, n_steps, _ptr(R), _stream(stream)))
        return R

    def run_to_peak(self, max_steps, stream=None, out=None):
        import torch
        if out is None:
            out = (torch.empty(self.B, dtype=torch.float64, device="cuda"),
                   torch.empty(self.B, dtype=torch.int32, device="cuda"),
                   torch.empty(self.B, dtype=torch.int32, device="cuda"))
        pk, ps, nd = out
        _check(lib().pd_run_to_peak(self.h, max_steps, _ptr(pk), _ptr(ps), _ptr(nd), _stream(stream)))
        return pk, ps, nd

    def adjoint(self, n_steps, obs_steps, dJ_dR, s0, kappa=None, ckpt_every=100, grad_kappa=True,
                stream=None):
        """Gradient of J = sum_o dJ_dR[:, o] R^{obs_steps[o]} over n_steps steps from the
        current state with respect to the node fields s0 and kappa (pd_adjoint).
        Returns (grad_s0, grad_kappa or None, R at the observation steps)."""
        import torch
        obs = (C.c_int32 * max(len(obs_steps), 1))(*[int(o) for o in obs_steps])
        gs = torch.empty((self.B, self.N), dtype=torch.float64, device="cuda")
        gk = torch.empty_like(gs) if grad_kappa else None
        R = torch.empty((self.B, len(obs_steps)), dtype=torch.float64, device="cuda")
        _check(lib().pd_adjoint(self.h, n_steps, ckpt_every, len(obs_steps), C.cast(obs, C.c_void_p),
                                _ptr(dJ_dR), _ptr(s0), _ptr(kappa), _ptr(gs), _ptr(gk), _ptr(R),
                                _stream(stream)))
        return gs, gk, R


def gf_coefficient(law, E, delta, G_F, k=25.0, alpha=0.25):
    """A of s_crit = s0 + A / s0 for a fracture energy G_F (pd_gf_coefficient)."""
    A = C.c_double()
    _check(lib().pd_gf_coefficient(law, E, delta, G_F, k, alpha, C.byref(A)))
    return A.value


def gf_coefficient_plane(law, model, E, delta, t, G_F, k=25.0, alpha=0.25):
    """A of s_crit = s0 + A / s0 for a plane model of thickness t (pd_gf_coefficient_plane)."""
    A = C.c_double()
    _check(lib().pd_gf_coefficient_plane(law, model, E, delta, t, G_F, k, alpha, C.byref(A)))
    return A.value


def run_to_peak_multi(states, max_steps, stream=None):
    """pd_run_to_peak_multi: run several states to their peaks together; returns
    [(peak, peak_step, n_done)] per state."""
    import torch
    n = len(states)
    outs = [(torch.empty(st.B, dtype=torch.float64, device="cuda"), torch.empty(st.B, dtype=torch.int32, device="cuda"),
             torch.empty(st.B, dtype=torch.int32, device="cuda")) for st in states]
    hs = (C.c_void_p * n)(*[st.h.value for st in states])
    ms = (C.c_int32 * n)(*max_steps)
    pk = (C.c_void_p * n)(*[o[0].data_ptr() for o in outs])
    ps = (C.c_void_p * n)(*[o[1].data_ptr() for o in outs])
    nd = (C.c_void_p * n)(*[o[2].data_ptr() for o in outs])
    _check(lib().pd_run_to_peak_multi(C.cast(hs, C.c_void_p), n, C.cast(ms, C.c_void_p), C.cast(pk, C.c_void_p),
                                      C.cast(ps, C.c_void_p), C.cast(nd, C.c_void_p), _stream(stream)))
    return outs


def autotune(g, row, col, mat, bc, batch=1, precision=PREC_MIXED, trial_steps=20, dt=0.0):
    """Fastest launch schedule (by, bz, q, ns) of a mesh and batch, and its time
    per step in microseconds (pd_autotune; cached per process)."""
    G, M, BCs = grid_struct(g), material_struct(mat, precision, dt), bc_struct(bc)
    best = Schedule()
    us = C.c_double()
    _check(lib().pd_autotune(C.byref(G), _ptr(row), _ptr(col), int(col.numel()), C.byref(M), C.byref(BCs), batch,
                             trial_steps, C.byref(best), C.byref(us)))
    return (best.by, best.bz, best.q, best.ns), us.value


def draw_xi(seed, level, sample_ids, n_modes, stream=None, out=None):
    import torch
    B = sample_ids.numel()
    xi = out if out is not None else torch.empty((B, n_modes), dtype=torch.float64, device="cuda")
    _check(lib().pd_draw_xi(seed, level, _ptr(sample_ids), B, n_modes, _ptr(xi), _stream(stream)))
    return xi


class Field:
    """Truncated KL random field on a hierarchy of nested grids (finest given)."""

    def __init__(self, finest, n_levels, cfg):
        import torch
        torch.cuda.synchronize()
        self._G, self._F = grid_struct(finest), field_struct(cfg)
        h = C.c_void_p()
        _check(lib().pd_field_create(C.byref(self._G), n_levels, C.byref(self._F), C.byref(h)))
        self.h = h
        self.K = cfg.n_modes
        # node counts per level, coarsest first (each coarser grid halves nx, ny, nz)
        # (a one-layer hierarchy halves nx and ny only)
        self.sizes = [(finest.nx >> s, finest.ny >> s, finest.nz if finest.nz == 1 else finest.nz >> s)
                      for s in range(n_levels - 1, -1, -1)]

    def close(self):
        """Free the field; raises if a sampling launch had given up waiting (PD_ERR_TIMEOUT)."""
        h = getattr(self, "h", None)
        if h:
            self.h = None
            _check(lib().pd_field_destroy(h))

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.h = None
            lib().pd_field_destroy(h)

    def adjoint(self, level, xi, dJ_ds0, stream=None):
        """dJ/dxi [B, K] from dJ/ds0 [B, N_level] (pd_field_adjoint)."""
        import torch
        B = xi.shape[0]
        out = torch.empty((B, self.K), dtype=torch.float64, device="cuda")
        _check(lib().pd_field_adjoint(self.h, level, _ptr(xi), B, _ptr(dJ_ds0), _ptr(out), _stream(stream)))
        return out

    def eigenvalues(self):
        import numpy as np
        lam = np.zeros(self.K)
        k = C.c_int32()
        _check(lib().pd_field_info(self.h, C.byref(k), lam.ctypes.data_as(C.c_void_p)))
        return lam

    def sample(self, level, xi, coarse=False, stream=None, out=None):
        import torch
        B = xi.shape[0]
        nf = self.sizes[level][0] * self.sizes[level][1] * self.sizes[level][2]
        f = out[0] if out is not None else torch.empty((B, nf), dtype=torch.float32, device="cuda")
        c = None
        if coarse:
            nc = self.sizes[level - 1][0] * self.sizes[level - 1][1] * self.sizes[level - 1][2]
            c = out[1] if out is not None else torch.empty((B, nc), dtype=torch.float32, device="cuda")
        _check(lib().pd_sample_field(self.h, level, _ptr(xi), B, _ptr(f), _ptr(c), _stream(stream)))
        return (f, c) if coarse else f


def mlmc_estimate(grids, bcs, max_steps, n_samples, mat, field, seed, batch, precision=PREC_MIXED,
                  first_sample=None, return_samples=False, tune_steps=0, stream=None):
    """Fixed-allocation MLMC over len(grids) nested levels (coarsest first).

    Returns per-level totals, the estimator, and the per-batch FP64 sums
    (n, sum Y, sum Y^2) in batch order (``batch_sums``), which is what
    ``shard.merge`` combines across processes."""
    import numpy as np
    L = len(grids)
    G = (Grid * L)(*[grid_struct(g) for g in grids])
    Bc = (BC * L)(*[bc_struct(b) for b in bcs])
    ms = (C.c_int32 * L)(*max_steps)
    ns = (C.c_int64 * L)(*n_samples)
    fs = (C.c_int64 * L)(*(first_sample if first_sample is not None else [0] * L))
    cfg = MlmcCfg(L, G, Bc, ms, ns, material_struct(mat, precision), field_struct(field), seed, batch, fs,
                  tune_steps)
    res = MlmcResult()
    tot = int(sum(n_samples))
    nbat = [(n + min(batch, max(n, 1)) - 1) // min(batch, max(n, 1)) for n in n_samples]
    qf = np.zeros(max(tot, 1))
    qc = np.zeros(max(tot, 1))
    bs = np.zeros((max(sum(nbat), 1), 3))
    _check(lib().mlmc_estimate(C.byref(cfg), C.byref(res), qf.ctypes.data_as(C.c_void_p),
                               qc.ctypes.data_as(C.c_void_p), bs.ctypes.data_as(C.c_void_p), _stream(stream)))
    levels = []
    for l in range(L):
        lv = res.level[l]
        levels.append(dict(n=lv.n, sum_y=lv.sum_y, sum_y2=lv.sum_y2, mean=lv.mean, var=lv.var,
                           var_unbiased=lv.var_unbiased, cost_s=lv.cost_s, steps=lv.steps,
                           bond_updates=lv.bond_updates))
    out = dict(levels=levels, q_ml=res.q_ml, var_ml=res.var_ml)
    o = 0
    out["batch_sums"] = []
    for l in range(L):
        out["batch_sums"].append(bs[o:o + nbat[l]].copy())
        o += nbat[l]
    if return_samples:
        out["q_fine"], out["q_coarse"] = qf[:tot], qc[:tot]
    return out


def mlmc_adaptive(grids, bcs, max_steps, mat, field, seed, batch, eps_s, eps_b, m_dof=8.0, alpha=1.0,
                  n_star=100, cost_model=None, first_sample=None, cap=1 << 20, precision=PREC_MIXED,
                  tune_steps=0, stream=None):
    """Adaptive MLMC (Algorithm MLMC) over up to len(grids) levels: returns the
    last level L, the bias estimate, per-level statistics, the estimator and
    every sample's (Q_l, Q_{l-1}) per level, in id order."""
    import numpy as np
    L = len(grids)
    G = (Grid * L)(*[grid_struct(g) for g in grids])
    Bc = (BC * L)(*[bc_struct(b) for b in bcs])
    ms = (C.c_int32 * L)(*max_steps)
    fs = (C.c_int64 * L)(*(first_sample if first_sample is not None else [0] * L))
    cfg = MlmcCfg(L, G, Bc, ms, None, material_struct(mat, precision), field_struct(field), seed, batch, fs,
                  tune_steps)
    cm = (C.c_double * L)(*cost_model) if cost_model is not None else None
    ad = AdaptiveCfg(eps_s, eps_b, m_dof, alpha, n_star, cm)
    res = MlmcResult()
    Lu, eb = C.c_int32(), C.c_double()
    qf = np.zeros(cap)
    qc = np.zeros(cap)
    _check(lib().mlmc_adaptive(C.byref(cfg), C.byref(ad), C.byref(res), C.byref(Lu), C.byref(eb),
                               qf.ctypes.data_as(C.c_void_p), qc.ctypes.data_as(C.c_void_p), cap,
                               _stream(stream)))
    levels, q = [], []
    o = 0
    for l in range(res.n_levels):
        lv = res.level[l]
        levels.append(dict(n=lv.n, sum_y=lv.sum_y, sum_y2=lv.sum_y2, mean=lv.mean, var=lv.var,
                           var_unbiased=lv.var_unbiased, cost_s=lv.cost_s, steps=lv.steps,
                           bond_updates=lv.bond_updates))
        q.append((qf[o:o + lv.n].copy(), qc[o:o + lv.n].copy()))
        o += lv.n
    return dict(L=Lu.value, bias=eb.value, levels=levels, q_ml=res.q_ml, var_ml=res.var_ml, samples=q)


def _levels_flat(levels):
    """[q0, (fine1, coarse1), ...] (device tensors) -> counts, flat fine, flat coarse."""
    import torch
    n = [int(levels[0].numel())] + [int(f.numel()) for f, _ in levels[1:]]
    qf = torch.cat([levels[0].double()] + [f.double() for f, _ in levels[1:]]).contiguous()
    qc = torch.cat([torch.zeros_like(levels[0], dtype=torch.float64)] +
                   [c.double() for _, c in levels[1:]]).contiguous()
    return (C.c_int64 * len(n))(*n), qf, qc


def ml_inverse_cdf(levels, u, stream=None):
    """F_L^-1(u) (pd_ml_inverse_cdf): levels = [Q_0, (Q_1, Q~_0), ...] device tensors."""
    import torch
    n, qf, qc = _levels_flat(levels)
    u = u.double().contiguous()
    out = torch.empty_like(u)
    _check(lib().pd_ml_inverse_cdf(len(levels), C.cast(n, C.c_void_p), _ptr(qf), _ptr(qc), u.numel(), _ptr(u),
                                   _ptr(out), _stream(stream)))
    return out


def ml_cdf(levels, x, n_u=1000, stream=None):
    """F(x) (pd_ml_cdf) on the points F_L^-1((i + 1/2) / n_u)."""
    import torch
    n, qf, qc = _levels_flat(levels)
    x = x.double().contiguous()
    F = torch.empty_like(x)
    _check(lib().pd_ml_cdf(len(levels), C.cast(n, C.c_void_p), _ptr(qf), _ptr(qc), n_u, x.numel(), _ptr(x),
                           _ptr(F), _stream(stream)))
    return F


def mlmc_merge(batch_sums_per_level):
    """Level totals and the estimator from per-batch sums (mlmc_merge):
    ``batch_sums_per_level[l]`` is an [n_batches, 3] array of (n, sum Y,
    sum Y^2) in sample order."""
    import numpy as np
    L = len(batch_sums_per_level)
    arrs = [np.asarray(b, np.float64).reshape(-1, 3) for b in batch_sums_per_level]
    nb = (C.c_int64 * L)(*[a.shape[0] for a in arrs])
    flat = np.ascontiguousarray(np.concatenate(arrs) if arrs else np.zeros((0, 3)))
    res = MlmcResult()
    _check(lib().mlmc_merge(L, nb, flat.ctypes.data_as(C.c_void_p) if flat.size else None, C.byref(res)))
    levels = []
    for l in range(L):
        lv = res.level[l]
        levels.append(dict(n=lv.n, sum_y=lv.sum_y, sum_y2=lv.sum_y2, mean=lv.mean, var=lv.var,
                           var_unbiased=lv.var_unbiased))
    return dict(levels=levels, q_ml=res.q_ml, var_ml=res.var_ml)


def mlmc_allocation(V, Cst, eps_s):
    import numpy as np
    V = np.ascontiguousarray(V, np.float64)
    Cs = np.ascontiguousarray(Cst, np.float64)
    N = np.zeros(V.size, np.int64)
    _check(lib().pd_mlmc_allocation(V.size, V.ctypes.data_as(C.c_void_p), Cs.ctypes.data_as(C.c_void_p),
                                    eps_s, N.ctypes.data_as(C.c_void_p)))
    return N


def reaction_at(xi_s, xi_k, state, field_s, field_k, level, n_steps, obs_steps, ckpt_every=100):
    """Reactions R^{obs_steps} [B, n_obs] of the samples whose strength field has
    KL coefficients xi_s (and stiffness field xi_k, or None), differentiable
    with respect to both coefficient sets: the backward pass runs pd_adjoint and
    pd_field_adjoint."""
    return _reaction_fn().apply(xi_s, xi_k, state, field_s, field_k, level, n_steps, list(obs_steps), ckpt_every)


_RFN = None


def _reaction_fn():
    global _RFN
    if _RFN is not None:
        return _RFN
    import torch

    class ReactionAt(torch.autograd.Function):
        @staticmethod
        def forward(ctx, xi_s, xi_k, state, field_s, field_k, level, n_steps, obs_steps, ckpt_every):
            s0 = field_s.sample(level, xi_s)
            kap = field_k.sample(level, xi_k) if xi_k is not None else None
            state.reset(s0, kap)
            R = state.step(n_steps)
            ctx.save_for_backward(xi_s, xi_k if xi_k is not None else torch.empty(0))
            ctx.args = (state, field_s, field_k, level, n_steps, obs_steps, ckpt_every, xi_k is not None)
            return R[:, obs_steps].contiguous()

        @staticmethod
        def backward(ctx, gR):
            xi_s, xi_k = ctx.saved_tensors
            state, field_s, field_k, level, n_steps, obs_steps, ckpt_every, has_k = ctx.args
            s0 = field_s.sample(level, xi_s)
            kap = field_k.sample(level, xi_k) if has_k else None
            state.reset(s0, kap)
            gs, gk, _ = state.adjoint(n_steps, obs_steps, gR.contiguous().to(torch.float64), s0, kap,
                                      ckpt_every=ckpt_every, grad_kappa=has_k)
            g_xs = field_s.adjoint(level, xi_s, gs)
            g_xk = field_k.adjoint(level, xi_k, gk) if has_k else None
            return g_xs, g_xk, None, None, None, None, None, None, None

    _RFN = ReactionAt
    return _RFN

