"""ctypes wrapper around ``pd_oracle.c`` (FP64 peridynamic reference).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Pins (tests under ``tests/test_oracle_*.py``):
* neighbour list: brute-force O(N^2) enumeration and a hand-checked notch case
  with exact rationals; exact bond counts of the workloads;
* bond laws: d(s0) = 0, d(s_crit) = 1, monotone d, and the closed-form bond
  fracture energy of Eq. exp_bond_energy against numerical quadrature;
* forces: zero under rigid translation and rotation; net internal force zero
  (antisymmetry); the interior force of a uniform stretch vanishes and its
  strain energy density matches the lattice closed form and, within the
  lattice error, the continuum value that defines the micromodulus;
* run: R(2U) = 2R(U) in the linear regime; damage monotone in time;
* reaction R_n: at static equilibrium it equals the axial force carried by
  the bonds crossing any interior section of a bar in tension, and the sum of
  the two (equal) support reactions of a beam in three-point bending, both
  from independent pair forces (tests/test_oracle_reaction.py);
* adjoint: central differences of the run with respect to node s0 and kappa
  (elastic and softening windows, both laws); s0 has no influence before a
  bond softens; linear in the observation weights.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain -O2, no FMA contraction, OpenMP)."""
    src = os.path.join(_HERE, "pd_oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared",
                               "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_double), ("m_ratio", C.c_double), ("notch", C.c_int32),
                ("notch_x2", C.c_int32), ("notch_y2", C.c_int32)]


class BC(C.Structure):
    _fields_ = [("type", C.c_int32), ("grip_planes", C.c_int32),
                ("support_x2", C.c_int32 * 2), ("load_x2", C.c_int32),
                ("u_max", C.c_double), ("n_ramp", C.c_int32)]


class Problem(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_double), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("c", C.c_double), ("rho", C.c_double), ("law", C.c_int32),
                ("s_ratio", C.c_double), ("k", C.c_double), ("alpha", C.c_double),
                ("dt", C.c_double), ("zeta", C.c_double), ("s0", C.c_void_p),
                ("kappa", C.c_void_p), ("bc", C.c_void_p), ("u_max", C.c_double),
                ("n_ramp", C.c_int32), ("gf_A", C.c_double), ("vol", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.or_build_bruteforce.argtypes = [C.POINTER(Grid), C.c_void_p, C.c_void_p,
                                          C.c_int64, C.POINTER(C.c_int64)]
        L.or_build_window.argtypes = L.or_build_bruteforce.argtypes
        L.or_bc_codes.argtypes = [C.POINTER(Grid), C.POINTER(BC), C.c_void_p]
        L.or_micromodulus_3d.argtypes = [C.c_double, C.c_double]
        L.or_micromodulus_3d.restype = C.c_double
        L.or_damage_law.argtypes = [C.c_int32, C.c_double, C.c_double, C.c_double,
                                    C.c_double, C.c_double]
        L.or_damage_law.restype = C.c_double
        L.or_stable_dt.argtypes = [C.POINTER(Grid), C.c_void_p, C.c_void_p, C.c_double,
                                   C.c_double, C.c_double]
        L.or_stable_dt.restype = C.c_double
        L.or_force.argtypes = [C.POINTER(Problem), C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_void_p]
        L.or_run.argtypes = [C.POINTER(Problem), C.c_int32, C.c_int32, C.c_int32,
                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                             C.POINTER(C.c_double), C.POINTER(C.c_int32),
                             C.POINTER(C.c_int32)]
        L.or_run_batch.argtypes = [C.POINTER(Problem), C.c_int32, C.c_int64, C.c_void_p,
                                   C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_max_threads.restype = C.c_int
        L.or_micromodulus_2d.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int32]
        L.or_micromodulus_2d.restype = C.c_double
        L.or_gf_coefficient_2d.argtypes = [C.c_int32] + [C.c_double] * 6
        L.or_gf_coefficient_2d.restype = C.c_double
        L.or_stable_dt_vol.argtypes = [C.POINTER(Grid), C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_double,
                                       C.c_double]
        L.or_stable_dt_vol.restype = C.c_double
        L.or_gf_coefficient.argtypes = [C.c_int32] + [C.c_double] * 5
        L.or_gf_coefficient.restype = C.c_double
        L.or_fracture_energy.argtypes = [C.c_int32] + [C.c_double] * 6
        L.or_fracture_energy.restype = C.c_double
        L.or_adjoint.argtypes = [C.POINTER(Problem), C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def make_grid(g) -> Grid:
    """From a ``pd_workloads.Grid``."""
    return Grid(g.nx, g.ny, g.nz, g.dx, g.m_ratio, g.notch, g.notch_x2, g.notch_y2)


def neighbours(g, brute: bool = False):
    """CSR (row_ptr int32[N+1], col int32[nb]) of the horizon (Eq. PD_Horizon)."""
    L = lib()
    G = make_grid(g)
    fn = L.or_build_bruteforce if brute else L.or_build_window
    nb = C.c_int64(0)
    n = g.nx * g.ny * g.nz
    row = np.zeros(n + 1, np.int32)
    fn(C.byref(G), _p(row), None, 0, C.byref(nb))
    col = np.zeros(max(nb.value, 1), np.int32)
    rc = fn(C.byref(G), _p(row), _p(col), nb.value, C.byref(nb))
    assert rc == 0
    return row, col[: nb.value]


def bc_codes(g, bc) -> np.ndarray:
    """Per-DOF boundary codes uint8[N, 3] from a ``pd_workloads.BC``."""
    L = lib()
    G = make_grid(g)
    B = BC(bc.type, bc.grip_planes, (C.c_int32 * 2)(*bc.support_x2), bc.load_x2,
           bc.u_max, bc.n_ramp)
    out = np.zeros((g.nx * g.ny * g.nz, 3), np.uint8)
    rc = L.or_bc_codes(C.byref(G), C.byref(B), _p(out))
    assert rc == 0
    return out


def micromodulus(E: float, delta: float) -> float:
    return lib().or_micromodulus_3d(E, delta)


def gf_coefficient(law: int, c: float, delta: float, G_F: float, k: float = 25.0, alpha: float = 0.25) -> float:
    """A of s_crit = s0 + A / s0 for a fracture energy G_F (or_gf_coefficient)."""
    return lib().or_gf_coefficient(law, c, delta, G_F, k, alpha)


def fracture_energy(law: int, c: float, delta: float, s0: float, sc: float, k: float = 25.0,
                    alpha: float = 0.25) -> float:
    """G_F of Eq. exp_fracture_energy (exp-linear) or of the bilinear law."""
    return lib().or_fracture_energy(law, c, delta, s0, sc, k, alpha)


def damage_law(law: int, s: float, s0: float, sc: float, k: float = 25.0,
               alpha: float = 0.25) -> float:
    return lib().or_damage_law(law, s, s0, sc, k, alpha)


def stable_dt(g, row, col, c, rho, safety, vol=0.0):
    G = make_grid(g)
    if vol > 0:
        return lib().or_stable_dt_vol(C.byref(G), _p(row), _p(col), c, rho, safety, vol)
    return lib().or_stable_dt(C.byref(G), _p(row), _p(col), c, rho, safety)


def micromodulus_2d(E: float, delta: float, t: float, plane_strain: bool) -> float:
    return lib().or_micromodulus_2d(E, delta, t, 1 if plane_strain else 0)


def gf_coefficient_2d(law: int, c: float, delta: float, t: float, G_F: float, k: float = 25.0,
                      alpha: float = 0.25) -> float:
    return lib().or_gf_coefficient_2d(law, c, delta, t, G_F, k, alpha)


class Model:
    """One mesh + material + boundary set-up of the oracle (owns its arrays)."""

    def __init__(self, w, row=None, col=None, s0=None, kappa=None, dt=None):
        g, m, bc = w.grid, w.mat, w.bc
        self.w = w
        if row is None:
            row, col = neighbours(g)
        self.row, self.col = np.ascontiguousarray(row), np.ascontiguousarray(col)
        self.n = g.nx * g.ny * g.nz
        self.nb = int(self.row[-1])
        model = getattr(m, "model", 0)
        if model == 0:
            self.c = micromodulus(m.E, g.m_ratio * g.dx)
            self.vol = 0.0
        else:
            self.c = micromodulus_2d(m.E, g.m_ratio * g.dx, m.thickness, model == 2)
            self.vol = g.dx * g.dx * m.thickness
        self.codes = np.ascontiguousarray(bc_codes(g, bc))
        self.dt = stable_dt(g, self.row, self.col, self.c, m.rho, m.dt_safety, self.vol) if dt is None else dt
        self.s0 = np.ascontiguousarray(
            np.full(self.n, np.float32(m.s0), np.float64) if s0 is None else np.asarray(s0, np.float64))
        self.kappa = None if kappa is None else np.ascontiguousarray(np.asarray(kappa, np.float64))
        self._mk()

    def _mk(self):
        g, m, bc = self.w.grid, self.w.mat, self.w.bc
        if m.G_F <= 0:
            gfA = 0.0
        elif getattr(m, "model", 0) == 0:
            gfA = gf_coefficient(m.law, self.c, g.m_ratio * g.dx, m.G_F, m.k, m.alpha)
        else:
            gfA = gf_coefficient_2d(m.law, self.c, g.m_ratio * g.dx, m.thickness, m.G_F, m.k, m.alpha)
        self.P = Problem(g.nx, g.ny, g.nz, g.dx, _p(self.row), _p(self.col), self.c, m.rho,
                         m.law, m.s_ratio, m.k, m.alpha, self.dt, m.zeta, _p(self.s0),
                         _p(self.kappa), _p(self.codes), bc.u_max, bc.n_ramp, gfA, self.vol)

    def set_field(self, s0, kappa=None):
        self.s0 = np.ascontiguousarray(np.asarray(s0, np.float64))
        self.kappa = None if kappa is None else np.ascontiguousarray(np.asarray(kappa, np.float64))
        self._mk()

    def zero_state(self):
        return (np.zeros((self.n, 3)), np.zeros((self.n, 3)), np.zeros(self.nb))

    def force(self, u, d):
        """F (N x 3) for displacement u and damage d (updated copy returned)."""
        u = np.ascontiguousarray(u, np.float64)
        d = np.array(d, np.float64, copy=True)
        F = np.zeros((self.n, 3))
        sm = C.c_double(0.0)
        lib().or_force(C.byref(self.P), _p(u), _p(d), _p(F), C.cast(C.pointer(sm), C.c_void_p))
        return F, d, sm.value

    def run(self, n_steps, state=None, step0=0, use_stop=False, peak=-np.inf, peak_step=-1):
        """Run n_steps from ``state`` = (u, v, d) (copied). Returns a dict."""
        u, v, d = self.zero_state() if state is None else [np.array(a, np.float64, copy=True)
                                                             for a in state]
        R = np.zeros(n_steps)
        sm = np.zeros(n_steps)
        pk = C.c_double(peak)
        ps = C.c_int32(peak_step)
        nd = C.c_int32(0)
        lib().or_run(C.byref(self.P), step0, n_steps, 1 if use_stop else 0, _p(u), _p(v),
                     _p(d), _p(R), _p(sm), C.byref(pk), C.byref(ps), C.byref(nd))
        k = nd.value
        return dict(u=u, v=v, d=d, reaction=R[:k], smax=sm[:k], peak=pk.value,
                    peak_step=ps.value, n_done=k)


    def adjoint(self, n_steps, obs_steps, weights):
        """Gradient of J = sum_o weights[o] R^{obs_steps[o]} over n_steps steps from the
        zero state with respect to the node fields s0 and (when set) kappa."""
        obs = np.ascontiguousarray(np.asarray(obs_steps, np.int32))
        wts = np.ascontiguousarray(np.asarray(weights, np.float64))
        gs = np.zeros(self.n)
        gk = np.zeros(self.n) if self.kappa is not None else None
        rc = lib().or_adjoint(C.byref(self.P), n_steps, obs.size, _p(obs), _p(wts), _p(gs), _p(gk))
        if rc != 0:
            raise RuntimeError(f"or_adjoint failed ({rc})")
        return gs, gk


def run_batch(model: Model, s0, n_steps, use_stop=True, kappa=None):
    """Independent samples (rows of s0, B x N) on OpenMP threads."""
    s0 = np.ascontiguousarray(np.asarray(s0, np.float64))
    B = s0.shape[0]
    n, nb = model.n, model.nb
    u = np.zeros((B, n, 3))
    v = np.zeros((B, n, 3))
    d = np.zeros((B, nb))
    pk = np.zeros(B)
    ps = np.zeros(B, np.int32)
    nd = np.zeros(B, np.int32)
    kap = None if kappa is None else np.ascontiguousarray(np.asarray(kappa, np.float64))
    lib().or_run_batch(C.byref(model.P), B, nb, _p(s0), _p(kap), n_steps, 1 if use_stop else 0,
                       _p(u), _p(v), _p(d), _p(pk), _p(ps), _p(nd))
    return dict(u=u, v=v, d=d, peak=pk, peak_step=ps, n_done=nd)


def max_threads() -> int:
    return lib().or_max_threads()
