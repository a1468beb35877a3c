"""Synthetic workload recipes and seeded input generators.

This module is shared by the CUDA path and by the FP64 oracle. It holds the
problem *statements* (grid sizes, material constants, boundary-condition
geometry, random-field settings, run lengths, seeds) and seeded generators of
arbitrary states for parity tests. It holds none of the method's arithmetic:
no neighbour search, no bond law, no integrator, no KL basis, no estimator.

Geometry is stated in integer "half-cell" units where the method needs exact
comparisons: a node with grid index ``ix`` sits at ``X = 2*ix + 1`` half-cells
(x = (ix + 1/2) dx), so a plane on a cell face has an even half-cell
coordinate and a plane through node centres an odd one.

Workloads (the paper's own experiments are 2D Gregoire-2013 concrete beams
with fib-derived properties, Section 6; neither the experimental data nor the
fib formulas are available, so synthetic 3D stand-ins with the paper's shapes
are used):

* ``bar``   -- 40x10x10 nodes, dx = 1 mm, uniaxial tension, FP64 path.
* ``beam``  -- notched three-point-bending beam 175x50x50 mm, dx = 2.5 mm,
               notch depth 0.2 D at mid-span, lognormal strength field.
* ``beam_levels(l)`` -- the same beam at dx = 5 / 2.5 / 1.25 mm (MLMC levels).
* ``sweep(D)`` -- geometrically similar notched beams of depth D.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np

# bond-law identifiers (shared numbering with the C ABI header)
LAW_BILINEAR = 0
LAW_EXPLINEAR = 1

# boundary-condition families
BC_BAR_TENSION = 1
BC_BEAM_3PT = 2

# per-DOF boundary codes
DOF_FREE = 0
DOF_FIXED = 1
DOF_PLUS = 2   # prescribed +U(n)
DOF_MINUS = 3  # prescribed -U(n)

# covariance kernels
COV_SQEXP = 0   # exp(-r^2 / l^2)
COV_EXP = 1     # exp(-r / l)  (the paper's Eq. for the exponential correlation)

MARG_LOGNORMAL = 0
MARG_WEIBULL = 1
MODEL_3D = 0
MODEL_PLANE_STRESS = 1
MODEL_PLANE_STRAIN = 2


@dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    nz: int
    dx: float            # node spacing [m]
    m_ratio: float       # horizon delta = m_ratio * dx
    notch: int = 0       # 1 if a notch plane is present
    notch_x2: int = 0    # notch plane x in half-cells (2 x / dx)
    notch_y2: int = 0    # notch depth from y = 0 in half-cells (2 a / dx)

    @property
    def n_nodes(self) -> int:
        return self.nx * self.ny * self.nz


@dataclass(frozen=True)
class Material:
    E: float = 30e9             # Young's modulus [Pa]
    rho: float = 2346.0         # density [kg/m^3] (Section 6.2)
    law: int = LAW_BILINEAR
    s0: float = 1e-4            # linear elastic limit stretch (mean of field)
    s_ratio: float = 10.0       # sf/s0 (bilinear) or sc/s0 (exp-linear)
    k: float = 25.0             # exp-linear decay rate (Section 6.2)
    alpha: float = 0.25         # exp-linear transition (Section 6.2)
    dt_safety: float = 0.5      # fraction of the stable time step
    zeta: float = 0.0           # mass-proportional damping rate [1/s]
    G_F: float = 0.0            # fracture energy [N/m]; > 0: s_crit from G_F per bond, s_ratio unused
    model: int = 0              # MODEL_3D, MODEL_PLANE_STRESS or MODEL_PLANE_STRAIN (grid with nz = 1)
    thickness: float = 0.0      # plane models: out-of-plane thickness t [m]


@dataclass(frozen=True)
class BC:
    type: int
    u_max: float                # prescribed displacement at the end of the ramp [m]
    n_ramp: int                 # steps of the linear ramp
    grip_planes: int = 3        # bar: node planes held at each end
    support_x2: tuple = (0, 0)  # beam: support lines, half-cells
    load_x2: int = 0            # beam: load line, half-cells


@dataclass(frozen=True)
class FieldCfg:
    kernel: int = COV_SQEXP
    length: float = 10e-3       # correlation length [m]
    n_modes: int = 64
    marginal: int = MARG_LOGNORMAL
    mean: float = 1e-4
    cov: float = 0.1            # coefficient of variation
    weibull_m: float = 3.0      # Weibull modulus (Section 6.2), when marginal = Weibull


@dataclass(frozen=True)
class Workload:
    name: str
    grid: Grid
    mat: Material
    bc: BC
    n_steps: int
    field: FieldCfg | None = None
    seed: int = 0
    batch: int = 1
    fp64: bool = False          # True: FP64 bond arithmetic; False: FP32 bonds, FP64 sums


def bar() -> Workload:
    """3D bar 40x10x10 nodes, dx = 1 mm, delta = 3.01 dx, bilinear law, 1,000 steps."""
    g = Grid(40, 10, 10, 1e-3, 3.01)
    mat = Material(E=30e9, law=LAW_BILINEAR, s0=1e-4, s_ratio=10.0, zeta=0.0)
    bc = BC(BC_BAR_TENSION, u_max=1.5e-5, n_ramp=1000, grip_planes=3)
    return Workload("bar_40x10x10_dx1mm", g, mat, bc, n_steps=1000, fp64=True)


def _beam_grid(D_mm: float, dx_mm: float, length_mm: float, thick_mm: float,
               notch: bool) -> Grid:
    nx = round(length_mm / dx_mm)
    ny = round(D_mm / dx_mm)
    nz = round(thick_mm / dx_mm)
    x_notch = length_mm / 2.0
    depth = 0.2 * D_mm
    return Grid(nx, ny, nz, dx_mm * 1e-3, 3.01, 1 if notch else 0,
                round(2 * x_notch / dx_mm), round(2 * depth / dx_mm))


def beam(dx_mm: float = 2.5, n_steps: int = 5000, seed: int = 1,
         law: int = LAW_BILINEAR) -> Workload:
    """Notched 3-point-bending beam 175x50x50 mm; span 2.5 D (the paper's span/depth, Section 6.2)."""
    D, L, T = 50.0, 175.0, 50.0
    g = _beam_grid(D, dx_mm, L, T, True)
    span = 2.5 * D
    sx = ((L - span) / 2.0, (L + span) / 2.0)
    bc = BC(BC_BEAM_3PT, u_max=4e-5, n_ramp=n_steps,
            support_x2=(round(2 * sx[0] / dx_mm), round(2 * sx[1] / dx_mm)),
            load_x2=round(2 * (L / 2.0) / dx_mm))
    s_ratio = 10.0 if law == LAW_BILINEAR else 25.0
    mat = Material(E=30e9, law=law, s0=1e-4, s_ratio=s_ratio, zeta=5e4)
    fld = FieldCfg(COV_SQEXP, 10e-3, 64, MARG_LOGNORMAL, 1e-4, 0.1)
    return Workload(f"notched_beam_175x50x50_dx{dx_mm}mm", g, mat, bc, n_steps, fld, seed)


def beam_type1(dx_mm: float = 2.5, n_steps: int = 5000, seed: int = 5, G_F: float = 20.0) -> Workload:
    """Unnotched (Type 1) three-point-bending beam 175x50x50 mm (Section 6.3's
    specimen type), exp-linear law with the critical stretch calibrated per
    bond from a fracture energy G_F [N/m] (Appendix A), same strength field."""
    D, L, T = 50.0, 175.0, 50.0
    g = _beam_grid(D, dx_mm, L, T, False)
    span = 2.5 * D
    sx = ((L - span) / 2.0, (L + span) / 2.0)
    bc = BC(BC_BEAM_3PT, u_max=6e-5, n_ramp=n_steps,
            support_x2=(round(2 * sx[0] / dx_mm), round(2 * sx[1] / dx_mm)),
            load_x2=round(2 * (L / 2.0) / dx_mm))
    mat = Material(E=30e9, law=LAW_EXPLINEAR, s0=1e-4, s_ratio=25.0, zeta=5e4, G_F=G_F)
    fld = FieldCfg(COV_SQEXP, 10e-3, 64, MARG_LOGNORMAL, 1e-4, 0.1)
    return Workload(f"unnotched_beam_175x50x50_dx{dx_mm}mm_GF{G_F:g}", g, mat, bc, n_steps, fld, seed)


def beam_levels():
    """MLMC hierarchy: the notched beam at dx = 5 / 2.5 / 1.25 mm; N_l = 1024 / 128 / 16.

    The ramp is scaled with the level so that the physical loading rate is the
    same on every level (the stable time step halves with dx)."""
    out = []
    for lvl, (dxm, nl) in enumerate(((5.0, 1024), (2.5, 128), (1.25, 16))):
        w = beam(dxm, n_steps=2500 * (2 ** lvl), seed=2)
        out.append(dataclasses.replace(w, batch=nl))
    return out


def small_beam_levels():
    """A two-level hierarchy of a small notched beam (80 x 25 x 10 mm, span 2.5 D,
    notch 0.2 D) at dx = 5 / 2.5 mm, for MLMC parity against the oracle:
    N_l = 6 / 4 samples, 600 / 1200 steps, the ramp scaled as in ``beam_levels``."""
    D, L, T = 25.0, 80.0, 10.0
    out = []
    for lvl, (dxm, nl) in enumerate(((5.0, 6), (2.5, 4))):
        n_steps = 600 * (2 ** lvl)
        g = _beam_grid(D, dxm, L, T, True)
        span = 2.5 * D
        sx = ((L - span) / 2.0, (L + span) / 2.0)
        bc = BC(BC_BEAM_3PT, u_max=2.5e-5, n_ramp=n_steps,
                support_x2=(round(2 * sx[0] / dxm), round(2 * sx[1] / dxm)),
                load_x2=round(2 * (L / 2.0) / dxm))
        mat = Material(E=30e9, law=LAW_BILINEAR, s0=1e-4, s_ratio=10.0, zeta=5e4)
        fld = FieldCfg(COV_SQEXP, 5e-3, 16, MARG_LOGNORMAL, 1e-4, 0.1)
        out.append(Workload(f"small_beam_80x25x10_dx{dxm}mm", g, mat, bc, n_steps, fld, 3, batch=nl))
    return out


def small_plane_levels(u_max: float = 3e-5):
    """A two-level plane-stress hierarchy (the paper's dimensionality): a notched
    80 x 25 mm beam, t = 50 mm, delta = pi dx, dx = 5 / 2.5 mm (16 x 5 and
    32 x 10 nodes), exp-linear law calibrated to G_F = 30 N/m, 6 / 4 samples,
    600 / 1200 steps (the ramp scaled with the level)."""
    import math
    D, L = 25.0, 80.0
    out = []
    for lvl, (dxm, nl) in enumerate(((5.0, 6), (2.5, 4))):
        n_steps = 600 * (2 ** lvl)
        nx, ny = round(L / dxm), round(D / dxm)
        g = Grid(nx, ny, 1, dxm * 1e-3, math.pi, 1, nx, round(2 * 0.2 * D / dxm))
        span = 2.5 * D
        sx = ((L - span) / 2.0, (L + span) / 2.0)
        bc = BC(BC_BEAM_3PT, u_max=u_max, n_ramp=n_steps,
                support_x2=(round(2 * sx[0] / dxm), round(2 * sx[1] / dxm)), load_x2=nx)
        mat = Material(E=30e9, law=LAW_EXPLINEAR, s0=1e-4, zeta=5e4, G_F=30.0, model=MODEL_PLANE_STRESS,
                       thickness=0.05)
        fld = FieldCfg(COV_SQEXP, 5e-3, 16, MARG_LOGNORMAL, 1e-4, 0.1)
        out.append(Workload(f"small_plane_beam_80x25_dx{dxm}mm", g, mat, bc, n_steps, fld, 3, batch=nl))
    return out


def sweep(D_mm: float, dx_mm: float = 2.5, n_steps: int = 5000) -> Workload:
    """Size-effect sweep member: depth D, span 3 D, length 3.5 D, thickness 50 mm."""
    L, T = 3.5 * D_mm, 50.0
    g = _beam_grid(D_mm, dx_mm, L, T, True)
    span = 3.0 * D_mm
    sx = ((L - span) / 2.0, (L + span) / 2.0)
    bc = BC(BC_BEAM_3PT, u_max=4e-5 * D_mm / 50.0, n_ramp=n_steps,
            support_x2=(round(2 * sx[0] / dx_mm), round(2 * sx[1] / dx_mm)),
            load_x2=round(2 * (L / 2.0) / dx_mm))
    mat = Material(E=30e9, law=LAW_BILINEAR, s0=1e-4, s_ratio=10.0, zeta=5e4 * 50.0 / D_mm)
    fld = FieldCfg(COV_SQEXP, 10e-3, 64, MARG_LOGNORMAL, 1e-4, 0.1)
    return Workload(f"sweep_D{int(D_mm)}mm_dx{dx_mm}mm", g, mat, bc, n_steps, fld, 3, 64)


def tiny_beam(nx=16, ny=6, nz=4, notch=True, dx_mm=2.5, n_steps=400) -> Workload:
    """A small notched beam for oracle-speed parity cases (several tiles plus a ragged tail)."""
    L, D, T = nx * dx_mm, ny * dx_mm, nz * dx_mm
    g = Grid(nx, ny, nz, dx_mm * 1e-3, 3.01, 1 if notch else 0, nx, 2)
    bc = BC(BC_BEAM_3PT, u_max=3e-6, n_ramp=n_steps,
            support_x2=(round(2 * 0.1 * L / dx_mm), round(2 * 0.9 * L / dx_mm)),
            load_x2=nx)
    mat = Material(E=30e9, law=LAW_BILINEAR, s0=1e-4, s_ratio=10.0, zeta=5e4)
    fld = FieldCfg(COV_SQEXP, 4 * dx_mm * 1e-3, 16, MARG_LOGNORMAL, 1e-4, 0.1)
    return Workload(f"tiny_beam_{nx}x{ny}x{nz}", g, mat, bc, n_steps, fld, 7)


# ---------------------------------------------------------------------------
# seeded generators of arbitrary states (inputs for parity tests only)
# ---------------------------------------------------------------------------

def random_state(n_nodes: int, batch: int, seed: int, u_scale: float = 1e-7):
    """Random displacements and velocities for single-step parity tests.

    Returns (u [B,N,3] f64, v [B,N,3] f64). Damage for such tests comes from
    ``pair_damage`` so that both directed copies of a bond agree.
    """
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((batch, n_nodes, 3)) * u_scale
    v = rng.standard_normal((batch, n_nodes, 3)) * 1e-3
    return u, v


def pair_damage(i: np.ndarray, j: np.ndarray, seed: int, batch: int,
                frac: float = 0.2) -> np.ndarray:
    """Damage in [0, 1) per directed bond (i -> j), symmetric in (i, j).

    A bond keyed by (min(i,j), max(i,j)) gets the same value in both directions.
    Roughly ``frac`` of bonds are damaged; the values are plain hash-derived numbers.
    """
    lo = np.minimum(i, j).astype(np.uint64)
    hi = np.maximum(i, j).astype(np.uint64)
    out = np.zeros((batch, i.size), dtype=np.float64)
    for b in range(batch):
        key = lo * np.uint64(2654435761) ^ (hi * np.uint64(40503) + np.uint64(seed * 7919 + b))
        key = (key ^ (key >> np.uint64(13))) * np.uint64(0x5bd1e995)
        key = key ^ (key >> np.uint64(15))
        r = (key % np.uint64(1 << 24)).astype(np.float64) / float(1 << 24)
        dmg = (r < frac)
        val = ((key >> np.uint64(24)) % np.uint64(1 << 20)).astype(np.float64) / float(1 << 20)
        out[b] = np.where(dmg, val, 0.0)
    return out


def lognormal_like_field(n_nodes: int, batch: int, seed: int, mean=1e-4, cov=0.1):
    """An arbitrary positive per-node strength field (not a KL sample) as FP32."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((batch, n_nodes))
    return (mean * np.exp(cov * g)).astype(np.float32)
