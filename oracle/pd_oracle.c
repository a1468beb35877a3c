/*
 * pd_oracle.c -- plain, slow FP64 reference of the bond-based peridynamic
 * explicit time step (Sections 2-3 and Appendix A of arXiv 2212.04415).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do. It shares no code, header, table or constant with the
 * CUDA path.
 *
 * Everything is written in the order the method states it, in double
 * precision, with one loop per definition and no blocking or fusion:
 *
 *   horizon        H_x = { x' : |x' - x| <= delta }                    (Eq. PD_Horizon)
 *   pair force     f = f(|xi+eta|, xi) (xi+eta)/|xi+eta|                (Eq. PD_Force_Function)
 *   stretch        s = (|xi+eta| - |xi|) / |xi|                          (Section 2.1)
 *   bond force     f = c (1 - d) s                                      (Eq. exp_scalar_force)
 *   micromodulus   c = 12 E / (pi delta^4)  (3D)                         (Eq. bond_stiffness_constant)
 *   softening      exponential-linear d(s)                              (Eq. exp_damage_parameter)
 *   motion         rho u'' = sum_j f_ij V_j + b                          (Eq. PD_EOM_Dynamic)
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - nodes sit at cell centres of a regular grid, V_j = dx^3, no surface
 *     or partial-volume correction;
 *   - the notch removes a bond whose segment strictly crosses the notch plane
 *     below the notch tip (a crossing exactly at the tip is kept);
 *   - the bilinear law d = 1 - s0 (sf - s) / (s (sf - s0)) on (s0, sf);
 *   - irreversibility d_n = max(d_{n-1}, d_law(s_n)); compression uses the
 *     stored d;
 *   - per-bond properties s0_ij = (s0_i + s0_j)/2, s_crit_ij = ratio * s0_ij
 *     or, calibrated to a fracture energy G_F, s_crit_ij = s0_ij + A / s0_ij
 *     (Eq. exp_fracture_energy solved for s_c; see or_gf_coefficient),
 *     c_ij = c (kappa_i + kappa_j)/2;
 *   - damped leapfrog (velocity-Verlet positions) integrator with
 *     mass-proportional damping zeta; stable step from the Silling-Askari
 *     bound dt_i = sqrt(2 rho / sum_j c V / |xi|) scaled by a safety factor;
 *   - displacement control U(n) = u_max * min(n, n_ramp) / n_ramp;
 *   - reaction R_n = -sum over prescribed DOFs of F * sign * V; peak load
 *     Q = max_n R_n (first step attaining it); optional stop once
 *     R_n < Q/2 and at least 100 steps have passed since the peak.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG -1
#define OR_ERR_CAP -2

typedef struct {
    int32_t nx, ny, nz;
    double dx;
    double m_ratio;
    int32_t notch;     /* 1 if the notch plane is present */
    int32_t notch_x2;  /* notch plane x, in half-cells */
    int32_t notch_y2;  /* notch depth from y = 0, in half-cells */
} or_grid;

typedef struct {
    int32_t type;        /* 1 bar tension (+x), 2 three-point bending (-y) */
    int32_t grip_planes; /* bar */
    int32_t support_x2[2];
    int32_t load_x2;
    double u_max;
    int32_t n_ramp;
} or_bc;

typedef struct {
    int32_t nx, ny, nz;
    double dx;
    const int32_t *row_ptr;
    const int32_t *col;
    double c;          /* micromodulus */
    double rho;
    int32_t law;       /* 0 bilinear, 1 exponential-linear */
    double s_ratio;    /* s_crit / s0 */
    double k, alpha;   /* exponential-linear parameters */
    double dt, zeta;
    const double *s0;     /* per-node linear-limit stretch, N */
    const double *kappa;  /* per-node stiffness multiplier, N, or NULL */
    const uint8_t *bc;    /* per-DOF codes, N*3: 0 free, 1 fixed, 2 +U(n), 3 -U(n) */
    double u_max;
    int32_t n_ramp;
    double gf_A;          /* > 0: s_crit = s0 + gf_A / s0 (from the fracture energy,
                             or_gf_coefficient); 0: s_crit = s_ratio * s0 */
    double vol;           /* node volume; 0: dx^3 (3D). Plane models: dx^2 t */
} or_problem;

/* ---------------------------------------------------------------- grid */

static void node_xyz(const or_grid *g, int64_t i, double *x) {
    int64_t ix = i % g->nx;
    int64_t iy = (i / g->nx) % g->ny;
    int64_t iz = i / ((int64_t)g->nx * g->ny);
    x[0] = (ix + 0.5) * g->dx;
    x[1] = (iy + 0.5) * g->dx;
    x[2] = (iz + 0.5) * g->dx;
}

/* Half-cell integer coordinates of node i: X = 2 ix + 1. */
static void node_half(const or_grid *g, int64_t i, int64_t *X) {
    int64_t ix = i % g->nx;
    int64_t iy = (i / g->nx) % g->ny;
    int64_t iz = i / ((int64_t)g->nx * g->ny);
    X[0] = 2 * ix + 1;
    X[1] = 2 * iy + 1;
    X[2] = 2 * iz + 1;
}

/* Is the pair (i, j) in the horizon: |x_j - x_i| <= m dx (Eq. PD_Horizon).
 * Offsets are whole numbers of cells, so the squared distance in cell units
 * is an exact integer; compare it with m^2 in double. */
static int in_horizon(const or_grid *g, int64_t i, int64_t j) {
    int64_t a[3], b[3];
    node_half(g, i, a);
    node_half(g, j, b);
    double d2 = 0.0;
    for (int c = 0; c < 3; ++c) {
        double o = (double)((b[c] - a[c]) / 2);
        d2 += o * o;
    }
    return d2 > 0.0 && d2 <= g->m_ratio * g->m_ratio;
}

/* Does the bond (i, j) cross the notch below its tip?  The notch is the
 * plane x = X_n (half-cells) for 0 <= y < Y_d, through the whole thickness.
 * The segment crosses iff (X_i - X_n)(X_j - X_n) < 0; the height where it
 * meets the plane is Y_i + (X_n - X_i)(Y_j - Y_i)/(X_j - X_i), compared with
 * Y_d exactly by cross-multiplying (integers only, so ties are exact). */
static int cut_by_notch(const or_grid *g, int64_t i, int64_t j) {
    if (!g->notch) return 0;
    int64_t a[3], b[3];
    node_half(g, i, a);
    node_half(g, j, b);
    int64_t Xn = g->notch_x2, Yd = g->notch_y2;
    if ((a[0] - Xn) * (b[0] - Xn) >= 0) return 0;
    int64_t dX = b[0] - a[0];
    int64_t num = a[1] * dX + (Xn - a[0]) * (b[1] - a[1]);  /* Y_cross * dX */
    int64_t rhs = Yd * dX;
    return dX > 0 ? (num < rhs) : (num > rhs);
}

/* Brute force over all O(N^2) pairs: the pin for the neighbour list. */
int or_build_bruteforce(const or_grid *g, int32_t *row_ptr, int32_t *col,
                        int64_t cap, int64_t *n_bonds) {
    int64_t n = (int64_t)g->nx * g->ny * g->nz;
    int64_t nb = 0;
    if (row_ptr) row_ptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            if (!in_horizon(g, i, j)) continue;
            if (cut_by_notch(g, i, j)) continue;
            if (col && nb < cap) col[nb] = (int32_t)j;
            ++nb;
        }
        if (row_ptr) row_ptr[i + 1] = (int32_t)nb;
    }
    *n_bonds = nb;
    return (col && nb > cap) ? OR_ERR_CAP : OR_OK;
}

/* The same list, scanning only the box of candidate cells within ceil(m)
 * of each node (faster for larger meshes; equal to the brute force above). */
int or_build_window(const or_grid *g, int32_t *row_ptr, int32_t *col,
                    int64_t cap, int64_t *n_bonds) {
    int64_t nx = g->nx, ny = g->ny, nz = g->nz;
    int64_t n = nx * ny * nz;
    int r = (int)ceil(g->m_ratio);
    int64_t nb = 0;
    if (row_ptr) row_ptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
        /* candidates in ascending linear index: z, then y, then x */
        for (int64_t jz = iz - r; jz <= iz + r; ++jz) {
            if (jz < 0 || jz >= nz) continue;
            for (int64_t jy = iy - r; jy <= iy + r; ++jy) {
                if (jy < 0 || jy >= ny) continue;
                for (int64_t jx = ix - r; jx <= ix + r; ++jx) {
                    if (jx < 0 || jx >= nx) continue;
                    int64_t j = jx + nx * (jy + ny * jz);
                    if (j == i) continue;
                    if (!in_horizon(g, i, j)) continue;
                    if (cut_by_notch(g, i, j)) continue;
                    if (col && nb < cap) col[nb] = (int32_t)j;
                    ++nb;
                }
            }
        }
        if (row_ptr) row_ptr[i + 1] = (int32_t)nb;
    }
    *n_bonds = nb;
    return (col && nb > cap) ? OR_ERR_CAP : OR_OK;
}

/* ---------------------------------------------------------- boundaries */

/* Per-DOF codes from the boundary description.
 * Bar (type 1): the first grip_planes x-planes fixed in all components; the
 * last grip_planes x-planes carry +U(n) along x and are held in y and z.
 * Beam (type 2): support lines = bottom layer (iy = 0) nodes whose centre is
 * within half a cell of a support x (both columns on a tie), fixed in y;
 * load line = top layer nodes within half a cell of the load x, carrying
 * -U(n) along y. */
int or_bc_codes(const or_grid *g, const or_bc *bc, uint8_t *codes) {
    int64_t nx = g->nx, ny = g->ny, nz = g->nz;
    int64_t n = nx * ny * nz;
    memset(codes, 0, (size_t)(3 * n));
    for (int64_t i = 0; i < n; ++i) {
        int64_t ix = i % nx, iy = (i / nx) % ny;
        int64_t X = 2 * ix + 1;
        if (bc->type == 1) {
            if (ix < bc->grip_planes) {
                codes[3 * i + 0] = 1;
                codes[3 * i + 1] = 1;
                codes[3 * i + 2] = 1;
            } else if (ix >= nx - bc->grip_planes) {
                codes[3 * i + 0] = 2;
                codes[3 * i + 1] = 1;
                codes[3 * i + 2] = 1;
            }
        } else if (bc->type == 2) {
            if (iy == 0) {
                for (int s = 0; s < 2; ++s) {
                    int64_t d = X - bc->support_x2[s];
                    if (d >= -1 && d <= 1) codes[3 * i + 1] = 1;
                }
            }
            if (iy == ny - 1) {
                int64_t d = X - bc->load_x2;
                if (d >= -1 && d <= 1) codes[3 * i + 1] = 3;
            }
        } else {
            return OR_ERR_ARG;
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------ material */

/* c = 12 E / (pi delta^4) in 3D (Eq. bond_stiffness_constant). */
double or_micromodulus_3d(double E, double delta) {
    return 12.0 * E / (M_PI * delta * delta * delta * delta);
}

/* Softening parameter of one bond for a stretch s above the elastic limit.
 * law 0 (bilinear): force falls linearly from c s0 at s0 to 0 at sf.
 * law 1 (exponential-linear, Eq. exp_damage_parameter). */
double or_damage_law(int32_t law, double s, double s0, double sc,
                     double k, double alpha) {
    if (s <= s0) return 0.0;
    if (s >= sc) return 1.0;
    if (law == 0) {
        return 1.0 - s0 * (sc - s) / (s * (sc - s0));
    }
    double t = (s - s0) / (sc - s0);
    double bracket = 1.0 - (1.0 - exp(-k * t)) / (1.0 - exp(-k)) + alpha * (1.0 - t);
    return 1.0 - (s0 / s) * bracket / (1.0 + alpha);
}

/* Plane models (Eq. bond_stiffness_constant): c = 9E / (pi t delta^3) for
 * plane stress, 48E / (5 pi t delta^3) for plane strain; t the thickness. The
 * grid has one node layer (nz = 1) and every node volume is dx^2 t. */
double or_micromodulus_2d(double E, double delta, double t, int32_t plane_strain) {
    double d3 = delta * delta * delta;
    return plane_strain ? 48.0 * E / (5.0 * M_PI * t * d3) : 9.0 * E / (M_PI * t * d3);
}

/* Two-dimensional calibration, Eq. exp_sc_2D as printed (it is consistent
 * with Eq. exp_fracture_energy_2D): its G_F term over s0 is A of
 * s_c = s0 + A / s0; for the bilinear law the same construction
 * (G_F = h c s0 delta^4 (s_c - s0) / 4) gives A = 4 G_F / (h c delta^4). */
double or_gf_coefficient_2d(int32_t law, double c, double delta, double h, double G_F, double k, double alpha) {
    double d4 = delta * delta * delta * delta;
    if (law == 0) return 4.0 * G_F / (h * c * d4);
    double ek = exp(k);
    double P = 2.0 * k - 2.0 * ek + alpha * k - alpha * k * ek + 2.0;
    return 4.0 * k * (1.0 - ek) * (1.0 + alpha) * G_F / (h * c * d4 * P);
}

/* Fracture-energy calibration of the critical stretch. The energy a bond
 * absorbs while softening, w = xi * int_{s0}^{s_c} f ds (Eq. exp_bond_energy),
 * integrated over the bonds crossing a unit area of a plane (the quadruple
 * integral of the three-dimensional case, equal to pi delta^5 / 5 times the
 * coefficient of xi in w) gives G_F:
 *   exp-linear (Eq. exp_fracture_energy):
 *     G_F = pi c s0 delta^5 (s0 - s_c) P / (10 k (e^k - 1) (1 + alpha)),
 *     P = 2k - 2e^k + alpha k - alpha k e^k + 2;
 *   bilinear (force c s0 at s0 falling linearly to 0 at s_c, w = c s0 xi (s_c - s0)/2):
 *     G_F = pi c s0 delta^5 (s_c - s0) / 10.
 * Both solve to s_c = s0 + A / s0; this returns A. Reading: the printed
 * Eq. exp_sc has (1 + alpha) s0 where Eq. exp_fracture_energy gives s0 (the
 * two-dimensional Eq. exp_sc_2D is consistent); the form that satisfies
 * Eq. exp_fracture_energy is used. */
double or_gf_coefficient(int32_t law, double c, double delta, double G_F, double k, double alpha) {
    double d5 = delta * delta * delta * delta * delta;
    if (law == 0) return 10.0 * G_F / (M_PI * c * d5);
    double ek = exp(k);
    double P = 2.0 * k - 2.0 * ek + alpha * k - alpha * k * ek + 2.0;
    return -10.0 * k * (ek - 1.0) * (1.0 + alpha) * G_F / (M_PI * c * d5 * P);
}

/* G_F of a bond family with elastic limit s0 and critical stretch s_c (the
 * closed forms above, before solving for s_c). */
double or_fracture_energy(int32_t law, double c, double delta, double s0, double sc, double k, double alpha) {
    double d5 = delta * delta * delta * delta * delta;
    if (law == 0) return M_PI * c * s0 * d5 * (sc - s0) / 10.0;
    double ek = exp(k);
    double P = 2.0 * k - 2.0 * ek + alpha * k - alpha * k * ek + 2.0;
    return M_PI * c * s0 * d5 * (s0 - sc) * P / (10.0 * k * (ek - 1.0) * (1.0 + alpha));
}

/* Stable time step, Silling-Askari bound with uniform c, times safety. */
double or_stable_dt_vol(const or_grid *g, const int32_t *row_ptr, const int32_t *col,
                        double c, double rho, double safety, double V) {
    int64_t n = (int64_t)g->nx * g->ny * g->nz;
    double best = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        double xi_[3], xj[3];
        node_xyz(g, i, xi_);
        double sum = 0.0;
        for (int32_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            node_xyz(g, col[p], xj);
            double L = sqrt((xj[0] - xi_[0]) * (xj[0] - xi_[0]) +
                            (xj[1] - xi_[1]) * (xj[1] - xi_[1]) +
                            (xj[2] - xi_[2]) * (xj[2] - xi_[2]));
            sum += c * V / L;
        }
        if (sum > 0.0) {
            double dti = sqrt(2.0 * rho / sum);
            if (dti < best) best = dti;
        }
    }
    return safety * best;
}

double or_stable_dt(const or_grid *g, const int32_t *row_ptr, const int32_t *col,
                    double c, double rho, double safety) {
    return or_stable_dt_vol(g, row_ptr, col, c, rho, safety, g->dx * g->dx * g->dx);
}

/* ------------------------------------------------------------- forces */

/* Internal force density F_i = sum_j f_ij V_j (Eq. PD_EOM_Dynamic, b = 0),
 * updating the damage of every bond from the current stretch first.
 * u: N*3 displacements; d: bond damage, updated in place; F: N*3 out;
 * smax: largest stretch of any bond (out, may be NULL). */
static void forces(const or_problem *p, const double *u, double *d, double *F,
                   double *smax) {
    int64_t n = (int64_t)p->nx * p->ny * p->nz;
    or_grid g = {p->nx, p->ny, p->nz, p->dx, 0.0, 0, 0, 0};
    double V = p->vol > 0.0 ? p->vol : p->dx * p->dx * p->dx;
    /* Nodes are independent (each sums its own row in CSR order and updates
     * only its own bonds' damage), so the node loop may run on OpenMP threads
     * without changing a single bit; the largest stretch is taken per node
     * and reduced afterwards in node order. Inside or_run_batch's parallel
     * region this loop runs on the calling thread alone. */
    double *smn = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double sm = -INFINITY;
        double xi_[3];
        node_xyz(&g, i, xi_);
        double Fi[3] = {0.0, 0.0, 0.0};
        for (int32_t q = p->row_ptr[i]; q < p->row_ptr[i + 1]; ++q) {
            int64_t j = p->col[q];
            double xj[3];
            node_xyz(&g, j, xj);
            double xi[3], eta[3], y[3];
            for (int c = 0; c < 3; ++c) {
                xi[c] = xj[c] - xi_[c];
                eta[c] = u[3 * j + c] - u[3 * i + c];
                y[c] = xi[c] + eta[c];
            }
            double L0 = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
            double L = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
            double s = (L - L0) / L0;
            if (s > sm) sm = s;
            double s0 = 0.5 * (p->s0[i] + p->s0[j]);
            double sc = p->gf_A > 0.0 ? s0 + p->gf_A / s0 : p->s_ratio * s0;
            double dl = or_damage_law(p->law, s, s0, sc, p->k, p->alpha);
            if (dl > d[q]) d[q] = dl;
            double cij = p->c;
            if (p->kappa) cij = p->c * 0.5 * (p->kappa[i] + p->kappa[j]);
            double f = cij * (1.0 - d[q]) * s;
            /* A fully damaged bond carries no force (f = c (1 - d) s = 0, the
             * bond law of Appendix A): its direction y / L is not needed, and
             * it is undefined once the bond has collapsed to zero length. */
            if (d[q] < 1.0)
                for (int c = 0; c < 3; ++c) Fi[c] += f * V * y[c] / L;
        }
        for (int c = 0; c < 3; ++c) F[3 * i + c] = Fi[c];
        smn[i] = sm;
    }
    double sm = -INFINITY;
    for (int64_t i = 0; i < n; ++i)
        if (smn[i] > sm) sm = smn[i];
    free(smn);
    if (smax) *smax = sm;
}

/* Prescribed displacement magnitude at step n. */
static double ramp(const or_problem *p, int64_t n) {
    int64_t m = n < p->n_ramp ? n : p->n_ramp;
    return p->u_max * (double)m / (double)p->n_ramp;
}

/* One evaluation of the internal force density and damage update, without
 * time integration (for single-step parity cases). */
int or_force(const or_problem *p, const double *u, double *d, double *F,
             double *smax) {
    forces(p, u, d, F, smax);
    return OR_OK;
}

/* Run n_steps explicit steps starting at step index step0 from the state
 * (u = u^n, v = v^{n-1/2}, d = d^{n-1}) of ONE sample.
 *
 * For each step n:
 *   F^n from u^n (damage updated from the stretch of u^n first);
 *   R^n = -sum over prescribed DOFs of F^n * sign * V;
 *   free DOF:   v^{n+1/2} = ((1 - zeta dt/2) v^{n-1/2} + dt F^n / rho) / (1 + zeta dt/2)
 *               u^{n+1}   = u^n + dt v^{n+1/2}
 *   fixed DOF:  u = v = 0
 *   prescribed: u^{n+1} = sign U(n+1), v^{n+1/2} = sign (U(n+1) - U(n)) / dt
 *   peak:       if R^n > Q then Q = R^n, n_peak = n
 *   stop rule:  if use_stop and Q > 0 and n - n_peak >= 100 and R^n < Q/2, stop
 *               after this step.
 * reaction[k] and smax[k] (k = step count within the call) are written when
 * non-NULL. peak/peak_step hold the running maximum on entry and exit (pass
 * -inf / -1 to start fresh). */
int or_run(const or_problem *p, int32_t step0, int32_t n_steps, int32_t use_stop,
           double *u, double *v, double *d, double *reaction, double *smax,
           double *peak, int32_t *peak_step, int32_t *n_done) {
    int64_t n = (int64_t)p->nx * p->ny * p->nz;
    double V = p->vol > 0.0 ? p->vol : p->dx * p->dx * p->dx;
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    if (!F) return OR_ERR_ARG;
    double Q = *peak;
    int32_t npk = *peak_step;
    int32_t done = 0;
    for (int32_t k = 0; k < n_steps; ++k) {
        int64_t step = (int64_t)step0 + k;
        double sm;
        forces(p, u, d, F, &sm);
        double R = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            for (int c = 0; c < 3; ++c) {
                uint8_t code = p->bc[3 * i + c];
                if (code == 2) R -= F[3 * i + c] * V;
                if (code == 3) R += F[3 * i + c] * V;
            }
        }
        if (reaction) reaction[k] = R;
        if (smax) smax[k] = sm;
        double Un = ramp(p, step), Un1 = ramp(p, step + 1);
        double a = 1.0 - 0.5 * p->zeta * p->dt;
        double b = 1.0 + 0.5 * p->zeta * p->dt;
        for (int64_t i = 0; i < n; ++i) {
            for (int c = 0; c < 3; ++c) {
                int64_t q = 3 * i + c;
                uint8_t code = p->bc[q];
                if (code == 0) {
                    v[q] = (a * v[q] + p->dt * F[q] / p->rho) / b;
                    u[q] = u[q] + p->dt * v[q];
                } else if (code == 1) {
                    u[q] = 0.0;
                    v[q] = 0.0;
                } else {
                    double sg = code == 2 ? 1.0 : -1.0;
                    v[q] = sg * (Un1 - Un) / p->dt;
                    u[q] = sg * Un1;
                }
            }
        }
        if (R > Q) {
            Q = R;
            npk = (int32_t)step;
        }
        done = k + 1;
        if (use_stop && Q > 0.0 && step - npk >= 100 && R < 0.5 * Q) break;
    }
    *peak = Q;
    *peak_step = npk;
    *n_done = done;
    free(F);
    return OR_OK;
}

/* Independent samples of the same mesh on OpenMP threads (one sample per
 * thread; every sample runs the single-thread loop above, so results do not
 * depend on the thread count). s0 and kappa are B x N; u, v are B x N x 3;
 * d is B x n_bonds. */
int or_run_batch(const or_problem *p, int32_t batch, int64_t n_bonds,
                 const double *s0, const double *kappa, int32_t n_steps,
                 int32_t use_stop, double *u, double *v, double *d,
                 double *peak, int32_t *peak_step, int32_t *n_done) {
    int64_t n = (int64_t)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t b = 0; b < batch; ++b) {
        or_problem q = *p;
        q.s0 = s0 + (int64_t)b * n;
        q.kappa = kappa ? kappa + (int64_t)b * n : NULL;
        peak[b] = -INFINITY;
        peak_step[b] = -1;
        or_run(&q, 0, n_steps, use_stop, u + (int64_t)b * 3 * n, v + (int64_t)b * 3 * n,
               d + (int64_t)b * n_bonds, NULL, NULL, &peak[b], &peak_step[b], &n_done[b]);
    }
    return OR_OK;
}

int or_max_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------ adjoint */

/* Derivatives of the softening law d = D(s; s0, sc) on (s0, sc), where the
 * critical stretch follows s0 with slope dsc_ds0 (ratio r, or 1 - A/s0^2 for
 * the fracture-energy calibration): dD/ds and the total dD/ds0 =
 * dD/ds0|sc + dsc_ds0 dD/dsc. Zero outside (s0, sc), where D is flat.
 *   bilinear:  D = 1 - s0 (sc - s) / (s (sc - s0))
 *              dD/ds = s0 sc / (s^2 (sc - s0))
 *              dD/ds0|sc = -(sc / s - 1) sc / (sc - s0)^2
 *              dD/dsc|s0 = -s0 (1 - s0 / s) / (sc - s0)^2
 *   exp-linear (Eq. exp_damage_parameter): D = 1 - (s0/s) beta(t) / (1 + alpha),
 *              t = (s - s0) / (sc - s0),
 *              beta(t) = 1 - (1 - e^{-k t}) / (1 - e^{-k}) + alpha (1 - t),
 *              beta'(t) = -k e^{-k t} / (1 - e^{-k}) - alpha,
 *              dt/ds = 1 / (sc - s0), dt/ds0 = (s - sc) / (sc - s0)^2,
 *              dt/dsc = -(s - s0) / (sc - s0)^2. */
static void law_derivs(int32_t law, double s, double s0, double sc, double dsc_ds0, double k, double alpha,
                       double *dDds, double *dDds0) {
    *dDds = 0.0;
    *dDds0 = 0.0;
    if (s <= s0 || s >= sc) return;
    double w = sc - s0;
    if (law == 0) {
        *dDds = s0 * sc / (s * s * w);
        double d_s0 = -(sc / s - 1.0) * sc / (w * w);
        double d_sc = -s0 * (1.0 - s0 / s) / (w * w);
        *dDds0 = d_s0 + dsc_ds0 * d_sc;
        return;
    }
    double t = (s - s0) / w;
    double beta = 1.0 - (1.0 - exp(-k * t)) / (1.0 - exp(-k)) + alpha * (1.0 - t);
    double dbeta = -k * exp(-k * t) / (1.0 - exp(-k)) - alpha;
    double dtds = 1.0 / w, dtds0 = (s - sc) / (w * w), dtdsc = -(s - s0) / (w * w);
    *dDds = (s0 * beta / (s * s) - (s0 / s) * dbeta * dtds) / (1.0 + alpha);
    double d_s0 = -(beta / s + (s0 / s) * dbeta * dtds0) / (1.0 + alpha);
    double d_sc = -(s0 / s) * dbeta * dtdsc / (1.0 + alpha);
    *dDds0 = d_s0 + dsc_ds0 * d_sc;
}

/* Reverse-mode derivative of J = sum_o w[o] R^{obs_step[o]} over a run of
 * n_steps steps from the zero state (no stop rule), with respect to the
 * per-node s0 (grad_s0, N) and kappa (grad_kappa, N, may be NULL; needs
 * p->kappa when non-NULL). The exact discrete adjoint of the step of or_run:
 * the branch of d_n = max(d_{n-1}, D(s_n)) taken forward is kept, so the
 * derivative follows D when it set the new value and d_{n-1} otherwise.
 *
 * The forward pass stores u^n and d^n of every step (test sizes only). With
 * h = s/L, the pair of directed forces of an undirected bond contributes
 *   Phi = lamF_i . f_ij + lamF_j . f_ji = -c_ij V (1 - d) h(y) (y . (lamF_j - lamF_i))
 * to the Lagrangian, and the reverse step n is:
 *   free DOF:    lv' = lamv^{n+1/2} + dt lamu^{n+1};  lamF^n = dt lv' / (rho b);
 *                lamv^{n-1/2} = a lv' / b;  lamu^n = lamu^{n+1} + bond terms
 *   prescribed:  lamF^n = -sign V sum_{o: obs_step[o] = n} w[o]
 *   bond (i,j):  lamd_tot = lamd + c_ij V h (y . dlam)
 *                lamy = dPhi/dy|_d + [active] lamd_tot D'(s) y / (L L0)
 *                lamu_i -= lamy   (the row of j adds +lamy for j)
 *                grad_s0_i += 0.5 [active] lamd_tot dD/ds0
 *                grad_kappa_i += 0.5 c dPhi/dc_ij,  dPhi/dc_ij = -V (1 - d) h (y . dlam)
 *                lamd <- [not active] lamd_tot */
int or_adjoint(const or_problem *p, int32_t n_steps, int32_t n_obs, const int32_t *obs_step,
               const double *w, double *grad_s0, double *grad_kappa) {
    int64_t n = (int64_t)p->nx * p->ny * p->nz;
    int64_t nb = p->row_ptr[n];
    double V = p->vol > 0.0 ? p->vol : p->dx * p->dx * p->dx;
    double a = 1.0 - 0.5 * p->zeta * p->dt;
    double b = 1.0 + 0.5 * p->zeta * p->dt;
    if (n_steps < 0 || (grad_kappa && !p->kappa)) return OR_ERR_ARG;
    double *U = (double *)malloc(sizeof(double) * 3 * (size_t)n * (size_t)(n_steps > 0 ? n_steps : 1));
    double *Dh = (double *)calloc((size_t)nb * (size_t)(n_steps + 1), sizeof(double));
    double *u = (double *)calloc(3 * (size_t)n, sizeof(double));
    double *v = (double *)calloc(3 * (size_t)n, sizeof(double));
    double *lu = (double *)calloc(3 * (size_t)n, sizeof(double));
    double *lun = (double *)calloc(3 * (size_t)n, sizeof(double));
    double *lv = (double *)calloc(3 * (size_t)n, sizeof(double));
    double *lF = (double *)calloc(3 * (size_t)n, sizeof(double));
    double *ld = (double *)calloc((size_t)nb, sizeof(double));
    double *F = (double *)calloc(3 * (size_t)n, sizeof(double));
    if (!U || !Dh || !u || !v || !lu || !lun || !lv || !lF || !ld || !F) return OR_ERR_ARG;
    /* forward, storing u^n and d^n (Dh[0] = d^{-1} = 0) */
    for (int32_t s = 0; s < n_steps; ++s) {
        memcpy(U + (size_t)s * 3 * n, u, sizeof(double) * 3 * (size_t)n);
        memcpy(Dh + (size_t)(s + 1) * nb, Dh + (size_t)s * nb, sizeof(double) * (size_t)nb);
        forces(p, u, Dh + (size_t)(s + 1) * nb, F, NULL);
        double Un = ramp(p, s), Un1 = ramp(p, s + 1);
        for (int64_t q = 0; q < 3 * n; ++q) {
            uint8_t code = p->bc[q];
            if (code == 0) {
                v[q] = (a * v[q] + p->dt * F[q] / p->rho) / b;
                u[q] = u[q] + p->dt * v[q];
            } else if (code == 1) {
                u[q] = 0.0;
                v[q] = 0.0;
            } else {
                double sg = code == 2 ? 1.0 : -1.0;
                v[q] = sg * (Un1 - Un) / p->dt;
                u[q] = sg * Un1;
            }
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        grad_s0[i] = 0.0;
        if (grad_kappa) grad_kappa[i] = 0.0;
    }
    or_grid g = {p->nx, p->ny, p->nz, p->dx, 0.0, 0, 0, 0};
    for (int32_t s = n_steps - 1; s >= 0; --s) {
        double wn = 0.0;
        for (int32_t o = 0; o < n_obs; ++o)
            if (obs_step[o] == s) wn += w[o];
        /* integrator */
        for (int64_t q = 0; q < 3 * n; ++q) {
            uint8_t code = p->bc[q];
            if (code == 0) {
                double lvp = lv[q] + p->dt * lu[q];
                lF[q] = p->dt * lvp / (p->rho * b);
                lv[q] = a * lvp / b;
                lun[q] = lu[q];
            } else if (code == 1) {
                lF[q] = 0.0;
                lv[q] = 0.0;
                lun[q] = 0.0;
            } else {
                double sg = code == 2 ? 1.0 : -1.0;
                lF[q] = -sg * V * wn;
                lv[q] = 0.0;
                lun[q] = 0.0;
            }
        }
        /* bonds, from u^s, d^{s-1} and d^s */
        const double *us = U + (size_t)s * 3 * n;
        const double *dprev = Dh + (size_t)s * nb;
        const double *dcur = Dh + (size_t)(s + 1) * nb;
        for (int64_t i = 0; i < n; ++i) {
            double xi_[3];
            node_xyz(&g, i, xi_);
            for (int32_t q = p->row_ptr[i]; q < p->row_ptr[i + 1]; ++q) {
                int64_t j = p->col[q];
                double xj[3], y[3], dl[3];
                node_xyz(&g, j, xj);
                double L0 = 0.0, L = 0.0, ydl = 0.0;
                for (int c = 0; c < 3; ++c) {
                    double xic = xj[c] - xi_[c];
                    y[c] = xic + (us[3 * j + c] - us[3 * i + c]);
                    dl[c] = lF[3 * j + c] - lF[3 * i + c];
                    L0 += xic * xic;
                    L += y[c] * y[c];
                    ydl += y[c] * dl[c];
                }
                L0 = sqrt(L0);
                L = sqrt(L);
                double sv = (L - L0) / L0;
                double h = sv / L;
                double s0 = 0.5 * (p->s0[i] + p->s0[j]);
                double cij = p->c;
                if (p->kappa) cij = p->c * 0.5 * (p->kappa[i] + p->kappa[j]);
                double sc = p->gf_A > 0.0 ? s0 + p->gf_A / s0 : p->s_ratio * s0;
                double dsc = p->gf_A > 0.0 ? 1.0 - p->gf_A / (s0 * s0) : p->s_ratio;
                double dD = or_damage_law(p->law, sv, s0, sc, p->k, p->alpha);
                int active = dD > dprev[q];
                double d = dcur[q];
                double lamd_tot = ld[q] + cij * V * h * ydl;
                double dDds = 0.0, dDds0 = 0.0;
                if (active) law_derivs(p->law, sv, s0, sc, dsc, p->k, p->alpha, &dDds, &dDds0);
                for (int c = 0; c < 3; ++c) {
                    double dh = y[c] / (L * L * L0) - sv * y[c] / (L * L * L);
                    double lamy = -cij * V * (1.0 - d) * (ydl * dh + h * dl[c]);
                    if (active) lamy += lamd_tot * dDds * y[c] / (L * L0);
                    lun[3 * i + c] -= lamy;
                }
                if (active) grad_s0[i] += 0.5 * lamd_tot * dDds0;
                if (grad_kappa) grad_kappa[i] += 0.5 * p->c * (-V * (1.0 - d) * h * ydl);
                ld[q] = active ? 0.0 : lamd_tot;
            }
        }
        memcpy(lu, lun, sizeof(double) * 3 * (size_t)n);
    }
    free(U);
    free(Dh);
    free(u);
    free(v);
    free(lu);
    free(lun);
    free(lv);
    free(lF);
    free(ld);
    free(F);
    return OR_OK;
}
