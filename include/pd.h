/*
 * pd.h -- C ABI of the GB300 bond-based peridynamic / multilevel Monte Carlo
 * hot path (arXiv 2212.04415, "A probabilistic peridynamic framework with an
 * application to the study of the statistical size effect").
 *
 * Conventions shared by every call:
 *  - Status: every call returns PD_OK (0) or a negative PD_ERR_* code. On an
 *    error nothing is written to the caller's output buffers, the call never
 *    aborts, and pd_last_error() returns a one-line description.
 *  - Device buffers are owned by the caller (allocated by the caller, for
 *    example as torch tensors, and passed as raw device pointers). Handles
 *    (pd_state, pd_field) own only their internal state, scratch and KL basis.
 *  - Every call that touches the GPU takes a CUDA stream (pd_stream, the same
 *    object as cudaStream_t; NULL = the legacy default stream) and is
 *    asynchronous on that stream unless its comment says "host-synchronous".
 *  - Units are SI (m, N, Pa, kg, s). Node i has grid index
 *    (ix, iy, iz) = (i % nx, (i / nx) % ny, i / (nx ny)) and sits at the cell
 *    centre ((ix + 1/2) dx, (iy + 1/2) dx, (iz + 1/2) dx).
 *  - Geometry that must compare exactly (notch, supports, load line) is given
 *    in integer half-cells: x = X dx / 2, so node ix sits at X = 2 ix + 1.
 *  - Arrays indexed by sample are sample-major: [B][N] or [B][N][3].
 */
#ifndef PD_GB300_H
#define PD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *pd_stream; /* == cudaStream_t */

#if defined(__GNUC__)
#define PD_API __attribute__((visibility("default")))
#else
#define PD_API
#endif

enum {
    PD_OK = 0,
    PD_ERR_ARG = -1,     /* invalid argument (sizes, NULL pointers, unsupported mode) */
    PD_ERR_CUDA = -2,    /* a CUDA runtime call failed */
    PD_ERR_OOM = -3,     /* device allocation failed */
    PD_ERR_TIMEOUT = -4, /* a bounded device wait gave up */
    PD_ERR_NAN = -5,     /* a non-finite value was detected */
    PD_ERR_CAP = -6      /* output capacity too small (the required size is reported) */
};

enum { PD_LAW_BILINEAR = 0, PD_LAW_EXPLINEAR = 1 };
enum { PD_PREC_FP64 = 0, PD_PREC_MIXED = 1 };
enum { PD_BC_BAR_TENSION = 1, PD_BC_BEAM_3PT = 2 };
enum { PD_COV_SQEXP = 0, PD_COV_EXP = 1 };
enum { PD_MARG_LOGNORMAL = 0, PD_MARG_WEIBULL = 1 };

/* Regular grid and horizon (Eq. PD_Horizon, Section 3.2: delta = m dx).
 * notch: 1 removes every bond whose segment strictly crosses the plane
 * X = notch_x2 (half-cells) at a height below Y = notch_y2 (half-cells); a
 * crossing exactly at the notch tip is kept. */
typedef struct pd_grid {
    int32_t nx, ny, nz; /* nodes per axis; nx, ny <= 2047, nz <= 1023 */
    double dx;          /* node spacing [m] */
    double m_ratio;     /* horizon / dx */
    int32_t notch;
    int32_t notch_x2;
    int32_t notch_y2;
} pd_grid;

/* Material and integrator (Appendix A; integrator readings in the design notes).
 * Micromodulus c = 12 E / (pi delta^4) (Eq. bond_stiffness_constant, 3D).
 * Bond force f = c_ij (1 - d) s (Eq. exp_scalar_force) with per-bond
 * s0_ij = (s0_i + s0_j)/2, s_crit_ij = s_ratio s0_ij, c_ij = c (kappa_i + kappa_j)/2.
 * law PD_LAW_BILINEAR: d = 1 - s0 (sf - s)/(s (sf - s0)) on (s0, sf);
 * law PD_LAW_EXPLINEAR: Eq. exp_damage_parameter with k, alpha.
 * Damage is irreversible: d_n = max(d_{n-1}, d_law(s_n)).
 * dt > 0 is used as given; dt <= 0 selects dt_safety x the Silling-Askari
 * stable step min_i sqrt(2 rho / sum_j c V / |xi_ij|).
 * zeta: mass-proportional damping rate [1/s] of the damped leapfrog update.
 * precision: PD_PREC_FP64 (all arithmetic FP64) or PD_PREC_MIXED (bond
 * kinematics and forces FP32; nodal sums, integration, reaction FP64). */
typedef struct pd_material {
    double E;
    double rho;
    int32_t law;
    double s_ratio;
    double k;
    double alpha;
    double dt;
    double dt_safety;
    double zeta;
    int32_t precision;
    double G_F;         /* fracture energy [N/m]; > 0: per-bond critical stretch
                           s_c = s0 + A / s0 with A from pd_gf_coefficient (s_ratio unused) */
    int32_t model;      /* PD_MODEL_3D, or a plane model on a one-layer grid (nz = 1) */
    double thickness;   /* plane models: out-of-plane thickness t [m] */
} pd_material;

/* Plane models (Eq. bond_stiffness_constant): c = 9E / (pi t delta^3) (plane
 * stress) or 48E / (5 pi t delta^3) (plane strain), node volume dx^2 t. */
enum { PD_MODEL_3D = 0, PD_MODEL_PLANE_STRESS = 1, PD_MODEL_PLANE_STRAIN = 2 };

/* A of the fracture-energy calibration s_c = s0 + A / s0 (Appendix A): Eq.
 * exp_fracture_energy solved for s_c for the exp-linear law (k, alpha), and
 * the same construction (bond energy c s0 xi (s_c - s0) / 2 over the bonds
 * crossing a unit plane, pi delta^5 / 5) for the bilinear law; c = 12E /
 * (pi delta^4). Reading: the printed Eq. exp_sc has (1 + alpha) s0 where Eq.
 * exp_fracture_energy gives s0; the consistent form is used. Host only. */
PD_API int pd_gf_coefficient(int32_t law, double E, double delta, double G_F, double k, double alpha,
                             double *A);

/* The same for a plane model of thickness t: Eq. exp_sc_2D,
 * A = 4k (e^k - 1)(1 + alpha) G_F / (t c delta^4 (-P)), P = 2k - 2e^k + alpha k
 * - alpha k e^k + 2 (exp-linear), A = 4 G_F / (t c delta^4) (bilinear), with c
 * the plane model's micromodulus. */
PD_API int pd_gf_coefficient_plane(int32_t law, int32_t model, double E, double delta, double t, double G_F,
                                   double k, double alpha, double *A);

/* Displacement control: prescribed magnitude U(n) = u_max min(n, n_ramp) / n_ramp.
 * PD_BC_BAR_TENSION: the first grip_planes x-planes are fixed; the last
 *   grip_planes x-planes move by +U(n) along x and are held in y and z.
 * PD_BC_BEAM_3PT: bottom-layer (iy = 0) nodes within half a cell of either
 *   support_x2 are held in y; top-layer nodes within half a cell of load_x2
 *   move by -U(n) along y. */
typedef struct pd_bc {
    int32_t type;
    int32_t grip_planes;
    int32_t support_x2[2];
    int32_t load_x2;
    double u_max;
    int32_t n_ramp;
} pd_bc;

/* Truncated Karhunen-Loeve random field (Section 5). */
typedef struct pd_field_cfg {
    int32_t kernel;   /* PD_COV_SQEXP: exp(-r^2/l^2) (separable); PD_COV_EXP: exp(-r/l) */
    double length;    /* correlation length l [m] */
    int32_t n_modes;  /* K, 1..256 */
    int32_t marginal; /* PD_MARG_LOGNORMAL or PD_MARG_WEIBULL */
    double mean;      /* mean of the marginal */
    double cov;       /* coefficient of variation (lognormal) */
    double weibull_m; /* Weibull modulus (Weibull) */
} pd_field_cfg;

typedef struct pd_state pd_state;
typedef struct pd_field pd_field;

/* One-line text of the last error raised on the calling thread. */
PD_API int pd_last_error(char *buf, size_t len);

/* Version string of the library (static storage). */
PD_API const char *pd_version(void);

/* ------------------------------------------------------------------ mesh */

/* Neighbour list of the horizon H_x = {x' : |x' - x| <= delta} (Eq. PD_Horizon),
 * minus notch-cut bonds, as CSR sorted by neighbour index within each row.
 * row_ptr: device int32[N+1] (always written); col: device int32[cap].
 * n_bonds (host out): number of directed bonds. If col == NULL only row_ptr
 * and n_bonds are produced; if cap < n_bonds, returns PD_ERR_CAP with
 * n_bonds set and col untouched. Host-synchronous (reads back n_bonds).
 * Bit-exact: the list is a pure integer function of the grid. */
PD_API int pd_build_neighbours(const pd_grid *g, int32_t *row_ptr, int32_t *col, int64_t cap,
                        int64_t *n_bonds, pd_stream stream);

/* The same neighbour list as pd_build_neighbours, computed without any device
 * allocation (the paper has no counterpart: this serves callers that cannot
 * call cudaMalloc, e.g. code running under an external memory manager that
 * owns all device memory). The one word of device scratch (the scan's
 * overflow flag) lives in a 256-byte static device array that every GPU
 * loading the library holds until exit; it is cleared on every call. Every
 * call looks up the array's address on the current device, so no address
 * outlives a cudaDeviceReset. The stream must belong to the current device
 * (PD_ERR_ARG otherwise). Calls that overlap on the GPU share the
 * array and race. Sizes: at most 2^31 - 2 nodes and 2^31 - 1 bonds; larger
 * grids return PD_ERR_ARG (a count-only call detects the bond overflow).
 * Arguments, outputs, synchronisation and errors are those of
 * pd_build_neighbours. */
PD_API int pd_build_neighbours_noalloc(const pd_grid *g, int32_t *row_ptr, int32_t *col, int64_t cap,
                                       int64_t *n_bonds, pd_stream stream);

/* Per-DOF boundary codes (device uint8[N*3]: 0 free, 1 fixed, 2 +U(n), 3 -U(n)). */
PD_API int pd_bc_codes(const pd_grid *g, const pd_bc *bc, uint8_t *codes, pd_stream stream);

/* ------------------------------------------------------------ time step */

/* Create the explicit-dynamics state of B independent samples on one mesh
 * (row_ptr/col: device CSR from pd_build_neighbours; copied, not retained).
 * Host-synchronous. The state starts at step 0 with u = v = d = 0 and a
 * uniform field s0 = 1e-4, kappa = 1; call pd_state_reset to set the fields. */
PD_API int pd_state_create(const pd_grid *g, const int32_t *row_ptr, const int32_t *col,
                    int64_t n_bonds, const pd_material *mat, const pd_bc *bc, int32_t batch,
                    pd_state **out);

/* Launch schedule of a state: bricks of 8 x by x bz nodes per block (by bz
 * even and <= 32 on the compile-time stencil path), q warps sharing each
 * row pair's half-stencil (1, 2 or 4; 0 = the built-in choice) and ns
 * samples per block on that path (1, or 2: a pair of samples computed
 * together on the paired FP32 instructions, bit-identical per sample to
 * ns = 1; 0 = the built-in choice, 1) and where each step's reaction force
 * is reduced on that path (1: in the step's own launch; 2: by every block of
 * the next launch, before it steps, so a single-wave launch has no serial
 * reduction tail; the last launch of every call reduces its own; results are
 * bit-identical; 0 = the built-in choice, 2 for launches of at most four
 * blocks per SM). A schedule changes the summation grouping, not the method:
 * results agree to rounding. The paper has no counterpart. */
typedef struct pd_schedule {
    int32_t by, bz, q, ns, reduce;
} pd_schedule;

/* pd_state_create with an explicit schedule (NULL: the built-in choice). */
PD_API int pd_state_create_sched(const pd_grid *g, const int32_t *row_ptr, const int32_t *col,
                                 int64_t n_bonds, const pd_material *mat, const pd_bc *bc,
                                 int32_t batch, const pd_schedule *sched, pd_state **out);

/* Autotuner: times trial_steps captured steps of every candidate schedule of
 * this mesh and batch (a state per candidate, uniform fields, CUDA events) and
 * returns the fastest with its time per step in microseconds (best_us may be
 * NULL). Results are cached per (grid, batch, law, precision, horizon) for the
 * life of the process, so repeated calls cost nothing. Host-synchronous;
 * allocates one candidate state at a time. */
PD_API int pd_autotune(const pd_grid *g, const int32_t *row_ptr, const int32_t *col, int64_t n_bonds,
                       const pd_material *mat, const pd_bc *bc, int32_t batch, int32_t trial_steps,
                       pd_schedule *best, double *best_us);
PD_API int pd_state_destroy(pd_state *st);

/* dt [s], micromodulus c, node and bond counts of a state (host outputs, any may be NULL). */
PD_API int pd_state_info(const pd_state *st, double *dt, double *c, int64_t *n_nodes,
                  int64_t *n_bonds);

/* Restart every sample at step 0 with u = v = d = 0, peak = -inf, and the
 * per-node fields s0 (device float[B][N], required) and kappa (device
 * float[B][N], or NULL for kappa = 1). */
PD_API int pd_state_reset(pd_state *st, const float *s0, const float *kappa, pd_stream stream);

/* pd_state_reset with the elastic-limit field s0 in FP64 (device
 * double[B][N], required): FP64-path states keep it in FP64 (so that the FP64
 * path is FP64 from the field on, e.g. for finite differences with respect to
 * the field), mixed-path states round it to FP32 as pd_state_reset does.
 * kappa as in pd_state_reset. */
PD_API int pd_state_reset_f64(pd_state *st, const double *s0, const float *kappa, pd_stream stream);

/* Overwrite u, v (device double[B][N][3]) and damage d (device double[B][n_bonds]
 * in CSR order, or NULL to keep) and set the step index of every sample. */
PD_API int pd_state_load(pd_state *st, const double *u, const double *v, const double *d,
                  int32_t step, pd_stream stream);

/* Copy u, v (device double[B][N][3]) and d (device double[B][n_bonds], CSR
 * order) out; any pointer may be NULL. */
PD_API int pd_state_store(const pd_state *st, double *u, double *v, double *d, pd_stream stream);

/* Internal force density F (device double[B][N][3]) of the current state,
 * F_i = sum_j f_ij V_j (Eq. PD_EOM_Dynamic with b = 0), updating the bond
 * damage from the current stretch exactly as a step does; u, v unchanged. */
PD_API int pd_force(pd_state *st, double *F, pd_stream stream);

/* Advance every sample n_steps explicit steps (Section 3; Eq. PD_EOM_Dynamic):
 * damage from the current stretch, bond forces, nodal sums, damped leapfrog
 * update with the prescribed displacements, and the reaction
 * R_n = -sum over prescribed DOFs of F sign V. reaction: device
 * double[B][n_steps] or NULL. Samples marked done by pd_run_to_peak do not move. */
PD_API int pd_step(pd_state *st, int32_t n_steps, double *reaction, pd_stream stream);

/* Run every sample until its peak-load rule stops it or max_steps steps have
 * been taken: Q = max_n R_n (first step attaining it); a sample stops once
 * R_n < Q/2 with Q > 0 and at least 100 steps after the peak.
 * Outputs (device): peak double[B], peak_step int32[B], n_done int32[B]
 * (steps executed). Host-synchronous (the host polls completion once per
 * chunk of captured steps). Errors after the run: PD_ERR_NAN if a sample's
 * reaction became non-finite; PD_ERR_CUDA if a staged box of the stencil
 * step did not arrive within its bounded wait, or if a sample was stepped at
 * a step parity other than the one its state's last reset or load implies
 * (both internal checks; the run's outputs are then not to be used). */
PD_API int pd_run_to_peak(pd_state *st, int32_t max_steps, double *peak, int32_t *peak_step,
                   int32_t *n_done, pd_stream stream);

/* ---------------------------------------------------------------- adjoint */

/* Reverse-mode gradient of J = sum_o dJ_dR[b][o] R^{n0 + obs_steps[o]} of every
 * sample b over a run of n_steps steps from the state's current content
 * (all samples at the same step index n0, as after pd_state_reset or
 * pd_state_load), with respect to the per-node fields s0 and kappa: the exact
 * discrete adjoint of the step (Eq. PD_EOM_Dynamic, Eq. exp_scalar_force,
 * Eq. exp_damage_parameter, the damped leapfrog update and the reaction), the
 * branch of d_n = max(d_{n-1}, D(s_n)) taken forward kept. The paper has no
 * counterpart; it serves parameter-importance studies of the random fields.
 *   obs_steps: host int32[n_obs], local step indices in [0, n_steps)
 *   dJ_dR:     device double[B][n_obs]
 *   s0, kappa: device float[B][N], the fields passed to pd_state_reset
 *              (kappa NULL: kappa = 1)
 *   grad_s0, grad_kappa: device double[B][N] out (grad_kappa may be NULL)
 *   R_obs:     device double[B][n_obs] out, the forward reactions, or NULL
 * Checkpoints (u, v, d) every ckpt_every steps (k) and recomputes each
 * segment. Device memory, allocated per call (PD_ERR_OOM when unavailable),
 * per sample: checkpoints (n_steps / k + 2) (6N + n_b) doubles and adjoint
 * state 12 N doubles; then for FP64-path states the segment's trajectory
 * k 3N + (k + 1) n_b doubles and n_b doubles of damage adjoint, for
 * mixed-path states 16 k N + 4 (k + 1) S bytes of FP32 trajectory (S the
 * slots of a sliced-ELL copy of the rows, slices of 32 nodes padded to the
 * longest row, about n_b), 8 S bytes of double-float damage adjoint and S
 * bytes marking the bonds whose damage grows in the run (only those carry a
 * damage adjoint).
 * Arithmetic: FP64 for FP64-path states; for mixed-path states the bond terms
 * in FP32 on the FP32 trajectory (the forward path's own precision class),
 * the damage adjoint in double-float, the node sums in FP64. The states come
 * from the state's own forward path. Host-synchronous. On return the state
 * holds the forward run's final state (step n0 + n_steps), as after
 * pd_step(n_steps). */
PD_API int pd_adjoint(pd_state *st, int32_t n_steps, int32_t ckpt_every, int32_t n_obs,
                      const int32_t *obs_steps, const double *dJ_dR, const float *s0,
                      const float *kappa, double *grad_s0, double *grad_kappa, double *R_obs,
                      pd_stream stream);

/* pd_run_to_peak for several states at once (meshes of different sizes, such as
 * the fine and coarse members of an MLMC level): each 64-step chunk is one
 * captured graph. Two states with the same launch shape (one sample per
 * block, brick rows and warp split alike, same law and stiffness-field mode)
 * step together in one launch per step, whose blocks cover both meshes;
 * other states run as graph branches, so the small meshes' launches overlap
 * the large ones'. One host poll per chunk covers every state. Per state i:
 * max_steps[i] and device outputs peak[i], peak_step[i], n_done[i] (the
 * pointer arrays are host arrays; each may be NULL). Results equal n_states
 * calls of pd_run_to_peak bit for bit. Host-synchronous; 1 <= n_states <= 16,
 * no state twice. */
PD_API int pd_run_to_peak_multi(pd_state *const *states, int32_t n_states, const int32_t *max_steps,
                                double *const *peak, int32_t *const *peak_step, int32_t *const *n_done,
                                pd_stream stream);

/* ---------------------------------------------------------- random field */

/* KL coefficients xi (device double[B][K]) of samples sample_ids (device
 * uint64[B]) on MLMC level `level`: Philox4x32-10 keyed by the seed, counter
 * (block, sample id, level), Box-Muller in FP64 (Section 4.2: the same xi
 * serves both members of a coupled pair). */
PD_API int pd_draw_xi(uint64_t seed, int32_t level, const uint64_t *sample_ids, int32_t B,
               int32_t n_modes, double *xi, pd_stream stream);

/* KL basis of the finest grid of a hierarchy of n_levels nested grids (each
 * coarser grid halves nx, ny, nz and doubles dx; level 0 is the coarsest).
 * Host-synchronous. The separable squared-exponential kernel works on any
 * size; the exponential kernel needs the dense covariance (finest N <= 4096). */
PD_API int pd_field_create(const pd_grid *finest, int32_t n_levels, const pd_field_cfg *cfg,
                    pd_field **out);
/* Synchronises the device; returns PD_ERR_TIMEOUT if a sampling launch of
 * this field gave up waiting for its tile copies or MMAs (that tile was
 * written as NaN). */
PD_API int pd_field_destroy(pd_field *f);

/* K and the KL eigenvalues (host double[K], may be NULL). */
PD_API int pd_field_info(const pd_field *f, int32_t *n_modes, double *lambda);

/* Chain rule of a node-field gradient back to the KL coefficients
 * (Section 5): dJ/dxi_k = sum_i dJ/ds0_i ds0_i/dg_i sqrt(lambda_k) phi_k(x_i),
 * with ds0/dg = sigma s0 (lognormal) or the Weibull copula's derivative;
 * g is recomputed in FP64 from xi. xi: device double[B][K]; dJ_ds0: device
 * double[B][N_level]; dJ_dxi: device double[B][K] out (FP64, fixed-order
 * sums). Host-synchronous. */
PD_API int pd_field_adjoint(const pd_field *f, int32_t level, const double *xi, int32_t B,
                            const double *dJ_ds0, double *dJ_dxi, pd_stream stream);

/* Field of B samples on grid `level`: g = Phi diag(sqrt(lambda)) xi, then the
 * marginal transform (Section 5.2). node_field: device float[B][N_level].
 * coarse_field (level > 0, or NULL): the same samples on grid level-1, from
 * the 2x2x2 mean of the Gaussian field before the transform (Section 4.2).
 * The product runs on the tensor cores in split TF32 (FP32-class accuracy).
 * A field's sampling calls must be ordered on one stream: each level keeps
 * one scratch buffer for the split coefficients (grown, with a device
 * synchronisation, when B exceeds every earlier call's). */
PD_API int pd_sample_field(pd_field *f, int32_t level, const double *xi, int32_t B,
                    float *node_field, float *coarse_field, pd_stream stream);

/* ------------------------------------------------------------------ MLMC */

#define PD_MAX_LEVELS 8

/* Fixed-allocation multilevel Monte Carlo (Section 4.2). Level l uses grid[l]
 * (coarsest first, dx halving) with bc[l] and max_steps[l]; level l > 0
 * draws each sample's field once on grid l and its 2x2x2 coarsening on grid
 * l-1 and runs both (Y_l = Q_l - Q_{l-1}); level 0 runs Q_0 alone. */
typedef struct pd_mlmc_cfg {
    int32_t n_levels;
    const pd_grid *grid;
    const pd_bc *bc;
    const int32_t *max_steps;
    const int64_t *n_samples;
    pd_material mat;
    pd_field_cfg field;
    uint64_t seed;
    int32_t batch;                /* samples per launch (<= 4096) */
    const int64_t *first_sample;  /* [n_levels] id of the first sample of each level, or NULL (0): a
                                     process of a sharded run takes ids first .. first + n - 1 */
    int32_t tune_steps;           /* > 0: schedules from pd_autotune with this many trial steps per
                                     candidate (fine and coarse states); 0: the built-in choice */
} pd_mlmc_cfg;

typedef struct pd_mlmc_level {
    int64_t n;           /* samples taken */
    double sum_y;        /* sum of Y (FP64, fixed order) */
    double sum_y2;       /* sum of Y^2 */
    double mean;         /* Y_hat = sum_y / n */
    double var;          /* s^2 = sum_y2/n - mean^2 (Eq. sample_variance) */
    double var_unbiased; /* s^2 n/(n-1) */
    double cost_s;       /* GPU seconds spent on the level */
    int64_t steps;       /* explicit steps executed (fine + coarse) */
    int64_t bond_updates;
} pd_mlmc_level;

typedef struct pd_mlmc_result {
    int32_t n_levels;
    pd_mlmc_level level[PD_MAX_LEVELS];
    double q_ml;   /* Q_hat^ML = sum_l Y_hat_l (Eq. MLMC_estimator) */
    double var_ml; /* sum_l var_l / n_l (Eq. MLMC_error, sampling part) */
} pd_mlmc_result;

/* Host-synchronous; owns its own device buffers. q_fine/q_coarse (host,
 * optional) receive every sample's Q_l and Q_{l-1} level after level
 * (sum_l n_samples[l] entries; q_coarse entries of level 0 are 0).
 * batch_sums (host, optional) receives, level after level and batch after
 * batch, the GPU's FP64 (n, sum Y, sum Y^2) of every batch of `batch`
 * consecutive samples: the level totals are these added in batch order, so
 * the batch sums of processes that each took whole batches of a level merge
 * (in sample order) to exactly the totals of a single-process run. */
PD_API int mlmc_estimate(const pd_mlmc_cfg *cfg, pd_mlmc_result *out, double *q_fine,
                  double *q_coarse, double *batch_sums, pd_stream stream);

/* Level totals and the estimator from the per-batch FP64 sums (n, sum Y,
 * sum Y^2) that mlmc_estimate returns (batch_sums), for one run or for
 * several processes that each took whole batches of every level (Section 4.2:
 * samples are independent, so a run shards by sample): batch_sums is host
 * double[sum_l n_batches[l]][3], level-major, each level's batches in sample
 * order. Each level's batch sums are added in the order given, from zero --
 * the additions a single run makes -- so the totals equal a single run's bit
 * for bit; then the mean, the sample variance (Eq. sample_variance, 1/n form,
 * and the unbiased form), Q_hat^ML = sum_l Y_hat_l (Eq. MLMC_estimator) and
 * var_ml = sum_l s_l^2 / n_l (Eq. MLMC_error). cost_s, steps and
 * bond_updates are 0 in out. Host only. */
PD_API int mlmc_merge(int32_t n_levels, const int64_t *n_batches, const double *batch_sums, pd_mlmc_result *out);

/* Optimal allocation N_l = floor(eps_s^-2 (sum_k sqrt(V_k C_k)) sqrt(V_l/C_l))
 * (Eq. sample_allocation), host arrays of length n_levels. */
PD_API int pd_mlmc_allocation(int32_t n_levels, const double *V, const double *C, double eps_s,
                       int64_t *N);

/* Multilevel inverse CDF of the peak load (Section 7):
 * F_L^-1(u) = R_0^[N_0 u] + sum_{l>=1} (R_l^[N_l u] - R~_{l-1}^[N_l u]), with R_l
 * and R~_{l-1} the fine and coarse members of level l's pairs sorted
 * ascending and R^[k] the k-th smallest. Readings: [N u] = ceil(N u),
 * 1-based, clamped to [1, N]; the coarse term of level l uses N_l.
 * n_per_level: host int64[n_levels] (>= 1 each); q_fine, q_coarse: device
 * double[sum N_l], level-major as mlmc_estimate returns them (q_coarse may be
 * NULL with one level; its level-0 entries are not read); values must be
 * finite. u, out: device double[n_u]. Host-synchronous (sorted copies are
 * allocated per call). */
PD_API int pd_ml_inverse_cdf(int32_t n_levels, const int64_t *n_per_level, const double *q_fine,
                             const double *q_coarse, int32_t n_u, const double *u, double *out,
                             pd_stream stream);

/* Multilevel CDF: F(x) = (1/n_u) #{i < n_u : F_L^-1((i + 1/2) / n_u) <= x} for
 * every x (device double[n_x]) into F (device double[n_x]); inputs as for
 * pd_ml_inverse_cdf. Host-synchronous. */
PD_API int pd_ml_cdf(int32_t n_levels, const int64_t *n_per_level, const double *q_fine,
                     const double *q_coarse, int32_t n_u, int32_t n_x, const double *x, double *F,
                     pd_stream stream);

/* Settings of the adaptive estimator (Algorithm MLMC, Section 4.2). */
typedef struct pd_mlmc_adaptive_cfg {
    double eps_s;              /* sampling tolerance of Eq. sample_allocation [units of Q] */
    double eps_b;              /* bias tolerance: stop once |Y_hat_L| / (m_dof^alpha - 1) < eps_b
                                  (Eq. bias_error with r = 1) */
    double m_dof;              /* ratio of degrees of freedom between levels (8 in 3D) */
    double alpha;              /* rate of |Y_hat_l| ~ M_l^-alpha (Eq. alpha_convergence_mlmc) */
    int32_t n_star;            /* warm-up samples on every new level (the paper uses 100) */
    const double *cost_model;  /* [n_levels] cost per sample, or NULL: the measured GPU time */
} pd_mlmc_adaptive_cfg;

/* Adaptive MLMC (Algorithm MLMC): start with level 0; on each new level L
 * take n_star samples; re-allocate N_l (Eq. sample_allocation, floor) for
 * l <= L from the level variances (Eq. sample_variance) and costs, and top
 * every level up to N_l with new sample ids (level l's samples are ids
 * first_sample[l] + 0, 1, ...); stop once the bias estimate of Eq.
 * bias_error falls below eps_b or L reaches cfg->n_levels - 1, else add a
 * level. cfg->n_samples is ignored (may be NULL). out receives the level
 * statistics of levels 0..L (n_levels = L + 1), L_used the last level,
 * bias the final bias estimate. q_fine/q_coarse (host, optional, capacity
 * cap entries) receive every sample's Q_l and Q_{l-1} level after level in
 * id order; PD_ERR_CAP (with out filled) when the run took more than cap
 * samples. Host-synchronous. */
PD_API int mlmc_adaptive(const pd_mlmc_cfg *cfg, const pd_mlmc_adaptive_cfg *ad, pd_mlmc_result *out,
                         int32_t *L_used, double *bias, double *q_fine, double *q_coarse, int64_t cap,
                         pd_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* PD_GB300_H */
