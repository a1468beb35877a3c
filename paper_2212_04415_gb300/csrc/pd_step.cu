// pd_step.cu -- the explicit bond-based peridynamic time step (Sections 2-3,
// Appendix A): bond kinematics, softening law with irreversible damage,
// deterministic nodal force sums, damped leapfrog update under displacement
// control, and the FP64 reaction / peak-load reduction.
//
// Layout (per state; B samples share one mesh):
//   * neighbour list as SELL-32: slices of 32 consecutive nodes, slot-major
//     inside a slice, so lane l of a warp reads slot k of node 32 s + l at
//     element off[s] + 32 k + l (one 128-byte line per warp per slot).
//     Padding slots hold -1 and trail each row.
//   * damage per directed bond in the same SELL order, per sample. Both
//     directed copies of a bond evolve identically: the stretch, the per-bond
//     properties and the law are symmetric in (i, j) bit for bit.
//   * a 32-byte gather record per node (double-buffered by step parity):
//       mixed: float4 (u_hi xyz, s0), float4 (u_lo xyz, packed grid coordinate)
//              where u = u_hi + u_lo (double-float), so u_j - u_i keeps FP64-like
//              accuracy with FP32 arithmetic;
//       fp64:  double u xyz, float s0, packed coordinate.
//   * FP64 u, v per node for the integrator (owner thread only).
// One thread owns one (sample, node) pair and walks its row in CSR order, so
// the nodal sum has a fixed order and needs no atomics. Blocks are ordered
// sample-fastest so that all samples of a batch stream the shared neighbour
// index through L2 together.
#include <cmath>
#include <vector>

#include "pd_internal.cuh"

namespace pdi {

struct RecMixed {
    float4 hi;  // u_hi.x, u_hi.y, u_hi.z, s0
    float4 lo;  // u_lo.x, u_lo.y, u_lo.z, coord bits
};
struct RecF64 {
    double ux, uy, uz;
    float s0;
    int32_t coord;
};
static_assert(sizeof(RecMixed) == 32 && sizeof(RecF64) == 32, "records are 32 bytes");

constexpr int kThreads = 256;
constexpr int kMaxQ = 64;  // largest squared stencil radius in cells (m <= 8)

struct StepArgs {
    long long N;
    int nblk;
    int B;
    const long long *sell_off;
    const int32_t *sell_w;
    const int32_t *sell_col;
    void *dmg;
    long long sell_len;
    double *u64;
    double *v64;
    void *rec0;
    void *rec1;
    const float *kappa;
    const uint8_t *codes;
    int32_t *step;
    int32_t *done;
    int32_t *status;
    double *peak;
    int32_t *peak_step;
    double *partial;
    unsigned int *ticket;
    double *reaction;
    int n_react;
    int k_local;
    double *F_out;
    double dt, rho, zeta, u_max;
    int n_ramp;
    int max_steps;
    int use_stop;
    double cV;  // micromodulus x node volume
    double V;
    double dx;
    double s_ratio, k, alpha, inv_1mek, inv_1pa;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T law_damage(int law, T s, T s0, T sc, T k, T alpha, T inv_1mek,
                                        T inv_1pa);

template <>
__device__ __forceinline__ float law_damage<float>(int law, float s, float s0, float sc, float k,
                                                   float alpha, float inv_1mek, float inv_1pa) {
    if (s >= sc) return 1.0f;
    if (law == PD_LAW_BILINEAR) return 1.0f - s0 * (sc - s) / (s * (sc - s0));
    const float t = (s - s0) / (sc - s0);
    const float br = 1.0f - (1.0f - expf(-k * t)) * inv_1mek + alpha * (1.0f - t);
    return 1.0f - (s0 / s) * br * inv_1pa;
}

template <>
__device__ __forceinline__ double law_damage<double>(int law, double s, double s0, double sc,
                                                     double k, double alpha, double inv_1mek,
                                                     double inv_1pa) {
    if (s >= sc) return 1.0;
    if (law == PD_LAW_BILINEAR) return 1.0 - s0 * (sc - s) / (s * (sc - s0));
    const double t = (s - s0) / (sc - s0);
    const double br = 1.0 - (1.0 - exp(-k * t)) * inv_1mek + alpha * (1.0 - t);
    return 1.0 - (s0 / s) * br * inv_1pa;
}

__device__ __forceinline__ double ramp(const StepArgs &a, int n) {
    const int m = n < a.n_ramp ? n : a.n_ramp;
    return a.u_max * (double)m / (double)a.n_ramp;
}

// One explicit step (or, with FORCE_ONLY, one force evaluation) of every
// (sample, node) pair. Grid: nblk * B blocks, sample index fastest.
template <bool F64, int LAW, bool KAPPA, bool FORCE_ONLY>
__global__ void __launch_bounds__(kThreads) k_step(const StepArgs a) {
    __shared__ float sL0f[kMaxQ + 1];
    __shared__ double sL0d[kMaxQ + 1];
    __shared__ double red[kThreads / 32];
    __shared__ int last_flag;

    for (int t = threadIdx.x; t <= kMaxQ; t += blockDim.x) {
        const double L0 = sqrt((double)t) * a.dx;
        sL0d[t] = L0;
        sL0f[t] = (float)L0;
    }
    __syncthreads();

    const int b = blockIdx.x % a.B;
    const int xb = blockIdx.x / a.B;
    const long long i = (long long)xb * kThreads + threadIdx.x;
    const bool done = FORCE_ONLY ? false : (a.done[b] != 0);
    const int n = a.step[b];
    double Rloc = 0.0;

    if (!done && i < a.N) {
        const size_t node = (size_t)b * a.N + i;
        const long long sl = i >> 5;
        const int lane = (int)(i & 31);
        const int w = a.sell_w[sl];
        const long long base = a.sell_off[sl] + lane;
        const size_t dbase = (size_t)b * a.sell_len;
        double Fx = 0.0, Fy = 0.0, Fz = 0.0;
        int32_t ci;
        float kap_i = 1.0f;
        if (KAPPA) kap_i = a.kappa[node];

        if (F64) {
            const RecF64 *rin = (const RecF64 *)((n & 1) ? a.rec1 : a.rec0) + (size_t)b * a.N;
            double *dm = (double *)a.dmg + dbase;
            const RecF64 me = rin[i];
            ci = me.coord;
            const int ix = ci & 2047, iy = (ci >> 11) & 2047, iz = ci >> 22;
            const double s0i = me.s0;
            for (int kk = 0; kk < w; ++kk) {
                const long long e = base + 32ll * kk;
                const int j = __ldg(a.sell_col + e);
                if (j < 0) break;
                const RecF64 rj = rin[j];
                const int cj = rj.coord;
                const int ddx = (cj & 2047) - ix, ddy = ((cj >> 11) & 2047) - iy, ddz = (cj >> 22) - iz;
                const int q = ddx * ddx + ddy * ddy + ddz * ddz;
                const double L0 = sL0d[q];
                const double xx = ddx * a.dx, xy = ddy * a.dx, xz = ddz * a.dx;
                const double ex = rj.ux - me.ux, ey = rj.uy - me.uy, ez = rj.uz - me.uz;
                const double yx = xx + ex, yy = xy + ey, yz = xz + ez;
                const double L = sqrt(yx * yx + yy * yy + yz * yz);
                const double s = (2.0 * (xx * ex + xy * ey + xz * ez) + (ex * ex + ey * ey + ez * ez)) /
                                 (L0 * (L + L0));
                const double s0 = 0.5 * (s0i + (double)rj.s0);
                double d = dm[e];
                if (s > s0) {
                    const double dl = law_damage<double>(LAW, s, s0, a.s_ratio * s0, a.k, a.alpha,
                                                         a.inv_1mek, a.inv_1pa);
                    if (dl > d) {
                        d = dl;
                        dm[e] = d;
                    }
                }
                double cv = a.cV;
                if (KAPPA) cv = a.cV * 0.5 * ((double)kap_i + (double)a.kappa[(size_t)b * a.N + j]);
                const double g = cv * (1.0 - d) * s / L;
                Fx += g * yx;
                Fy += g * yy;
                Fz += g * yz;
            }
        } else {
            const RecMixed *rin = (const RecMixed *)((n & 1) ? a.rec1 : a.rec0) + (size_t)b * a.N;
            float *dm = (float *)a.dmg + dbase;
            const float4 hi = __ldg(&rin[i].hi);
            const float4 lo = __ldg(&rin[i].lo);
            ci = __float_as_int(lo.w);
            const int ix = ci & 2047, iy = (ci >> 11) & 2047, iz = ci >> 22;
            const float dxf = (float)a.dx;
            const float cVf = (float)a.cV;
            const float sr = (float)a.s_ratio, kf = (float)a.k, af = (float)a.alpha;
            const float i1 = (float)a.inv_1mek, i2 = (float)a.inv_1pa;
            for (int kk = 0; kk < w; ++kk) {
                const long long e = base + 32ll * kk;
                const int j = __ldg(a.sell_col + e);
                if (j < 0) break;
                const float4 hj = __ldg(&rin[j].hi);
                const float4 lj = __ldg(&rin[j].lo);
                const int cj = __float_as_int(lj.w);
                const int ddx = (cj & 2047) - ix, ddy = ((cj >> 11) & 2047) - iy, ddz = (cj >> 22) - iz;
                const int q = ddx * ddx + ddy * ddy + ddz * ddz;
                const float L0 = sL0f[q];
                const float xx = (float)ddx * dxf, xy = (float)ddy * dxf, xz = (float)ddz * dxf;
                const float ex = (hj.x - hi.x) + (lj.x - lo.x);
                const float ey = (hj.y - hi.y) + (lj.y - lo.y);
                const float ez = (hj.z - hi.z) + (lj.z - lo.z);
                const float yx = xx + ex, yy = xy + ey, yz = xz + ez;
                const float L = sqrtf(yx * yx + yy * yy + yz * yz);
                const float s = (2.0f * (xx * ex + xy * ey + xz * ez) + (ex * ex + ey * ey + ez * ez)) /
                                (L0 * (L + L0));
                const float s0 = 0.5f * (hi.w + hj.w);
                float d = dm[e];
                if (s > s0) {
                    const float dl = law_damage<float>(LAW, s, s0, sr * s0, kf, af, i1, i2);
                    if (dl > d) {
                        d = dl;
                        dm[e] = d;
                    }
                }
                float cv = cVf;
                if (KAPPA) cv = cVf * 0.5f * (kap_i + a.kappa[(size_t)b * a.N + j]);
                const float g = cv * (1.0f - d) * s / L;
                Fx += (double)(g * yx);
                Fy += (double)(g * yy);
                Fz += (double)(g * yz);
            }
        }

        if (FORCE_ONLY) {
            a.F_out[3 * node + 0] = Fx;
            a.F_out[3 * node + 1] = Fy;
            a.F_out[3 * node + 2] = Fz;
        } else {
            const double F[3] = {Fx, Fy, Fz};
            const double U0 = ramp(a, n), U1 = ramp(a, n + 1);
            const double ca = 1.0 - 0.5 * a.zeta * a.dt;
            const double cb = 1.0 + 0.5 * a.zeta * a.dt;
            double un[3];
            double *u = a.u64 + 3 * node;
            double *v = a.v64 + 3 * node;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const uint8_t code = a.codes[3 * i + c];
                double uc = u[c], vc = v[c];
                if (code == 0) {
                    vc = (ca * vc + a.dt * F[c] / a.rho) / cb;
                    uc = uc + a.dt * vc;
                } else if (code == 1) {
                    uc = 0.0;
                    vc = 0.0;
                } else {
                    const double sg = code == 2 ? 1.0 : -1.0;
                    Rloc += (code == 2 ? -F[c] : F[c]) * a.V;
                    vc = sg * (U1 - U0) / a.dt;
                    uc = sg * U1;
                }
                u[c] = uc;
                v[c] = vc;
                un[c] = uc;
            }
            if (F64) {
                RecF64 *rout = (RecF64 *)((n & 1) ? a.rec0 : a.rec1) + (size_t)b * a.N;
                const RecF64 *rin = (const RecF64 *)((n & 1) ? a.rec1 : a.rec0) + (size_t)b * a.N;
                RecF64 r;
                r.ux = un[0];
                r.uy = un[1];
                r.uz = un[2];
                r.s0 = rin[i].s0;
                r.coord = ci;
                rout[i] = r;
            } else {
                RecMixed *rout = (RecMixed *)((n & 1) ? a.rec0 : a.rec1) + (size_t)b * a.N;
                const RecMixed *rin = (const RecMixed *)((n & 1) ? a.rec1 : a.rec0) + (size_t)b * a.N;
                const float hx = (float)un[0], hy = (float)un[1], hz = (float)un[2];
                RecMixed r;
                r.hi = make_float4(hx, hy, hz, rin[i].hi.w);
                r.lo = make_float4((float)(un[0] - (double)hx), (float)(un[1] - (double)hy),
                                   (float)(un[2] - (double)hz), __int_as_float(ci));
                rout[i] = r;
            }
        }
    }

    if (FORCE_ONLY || done) return;  // uniform per block

    // deterministic reaction reduction: warp tree, then warps in order
    Rloc = warp_sum(Rloc);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = Rloc;
    __syncthreads();
    if (warp == 0) {
        double v = lane < kThreads / 32 ? red[lane] : 0.0;
        v = warp_sum(v);
        if (lane == 0) {
            a.partial[(size_t)b * a.nblk + xb] = v;
            __threadfence();
            const unsigned t = atomicAdd(&a.ticket[b], 1u);
            last_flag = (t == (unsigned)(a.nblk - 1));
        }
    }
    __syncthreads();
    if (!last_flag) return;
    if (warp == 0) {
        __threadfence();
        const volatile double *p = a.partial + (size_t)b * a.nblk;
        double v = 0.0;
        for (int t = lane; t < a.nblk; t += 32) v += p[t];
        v = warp_sum(v);
        if (lane == 0) {
            const double R = v;
            if (!isfinite(R)) a.status[b] |= 1;
            if (a.reaction) a.reaction[(size_t)b * a.n_react + a.k_local] = R;
            double Q = a.peak[b];
            int np = a.peak_step[b];
            if (R > Q) {
                Q = R;
                np = n;
                a.peak[b] = Q;
                a.peak_step[b] = np;
            }
            a.step[b] = n + 1;
            if (a.use_stop) {
                if ((Q > 0.0 && n - np >= 100 && R < 0.5 * Q) || n + 1 >= a.max_steps || !isfinite(R))
                    a.done[b] = 1;
            }
            a.ticket[b] = 0u;
        }
    }
}

// ---------------------------------------------------------------- set-up

__global__ void k_slice_width(const int32_t *row_ptr, long long N, long long n_slices, int32_t *w) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_slices) return;
    int m = 0;
    for (int l = 0; l < 32; ++l) {
        const long long i = s * 32 + l;
        if (i < N) m = max(m, row_ptr[i + 1] - row_ptr[i]);
    }
    w[s] = m;
}

__global__ void k_fill_sell(const int32_t *row_ptr, const int32_t *col, long long N,
                            long long n_slices, const long long *off, const int32_t *w,
                            int32_t *sell_col) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_slices * 32) return;
    const long long s = t >> 5;
    const int lane = (int)(t & 31);
    const long long i = s * 32 + lane;
    const int len = i < N ? row_ptr[i + 1] - row_ptr[i] : 0;
    const long long r0 = i < N ? row_ptr[i] : 0;
    for (int k = 0; k < w[s]; ++k) sell_col[off[s] + 32ll * k + lane] = k < len ? col[r0 + k] : -1;
}

__global__ void k_coords(int nx, int ny, long long N, int32_t *coord) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((long long)nx * ny));
    coord[i] = pack_coord(ix, iy, iz);
}

// Per-node Silling-Askari stable step sqrt(2 rho / sum_j c V / |xi_ij|), sum in CSR order.
__global__ void k_dt_sum(const int32_t *row_ptr, const int32_t *col, const int32_t *coord,
                         long long N, double cV, double dx, double rho, double *dti) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int ci = coord[i];
    double sum = 0.0;
    for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
        const int cj = coord[col[p]];
        const int ddx = (cj & 2047) - (ci & 2047), ddy = ((cj >> 11) & 2047) - ((ci >> 11) & 2047),
                  ddz = (cj >> 22) - (ci >> 22);
        const double L = sqrt((double)(ddx * ddx + ddy * ddy + ddz * ddz)) * dx;
        sum += cV / L;
    }
    dti[i] = sum > 0.0 ? sqrt(2.0 * rho / sum) : INFINITY;
}

__global__ void k_min(const double *x, long long n, double *out) {
    __shared__ double sm[1024];
    double m = INFINITY;
    for (long long t = threadIdx.x; t < n; t += blockDim.x) m = fmin(m, x[t]);
    sm[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] = fmin(sm[threadIdx.x], sm[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sm[0];
}

template <bool F64>
__global__ void k_reset(long long N, int B, const float *s0, const int32_t *coord, double *u64,
                        double *v64, void *rec0, void *rec1) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * B) return;
    const long long i = t % N;
    for (int c = 0; c < 3; ++c) {
        u64[3 * t + c] = 0.0;
        v64[3 * t + c] = 0.0;
    }
    if (F64) {
        RecF64 r;
        r.ux = r.uy = r.uz = 0.0;
        r.s0 = s0 ? s0[t] : 1e-4f;
        r.coord = coord[i];
        ((RecF64 *)rec0)[t] = r;
        ((RecF64 *)rec1)[t] = r;
    } else {
        RecMixed r;
        r.hi = make_float4(0.f, 0.f, 0.f, s0 ? s0[t] : 1e-4f);
        r.lo = make_float4(0.f, 0.f, 0.f, __int_as_float(coord[i]));
        ((RecMixed *)rec0)[t] = r;
        ((RecMixed *)rec1)[t] = r;
    }
}

__global__ void k_reset_run(int B, int32_t *step, int32_t *done, int32_t *status, double *peak,
                            int32_t *peak_step, unsigned *ticket, int step0) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    step[b] = step0;
    done[b] = 0;
    status[b] = 0;
    peak[b] = -INFINITY;
    peak_step[b] = -1;
    ticket[b] = 0u;
}

// Load u (and the gather record of the current parity) from caller arrays.
template <bool F64>
__global__ void k_load_u(long long N, int B, const double *u, const double *v, double *u64,
                         double *v64, const int32_t *step, void *rec0, void *rec1) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * B) return;
    const int b = (int)(t / N);
    const int par = step[b] & 1;
    double uu[3];
    for (int c = 0; c < 3; ++c) {
        uu[c] = u ? u[3 * t + c] : u64[3 * t + c];
        u64[3 * t + c] = uu[c];
        if (v) v64[3 * t + c] = v[3 * t + c];
    }
    if (F64) {
        RecF64 *r = (RecF64 *)(par ? rec1 : rec0) + t;
        r->ux = uu[0];
        r->uy = uu[1];
        r->uz = uu[2];
    } else {
        RecMixed *r = (RecMixed *)(par ? rec1 : rec0) + t;
        const float hx = (float)uu[0], hy = (float)uu[1], hz = (float)uu[2];
        float4 hi = r->hi, lo = r->lo;
        hi.x = hx;
        hi.y = hy;
        hi.z = hz;
        lo.x = (float)(uu[0] - (double)hx);
        lo.y = (float)(uu[1] - (double)hy);
        lo.z = (float)(uu[2] - (double)hz);
        r->hi = hi;
        r->lo = lo;
    }
}

// Copy the s0 field into both parities of the record (after a load).
template <bool F64>
__global__ void k_copy_s0_other(long long N, int B, const int32_t *step, void *rec0, void *rec1) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * B) return;
    const int b = (int)(t / N);
    const int par = step[b] & 1;
    if (F64) {
        RecF64 *src = (RecF64 *)(par ? rec1 : rec0) + t;
        RecF64 *dst = (RecF64 *)(par ? rec0 : rec1) + t;
        *dst = *src;
    } else {
        RecMixed *src = (RecMixed *)(par ? rec1 : rec0) + t;
        RecMixed *dst = (RecMixed *)(par ? rec0 : rec1) + t;
        *dst = *src;
    }
}

// CSR-ordered damage <-> SELL-ordered damage.
template <typename T, bool TO_SELL>
__global__ void k_dmg_map(const int32_t *row_ptr, long long N, int B, long long nb,
                          const long long *off, long long sell_len, T *sell, double *csr) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * B) return;
    const int b = (int)(t / N);
    const long long i = t % N;
    const long long s = i >> 5;
    const int lane = (int)(i & 31);
    const int r0 = row_ptr[i], len = row_ptr[i + 1] - r0;
    for (int k = 0; k < len; ++k) {
        const long long e = (size_t)b * sell_len + off[s] + 32ll * k + lane;
        const long long c = (size_t)b * nb + r0 + k;
        if (TO_SELL)
            sell[e] = (T)csr[c];
        else
            csr[c] = (double)sell[e];
    }
}

__global__ void k_store_u(long long N, int B, const double *u64, const double *v64, double *u,
                          double *v) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * N * B) return;
    if (u) u[t] = u64[t];
    if (v) v[t] = v64[t];
}

__global__ void k_run_init(int B, const int32_t *step, int32_t *done, int max_steps) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    if (step[b] >= max_steps) done[b] = 1;
}

__global__ void k_count_active(int B, const int32_t *done, int32_t *host_flag) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int c = 0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) c += done[b] == 0;
    atomicAdd(&cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) *(volatile int32_t *)host_flag = cnt;
}

__global__ void k_copy_out(int B, const double *peak, const int32_t *peak_step,
                           const int32_t *step, double *o_peak, int32_t *o_ps, int32_t *o_nd) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    if (o_peak) o_peak[b] = peak[b];
    if (o_ps) o_ps[b] = peak_step[b];
    if (o_nd) o_nd[b] = step[b];
}

// ------------------------------------------------------------- dispatch

typedef void (*StepKernel)(const StepArgs);

template <bool F64, bool FO>
static StepKernel pick3(int law, bool kappa) {
    if (law == PD_LAW_BILINEAR)
        return kappa ? k_step<F64, 0, true, FO> : k_step<F64, 0, false, FO>;
    return kappa ? k_step<F64, 1, true, FO> : k_step<F64, 1, false, FO>;
}

static StepKernel pick(const pd_state *st, bool force_only) {
    const bool f64 = st->mat.precision == PD_PREC_FP64;
    if (f64) return force_only ? pick3<true, true>(st->mat.law, st->has_kappa)
                               : pick3<true, false>(st->mat.law, st->has_kappa);
    return force_only ? pick3<false, true>(st->mat.law, st->has_kappa)
                      : pick3<false, false>(st->mat.law, st->has_kappa);
}

static StepArgs make_args(const pd_state *st) {
    StepArgs a;
    memset(&a, 0, sizeof(a));
    a.N = st->N;
    a.nblk = st->nblk;
    a.B = st->B;
    a.sell_off = st->sell_off;
    a.sell_w = st->sell_w;
    a.sell_col = st->sell_col;
    a.dmg = st->dmg;
    a.sell_len = st->sell_len;
    a.u64 = st->u64;
    a.v64 = st->v64;
    a.rec0 = st->rec[0];
    a.rec1 = st->rec[1];
    a.kappa = st->kappa;
    a.codes = st->codes;
    a.step = st->step;
    a.done = st->done;
    a.status = st->status;
    a.peak = st->peak;
    a.peak_step = st->peak_step;
    a.partial = st->partial;
    a.ticket = st->ticket;
    a.dt = st->dt;
    a.rho = st->mat.rho;
    a.zeta = st->mat.zeta;
    a.u_max = st->bc.u_max;
    a.n_ramp = st->bc.n_ramp;
    a.max_steps = 0x7fffffff;
    a.use_stop = 0;
    a.cV = st->c * st->V;
    a.V = st->V;
    a.dx = st->g.dx;
    a.s_ratio = st->mat.s_ratio;
    a.k = st->mat.k;
    a.alpha = st->mat.alpha;
    a.inv_1mek = 1.0 / (1.0 - std::exp(-st->mat.k));
    a.inv_1pa = 1.0 / (1.0 + st->mat.alpha);
    return a;
}

static int launch_step(const pd_state *st, const StepArgs &a, bool force_only, cudaStream_t s) {
    StepKernel k = pick(st, force_only);
    const unsigned grid = (unsigned)st->nblk * (unsigned)st->B;
    k<<<grid, kThreads, 0, s>>>(a);
    PD_CHECK_LAUNCH();
    return PD_OK;
}

static unsigned blocks_for(long long n, int bs = 256) { return (unsigned)((n + bs - 1) / bs); }

static void free_state(pd_state *st) {
    if (!st) return;
    cudaFree(st->row_ptr);
    cudaFree(st->sell_off);
    cudaFree(st->sell_w);
    cudaFree(st->sell_col);
    cudaFree(st->dmg);
    cudaFree(st->u64);
    cudaFree(st->v64);
    cudaFree(st->rec[0]);
    cudaFree(st->rec[1]);
    cudaFree(st->kappa);
    cudaFree(st->codes);
    cudaFree(st->coord);
    cudaFree(st->step);
    cudaFree(st->done);
    cudaFree(st->status);
    cudaFree(st->peak);
    cudaFree(st->peak_step);
    cudaFree(st->partial);
    cudaFree(st->ticket);
    if (st->chunk_exec) cudaGraphExecDestroy(st->chunk_exec);
    if (st->host_flag) cudaFreeHost(st->host_flag);
    if (st->ev[0]) cudaEventDestroy(st->ev[0]);
    if (st->ev[1]) cudaEventDestroy(st->ev[1]);
    delete st;
}

static int build_state(pd_state *st, const int32_t *row_ptr, const int32_t *col) {
    const long long N = st->N;
    const int B = st->B;
    cudaStream_t s = 0;
    PD_TRY(dalloc(&st->row_ptr, N + 1));
    PD_CHECK_CUDA(cudaMemcpy(st->row_ptr, row_ptr, (N + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice));
    int32_t last = 0;
    PD_CHECK_CUDA(cudaMemcpy(&last, st->row_ptr + N, sizeof(int32_t), cudaMemcpyDeviceToHost));
    PD_REQUIRE((long long)last == st->nb, "row_ptr[N] = %d does not match n_bonds = %lld", last,
               (long long)st->nb);
    // SELL-32 layout
    st->n_slices = (N + 31) / 32;
    PD_TRY(dalloc(&st->sell_w, st->n_slices));
    PD_TRY(dalloc(&st->sell_off, st->n_slices));
    k_slice_width<<<blocks_for(st->n_slices), 256, 0, s>>>(st->row_ptr, N, st->n_slices, st->sell_w);
    PD_CHECK_LAUNCH();
    std::vector<int32_t> w(st->n_slices);
    std::vector<long long> off(st->n_slices);
    PD_CHECK_CUDA(cudaMemcpy(w.data(), st->sell_w, w.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    long long acc = 0;
    for (long long q = 0; q < st->n_slices; ++q) {
        off[q] = acc;
        acc += 32ll * w[q];
    }
    st->sell_len = acc;
    PD_CHECK_CUDA(cudaMemcpy(st->sell_off, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice));
    PD_TRY(dalloc(&st->sell_col, st->sell_len));
    k_fill_sell<<<blocks_for(st->n_slices * 32), 256, 0, s>>>(st->row_ptr, col, N, st->n_slices,
                                                               st->sell_off, st->sell_w, st->sell_col);
    PD_CHECK_LAUNCH();
    // per-node constants
    PD_TRY(dalloc(&st->coord, N));
    k_coords<<<blocks_for(N), 256, 0, s>>>(st->g.nx, st->g.ny, N, st->coord);
    PD_CHECK_LAUNCH();
    PD_TRY(dalloc(&st->codes, 3 * N));
    PD_TRY(pd_bc_codes(&st->g, &st->bc, st->codes, (pd_stream)s));
    // time step
    if (st->mat.dt > 0.0) {
        st->dt = st->mat.dt;
    } else {
        double *dti = nullptr, *dmin = nullptr;
        PD_TRY(dalloc(&dti, N));
        PD_TRY(dalloc(&dmin, 1));
        k_dt_sum<<<blocks_for(N), 256, 0, s>>>(st->row_ptr, col, st->coord, N, st->c * st->V, st->g.dx,
                                               st->mat.rho, dti);
        k_min<<<1, 1024, 0, s>>>(dti, N, dmin);
        double h = 0.0;
        cudaError_t e = cudaMemcpy(&h, dmin, sizeof(double), cudaMemcpyDeviceToHost);
        cudaFree(dti);
        cudaFree(dmin);
        PD_CHECK_CUDA(e);
        PD_REQUIRE(std::isfinite(h) && h > 0.0, "no bonds: stable time step undefined");
        st->dt = st->mat.dt_safety * h;
    }
    // per-sample arrays
    const bool f64 = st->mat.precision == PD_PREC_FP64;
    const size_t dsz = f64 ? sizeof(double) : sizeof(float);
    PD_CHECK_CUDA(cudaMalloc(&st->dmg, (size_t)B * st->sell_len * dsz));
    PD_TRY(dalloc(&st->u64, 3 * N * B));
    PD_TRY(dalloc(&st->v64, 3 * N * B));
    PD_CHECK_CUDA(cudaMalloc(&st->rec[0], (size_t)B * N * 32));
    PD_CHECK_CUDA(cudaMalloc(&st->rec[1], (size_t)B * N * 32));
    st->nblk = (int)((N + kThreads - 1) / kThreads);
    PD_TRY(dalloc(&st->step, B));
    PD_TRY(dalloc(&st->done, B));
    PD_TRY(dalloc(&st->status, B));
    PD_TRY(dalloc(&st->peak, B));
    PD_TRY(dalloc(&st->peak_step, B));
    PD_TRY(dalloc(&st->partial, (size_t)B * st->nblk));
    PD_TRY(dalloc(&st->ticket, B));
    PD_CHECK_CUDA(cudaHostAlloc((void **)&st->host_flag, 4 * sizeof(int32_t), cudaHostAllocMapped));
    PD_CHECK_CUDA(cudaHostGetDevicePointer((void **)&st->host_flag_dev, st->host_flag, 0));
    PD_CHECK_CUDA(cudaEventCreateWithFlags(&st->ev[0], cudaEventDisableTiming));
    PD_CHECK_CUDA(cudaEventCreateWithFlags(&st->ev[1], cudaEventDisableTiming));
    PD_TRY(pd_state_reset(st, nullptr, nullptr, (pd_stream)s));
    PD_CHECK_CUDA(cudaDeviceSynchronize());
    return PD_OK;
}

}  // namespace pdi

using namespace pdi;

extern "C" int pd_state_create(const pd_grid *g, const int32_t *row_ptr, const int32_t *col,
                               int64_t n_bonds, const pd_material *mat, const pd_bc *bc,
                               int32_t batch, pd_state **out) {
    PD_REQUIRE(out != nullptr, "out is NULL");
    *out = nullptr;
    PD_TRY(validate_grid(g));
    PD_REQUIRE(row_ptr && col && mat && bc, "row_ptr, col, mat and bc are required");
    PD_REQUIRE(batch >= 1 && batch <= 65536, "batch must be in [1, 65536]");
    PD_REQUIRE(n_bonds >= 0 && n_bonds < (1ll << 31), "n_bonds out of range");
    PD_REQUIRE(mat->law == PD_LAW_BILINEAR || mat->law == PD_LAW_EXPLINEAR, "unknown law %d", mat->law);
    PD_REQUIRE(mat->precision == PD_PREC_FP64 || mat->precision == PD_PREC_MIXED, "unknown precision");
    PD_REQUIRE(mat->E > 0 && mat->rho > 0 && mat->s_ratio > 1.0, "E, rho > 0 and s_ratio > 1 required");
    PD_REQUIRE(mat->dt > 0 || mat->dt_safety > 0, "dt or dt_safety must be positive");
    PD_REQUIRE(mat->zeta >= 0, "zeta must be >= 0");
    PD_REQUIRE(bc->type == PD_BC_BAR_TENSION || bc->type == PD_BC_BEAM_3PT, "unknown bc type");
    PD_REQUIRE(bc->n_ramp >= 1, "n_ramp must be >= 1");
    PD_REQUIRE(g->m_ratio * g->m_ratio <= 64.0, "m_ratio^2 must be <= 64");
    pd_state *st = new pd_state();
    memset(st, 0, sizeof(*st));
    st->g = *g;
    st->mat = *mat;
    st->bc = *bc;
    st->B = batch;
    st->N = (int64_t)g->nx * g->ny * g->nz;
    st->nb = n_bonds;
    const double delta = g->m_ratio * g->dx;
    st->c = 12.0 * mat->E / (M_PI * delta * delta * delta * delta);
    st->V = g->dx * g->dx * g->dx;
    int rc = build_state(st, row_ptr, col);
    if (rc != PD_OK) {
        free_state(st);
        return rc;
    }
    *out = st;
    return PD_OK;
}

extern "C" int pd_state_destroy(pd_state *st) {
    if (st) {
        cudaDeviceSynchronize();
        free_state(st);
    }
    return PD_OK;
}

extern "C" int pd_state_info(const pd_state *st, double *dt, double *c, int64_t *n_nodes,
                             int64_t *n_bonds) {
    PD_REQUIRE(st != nullptr, "state is NULL");
    if (dt) *dt = st->dt;
    if (c) *c = st->c;
    if (n_nodes) *n_nodes = st->N;
    if (n_bonds) *n_bonds = st->nb;
    return PD_OK;
}

extern "C" int pd_state_reset(pd_state *st, const float *s0, const float *kappa, pd_stream stream) {
    PD_REQUIRE(st != nullptr, "state is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const long long NB = st->N * st->B;
    const bool f64 = st->mat.precision == PD_PREC_FP64;
    const size_t dsz = f64 ? sizeof(double) : sizeof(float);
    PD_CHECK_CUDA(cudaMemsetAsync(st->dmg, 0, (size_t)st->B * st->sell_len * dsz, s));
    if (f64)
        k_reset<true><<<blocks_for(NB), 256, 0, s>>>(st->N, st->B, s0, st->coord, st->u64, st->v64,
                                                     st->rec[0], st->rec[1]);
    else
        k_reset<false><<<blocks_for(NB), 256, 0, s>>>(st->N, st->B, s0, st->coord, st->u64, st->v64,
                                                      st->rec[0], st->rec[1]);
    PD_CHECK_LAUNCH();
    if (kappa) {
        if (!st->kappa) PD_TRY(dalloc(&st->kappa, (size_t)NB));
        PD_CHECK_CUDA(cudaMemcpyAsync(st->kappa, kappa, (size_t)NB * sizeof(float), cudaMemcpyDeviceToDevice, s));
        st->has_kappa = true;
    } else {
        st->has_kappa = false;
    }
    if (st->chunk_exec) {  // the captured chunk bakes has_kappa into the kernel choice
        cudaGraphExecDestroy(st->chunk_exec);
        st->chunk_exec = nullptr;
    }
    k_reset_run<<<blocks_for(st->B), 256, 0, s>>>(st->B, st->step, st->done, st->status, st->peak,
                                                  st->peak_step, st->ticket, 0);
    PD_CHECK_LAUNCH();
    return PD_OK;
}

extern "C" int pd_state_load(pd_state *st, const double *u, const double *v, const double *d,
                             int32_t step, pd_stream stream) {
    PD_REQUIRE(st != nullptr, "state is NULL");
    PD_REQUIRE(step >= 0, "step must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    const long long NB = st->N * st->B;
    const bool f64 = st->mat.precision == PD_PREC_FP64;
    k_reset_run<<<blocks_for(st->B), 256, 0, s>>>(st->B, st->step, st->done, st->status, st->peak,
                                                  st->peak_step, st->ticket, step);
    PD_CHECK_LAUNCH();
    if (f64) {
        k_load_u<true><<<blocks_for(NB), 256, 0, s>>>(st->N, st->B, u, v, st->u64, st->v64, st->step,
                                                      st->rec[0], st->rec[1]);
        k_copy_s0_other<true><<<blocks_for(NB), 256, 0, s>>>(st->N, st->B, st->step, st->rec[0], st->rec[1]);
    } else {
        k_load_u<false><<<blocks_for(NB), 256, 0, s>>>(st->N, st->B, u, v, st->u64, st->v64, st->step,
                                                       st->rec[0], st->rec[1]);
        k_copy_s0_other<false><<<blocks_for(NB), 256, 0, s>>>(st->N, st->B, st->step, st->rec[0], st->rec[1]);
    }
    PD_CHECK_LAUNCH();
    if (d) {
        if (f64)
            k_dmg_map<double, true><<<blocks_for(NB), 256, 0, s>>>(
                st->row_ptr, st->N, st->B, st->nb, st->sell_off, st->sell_len, (double *)st->dmg, (double *)d);
        else
            k_dmg_map<float, true><<<blocks_for(NB), 256, 0, s>>>(
                st->row_ptr, st->N, st->B, st->nb, st->sell_off, st->sell_len, (float *)st->dmg, (double *)d);
        PD_CHECK_LAUNCH();
    }
    return PD_OK;
}

extern "C" int pd_state_store(const pd_state *st, double *u, double *v, double *d, pd_stream stream) {
    PD_REQUIRE(st != nullptr, "state is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const long long NB = st->N * st->B;
    if (u || v) {
        k_store_u<<<blocks_for(3 * NB), 256, 0, s>>>(st->N, st->B, st->u64, st->v64, u, v);
        PD_CHECK_LAUNCH();
    }
    if (d) {
        if (st->mat.precision == PD_PREC_FP64)
            k_dmg_map<double, false><<<blocks_for(NB), 256, 0, s>>>(
                st->row_ptr, st->N, st->B, st->nb, st->sell_off, st->sell_len, (double *)st->dmg, d);
        else
            k_dmg_map<float, false><<<blocks_for(NB), 256, 0, s>>>(
                st->row_ptr, st->N, st->B, st->nb, st->sell_off, st->sell_len, (float *)st->dmg, d);
        PD_CHECK_LAUNCH();
    }
    return PD_OK;
}

extern "C" int pd_force(pd_state *st, double *F, pd_stream stream) {
    PD_REQUIRE(st != nullptr && F != nullptr, "state and F are required");
    StepArgs a = make_args(st);
    a.F_out = F;
    return launch_step(st, a, true, (cudaStream_t)stream);
}

extern "C" int pd_step(pd_state *st, int32_t n_steps, double *reaction, pd_stream stream) {
    PD_REQUIRE(st != nullptr, "state is NULL");
    PD_REQUIRE(n_steps >= 0, "n_steps must be >= 0");
    StepArgs a = make_args(st);
    a.reaction = reaction;
    a.n_react = n_steps;
    for (int k = 0; k < n_steps; ++k) {
        a.k_local = k;
        PD_TRY(launch_step(st, a, false, (cudaStream_t)stream));
    }
    return PD_OK;
}

extern "C" int pd_run_to_peak(pd_state *st, int32_t max_steps, double *peak, int32_t *peak_step,
                              int32_t *n_done, pd_stream stream) {
    PD_REQUIRE(st != nullptr, "state is NULL");
    PD_REQUIRE(max_steps >= 0, "max_steps must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    const int chunk = 64;
    if (!st->chunk_exec || st->chunk_max_steps != max_steps) {
        if (st->chunk_exec) {
            cudaGraphExecDestroy(st->chunk_exec);
            st->chunk_exec = nullptr;
        }
        cudaStream_t cs;
        PD_CHECK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        StepArgs a = make_args(st);
        a.use_stop = 1;
        a.max_steps = max_steps;
        StepKernel k = pick(st, false);
        const unsigned grid = (unsigned)st->nblk * (unsigned)st->B;
        cudaGraph_t graph;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int q = 0; q < chunk; ++q) k<<<grid, kThreads, 0, cs>>>(a);
            e = cudaStreamEndCapture(cs, &graph);
        }
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(&st->chunk_exec, graph, 0);
            cudaGraphDestroy(graph);
        }
        cudaStreamDestroy(cs);
        PD_CHECK_CUDA(e);
        st->chunk_steps = chunk;
        st->chunk_max_steps = max_steps;
    }
    k_run_init<<<blocks_for(st->B), 256, 0, s>>>(st->B, st->step, st->done, max_steps);
    PD_CHECK_LAUNCH();
    const int n_chunks = max_steps / chunk + 1;
    for (int c = 0; c < n_chunks; ++c) {
        PD_CHECK_CUDA(cudaGraphLaunch(st->chunk_exec, s));
        k_count_active<<<1, 256, 0, s>>>(st->B, st->done, st->host_flag_dev + (c & 1));
        PD_CHECK_LAUNCH();
        PD_CHECK_CUDA(cudaEventRecord(st->ev[c & 1], s));
        if (c >= 1) {
            PD_CHECK_CUDA(cudaEventSynchronize(st->ev[(c - 1) & 1]));
            if (((volatile int32_t *)st->host_flag)[(c - 1) & 1] == 0) break;
        }
    }
    k_copy_out<<<blocks_for(st->B), 256, 0, s>>>(st->B, st->peak, st->peak_step, st->step, peak,
                                                  peak_step, n_done);
    PD_CHECK_LAUNCH();
    std::vector<int32_t> status(st->B);
    PD_CHECK_CUDA(cudaMemcpyAsync(status.data(), st->status, st->B * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PD_CHECK_CUDA(cudaStreamSynchronize(s));
    for (int b = 0; b < st->B; ++b)
        if (status[b] & 1) {
            set_error("non-finite reaction in sample %d", b);
            return PD_ERR_NAN;
        }
    return PD_OK;
}
