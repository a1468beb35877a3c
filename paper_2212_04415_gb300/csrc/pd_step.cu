// pd_step.cu -- the explicit bond-based peridynamic time step (Sections 2-3,
// Appendix A): bond kinematics, softening law with irreversible damage,
// deterministic nodal force sums, damped leapfrog update under displacement
// control, and the FP64 reaction / peak-load reduction.
//
// Layout (per state; B samples share one mesh):
//   * The grid is regular, so every bond of node i is one of the n_off
//     stencil offsets k (|k|^2 <= m^2, xi = dx k). The CSR neighbour list is
//     stored as one byte per directed bond (the stencil id).
//   * Nodes are grouped in bricks of 8 x BY x BZ; a slice is the 8
//     x-consecutive nodes of one brick row. Slots are slot-major inside a
//     slice (SELL-8) and rows are padded with id 0xFF to a multiple of 4.
//     A warp serves one slice at a time: lane L takes node c = L % 8 and
//     sub-lane t = L / 8, i.e. slots t, t + 4, t + 8, ...; round m of the warp
//     reads the 32 consecutive elements off[s] + 32 m + L (one id byte and one
//     damage word per lane: coalesced).
//   * Damage per directed bond in the same order, per sample. Both directed
//     copies of a bond evolve identically: the stretch, the per-bond
//     properties and the law are symmetric in (i, j) bit for bit.
//   * Gather records per node, double-buffered by step parity:
//       mixed: float4 hi = (u_hi, s0), float4 lo = (u_lo, kappa), u = u_hi + u_lo
//              (double-float), so u_j - u_i keeps FP64-like accuracy in FP32;
//       fp64:  double4 (u, s0).
//   * Mixed path: one block per (brick, sample) stages the brick's records
//     and a halo of the stencil radius in shared memory, so every bond
//     gathers from shared memory (brick-local stencil offsets); only the id
//     and damage streams and the owner's update touch global memory.
//   * velocities: mixed path double-float float4 hi/lo pairs, fp64 path FP64
//     (the fp64 path also keeps FP64 u next to its records).
// Arithmetic: GB300 runs FP64 at about 1/64 of the FP32 rate, so the mixed
// path issues no FP64 instruction per bond or per node. Each lane sums its
// bonds in FP32 over groups of 4 rounds and adds each group to a compensated
// (TwoSum) accumulator, the 4 lane partials are added in double-float along a
// fixed xor tree (TwoSum is exact, so every sub-lane ends with the same
// total), and sub-lane t integrates component t of its node in double-float
// arithmetic (about 48 significant bits). FP64 is used for the reaction of
// prescribed DOFs and its reduction only. The fp64 path does everything in
// FP64 with global gathers. Order is fixed everywhere, so results are
// deterministic with no atomics. Blocks are ordered sample-fastest so that
// the samples of a batch stream the shared stencil ids through L2 together.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "pd_device.cuh"

namespace pdi {

// One explicit step (or, with FORCE_ONLY, one force evaluation) of every
// (sample, node) pair. Grid: n_bricks * B blocks, sample fastest; the warps of
// a block take the brick's slices in turn. After the bond loop every sub-lane
// of a node holds the node's total force; sub-lane t integrates component t.
template <bool F64, int LAW, bool KAPPA, bool FORCE_ONLY>
__global__ void __launch_bounds__(kThreads, 2) k_step(const StepArgs a) {
    constexpr int T = kLanes, C = kSlice;
    extern __shared__ float4 s_rec[];  // mixed: staged hi[Wtot] then lo[Wtot]
    __shared__ float4 s_xi[kTab];
    __shared__ int s_off[kTab];
    __shared__ double4_32a s_xid[F64 ? kTab : 1];
    __shared__ double red[kWarps];
    __shared__ double s_U[2];
    __shared__ float s_pre[4];
    __shared__ unsigned s_cnt;

    const int b = blockIdx.x % a.B;
    const int brick = blockIdx.x / a.B;
    const bool done = FORCE_ONLY ? false : (a.done[a.par * a.B + b] != 0);
    const int n = a.step[a.par * a.B + b];
    if (done) {  // block-uniform
        if (brick == 0 && threadIdx.x == 0) carry_done(a, b);
        return;
    }
    for (int q = threadIdx.x; q < kTab; q += kThreads) {
        s_xi[q] = a.xi_tab[q];
        s_off[q] = a.off_tab[q];
        if (F64) s_xid[q] = a.xid_tab[q];
    }
    if (threadIdx.x < kWarps) red[threadIdx.x] = 0.0;
    if (threadIdx.x == 0) {
        if (F64) {
            s_U[0] = ramp(a, n);
            s_U[1] = ramp(a, n + 1);
        } else {
            df U1, vp;
            prescribed(a, n, U1, vp);
            s_pre[0] = U1.hi;
            s_pre[1] = U1.lo;
            s_pre[2] = vp.hi;
            s_pre[3] = vp.lo;
        }
        s_cnt = 0u;
    }
    const int bx = brick % a.nbx, by = (brick / a.nbx) % a.nby, bz = brick / (a.nbx * a.nby);
    const int x0 = kSlice * bx, y0 = a.BY * by, z0 = a.BZ * bz;
    const size_t BN = (size_t)a.B * a.N;
    const int Wtot = a.Wx * a.Wy * a.Wz;
    float4 *s_hi = s_rec, *s_lo = s_rec + Wtot;
    if (!F64 && !done) {
        // stage the brick and its halo (cells outside the grid are never read)
        const float4 *rhi = (const float4 *)((n & 1) ? a.rec1 : a.rec0) + (size_t)b * a.N;
        const float4 *rlo = rhi + BN;
        for (int q = threadIdx.x; q < Wtot; q += kThreads) {
            const int lx = q % a.Wx, ly = (q / a.Wx) % a.Wy, lz = q / (a.Wx * a.Wy);
            const int gx = x0 - a.H + lx, gy = y0 - a.H + ly, gz = z0 - a.H + lz;
            float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
            if (gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz) {
                const int gi = gx + a.nx * (gy + a.ny * gz);
                h = __ldg(rhi + gi);
                l = __ldg(rlo + gi);
            }
            s_hi[q] = h;
            s_lo[q] = l;
        }
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = lane % C, t = lane / C;
    double Rloc = 0.0;  // this thread's share of the reaction (FP64)

    if (!done) {
        for (int r = warp; r < a.BY * a.BZ; r += kWarps) {
            const long long sl = (long long)brick * (a.BY * a.BZ) + r;
            const int nv = a.slice_nv[sl];
            if (nv == 0) continue;  // warp-uniform: a brick row outside the grid
            const bool own = c < nv;
            const int ii = a.slice_i0[sl] + c;
            const size_t node = (size_t)b * a.N + ii;
            const int M = a.sell_m[sl];
            const uint8_t *ids = a.ids + a.sell_off[sl] + lane;
            if (F64) {
                double Fx = 0.0, Fy = 0.0, Fz = 0.0;
                const double4_32a *rin = (const double4_32a *)((n & 1) ? a.rec1 : a.rec0) + (size_t)b * a.N;
                if (own) {
                    double *dm = (double *)a.dmg + (size_t)b * a.sell_len + a.sell_off[sl] + lane;
                    const double4_32a me = rin[ii];
                    const double kap_i = KAPPA ? (double)a.kappa[node] : 1.0;
                    for (int m = 0; m < M; ++m) {
                        const int id = ids[32 * m];
                        const int j = ii + s_off[id];
                        const double4_32a xl = s_xid[id];
                        const double4_32a rj = rin[j];
                        const double ex = rj.x - me.x, ey = rj.y - me.y, ez = rj.z - me.z;
                        const double yx = xl.x + ex, yy = xl.y + ey, yz = xl.z + ez;
                        const double L = sqrt(yx * yx + yy * yy + yz * yz);
                        const double s = (2.0 * (xl.x * ex + xl.y * ey + xl.z * ez) + (ex * ex + ey * ey + ez * ez)) /
                                         (xl.w * (L + xl.w));
                        const double s0 = 0.5 * (me.w + rj.w);
                        double d = dm[32 * m];
                        if (s > s0) {
                            const double dl =
                                law_damage<double>(LAW, s, s0, crit_stretch(s0, a.s_ratio, a.gfA), a.k, a.alpha,
                                                   a.inv_1mek, a.inv_1pa);
                            if (dl > d) {
                                d = dl;
                                dm[32 * m] = d;
                            }
                        }
                        double cv = a.cV;
                        if (KAPPA) cv = a.cV * 0.5 * (kap_i + (double)a.kappa[(size_t)b * a.N + j]);
                        // a broken bond carries no force (its direction is undefined at L = 0)
                        const double g = d < 1.0 ? cv * (1.0 - d) * s / L : 0.0;
                        Fx += g * yx;
                        Fy += g * yy;
                        Fz += g * yz;
                    }
                }
#pragma unroll
                for (int o = C; o < 32; o <<= 1) {
                    Fx += __shfl_xor_sync(0xffffffffu, Fx, o);
                    Fy += __shfl_xor_sync(0xffffffffu, Fy, o);
                    Fz += __shfl_xor_sync(0xffffffffu, Fz, o);
                }
                if (own) {
                    for (int q = t; q < 3; q += T) {
                        const double F = pick3(Fx, Fy, Fz, q);
                        if (FORCE_ONLY) {
                            a.F_out[3 * node + q] = F;
                            continue;
                        }
                        const uint8_t code = a.codes[3 * (size_t)ii + q];
                        double uc = a.u64[3 * node + q], vc = a.v64[3 * node + q];
                        if (code == 0) {
                            vc = (a.ca * vc + a.dtr * F) * a.icb;
                            uc = uc + a.dt * vc;
                        } else if (code == 1) {
                            uc = 0.0;
                            vc = 0.0;
                        } else {
                            const double sg = code == 2 ? 1.0 : -1.0;
                            Rloc -= sg * F;
                            vc = sg * (s_U[1] - s_U[0]) * a.idt;
                            uc = sg * s_U[1];
                        }
                        a.u64[3 * node + q] = uc;
                        a.v64[3 * node + q] = vc;
                        double *ro = (double *)((double4_32a *)((n & 1) ? a.rec0 : a.rec1) + node);
                        ro[q] = uc;
                    }
                }
            } else {
                float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
                const int ly = r % a.BY, lz = r / a.BY;
                const int il = (a.H + c) + a.Wx * ((a.H + ly) + a.Wy * (a.H + lz));
                const float4 hi = s_hi[il], lo = s_lo[il];
                if (own) {
                    float *dm = (float *)a.dmg + (size_t)b * a.sell_len + a.sell_off[sl] + lane;
                    const float cVf = a.cVf;
                    const float sr = a.s_ratio_f, kf = a.k_f, af = a.alpha_f;
                    const float i1 = a.inv_1mek_f, i2 = a.inv_1pa_f;
                    // Padding slots (id 0xFF) point at the node itself with |xi| = dx:
                    // zero stretch, zero force, no damage write, no branch.
                    // Bonds are summed in plain FP32 over groups of 4 rounds and each
                    // group sum is added to the compensated (TwoSum) accumulator.
                    for (int m0 = 0; m0 < M; m0 += 4) {
                        float px = 0.f, py = 0.f, pz = 0.f;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int m = m0 + q;
                            if (m < M) {
                                const int id = __ldg(ids + 32 * m);
                                const int jl = il + s_off[id];
                                const float4 xl = s_xi[id];
                                const float4 hj = s_hi[jl];
                                const float4 lj = s_lo[jl];
                                const float ex = (hj.x - hi.x) + (lj.x - lo.x);
                                const float ey = (hj.y - hi.y) + (lj.y - lo.y);
                                const float ez = (hj.z - hi.z) + (lj.z - lo.z);
                                const float yx = xl.x + ex, yy = xl.y + ey, yz = xl.z + ez;
                                const float y2 = yx * yx + yy * yy + yz * yz;
                                const float rL = rsqrtf(y2);
                                const float L = y2 * rL;
                                const float s = __fdividef(
                                    2.0f * (xl.x * ex + xl.y * ey + xl.z * ez) + (ex * ex + ey * ey + ez * ez),
                                    xl.w * (L + xl.w));
                                const float s0 = 0.5f * (hi.w + hj.w);
                                float d = dm[32 * m];
                                if (s > s0) {
                                    const float dl = law_damage<float>(LAW, s, s0, crit_stretch(s0, sr, a.gfA_f), kf, af, i1, i2);
                                    if (dl > d) {
                                        d = dl;
                                        dm[32 * m] = d;
                                    }
                                }
                                float cv = cVf;
                                if (KAPPA) cv = cVf * 0.5f * (lo.w + lj.w);
                                // a broken bond carries no force (its direction is undefined at |y| = 0)
                                const float g = d < 1.0f ? cv * (1.0f - d) * s * rL : 0.0f;
                                px += g * yx;
                                py += g * yy;
                                pz += g * yz;
                            }
                        }
                        two_sum_acc(sx, cx, px);
                        two_sum_acc(sy, cy, py);
                        two_sum_acc(sz, cz, pz);
                    }
                }
                // add the 4 sub-lane partials of each node in double-float (fixed
                // xor tree; TwoSum is exact, so partners get identical totals)
#pragma unroll
                for (int o = C; o < 32; o <<= 1) {
                    const float px = __shfl_xor_sync(0xffffffffu, sx, o), qx = __shfl_xor_sync(0xffffffffu, cx, o);
                    const float py = __shfl_xor_sync(0xffffffffu, sy, o), qy = __shfl_xor_sync(0xffffffffu, cy, o);
                    const float pz = __shfl_xor_sync(0xffffffffu, sz, o), qz = __shfl_xor_sync(0xffffffffu, cz, o);
                    df rr = two_sum(sx, px);
                    sx = rr.hi;
                    cx = rr.lo + (cx + qx);
                    rr = two_sum(sy, py);
                    sy = rr.hi;
                    cy = rr.lo + (cy + qy);
                    rr = two_sum(sz, pz);
                    sz = rr.hi;
                    cz = rr.lo + (cz + qz);
                }
                if (own) {
                    for (int q = t; q < 3; q += T) {
                        const df F = two_sum(pick3(sx, sy, sz, q), pick3(cx, cy, cz, q));
                        if (FORCE_ONLY) {
                            a.F_out[3 * node + q] = (double)F.hi + (double)F.lo;
                            continue;
                        }
                        const uint8_t code = a.codes[3 * (size_t)ii + q];
                        df u = {pick3(hi.x, hi.y, hi.z, q), pick3(lo.x, lo.y, lo.z, q)};
                        float *vh = (float *)(a.vdf + node);
                        float *vl = (float *)(a.vdf + BN + node);
                        df v = {vh[q], vl[q]};
                        if (code == 0) {
                            v = df_mul(df_add(df_mul(a.ca_df, v), df_mul(a.dtr_df, F)), a.icb_df);
                            u = df_add(u, df_mul(a.dt_df, v));
                        } else if (code == 1) {
                            u = {0.f, 0.f};
                            v = {0.f, 0.f};
                        } else {
                            const float sg = code == 2 ? 1.0f : -1.0f;
                            Rloc -= (double)sg * ((double)F.hi + (double)F.lo);
                            v = df{sg * s_pre[2], sg * s_pre[3]};
                            u = df{sg * s_pre[0], sg * s_pre[1]};
                        }
                        vh[q] = v.hi;
                        vl[q] = v.lo;
                        float *oh = (float *)((float4 *)((n & 1) ? a.rec0 : a.rec1) + node);
                        float *ol = (float *)((float4 *)((n & 1) ? a.rec0 : a.rec1) + BN + node);
                        oh[q] = u.hi;
                        ol[q] = u.lo;
                    }
                }
            }
        }
    }

    if (FORCE_ONLY || done) return;  // uniform per block

    const int ridx = a.brick_ridx[brick];
    if (ridx >= 0) {
        // this path never defers its reaction: the view is the buffer as read
        RunView rv;
        rv.n = n;
        rv.dn = 0;
        rv.Q = 0.0;  // read from the buffer by the finishing block
        rv.np = 0;
        rv.Rp = 0.0;
        rv.have = 0;
        reaction_finish(a, Rloc, b, ridx, warp, lane, kWarps, red, &s_cnt, rv);
    }
}

// ---------------------------------------------------------------- set-up

// Rounds per slice: ceil(max row length / 4).
__global__ void k_slice_rounds(const int32_t *row_ptr, const int32_t *i0, const int32_t *nv, long long n_slices,
                               int32_t *m) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_slices) return;
    int w = 0;
    for (int l = 0; l < nv[s]; ++l) {
        const int i = i0[s] + l;
        w = max(w, row_ptr[i + 1] - row_ptr[i]);
    }
    m[s] = (w + kLanes - 1) / kLanes;
}

// Stencil id of every slot; flags neighbours that are not stencil offsets.
__global__ void k_fill_ids(const int32_t *row_ptr, const int32_t *col, const int32_t *coord, const int32_t *i0,
                           const int32_t *nv, long long n_slices, const long long *off, const int32_t *m,
                           const int16_t *box, int R, uint8_t *ids, int32_t *bad) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_slices * kSlice) return;
    const long long s = q / kSlice;
    const int c = (int)(q % kSlice);
    const bool valid = c < nv[s];
    const int i = i0[s] + c;
    const int len = valid ? row_ptr[i + 1] - row_ptr[i] : 0;
    const int W = kLanes * m[s];
    const int ci = valid ? coord[i] : 0;
    const int D = 2 * R + 1;
    for (int k = 0; k < W; ++k) {
        uint8_t id = kPad;
        if (k < len) {
            const int cj = coord[col[row_ptr[i] + k]];
            const int dx = (cj & 2047) - (ci & 2047), dy = ((cj >> 11) & 2047) - ((ci >> 11) & 2047),
                      dz = (cj >> 22) - (ci >> 22);
            int v = -1;
            if (abs(dx) <= R && abs(dy) <= R && abs(dz) <= R) v = box[(dz + R) * D * D + (dy + R) * D + (dx + R)];
            if (v < 0) {
                *bad = 1;
                v = kPad;
            }
            id = (uint8_t)v;
        }
        ids[off[s] + (long long)k * kSlice + c] = id;
    }
}

__global__ void k_coords(int nx, int ny, long long N, int32_t *coord) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((long long)nx * ny));
    coord[i] = pack_coord(ix, iy, iz);
}

// Per-node Silling-Askari stable step sqrt(2 rho / sum_j c V / |xi_ij|), sum in CSR order.
__global__ void k_dt_sum(const int32_t *row_ptr, const int32_t *col, const int32_t *coord, long long N, double cV,
                         double dx, double rho, double *dti) {
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
__global__ void k_reset(long long N, int B, const float *s0, const double *s0d, const float *kappa, double *u64,
                        double *v64, float4 *vdf, void *rec0, void *rec1) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * B) return;
    const float s = s0d ? (float)s0d[t] : (s0 ? s0[t] : 1e-4f);
    if (F64) {
        for (int c = 0; c < 3; ++c) {
            u64[3 * t + c] = 0.0;
            v64[3 * t + c] = 0.0;
        }
        const double4_32a r = make_double4_32a(0.0, 0.0, 0.0, s0d ? s0d[t] : (double)s);
        ((double4_32a *)rec0)[t] = r;
        ((double4_32a *)rec1)[t] = r;
    } else {
        const size_t BN = (size_t)N * B;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 hi = make_float4(0.f, 0.f, 0.f, s);
        const float4 lo = make_float4(0.f, 0.f, 0.f, kappa ? kappa[t] : 1.0f);
        vdf[t] = z;
        vdf[BN + t] = z;
        ((float4 *)rec0)[t] = hi;
        ((float4 *)rec1)[t] = hi;
        ((float4 *)rec0)[BN + t] = lo;
        ((float4 *)rec1)[BN + t] = lo;
    }
}

__global__ void k_reset_run(int B, int32_t *step, int32_t *done, int32_t *pend, double *pk2, int32_t *ps2,
                            int32_t *status, double *peak, int32_t *peak_step, unsigned *ticket, int step0) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    for (int p = 0; p < 2; ++p) {
        step[p * B + b] = step0;
        done[p * B + b] = 0;
        pend[p * B + b] = 0;
        pk2[p * B + b] = -INFINITY;
        ps2[p * B + b] = -1;
    }
    status[b] = 0;
    peak[b] = -INFINITY;
    peak_step[b] = -1;
    ticket[b] = 0u;
}

// Load u, v from caller arrays (NULL keeps the current values) and refresh
// both parities of the gather records; mixed path splits into double-float.
template <bool F64>
__global__ void k_load_u(long long N, int B, const double *u, const double *v, double *u64, double *v64,
                         float4 *vdf, const int32_t *step, void *rec0, void *rec1) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * B) return;
    const size_t BN = (size_t)N * B;
    if (F64) {
        double uu[3];
        for (int c = 0; c < 3; ++c) {
            uu[c] = u ? u[3 * t + c] : u64[3 * t + c];
            u64[3 * t + c] = uu[c];
            if (v) v64[3 * t + c] = v[3 * t + c];
        }
        for (int p = 0; p < 2; ++p) {
            double4_32a *r = (double4_32a *)(p ? rec1 : rec0) + t;
            r->x = uu[0];
            r->y = uu[1];
            r->z = uu[2];
        }
    } else {
        const int par = step[t / N] & 1;
        const float4 *cur_h = (const float4 *)(par ? rec1 : rec0) + t;
        const float4 *cur_l = (const float4 *)(par ? rec1 : rec0) + BN + t;
        float hx[3], lx[3];
        for (int c = 0; c < 3; ++c) {
            if (u) {
                const df d = df_split(u[3 * t + c]);
                hx[c] = d.hi;
                lx[c] = d.lo;
            } else {
                hx[c] = ((const float *)cur_h)[c];
                lx[c] = ((const float *)cur_l)[c];
            }
        }
        for (int p = 0; p < 2; ++p) {
            float4 *h = (float4 *)(p ? rec1 : rec0) + t;
            float4 *l = (float4 *)(p ? rec1 : rec0) + BN + t;
            h->x = hx[0];
            h->y = hx[1];
            h->z = hx[2];
            l->x = lx[0];
            l->y = lx[1];
            l->z = lx[2];
        }
        if (v) {
            const df a = df_split(v[3 * t + 0]), b = df_split(v[3 * t + 1]), c = df_split(v[3 * t + 2]);
            vdf[t] = make_float4(a.hi, b.hi, c.hi, 0.f);
            vdf[BN + t] = make_float4(a.lo, b.lo, c.lo, 0.f);
        }
    }
}

// Slice and lane of node i in the brick layout.
__device__ __forceinline__ long long slice_of(int i, int nx, int ny, int BY, int BZ, int nbx, int nby, int *lane) {
    const int ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
    const long long brick = (ix / kSlice) + (long long)nbx * ((iy / BY) + (long long)nby * (iz / BZ));
    *lane = ix % kSlice;
    return brick * (BY * BZ) + (iy % BY) + BY * (iz % BZ);
}

// CSR-ordered damage <-> SELL-ordered damage.
template <typename T, bool TO_SELL>
__global__ void k_dmg_map(const int32_t *row_ptr, long long N, int B, long long nb, int nx, int ny, int BY, int BZ,
                          int nbx, int nby, const long long *off, long long sell_len, T *sell, double *csr) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * B) return;
    const int b = (int)(t / N);
    const int i = (int)(t % N);
    int c;
    const long long s = slice_of(i, nx, ny, BY, BZ, nbx, nby, &c);
    const int r0 = row_ptr[i], len = row_ptr[i + 1] - r0;
    for (int k = 0; k < len; ++k) {
        const long long e = (long long)b * sell_len + off[s] + (long long)k * kSlice + c;
        const long long q = (long long)b * nb + r0 + k;
        if (TO_SELL)
            sell[e] = (T)csr[q];
        else
            csr[q] = (double)sell[e];
    }
}

// Copy u, v out as FP64 (the mixed path adds its double-float pairs).
template <bool F64>
__global__ void k_store_u(long long N, int B, const double *u64, const double *v64, const float4 *vdf,
                          const int32_t *step, const void *rec0, const void *rec1, double *u, double *v) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * B) return;
    const size_t BN = (size_t)N * B;
    if (F64) {
        for (int c = 0; c < 3; ++c) {
            if (u) u[3 * t + c] = u64[3 * t + c];
            if (v) v[3 * t + c] = v64[3 * t + c];
        }
    } else {
        const int par = step[t / N] & 1;
        const float *h = (const float *)((const float4 *)(par ? rec1 : rec0) + t);
        const float *l = (const float *)((const float4 *)(par ? rec1 : rec0) + BN + t);
        const float *vh = (const float *)(vdf + t);
        const float *vl = (const float *)(vdf + BN + t);
        for (int c = 0; c < 3; ++c) {
            if (u) u[3 * t + c] = (double)h[c] + (double)l[c];
            if (v) v[3 * t + c] = (double)vh[c] + (double)vl[c];
        }
    }
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

__global__ void k_copy_out(int B, const double *peak, const int32_t *peak_step, const int32_t *step,
                           double *o_peak, int32_t *o_ps, int32_t *o_nd) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    if (o_peak) o_peak[b] = peak[b];
    if (o_ps) o_ps[b] = peak_step[b];
    if (o_nd) o_nd[b] = step[b];
}

// ------------------------------------------------------------- dispatch

typedef void (*StepKernel)(const StepArgs);

template <bool F64, bool FO>
static StepKernel pick_law(int law, bool kappa) {
    if (law == PD_LAW_BILINEAR) return kappa ? k_step<F64, 0, true, FO> : k_step<F64, 0, false, FO>;
    return kappa ? k_step<F64, 1, true, FO> : k_step<F64, 1, false, FO>;
}

static StepKernel pick(const pd_state *st, bool fo) {
    const bool f64 = st->mat.precision == PD_PREC_FP64;
    if (f64) return fo ? pick_law<true, true>(st->mat.law, st->has_kappa)
                       : pick_law<true, false>(st->mat.law, st->has_kappa);
    return fo ? pick_law<false, true>(st->mat.law, st->has_kappa) : pick_law<false, false>(st->mat.law, st->has_kappa);
}

static StepArgs make_args(const pd_state *st) {
    StepArgs a;
    memset(&a, 0, sizeof(a));
    a.N = st->N;
    a.n_slices = st->n_slices;
    a.nblk = st->nrb;
    a.par = st->bk_par;
    a.brick_ridx = st->brick_ridx;
    a.B = st->B;
    a.sell_off = st->sell_off;
    a.sell_m = st->sell_m;
    a.slice_i0 = st->slice_i0;
    a.slice_nv = st->slice_nv;
    a.nx = st->g.nx;
    a.ny = st->g.ny;
    a.nz = st->g.nz;
    a.BY = st->by;
    a.BZ = st->bz;
    a.nbx = st->nbx;
    a.nby = st->nby;
    a.H = st->halo;
    a.Wx = kSlice + 2 * st->halo;
    a.Wy = st->by + 2 * st->halo;
    a.Wz = st->bz + 2 * st->halo;
    a.ids = st->ids;
    a.xi_tab = st->xi_tab;
    a.xid_tab = st->xid_tab;
    a.off_tab = st->off_tab;
    a.n_off = st->n_off;
    a.dmg = st->dmg;
    a.sell_len = st->stencil ? st->st_len : st->sell_len;
    a.dxf = (float)st->g.dx;
    a.st_wpb = st->st_wpb;
    if (st->stencil) stencil_fill_args(st, a);
    for (int q = 0; q < 10; ++q) a.L0q[q] = (float)(std::sqrt((double)q) * st->g.dx);
    a.u64 = st->u64;
    a.v64 = st->v64;
    a.rec0 = st->rec[0];
    a.rec1 = st->rec[1];
    a.kappa = st->kappa;
    a.codes = st->codes;
    a.step = st->step;
    a.done = st->done;
    a.pend = st->pend;
    a.pk2 = st->pk2;
    a.ps2 = st->ps2;
    a.defer = 0;
    a.pendable = st->stencil && st->st_defer;
    a.rec_off = st->rec_off;
    a.status = st->status;
    a.peak = st->peak;
    a.peak_step = st->peak_step;
    a.partial = st->partial;
    a.ticket = st->ticket;
    a.dt = st->dt;
    a.rho = st->mat.rho;
    a.zeta = st->mat.zeta;
    a.ca = 1.0 - 0.5 * st->mat.zeta * st->dt;
    a.dtr = st->dt / st->mat.rho;
    a.icb = 1.0 / (1.0 + 0.5 * st->mat.zeta * st->dt);
    a.idt = 1.0 / st->dt;
    a.du_df = df_split(st->bc.u_max / (double)st->bc.n_ramp);
    a.dudt_df = df_split(st->bc.u_max / ((double)st->bc.n_ramp * st->dt));
    a.ca_df = df_split(a.ca);
    a.dtr_df = df_split(a.dtr);
    a.icb_df = df_split(a.icb);
    a.dt_df = df_split(a.dt);
    a.vdf = st->vdf;
    a.u_max = st->bc.u_max;
    a.n_ramp = st->bc.n_ramp;
    a.max_steps = 0x7fffffff;
    a.use_stop = 0;
    a.cV = st->c * st->V;
    a.V = st->V;
    a.s_ratio = st->mat.s_ratio;
    a.k = st->mat.k;
    a.alpha = st->mat.alpha;
    a.inv_1mek = 1.0 / (1.0 - std::exp(-st->mat.k));
    a.inv_1pa = 1.0 / (1.0 + st->mat.alpha);
    a.gfA = st->gfA;
    a.gfA_f = (float)st->gfA;
    a.cVf = (float)a.cV;
    a.cV_df = df_split(a.cV);
    a.cVh_df = df_split(0.5 * a.cV);
    a.va_df = df_split(a.ca * a.icb);
    a.vf_df = df_split(a.dtr * a.icb * a.cV);
    a.vfh_df = df_split(a.dtr * a.icb * (0.5 * a.cV));
    a.s_ratio_f = (float)a.s_ratio;
    a.k_f = (float)a.k;
    a.alpha_f = (float)a.alpha;
    a.inv_1mek_f = (float)a.inv_1mek;
    a.inv_1pa_f = (float)a.inv_1pa;
    return a;
}

static int launch_step(const pd_state *st, const StepArgs &a, bool force_only, cudaStream_t s) {
    if (st->stencil) return stencil_launch(st, a, force_only, s);
    StepKernel k = pick(st, force_only);
    const unsigned grid = (unsigned)st->nblk * (unsigned)st->B;
    k<<<grid, kThreads, st->smem_bytes, s>>>(a);
    PD_CHECK_LAUNCH();
    return PD_OK;
}

// Dynamic shared memory limit of every generic step kernel (set at state
// creation, outside any stream capture). It only ever grows (per device):
// states of several meshes coexist and each launches with its own size.
static int generic_set_attributes(size_t smem) {
    static std::mutex mu;
    static size_t limit[64] = {};
    int dev = 0;
    PD_CHECK_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && smem <= limit[dev]) return PD_OK;
    for (int f = 0; f < 2; ++f)
        for (int fo = 0; fo < 2; ++fo)
            for (int law = 0; law < 2; ++law)
                for (int kap = 0; kap < 2; ++kap) {
                    StepKernel k = f ? (fo ? pick_law<true, true>(law, kap) : pick_law<true, false>(law, kap))
                                     : (fo ? pick_law<false, true>(law, kap) : pick_law<false, false>(law, kap));
                    PD_CHECK_CUDA(
                        cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
                }
    if (dev >= 0 && dev < 64) limit[dev] = smem;
    return PD_OK;
}

static unsigned blocks_for(long long n, int bs = 256) { return (unsigned)((n + bs - 1) / bs); }

static void free_state(pd_state *st) {
    if (!st) return;
    cudaFree(st->row_ptr);
    cudaFree(st->sell_off);
    cudaFree(st->sell_m);
    cudaFree(st->slice_i0);
    cudaFree(st->slice_nv);
    cudaFree(st->ids);
    cudaFree(st->st_tmpl);
    cudaFree(st->st_dirty);
    cudaFree(st->st_box);
    cudaFree(st->col_csr);
    cudaFree(st->xi_tab);
    cudaFree(st->xid_tab);
    cudaFree(st->off_tab);
    cudaFree(st->dmg);
    cudaFree(st->u64);
    cudaFree(st->v64);
    cudaFree(st->vdf);
    cudaFree(st->rec[0]);
    cudaFree(st->rec[1]);
    cudaFree(st->grec[0]);
    cudaFree(st->grec[1]);
    cudaFree(st->grecR[0]);
    cudaFree(st->grecR[1]);
    cudaFree(st->kappa);
    cudaFree(st->codes);
    cudaFree(st->coord);
    cudaFree(st->step);
    cudaFree(st->done);
    cudaFree(st->pend);
    cudaFree(st->pk2);
    cudaFree(st->ps2);
    cudaFree(st->brick_ridx);
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

// Stencil of the horizon: integer offsets with 0 < |k|^2 <= m^2, ordered by
// ascending linear index offset (z, then y, then x), so a CSR row (sorted by
// neighbour index) visits ids in ascending order.
static int build_stencil(pd_state *st, int16_t **box_dev, int *R_out) {
    const pd_grid &g = st->g;
    const double m2 = g.m_ratio * g.m_ratio;
    const int R = (int)std::ceil(g.m_ratio);
    const int D = 2 * R + 1;
    std::vector<int16_t> box((size_t)D * D * D, -1);
    std::vector<float4> xt;
    std::vector<double4_32a> xd;
    std::vector<int32_t> ot;
    std::vector<std::array<int, 3>> off_comp;
    int halo = 0;
    for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                const int q = dx * dx + dy * dy + dz * dz;
                if (q == 0 || (double)q > m2) continue;
                const double L0 = std::sqrt((double)q) * g.dx;
                box[(size_t)(dz + R) * D * D + (dy + R) * D + (dx + R)] = (int16_t)xt.size();
                xt.push_back(make_float4((float)dx * (float)g.dx, (float)dy * (float)g.dx, (float)dz * (float)g.dx,
                                         (float)L0));
                xd.push_back(make_double4_32a(dx * g.dx, dy * g.dx, dz * g.dx, L0));
                off_comp.push_back({dx, dy, dz});
                halo = std::max(halo, std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))));
            }
    PD_REQUIRE(xt.size() <= (size_t)kPad, "horizon stencil has %zu offsets (at most 255 supported)", xt.size());
    st->n_off = (int32_t)xt.size();
    st->halo = halo;
    // neighbour offsets: global linear index (fp64 path) or index inside the
    // staged brick of (8 + 2 halo) x (by + 2 halo) x (bz + 2 halo) records (mixed)
    const bool f64 = st->mat.precision == PD_PREC_FP64;
    const int Wx = kSlice + 2 * halo, Wy = st->by + 2 * halo;
    for (const auto &k : off_comp)
        ot.push_back(f64 ? k[0] + g.nx * (k[1] + g.ny * k[2]) : k[0] + Wx * (k[1] + Wy * k[2]));
    // unused ids and the padding id: the node itself at distance dx (zero stretch)
    while (xt.size() < (size_t)kTab) {
        xt.push_back(make_float4((float)g.dx, 0.f, 0.f, (float)g.dx));
        xd.push_back(make_double4_32a(g.dx, 0.0, 0.0, g.dx));
        ot.push_back(0);
    }
    PD_TRY(dalloc(&st->xi_tab, xt.size()));
    PD_TRY(dalloc(&st->xid_tab, xd.size()));
    PD_TRY(dalloc(&st->off_tab, ot.size()));
    PD_TRY(dalloc(box_dev, box.size()));
    PD_CHECK_CUDA(cudaMemcpy(st->xi_tab, xt.data(), xt.size() * sizeof(float4), cudaMemcpyHostToDevice));
    PD_CHECK_CUDA(cudaMemcpy(st->xid_tab, xd.data(), xd.size() * sizeof(double4_32a), cudaMemcpyHostToDevice));
    PD_CHECK_CUDA(cudaMemcpy(st->off_tab, ot.data(), ot.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    PD_CHECK_CUDA(cudaMemcpy(*box_dev, box.data(), box.size() * sizeof(int16_t), cudaMemcpyHostToDevice));
    *R_out = R;
    return PD_OK;
}

static int build_state(pd_state *st, const int32_t *row_ptr, const int32_t *col) {
    const long long N = st->N;
    const int B = st->B;
    cudaStream_t s = 0;
    PD_TRY(dalloc(&st->row_ptr, N + 1));
    PD_CHECK_CUDA(cudaMemcpy(st->row_ptr, row_ptr, (N + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice));
    int32_t last = 0;
    PD_CHECK_CUDA(cudaMemcpy(&last, st->row_ptr + N, sizeof(int32_t), cudaMemcpyDeviceToHost));
    PD_REQUIRE((long long)last == st->nb, "row_ptr[N] = %d does not match n_bonds = %lld", last, (long long)st->nb);
    PD_TRY(dalloc(&st->coord, N));
    k_coords<<<blocks_for(N), 256, 0, s>>>(st->g.nx, st->g.ny, N, st->coord);
    PD_CHECK_LAUNCH();
    // brick-ordered SELL-8 layout of stencil ids
    const pd_grid &g = st->g;
    st->nbx = (g.nx + kSlice - 1) / kSlice;
    st->nby = (g.ny + st->by - 1) / st->by;
    st->nbz = (g.nz + st->bz - 1) / st->bz;
    st->n_bricks = (long long)st->nbx * st->nby * st->nbz;
    st->n_slices = st->n_bricks * st->by * st->bz;
    PD_REQUIRE(st->n_bricks * st->B < (1ll << 31), "too many blocks");
    {
        std::vector<int32_t> i0(st->n_slices), nv(st->n_slices);
        for (long long br = 0; br < st->n_bricks; ++br) {
            const int bx = (int)(br % st->nbx), by = (int)((br / st->nbx) % st->nby), bz = (int)(br / ((long long)st->nbx * st->nby));
            for (int r = 0; r < st->by * st->bz; ++r) {
                const int y = by * st->by + r % st->by, z = bz * st->bz + r / st->by, x0 = bx * kSlice;
                const long long sidx = br * st->by * st->bz + r;
                const bool in = y < g.ny && z < g.nz;
                i0[sidx] = in ? x0 + g.nx * (y + g.ny * z) : 0;
                nv[sidx] = in ? std::min(kSlice, g.nx - x0) : 0;
            }
        }
        PD_TRY(dalloc(&st->slice_i0, st->n_slices));
        PD_TRY(dalloc(&st->slice_nv, st->n_slices));
        PD_CHECK_CUDA(cudaMemcpy(st->slice_i0, i0.data(), i0.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        PD_CHECK_CUDA(cudaMemcpy(st->slice_nv, nv.data(), nv.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    PD_TRY(dalloc(&st->sell_m, st->n_slices));
    PD_TRY(dalloc(&st->sell_off, st->n_slices));
    k_slice_rounds<<<blocks_for(st->n_slices), 256, 0, s>>>(st->row_ptr, st->slice_i0, st->slice_nv, st->n_slices,
                                                            st->sell_m);
    PD_CHECK_LAUNCH();
    std::vector<int32_t> m(st->n_slices);
    std::vector<long long> off(st->n_slices);
    PD_CHECK_CUDA(cudaMemcpy(m.data(), st->sell_m, m.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    long long acc = 0;
    for (long long q = 0; q < st->n_slices; ++q) {
        off[q] = acc;
        acc += 32ll * m[q];
    }
    st->sell_len = acc;
    PD_CHECK_CUDA(cudaMemcpy(st->sell_off, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice));
    int16_t *box = nullptr;
    int R = 0;
    int rc = build_stencil(st, &box, &R);
    if (rc != PD_OK) {
        cudaFree(box);
        return rc;
    }
    st->smem_bytes = st->mat.precision == PD_PREC_FP64
                         ? 0
                         : 2 * sizeof(float4) * (size_t)(kSlice + 2 * st->halo) * (st->by + 2 * st->halo) *
                               (st->bz + 2 * st->halo);
    PD_REQUIRE(st->smem_bytes <= 200 * 1024, "brick %dx%dx%d with halo %d needs %zu bytes of shared memory", kSlice,
               st->by, st->bz, st->halo, st->smem_bytes);
    int32_t *bad = nullptr;
    if ((rc = dalloc(&st->ids, st->sell_len)) != PD_OK || (rc = dalloc(&bad, 1)) != PD_OK) {
        cudaFree(box);
        cudaFree(bad);
        return rc;
    }
    cudaMemset(bad, 0, sizeof(int32_t));
    k_fill_ids<<<blocks_for(st->n_slices * kSlice), 256, 0, s>>>(st->row_ptr, col, st->coord, st->slice_i0,
                                                                st->slice_nv, st->n_slices, st->sell_off, st->sell_m,
                                                                box, R, st->ids, bad);
    int32_t hbad = 0;
    cudaError_t e = cudaMemcpy(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost);
    cudaFree(box);
    cudaFree(bad);
    PD_CHECK_CUDA(e);
    PD_REQUIRE(!hbad, "a CSR neighbour is not a horizon stencil offset of the grid");
    PD_TRY(dalloc(&st->col_csr, st->nb));
    PD_CHECK_CUDA(cudaMemcpy(st->col_csr, col, st->nb * sizeof(int32_t), cudaMemcpyDeviceToDevice));
    PD_TRY(generic_set_attributes(st->smem_bytes));
    st->stencil = stencil_applicable(st);
    if (st->stencil) PD_TRY(stencil_build(st, col));
    PD_TRY(dalloc(&st->codes, 3 * N));
    PD_TRY(pd_bc_codes(&st->g, &st->bc, st->codes, (pd_stream)s));
    // time step
    if (st->mat.dt > 0.0) {
        st->dt = st->mat.dt;
    } else {
        double *dti = nullptr, *dmin = nullptr;
        PD_TRY(dalloc(&dti, N));
        PD_TRY(dalloc(&dmin, 1));
        k_dt_sum<<<blocks_for(N), 256, 0, s>>>(st->row_ptr, col, st->coord, N, st->c * st->V, st->g.dx, st->mat.rho,
                                               dti);
        k_min<<<1, 1024, 0, s>>>(dti, N, dmin);
        double h = 0.0;
        e = cudaMemcpy(&h, dmin, sizeof(double), cudaMemcpyDeviceToHost);
        cudaFree(dti);
        cudaFree(dmin);
        PD_CHECK_CUDA(e);
        PD_REQUIRE(std::isfinite(h) && h > 0.0, "no bonds: stable time step undefined");
        st->dt = st->mat.dt_safety * h;
    }
    // per-sample arrays
    const bool f64 = st->mat.precision == PD_PREC_FP64;
    (void)g;
    const size_t dsz = f64 ? sizeof(double) : sizeof(float);
    PD_CHECK_CUDA(cudaMalloc(&st->dmg, (size_t)B * (st->stencil ? st->st_len : st->sell_len) * dsz));
    if (f64) {
        PD_TRY(dalloc(&st->u64, 3 * N * B));
        PD_TRY(dalloc(&st->v64, 3 * N * B));
    } else {
        PD_TRY(dalloc(&st->vdf, 2 * N * B));
    }
    PD_CHECK_CUDA(cudaMalloc(&st->rec[0], (size_t)B * N * 32));
    PD_CHECK_CUDA(cudaMalloc(&st->rec[1], (size_t)B * N * 32));
    st->nblk = (int)st->n_bricks;
    PD_TRY(dalloc(&st->step, 2 * B));
    PD_TRY(dalloc(&st->done, 2 * B));
    PD_TRY(dalloc(&st->pend, 2 * B));
    PD_TRY(dalloc(&st->pk2, 2 * B));
    PD_TRY(dalloc(&st->ps2, 2 * B));
    // a state steps only after pd_state_reset / pd_state_load; until then no
    // reaction is pending and no sample counts as done
    PD_CHECK_CUDA(cudaMemset(st->pend, 0, 2 * (size_t)B * sizeof(int32_t)));
    PD_CHECK_CUDA(cudaMemset(st->done, 0, 2 * (size_t)B * sizeof(int32_t)));
    PD_CHECK_CUDA(cudaMemset(st->step, 0, 2 * (size_t)B * sizeof(int32_t)));
    st->bk_par = 0;
    st->rec_off = 0;
    // reaction bricks: those holding a prescribed DOF, plus brick 0
    {
        std::vector<uint8_t> hc((size_t)3 * N);
        PD_CHECK_CUDA(cudaMemcpy(hc.data(), st->codes, hc.size(), cudaMemcpyDeviceToHost));
        std::vector<int32_t> ridx(st->n_bricks, -1);
        ridx[0] = 0;
        for (long long i = 0; i < N; ++i) {
            if (hc[3 * i] < 2 && hc[3 * i + 1] < 2 && hc[3 * i + 2] < 2) continue;
            const int ix = (int)(i % g.nx), iy = (int)((i / g.nx) % g.ny), iz = (int)(i / ((long long)g.nx * g.ny));
            const long long br = (ix / kSlice) + (long long)st->nbx * ((iy / st->by) + (long long)st->nby * (iz / st->bz));
            ridx[br] = 0;
        }
        int cnt = 0;
        for (auto &v : ridx)
            if (v >= 0) v = cnt++;
        st->nrb = cnt;
        PD_TRY(dalloc(&st->brick_ridx, ridx.size()));
        PD_CHECK_CUDA(cudaMemcpy(st->brick_ridx, ridx.data(), ridx.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    PD_TRY(dalloc(&st->status, B));
    PD_TRY(dalloc(&st->peak, B));
    PD_TRY(dalloc(&st->peak_step, B));
    PD_TRY(dalloc(&st->partial, (size_t)2 * B * st->nrb));
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

extern "C" int pd_state_create_sched(const pd_grid *g, const int32_t *row_ptr, const int32_t *col,
                                     int64_t n_bonds, const pd_material *mat, const pd_bc *bc, int32_t batch,
                                     const pd_schedule *sched, pd_state **out) {
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
    const long long NB = (long long)g->nx * g->ny * g->nz * batch;
    PD_REQUIRE(NB < (1ll << 31), "nodes x batch must be below 2^31");
    pd_state *st = new pd_state();
    memset(st, 0, sizeof(*st));
    st->g = *g;
    st->mat = *mat;
    st->bc = *bc;
    st->B = batch;
    st->N = (int64_t)g->nx * g->ny * g->nz;
    st->nb = n_bonds;
    // brick rows (a schedule overrides them)
    {
        static const int cand_generic[][2] = {{8, 8}, {8, 4}, {4, 4}, {4, 2}, {2, 2}, {2, 1}, {1, 1}};
        const double m2 = g->m_ratio * g->m_ratio;
        const bool stencil = mat->precision == PD_PREC_MIXED && m2 >= 9.0 && m2 < 10.0;
        st->by = 1;
        st->bz = 1;
        if (stencil) {
            // measured on GB300 (28k-node beam): 4x4 bricks for batches of at least
            // ~0.4M nodes, 4x2 bricks (with the half-stencil split over two warps)
            // below that, 2x2 / 2x1 for small grids
            const long long nodes = (long long)g->nx * g->ny * g->nz * batch;
            st->by = 4;
            st->bz = nodes >= 400000 ? 4 : 2;
            if (g->nz == 1) {  // one layer (plane models): bricks of 8 x by x 1
                st->by = g->ny >= 8 ? 8 : (g->ny >= 4 ? 4 : 2);
                st->bz = 1;
            } else if (g->ny < 4 || g->nz < 2) {
                st->by = 2;
                st->bz = 2;
            }
        } else {
            // the largest brick that still gives at least two blocks per SM
            for (const auto &cb : cand_generic) {
                const long long nbr =
                    (long long)((g->nx + 7) / 8) * ((g->ny + cb[0] - 1) / cb[0]) * ((g->nz + cb[1] - 1) / cb[1]);
                if (nbr * batch >= 304) {
                    st->by = cb[0];
                    st->bz = cb[1];
                    break;
                }
            }
        }
        if (sched && (sched->by > 0 || sched->bz > 0)) {
            if (sched->by < 1 || sched->by > 16 || sched->bz < 1 || sched->bz > 16) {
                delete st;
                set_error("schedule bricks %d x %d outside [1, 16]", sched->by, sched->bz);
                return PD_ERR_ARG;
            }
            st->by = sched->by;
            st->bz = sched->bz;
        }
        st->q_req = sched ? sched->q : 0;
        if (st->q_req != 0 && st->q_req != 1 && st->q_req != 2 && st->q_req != 4) {
            const int q = st->q_req;
            delete st;
            set_error("schedule q = %d is not 0, 1, 2 or 4", q);
            return PD_ERR_ARG;
        }
        st->ns_req = sched ? sched->ns : 0;
        st->reduce_req = sched ? sched->reduce : 0;
        if (st->ns_req < 0 || st->ns_req > 2 || st->reduce_req < 0 || st->reduce_req > 2) {
            const int v = st->ns_req, w = st->reduce_req;
            delete st;
            set_error("schedule ns = %d / reduce = %d is not 0, 1 or 2", v, w);
            return PD_ERR_ARG;
        }
    }
    const double delta = g->m_ratio * g->dx;
    if (mat->model != PD_MODEL_3D) {
        if ((mat->model != PD_MODEL_PLANE_STRESS && mat->model != PD_MODEL_PLANE_STRAIN) || g->nz != 1 ||
            !(mat->thickness > 0)) {
            delete st;
            set_error("plane models need model 1 or 2, a one-layer grid (nz = 1) and thickness > 0");
            return PD_ERR_ARG;
        }
    }
    const double d3 = delta * delta * delta;
    if (mat->model == PD_MODEL_3D) {
        st->c = 12.0 * mat->E / (M_PI * d3 * delta);
        st->V = g->dx * g->dx * g->dx;
    } else {
        st->c = mat->model == PD_MODEL_PLANE_STRESS ? 9.0 * mat->E / (M_PI * mat->thickness * d3)
                                                    : 48.0 * mat->E / (5.0 * M_PI * mat->thickness * d3);
        st->V = g->dx * g->dx * mat->thickness;
    }
    st->gfA = 0.0;
    if (mat->G_F > 0.0) {
        const int grc = mat->model == PD_MODEL_3D
                            ? pd_gf_coefficient(mat->law, mat->E, delta, mat->G_F, mat->k, mat->alpha, &st->gfA)
                            : pd_gf_coefficient_plane(mat->law, mat->model, mat->E, delta, mat->thickness,
                                                      mat->G_F, mat->k, mat->alpha, &st->gfA);
        if (grc != PD_OK) {
            delete st;
            return grc;
        }
    }
    int rc = build_state(st, row_ptr, col);
    if (rc != PD_OK) {
        free_state(st);
        return rc;
    }
    *out = st;
    return PD_OK;
}

extern "C" int pd_gf_coefficient(int32_t law, double E, double delta, double G_F, double k, double alpha,
                                 double *A) {
    PD_REQUIRE(A != nullptr, "A is NULL");
    PD_REQUIRE(law == PD_LAW_BILINEAR || law == PD_LAW_EXPLINEAR, "unknown law %d", law);
    PD_REQUIRE(E > 0 && delta > 0 && G_F >= 0, "E, delta > 0 and G_F >= 0 required");
    PD_REQUIRE(law == PD_LAW_BILINEAR || (k > 0 && k < 700 && alpha >= 0), "0 < k < 700 and alpha >= 0 required");
    const double c = 12.0 * E / (M_PI * delta * delta * delta * delta);
    const double pc5 = M_PI * c * delta * delta * delta * delta * delta;  // pi c delta^5
    if (law == PD_LAW_BILINEAR) {
        *A = 10.0 * G_F / pc5;  // G_F = pi c s0 delta^5 (s_c - s0) / 10
        return PD_OK;
    }
    const double ek = std::exp(k);
    const double P = 2.0 * k - 2.0 * ek + alpha * k - alpha * k * ek + 2.0;  // < 0
    // G_F = pi c s0 delta^5 (s0 - s_c) P / (10 k (e^k - 1)(1 + alpha))
    *A = 10.0 * k * (ek - 1.0) * (1.0 + alpha) * G_F / (pc5 * -P);
    return PD_OK;
}

extern "C" int pd_gf_coefficient_plane(int32_t law, int32_t model, double E, double delta, double t, double G_F,
                                       double k, double alpha, double *A) {
    PD_REQUIRE(A != nullptr, "A is NULL");
    PD_REQUIRE(law == PD_LAW_BILINEAR || law == PD_LAW_EXPLINEAR, "unknown law %d", law);
    PD_REQUIRE(model == PD_MODEL_PLANE_STRESS || model == PD_MODEL_PLANE_STRAIN, "model must be a plane model");
    PD_REQUIRE(E > 0 && delta > 0 && t > 0 && G_F >= 0, "E, delta, t > 0 and G_F >= 0 required");
    PD_REQUIRE(law == PD_LAW_BILINEAR || (k > 0 && k < 700 && alpha >= 0), "0 < k < 700 and alpha >= 0 required");
    const double d3 = delta * delta * delta;
    const double c = model == PD_MODEL_PLANE_STRESS ? 9.0 * E / (M_PI * t * d3) : 48.0 * E / (5.0 * M_PI * t * d3);
    const double tcd4 = t * c * d3 * delta;  // t c delta^4
    if (law == PD_LAW_BILINEAR) {
        *A = 4.0 * G_F / tcd4;  // G_F = t c s0 delta^4 (s_c - s0) / 4
        return PD_OK;
    }
    const double ek = std::exp(k);
    const double P = 2.0 * k - 2.0 * ek + alpha * k - alpha * k * ek + 2.0;
    *A = 4.0 * k * (ek - 1.0) * (1.0 + alpha) * G_F / (tcd4 * -P);
    return PD_OK;
}

extern "C" int pd_state_create(const pd_grid *g, const int32_t *row_ptr, const int32_t *col, int64_t n_bonds,
                               const pd_material *mat, const pd_bc *bc, int32_t batch, pd_state **out) {
    return pd_state_create_sched(g, row_ptr, col, n_bonds, mat, bc, batch, nullptr, out);
}

extern "C" int pd_state_destroy(pd_state *st) {
    if (st) {
        cudaDeviceSynchronize();
        free_state(st);
    }
    return PD_OK;
}

extern "C" int pd_state_info(const pd_state *st, double *dt, double *c, int64_t *n_nodes, int64_t *n_bonds) {
    PD_REQUIRE(st != nullptr, "state is NULL");
    if (dt) *dt = st->dt;
    if (c) *c = st->c;
    if (n_nodes) *n_nodes = st->N;
    if (n_bonds) *n_bonds = st->nb;
    return PD_OK;
}

static int state_reset(pd_state *st, const float *s0, const double *s0d, const float *kappa, pd_stream stream) {
    PD_REQUIRE(st != nullptr, "state is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const long long NB = st->N * st->B;
    const bool f64 = st->mat.precision == PD_PREC_FP64;
    const size_t dsz = f64 ? sizeof(double) : sizeof(float);
    if (st->stencil)
        PD_TRY(stencil_reset_damage(st, s));
    else
        PD_CHECK_CUDA(cudaMemsetAsync(st->dmg, 0, (size_t)st->B * st->sell_len * dsz, s));
    const bool had = st->has_kappa;
    if (kappa) {
        if (!st->kappa) PD_TRY(dalloc(&st->kappa, (size_t)NB));
        PD_CHECK_CUDA(cudaMemcpyAsync(st->kappa, kappa, (size_t)NB * sizeof(float), cudaMemcpyDeviceToDevice, s));
        st->has_kappa = true;
    } else {
        st->has_kappa = false;
    }
    if (f64)
        k_reset<true><<<blocks_for(NB), 256, 0, s>>>(st->N, st->B, s0, s0d, kappa, st->u64, st->v64, st->vdf,
                                                     st->rec[0], st->rec[1]);
    else
        k_reset<false><<<blocks_for(NB), 256, 0, s>>>(st->N, st->B, s0, s0d, kappa, st->u64, st->v64, st->vdf,
                                                      st->rec[0], st->rec[1]);
    PD_CHECK_LAUNCH();
    if (st->stencil) PD_TRY(stencil_refresh_grec(st, s));
    if (st->chunk_exec && had != st->has_kappa) {  // the captured chunk bakes the kernel choice
        cudaGraphExecDestroy(st->chunk_exec);
        st->chunk_exec = nullptr;
    }
    k_reset_run<<<blocks_for(st->B), 256, 0, s>>>(st->B, st->step, st->done, st->pend, st->pk2, st->ps2,
                                                  st->status, st->peak, st->peak_step,
                                                  st->ticket, 0);
    PD_CHECK_LAUNCH();
    st->rec_off = st->bk_par;  // step 0 at the next launch's parity
    return PD_OK;
}

extern "C" int pd_state_reset(pd_state *st, const float *s0, const float *kappa, pd_stream stream) {
    return state_reset(st, s0, nullptr, kappa, stream);
}

extern "C" int pd_state_reset_f64(pd_state *st, const double *s0, const float *kappa, pd_stream stream) {
    PD_REQUIRE(s0 != nullptr, "s0 is required");
    return state_reset(st, nullptr, s0, kappa, stream);
}

extern "C" int pd_state_load(pd_state *st, const double *u, const double *v, const double *d, int32_t step,
                             pd_stream stream) {
    PD_REQUIRE(st != nullptr, "state is NULL");
    PD_REQUIRE(step >= 0, "step must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    const long long NB = st->N * st->B;
    const bool f64 = st->mat.precision == PD_PREC_FP64;
    k_reset_run<<<blocks_for(st->B), 256, 0, s>>>(st->B, st->step, st->done, st->pend, st->pk2, st->ps2,
                                                  st->status, st->peak, st->peak_step,
                                                  st->ticket, step);
    PD_CHECK_LAUNCH();
    st->rec_off = st->bk_par ^ (step & 1);
    if (f64)
        k_load_u<true><<<blocks_for(NB), 256, 0, s>>>(st->N, st->B, u, v, st->u64, st->v64, st->vdf, st->step + st->bk_par * st->B,
                                                      st->rec[0], st->rec[1]);
    else
        k_load_u<false><<<blocks_for(NB), 256, 0, s>>>(st->N, st->B, u, v, st->u64, st->v64, st->vdf, st->step + st->bk_par * st->B,
                                                       st->rec[0], st->rec[1]);
    PD_CHECK_LAUNCH();
    if (st->stencil) PD_TRY(stencil_refresh_grec(st, s));
    if (d && st->stencil) {
        PD_TRY(stencil_map_damage(st, (double *)d, true, s));
    } else if (d) {
        if (f64)
            k_dmg_map<double, true><<<blocks_for(NB), 256, 0, s>>>(
                st->row_ptr, st->N, st->B, st->nb, st->g.nx, st->g.ny, st->by, st->bz, st->nbx, st->nby, st->sell_off,
                st->sell_len, (double *)st->dmg, (double *)d);
        else
            k_dmg_map<float, true><<<blocks_for(NB), 256, 0, s>>>(
                st->row_ptr, st->N, st->B, st->nb, st->g.nx, st->g.ny, st->by, st->bz, st->nbx, st->nby, st->sell_off,
                st->sell_len, (float *)st->dmg, (double *)d);
        PD_CHECK_LAUNCH();
    }
    return PD_OK;
}

extern "C" int pd_state_store(const pd_state *st, double *u, double *v, double *d, pd_stream stream) {
    PD_REQUIRE(st != nullptr, "state is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const long long NB = st->N * st->B;
    if (u || v) {
        if (st->mat.precision == PD_PREC_FP64)
            k_store_u<true><<<blocks_for(NB), 256, 0, s>>>(st->N, st->B, st->u64, st->v64, st->vdf, st->step + st->bk_par * st->B,
                                                           st->rec[0], st->rec[1], u, v);
        else
            k_store_u<false><<<blocks_for(NB), 256, 0, s>>>(st->N, st->B, st->u64, st->v64, st->vdf, st->step + st->bk_par * st->B,
                                                            st->rec[0], st->rec[1], u, v);
        PD_CHECK_LAUNCH();
    }
    if (d && st->stencil) {
        PD_TRY(stencil_map_damage(st, d, false, s));
    } else if (d) {
        if (st->mat.precision == PD_PREC_FP64)
            k_dmg_map<double, false><<<blocks_for(NB), 256, 0, s>>>(
                st->row_ptr, st->N, st->B, st->nb, st->g.nx, st->g.ny, st->by, st->bz, st->nbx, st->nby, st->sell_off,
                st->sell_len, (double *)st->dmg, d);
        else
            k_dmg_map<float, false><<<blocks_for(NB), 256, 0, s>>>(
                st->row_ptr, st->N, st->B, st->nb, st->g.nx, st->g.ny, st->by, st->bz, st->nbx, st->nby, st->sell_off,
                st->sell_len, (float *)st->dmg, d);
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
        a.par = st->bk_par;
        a.defer = st->stencil && st->st_defer && k + 1 < n_steps;  // the last launch finishes every reaction
        PD_TRY(launch_step(st, a, false, (cudaStream_t)stream));
        st->bk_par ^= 1;
    }
    return PD_OK;
}

extern "C" int pd_run_to_peak(pd_state *st, int32_t max_steps, double *peak, int32_t *peak_step, int32_t *n_done,
                              pd_stream stream) {
    PD_REQUIRE(st != nullptr, "state is NULL");
    PD_REQUIRE(max_steps >= 0, "max_steps must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    const int chunk = 64;
    if (!st->chunk_exec || st->chunk_max_steps != max_steps || st->chunk_par != st->bk_par ||
        st->chunk_rec_off != st->rec_off) {
        if (st->chunk_exec) {
            cudaGraphExecDestroy(st->chunk_exec);
            st->chunk_exec = nullptr;
        }
        cudaStream_t cs;
        PD_CHECK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        StepArgs a = make_args(st);
        a.use_stop = 1;
        a.max_steps = max_steps;
        cudaGraph_t graph;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            int lrc = PD_OK;
            for (int q = 0; q < chunk && lrc == PD_OK; ++q) {
                a.par = st->bk_par ^ (q & 1);  // the chunk is even, so it ends on the parity it starts from
                a.defer = st->stencil && st->st_defer && q + 1 < chunk;  // the last launch finishes
                lrc = launch_step(st, a, false, cs);
            }
            e = cudaStreamEndCapture(cs, &graph);
            if (lrc != PD_OK && e == cudaSuccess) {
                cudaGraphDestroy(graph);
                cudaStreamDestroy(cs);
                return lrc;
            }
        }
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(&st->chunk_exec, graph, 0);
            cudaGraphDestroy(graph);
        }
        cudaStreamDestroy(cs);
        PD_CHECK_CUDA(e);
        st->chunk_steps = chunk;
        st->chunk_max_steps = max_steps;
        st->chunk_par = st->bk_par;
        st->chunk_rec_off = st->rec_off;
    }
    k_run_init<<<blocks_for(st->B), 256, 0, s>>>(st->B, st->step + st->bk_par * st->B, st->done + st->bk_par * st->B,
                                                 max_steps);
    PD_CHECK_LAUNCH();
    const int n_chunks = max_steps / chunk + 1;
    for (int c = 0; c < n_chunks; ++c) {
        PD_CHECK_CUDA(cudaGraphLaunch(st->chunk_exec, s));
        k_count_active<<<1, 256, 0, s>>>(st->B, st->done + st->bk_par * st->B, st->host_flag_dev + (c & 1));
        PD_CHECK_LAUNCH();
        PD_CHECK_CUDA(cudaEventRecord(st->ev[c & 1], s));
        if (c >= 1) {
            PD_CHECK_CUDA(cudaEventSynchronize(st->ev[(c - 1) & 1]));
            if (((volatile int32_t *)st->host_flag)[(c - 1) & 1] == 0) break;
        }
    }
    k_copy_out<<<blocks_for(st->B), 256, 0, s>>>(st->B, st->peak, st->peak_step, st->step + st->bk_par * st->B, peak,
                                                  peak_step, n_done);
    PD_CHECK_LAUNCH();
    std::vector<int32_t> status(st->B);
    PD_CHECK_CUDA(cudaMemcpyAsync(status.data(), st->status, st->B * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PD_CHECK_CUDA(cudaStreamSynchronize(s));
    for (int b = 0; b < st->B; ++b)
        if (status[b] & 2) {
            set_error("the staged box of a stencil step of sample %d did not arrive (bounded wait expired)", b);
            return PD_ERR_CUDA;
        } else if (status[b] & 4) {
            set_error("sample %d was staged from the records of the wrong step parity", b);
            return PD_ERR_CUDA;
        } else if (status[b] & 1) {
            set_error("non-finite reaction in sample %d", b);
            return PD_ERR_NAN;
        }
    return PD_OK;
}

// Several states (meshes of different sizes, e.g. the fine and coarse members
// of an MLMC level) run to their peaks together: one captured graph per 64-step
// chunk holds every state's step launches as independent branches, so the
// GPU overlaps the small meshes' launches with the large ones', and one host
// poll per chunk covers all states.
extern "C" int pd_run_to_peak_multi(pd_state *const *states, int32_t n_states, const int32_t *max_steps,
                                    double *const *peak, int32_t *const *peak_step, int32_t *const *n_done,
                                    pd_stream stream) {
    PD_REQUIRE(states && max_steps && n_states >= 1 && n_states <= 16, "1 to 16 states and max_steps required");
    for (int i = 0; i < n_states; ++i) {
        PD_REQUIRE(states[i] != nullptr, "state %d is NULL", i);
        PD_REQUIRE(max_steps[i] >= 0, "max_steps[%d] must be >= 0", i);
        for (int j = 0; j < i; ++j) PD_REQUIRE(states[j] != states[i], "state %d appears twice", i);
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int chunk = 64;
    int rc = PD_OK;
    cudaStream_t cs = nullptr, br[16] = {};
    cudaEvent_t fork = nullptr, join[16] = {};
    cudaGraphExec_t exec = nullptr;
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        for (int i = 0; i < n_states; ++i) {
            if (br[i]) cudaStreamDestroy(br[i]);
            if (join[i]) cudaEventDestroy(join[i]);
        }
        if (fork) cudaEventDestroy(fork);
        if (cs) cudaStreamDestroy(cs);
    };
    bool ok = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 1; i < n_states && ok; ++i)
        ok = cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cleanup();
        set_error("stream or event creation failed");
        return PD_ERR_CUDA;
    }
    // the chunk graph: two states with the same launch shape (the members of an
    // MLMC pair) step together, one launch per step; otherwise state 0 runs on
    // the capture stream and the others on forked branches
    const bool paired = n_states == 2 && stencil_pairable(states[0], states[1]);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess && paired) {
        int lrc = PD_OK;
        StepArgs a0 = make_args(states[0]), a1 = make_args(states[1]);
        a0.use_stop = a1.use_stop = 1;
        a0.max_steps = max_steps[0];
        a1.max_steps = max_steps[1];
        for (int q = 0; q < chunk && lrc == PD_OK; ++q) {
            a0.par = states[0]->bk_par ^ (q & 1);  // even chunk: ends on the parity it starts from
            a1.par = states[1]->bk_par ^ (q & 1);
            a0.defer = states[0]->st_defer && q + 1 < chunk;  // the last launch finishes
            a1.defer = states[1]->st_defer && q + 1 < chunk;
            lrc = stencil_launch_pair(states[0], a0, states[1], a1, cs);
        }
        e = cudaStreamEndCapture(cs, &graph);
        if (lrc != PD_OK) rc = lrc;
    } else if (e == cudaSuccess) {
        int lrc = PD_OK;
        if (n_states > 1) cudaEventRecord(fork, cs);
        for (int i = 0; i < n_states && lrc == PD_OK; ++i) {
            pd_state *st = states[i];
            cudaStream_t ls = i == 0 ? cs : br[i];
            if (i > 0) cudaStreamWaitEvent(ls, fork, 0);
            StepArgs a = make_args(st);
            a.use_stop = 1;
            a.max_steps = max_steps[i];
            for (int q = 0; q < chunk && lrc == PD_OK; ++q) {
                a.par = st->bk_par ^ (q & 1);  // even chunk: ends on the parity it starts from
                a.defer = st->stencil && st->st_defer && q + 1 < chunk;  // the last launch finishes
                lrc = launch_step(st, a, false, ls);
            }
            if (i > 0) {
                cudaEventRecord(join[i], ls);
                cudaStreamWaitEvent(cs, join[i], 0);
            }
        }
        e = cudaStreamEndCapture(cs, &graph);
        if (lrc != PD_OK) rc = lrc;
    }
    if (rc == PD_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (rc == PD_OK && e != cudaSuccess) {
        set_error("chunk graph of %d states: %s", n_states, cudaGetErrorString(e));
        rc = PD_ERR_CUDA;
    }
    if (rc != PD_OK) {
        cleanup();
        return rc;
    }
    for (int i = 0; i < n_states; ++i) {
        pd_state *st = states[i];
        k_run_init<<<blocks_for(st->B), 256, 0, s>>>(st->B, st->step + st->bk_par * st->B,
                                                     st->done + st->bk_par * st->B, max_steps[i]);
    }
    int max_all = 0;
    for (int i = 0; i < n_states; ++i) max_all = std::max(max_all, (int)max_steps[i]);
    const int n_chunks = max_all / chunk + 1;
    for (int c = 0; c < n_chunks && rc == PD_OK; ++c) {
        if (cudaGraphLaunch(exec, s) != cudaSuccess) {
            rc = PD_ERR_CUDA;
            break;
        }
        for (int i = 0; i < n_states; ++i) {
            pd_state *st = states[i];
            k_count_active<<<1, 256, 0, s>>>(st->B, st->done + st->bk_par * st->B, st->host_flag_dev + (c & 1));
        }
        if (cudaEventRecord(states[0]->ev[c & 1], s) != cudaSuccess) {
            rc = PD_ERR_CUDA;
            break;
        }
        if (c >= 1) {
            if (cudaEventSynchronize(states[0]->ev[(c - 1) & 1]) != cudaSuccess) {
                rc = PD_ERR_CUDA;
                break;
            }
            int live = 0;
            for (int i = 0; i < n_states; ++i) live += ((volatile int32_t *)states[i]->host_flag)[(c - 1) & 1];
            if (live == 0) break;
        }
    }
    if (rc != PD_OK) {
        set_error("multi-state run failed: %s", cudaGetErrorString(cudaGetLastError()));
        cudaStreamSynchronize(s);
        cleanup();
        return rc;
    }
    for (int i = 0; i < n_states; ++i) {
        pd_state *st = states[i];
        k_copy_out<<<blocks_for(st->B), 256, 0, s>>>(st->B, st->peak, st->peak_step, st->step + st->bk_par * st->B,
                                                      peak ? peak[i] : nullptr, peak_step ? peak_step[i] : nullptr,
                                                      n_done ? n_done[i] : nullptr);
    }
    std::vector<std::vector<int32_t>> status(n_states);
    for (int i = 0; i < n_states; ++i) {
        status[i].resize(states[i]->B);
        cudaMemcpyAsync(status[i].data(), states[i]->status, states[i]->B * sizeof(int32_t), cudaMemcpyDeviceToHost,
                        s);
    }
    const cudaError_t se = cudaStreamSynchronize(s);
    cleanup();
    PD_CHECK_CUDA(se);
    for (int i = 0; i < n_states; ++i)
        for (int b = 0; b < states[i]->B; ++b)
            if (status[i][b] & 2) {
                set_error("the staged box of a stencil step of sample %d of state %d did not arrive (bounded wait "
                          "expired)", b, i);
                return PD_ERR_CUDA;
            } else if (status[i][b] & 4) {
                set_error("sample %d of state %d was staged from the records of the wrong step parity", b, i);
                return PD_ERR_CUDA;
            } else if (status[i][b] & 1) {
                set_error("non-finite reaction in sample %d of state %d", b, i);
                return PD_ERR_NAN;
            }
    return PD_OK;
}
