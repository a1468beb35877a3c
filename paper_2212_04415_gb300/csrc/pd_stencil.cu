// pd_stencil.cu -- the mixed-precision step for the 122-offset horizon
// (|k|^2 <= 9 in cell units: m in [3, sqrt(10)), which covers m = 3.01, 3.14
// and pi of the workloads), with the stencil fixed at compile time.
//
// Every node keeps one damage slot for each of the 122 stencil offsets. A slot
// whose neighbour does not exist (outside the body, or across the notch) is a
// permanently broken bond (d = 1): its force (1 - d) c s is exactly zero, so
// the node sums equal those over the neighbour list alone, and the bond loop
// has no ids, no tables and no padding. Two sub-lanes share a node: sub-lane 0
// takes the 61 offsets +k of the positive half-stencil, sub-lane 1 the mirrored
// offsets -k, in the same code with a sign register, so the two directed
// copies of a bond are computed by identical instruction sequences on exactly
// negated operands (bitwise-symmetric stretch and damage).
//
// Layout per sample: [brick][warp][64 rounds][32 lanes] damage words (the 61
// offsets padded to 64); lane L = 16 t + 8 r + c serves node (x0 + c, brick
// row 2 w + r) and sub-lane t. A block (one brick of 8 x BY x BZ nodes, one
// sample) stages the brick's gather records and a 3-cell halo in shared memory
// (cells outside the grid read as zero displacement), so all gathers are
// shared-memory loads with compile-time offsets.
//
// A one-layer grid (nz = 1, the plane models) has only the 28 in-plane
// offsets: the same kernel is compiled for that shape (14 offsets per sign,
// padded to 16 rounds, no z-halo), so a plane node costs 16 rounds, not 64.
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <utility>
#include <vector>

#include "pd_device.cuh"

namespace pdi {

namespace {

constexpr int kHalo = 3;             // largest offset component (x and y)
constexpr int kWx = kSlice + 2 * kHalo;

// Stencil shape by dimension: the positive half of the horizon (61 of the 122
// offsets in 3D; 14 of the 28 offsets of a one-layer grid, where no bond
// leaves the layer), padded to a multiple of 16 rounds (the padding points at
// the node itself), and the z-halo staged in shared memory.
template <int DIM>
struct Sten;
template <>
struct Sten<3> {
    static constexpr int kHalf = 61, kRounds = 64, kHaloZ = 3;
};
template <>
struct Sten<2> {
    static constexpr int kHalf = 14, kRounds = 16, kHaloZ = 0;
};

struct I3 {
    int x, y, z;
};

__host__ __device__ constexpr bool positive_half(int x, int y, int z) {
    return z > 0 || (z == 0 && (y > 0 || (y == 0 && x > 0)));
}

// m-th offset of the positive half-stencil, in ascending linear order (z, y, x);
// the planar stencil is the z = 0 part of the same order.
template <int DIM>
__host__ __device__ constexpr I3 half_off(int m) {
    int cnt = 0;
    for (int z = 0; z <= (DIM == 3 ? 3 : 0); ++z)
        for (int y = -3; y <= 3; ++y)
            for (int x = -3; x <= 3; ++x)
                if (positive_half(x, y, z) && x * x + y * y + z * z <= 9) {
                    if (cnt == m) return I3{x, y, z};
                    ++cnt;
                }
    return I3{0, 0, 0};
}

// One bond of this lane: stencil entry m of the lane's sign table (xi, |xi|
// and the byte offset of the neighbour's staged record), damage d.
template <int LAW, bool KAPPA>
__device__ __forceinline__ void stencil_bond(int m, float d, const float4 *tab, const int *offb, const char *own,
                                             float4 hi, float4 lo, float *dm, float cV, float sr, float kf, float af,
                                             float i1, float i2, float gfa, float &px, float &py, float &pz) {
    const float4 k = tab[m];
    const char *rj = own + offb[m];
    const float4 hj = *(const float4 *)rj;
    const float4 lj = *(const float4 *)(rj + 16);
    const float ex = (hj.x - hi.x) + (lj.x - lo.x);
    const float ey = (hj.y - hi.y) + (lj.y - lo.y);
    const float ez = (hj.z - hi.z) + (lj.z - lo.z);
    const float yx = k.x + ex, yy = k.y + ey, yz = k.z + ez;
    const float y2 = yx * yx + yy * yy + yz * yz;
    const float rL = rsqrtf(y2);
    const float L = y2 * rL;
    const float s = __fdividef(2.0f * (k.x * ex + k.y * ey + k.z * ez) + (ex * ex + ey * ey + ez * ez), k.w * (L + k.w));
    const float s0 = 0.5f * (hi.w + hj.w);
    if (s > s0) {
        const float dl = law_damage<float>(LAW, s, s0, crit_stretch(s0, sr, gfa), kf, af, i1, i2);
        if (dl > d) {
            d = dl;
            dm[32 * m] = d;
        }
    }
    float cv = cV;
    if (KAPPA) cv = cV * 0.5f * (lo.w + lj.w);
    const float gg = cv * (1.0f - d) * s * rL;
    px = fmaf(gg, yx, px);
    py = fmaf(gg, yy, py);
    pz = fmaf(gg, yz, pz);
}

// Bonds [m0, m0 + 8 G) of the padded half-stencil for one lane, in groups of
// 8: the FP32 sum of a group is added to the compensated (TwoSum)
// accumulator, and the next group's damage words are requested while the
// current group computes (two register sets in turn). The sign tables hold
// xi = +k dx for sub-lane 0 and -k dx for sub-lane 1 (exact negations), so
// both directed copies of a bond run the same instructions on negated operands.
template <int G, int LAW, bool KAPPA>
__device__ __forceinline__ void bond_span(int m0, const float4 *tab, const int *offb, const char *own, float4 hi,
                                          float4 lo, float *dm, float cV, float sr, float kf, float af, float i1,
                                          float i2, float gfa, float *acc) {
    static_assert(G % 2 == 0, "even number of groups");
    float da[8], db[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) da[u] = dm[32 * (m0 + u)];
#pragma unroll 1
    for (int g = 0; g < G; g += 2) {
        const int ma = m0 + 8 * g, mb = ma + 8;
#pragma unroll
        for (int u = 0; u < 8; ++u) db[u] = dm[32 * (mb + u)];
        float px = 0.f, py = 0.f, pz = 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            stencil_bond<LAW, KAPPA>(ma + u, da[u], tab, offb, own, hi, lo, dm, cV, sr, kf, af, i1, i2, gfa, px, py, pz);
        two_sum_acc(acc[0], acc[3], px);
        two_sum_acc(acc[1], acc[4], py);
        two_sum_acc(acc[2], acc[5], pz);
        if (g + 2 < G) {
#pragma unroll
            for (int u = 0; u < 8; ++u) da[u] = dm[32 * (mb + 8 + u)];
        }
        px = py = pz = 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            stencil_bond<LAW, KAPPA>(mb + u, db[u], tab, offb, own, hi, lo, dm, cV, sr, kf, af, i1, i2, gfa, px, py, pz);
        two_sum_acc(acc[0], acc[3], px);
        two_sum_acc(acc[1], acc[4], py);
        two_sum_acc(acc[2], acc[5], pz);
    }
}

// Warps of a block: wpb row pairs x Q parts of the half-stencil. Part 0's warp
// of a row pair adds the other parts' sums (fixed order) and integrates.
template <int DIM, int Q, int LAW, bool KAPPA, bool FORCE_ONLY>
__global__ void __launch_bounds__(512, 2) k_step_stencil(const StepArgs a) {
    using S = Sten<DIM>;
    constexpr int kHalf = S::kHalf, kRounds = S::kRounds, kHaloZ = S::kHaloZ;
    extern __shared__ float4 s_rec[];
    __shared__ float2 red[16];
    __shared__ float s_pre[4];  // U(n+1) and the prescribed velocity, double-float
    __shared__ unsigned s_cnt;
    __shared__ float4 s_tab[2][kRounds];  // per sub-lane sign: xi (x, y, z) and |xi|
    __shared__ int s_offb[2][kRounds];    // per sign: byte offset of the neighbour's staged record

    const int nwarps = blockDim.x >> 5;
    const int wpb = a.st_wpb;
    const int b = blockIdx.x % a.B;
    const int brick = blockIdx.x / a.B;
    const bool done = FORCE_ONLY ? false : (a.done[a.par * a.B + b] != 0);
    const int n = a.step[a.par * a.B + b];
    if (done) {  // block-uniform
        if (brick == 0 && threadIdx.x == 0) carry_done(a, b);
        return;
    }
    if (threadIdx.x < 16) red[threadIdx.x] = make_float2(0.f, 0.f);
    if (threadIdx.x == 0) {
        df U1, vp;
        prescribed(a, n, U1, vp);
        s_pre[0] = U1.hi;
        s_pre[1] = U1.lo;
        s_pre[2] = vp.hi;
        s_pre[3] = vp.lo;
        s_cnt = 0u;
    }
    const int bx = brick % a.nbx, by = (brick / a.nbx) % a.nby, bz = brick / (a.nbx * a.nby);
    const int x0 = kSlice * bx, y0 = a.BY * by, z0 = a.BZ * bz;
    const size_t BN = (size_t)a.B * a.N;
    const int Wy = a.BY + 2 * kHalo, Wz = a.BZ + 2 * kHaloZ;
    const int Wtot = kWx * Wy * Wz;
    float *s_part = (float *)(s_rec + 2 * Wtot);  // [Q-1][wpb][16][6]
    for (int m = threadIdx.x; m < kRounds; m += blockDim.x) {
        if (m < kHalf) {
            const float4 k = a.half_tab[m];
            const int lo_ = a.half_off[0][m] + kWx * a.half_off[1][m] + kWx * Wy * a.half_off[2][m];
            s_tab[0][m] = k;
            s_tab[1][m] = make_float4(-k.x, -k.y, -k.z, k.w);
            s_offb[0][m] = 32 * lo_;
            s_offb[1][m] = -32 * lo_;
        } else {  // padding: the node itself (zero stretch, zero force)
            s_tab[0][m] = s_tab[1][m] = make_float4(a.dxf, 0.f, 0.f, a.dxf);
            s_offb[0][m] = s_offb[1][m] = 0;
        }
    }
    const float4 *rhi = (const float4 *)((n & 1) ? a.rec1 : a.rec0) + (size_t)b * a.N;
    const float4 *rlo = rhi + BN;
    if (!done) {
        // stage the brick and its halo with asynchronous copies, all requested
        // at once (cells outside the grid are zero-filled)
        for (int q = threadIdx.x; q < Wtot; q += blockDim.x) {
            const int lx = q % kWx, ly = (q / kWx) % Wy, lz = q / (kWx * Wy);
            const int gx = x0 - kHalo + lx, gy = y0 - kHalo + ly, gz = z0 - kHaloZ + lz;
            const bool in = gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz;
            const int gi = in ? gx + a.nx * (gy + a.ny * gz) : 0;
            cp_async16(s_rec + 2 * q, rhi + gi, in ? 16 : 0);  // records interleaved: hi, lo
            cp_async16(s_rec + 2 * q + 1, rlo + gi, in ? 16 : 0);
        }
        cp_async_wait_all();
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rp = warp % wpb, part = warp / wpb;
    const int t = lane >> 4, r = (lane >> 3) & 1, c = lane & 7;
    df Rloc = {0.f, 0.f};
    const int row = 2 * rp + r;
    const int ly = row % a.BY, lz = row / a.BY;
    const int gx = x0 + c, gy = y0 + ly, gz = z0 + lz;
    const bool own = gx < a.nx && gy < a.ny && gz < a.nz;
    const int ii = gx + a.nx * (gy + a.ny * gz);
    const size_t node = (size_t)b * a.N + ii;
    const int il = (kHalo + c) + kWx * ((kHalo + ly) + Wy * (kHaloZ + lz));
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // sx, sy, sz, cx, cy, cz
    const float4 hi = s_rec[2 * il], lo = s_rec[2 * il + 1];
    if (!done) {
        if (own) {
            constexpr int R = kRounds / Q;
            float *dm = (float *)a.dmg + (size_t)b * a.sell_len + ((size_t)brick * wpb + rp) * (kRounds * 32) + lane;
            bond_span<R / 8, LAW, KAPPA>(part * R, s_tab[t], s_offb[t], (const char *)(s_rec + 2 * il), hi, lo, dm,
                                         a.cVf, a.s_ratio_f, a.k_f, a.alpha_f, a.inv_1mek_f, a.inv_1pa_f, a.gfA_f,
                                         acc);
        }
        // add the two sub-lane partials in double-float (TwoSum is exact, so
        // both sub-lanes end with the same total)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float p = __shfl_xor_sync(0xffffffffu, acc[q], 16);
            const float pc = __shfl_xor_sync(0xffffffffu, acc[3 + q], 16);
            const df rr = two_sum(acc[q], p);
            acc[q] = rr.hi;
            acc[3 + q] = rr.lo + (acc[3 + q] + pc);
        }
    }
    if (Q > 1) {
        if (!done && part > 0 && t == 0) {
            float *dst = s_part + (((size_t)(part - 1) * wpb + rp) * 16 + (lane & 15)) * 6;
#pragma unroll
            for (int q = 0; q < 6; ++q) dst[q] = acc[q];
        }
        __syncthreads();
        if (!done && part == 0) {
            for (int pp = 1; pp < Q; ++pp) {
                const float *src = s_part + (((size_t)(pp - 1) * wpb + rp) * 16 + (lane & 15)) * 6;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const df rr = two_sum(acc[q], src[q]);
                    acc[q] = rr.hi;
                    acc[3 + q] = rr.lo + (acc[3 + q] + src[3 + q]);
                }
            }
        }
    }
    if (!done && own && part == 0) {
        for (int q = t; q < 3; q += 2) {
            const float sq = q == 0 ? acc[0] : (q == 1 ? acc[1] : acc[2]);
            const float cq = q == 0 ? acc[3] : (q == 1 ? acc[4] : acc[5]);
            const df F = two_sum(sq, cq);
            if (FORCE_ONLY) {
                a.F_out[3 * node + q] = (double)F.hi + (double)F.lo;
                continue;
            }
            const uint8_t code = a.codes[3 * (size_t)ii + q];
            df u = {q == 0 ? hi.x : (q == 1 ? hi.y : hi.z), q == 0 ? lo.x : (q == 1 ? lo.y : lo.z)};
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
                Rloc = df_add(Rloc, df{-sg * F.hi, -sg * F.lo});
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
    if (FORCE_ONLY || done) return;

    const int ridx = a.brick_ridx[brick];
    if (ridx >= 0) reaction_finish(a, Rloc, b, ridx, warp, lane, nwarps, red, &s_cnt, n);
}

// Slot of node i, stencil code (2 m + t), in the per-sample damage array.
__device__ __forceinline__ long long slot_of(int i, int code, int nx, int ny, int BY, int BZ, int nbx, int nby,
                                             int wpb, int rounds) {
    const int ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
    const long long brick = (ix / kSlice) + (long long)nbx * ((iy / BY) + (long long)nby * (iz / BZ));
    const int row = (iy % BY) + BY * (iz % BZ);
    const int w = row >> 1, rr = row & 1, c = ix % kSlice;
    const int m = code >> 1, t = code & 1;
    return ((brick * wpb + w) * rounds + m) * 32 + (16 * t + 8 * rr + c);
}

// code of the CSR neighbour j of i: 2 m + t, or -1 if not a stencil offset
__device__ __forceinline__ int code_of(const int32_t *coord, int i, int j, const int16_t *box) {
    const int ci = coord[i], cj = coord[j];
    const int dx = (cj & 2047) - (ci & 2047), dy = ((cj >> 11) & 2047) - ((ci >> 11) & 2047), dz = (cj >> 22) - (ci >> 22);
    if (dx < -3 || dx > 3 || dy < -3 || dy > 3 || dz < -3 || dz > 3) return -1;
    return box[(dz + 3) * 49 + (dy + 3) * 7 + (dx + 3)];
}

// Damage template: 0 for every slot of a CSR bond, 1 (absent bond) elsewhere.
__global__ void k_stencil_template(const int32_t *row_ptr, const int32_t *col, const int32_t *coord, long long N,
                                   int nx, int ny, int BY, int BZ, int nbx, int nby, int wpb, int rounds,
                                   const int16_t *box, float *tmpl, int32_t *bad) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
        const int code = code_of(coord, (int)i, col[p], box);
        if (code < 0) {
            *bad = 1;
            continue;
        }
        tmpl[slot_of((int)i, code, nx, ny, BY, BZ, nbx, nby, wpb, rounds)] = 0.0f;
    }
}

__global__ void k_fill_float(float *p, long long n, float v) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) p[t] = v;
}

__global__ void k_stencil_reset(long long len, int B, const float *tmpl, float *dmg) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= len * B) return;
    dmg[t] = tmpl[t % len];
}

template <bool TO_STATE>
__global__ void k_stencil_map(const int32_t *row_ptr, const int32_t *col, const int32_t *coord, long long N, int B,
                              long long nb, int nx, int ny, int BY, int BZ, int nbx, int nby, int wpb, int rounds,
                              long long len, const int16_t *box, float *dmg, double *csr) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * B) return;
    const int b = (int)(t / N);
    const int i = (int)(t % N);
    for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
        const int code = code_of(coord, i, col[p], box);
        if (code < 0) continue;
        const long long e = (long long)b * len + slot_of(i, code, nx, ny, BY, BZ, nbx, nby, wpb, rounds);
        const long long q = (long long)b * nb + p;
        if (TO_STATE)
            dmg[e] = (float)csr[q];
        else
            csr[q] = (double)dmg[e];
    }
}

typedef void (*StencilKernel)(const StepArgs);

template <int DIM, int Q>
StencilKernel pick_q(int law, bool kappa, bool fo) {
    if (law == PD_LAW_BILINEAR) {
        if (fo) return kappa ? k_step_stencil<DIM, Q, 0, true, true> : k_step_stencil<DIM, Q, 0, false, true>;
        return kappa ? k_step_stencil<DIM, Q, 0, true, false> : k_step_stencil<DIM, Q, 0, false, false>;
    }
    if (fo) return kappa ? k_step_stencil<DIM, Q, 1, true, true> : k_step_stencil<DIM, Q, 1, false, true>;
    return kappa ? k_step_stencil<DIM, Q, 1, true, false> : k_step_stencil<DIM, Q, 1, false, false>;
}

// The planar stencil's 16 rounds make two groups of 8 at Q = 1 only.
StencilKernel pick_stencil(int dim, int q, int law, bool kappa, bool fo) {
    if (dim == 2) return pick_q<2, 1>(law, kappa, fo);
    if (q == 4) return pick_q<3, 4>(law, kappa, fo);
    if (q == 2) return pick_q<3, 2>(law, kappa, fo);
    return pick_q<3, 1>(law, kappa, fo);
}

unsigned blocks_of(long long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

bool stencil_applicable(const pd_state *st) {
    const double m2 = st->g.m_ratio * st->g.m_ratio;
    return st->mat.precision == PD_PREC_MIXED && m2 >= 9.0 && m2 < 10.0 && ((st->by * st->bz) % 2 == 0) &&
           st->by * st->bz <= 32;
}

// The dynamic shared-memory limit of the stencil kernels only ever grows (per
// device): states of several meshes coexist (the fine and coarse members of
// MLMC pairs) and each launches with its own brick size.
int stencil_set_attributes(size_t smem) {
    static std::mutex mu;
    static size_t limit[64] = {};
    int dev = 0;
    PD_CHECK_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && smem <= limit[dev]) return PD_OK;
    for (int dim = 2; dim <= 3; ++dim)
        for (int q = 1; q <= 4; q *= 2)
            for (int law = 0; law < 2; ++law)
                for (int kap = 0; kap < 2; ++kap)
                    for (int fo = 0; fo < 2; ++fo)
                        PD_CHECK_CUDA(cudaFuncSetAttribute((const void *)pick_stencil(dim, q, law, kap, fo),
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (dev >= 0 && dev < 64) limit[dev] = smem;
    return PD_OK;
}

int stencil_build(pd_state *st, const int32_t *col) {
    const long long N = st->N;
    st->st_wpb = st->by * st->bz / 2;
    st->st_dim = st->g.nz == 1 ? 2 : 3;  // a one-layer grid has only the planar offsets
    const int rounds = st->st_dim == 3 ? Sten<3>::kRounds : Sten<2>::kRounds;
    const int haloz = st->st_dim == 3 ? Sten<3>::kHaloZ : Sten<2>::kHaloZ;
    st->st_len = st->n_bricks * st->st_wpb * (long long)rounds * 32;
    // staged records of the brick and its halo: float4 hi and lo per node
    st->smem_bytes = 2 * sizeof(float4) * (size_t)kWx * (st->by + 2 * kHalo) * (st->bz + 2 * haloz);
    // split the half-stencil over Q warps when the mesh gives too few warps per SM
    // (measured on GB300: Q = 2 for single samples of the 28k-node beam, 1 for batches)
    const long long warps1 = st->n_bricks * st->B * st->st_wpb;
    st->st_q = warps1 >= 152ll * 24 ? 1 : 2;
    if (const char *e = std::getenv("PD_STENCIL_Q")) {
        const int v = std::atoi(e);
        if (v == 1 || v == 2 || v == 4) st->st_q = v;
    }
    if (st->q_req) st->st_q = st->q_req;
    if (st->st_dim == 2) st->st_q = 1;
    while (st->st_q > 1 && 32 * st->st_wpb * st->st_q > 512) st->st_q /= 2;
    st->smem_bytes += (size_t)(st->st_q - 1) * st->st_wpb * 16 * 6 * sizeof(float);
    std::vector<int16_t> box(343, -1);
    const int half = st->st_dim == 3 ? Sten<3>::kHalf : Sten<2>::kHalf;
    for (int m = 0; m < half; ++m) {
        const I3 k = st->st_dim == 3 ? half_off<3>(m) : half_off<2>(m);
        box[(k.z + 3) * 49 + (k.y + 3) * 7 + (k.x + 3)] = (int16_t)(2 * m);
        box[(-k.z + 3) * 49 + (-k.y + 3) * 7 + (-k.x + 3)] = (int16_t)(2 * m + 1);
    }
    PD_TRY(dalloc(&st->st_box, box.size()));
    PD_CHECK_CUDA(cudaMemcpy(st->st_box, box.data(), box.size() * sizeof(int16_t), cudaMemcpyHostToDevice));
    PD_TRY(dalloc(&st->st_tmpl, st->st_len));
    // every slot starts as an absent (broken) bond; the slots of real bonds are cleared
    k_fill_float<<<blocks_of(st->st_len), 256>>>(st->st_tmpl, st->st_len, 1.0f);
    PD_CHECK_LAUNCH();
    int32_t *bad = nullptr;
    PD_TRY(dalloc(&bad, 1));
    cudaMemset(bad, 0, sizeof(int32_t));
    k_stencil_template<<<blocks_of(N), 256>>>(st->row_ptr, col, st->coord, N, st->g.nx, st->g.ny, st->by, st->bz,
                                              st->nbx, st->nby, st->st_wpb, rounds, st->st_box, st->st_tmpl, bad);
    int32_t hbad = 0;
    const cudaError_t e = cudaMemcpy(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost);
    cudaFree(bad);
    PD_CHECK_CUDA(e);
    PD_REQUIRE(!hbad, "a CSR neighbour is not a horizon stencil offset of the grid");
    return stencil_set_attributes(st->smem_bytes);
}

void stencil_fill_args(const pd_state *st, StepArgs &a) {
    const float dxf = (float)st->g.dx;
    const int half = st->st_dim == 3 ? Sten<3>::kHalf : Sten<2>::kHalf;
    for (int m = 0; m < half; ++m) {
        const I3 k = st->st_dim == 3 ? half_off<3>(m) : half_off<2>(m);
        const int q = k.x * k.x + k.y * k.y + k.z * k.z;
        a.half_tab[m] = make_float4((float)k.x * dxf, (float)k.y * dxf, (float)k.z * dxf,
                                    (float)(std::sqrt((double)q) * st->g.dx));
        a.half_off[0][m] = k.x;
        a.half_off[1][m] = k.y;
        a.half_off[2][m] = k.z;
    }
}

int stencil_reset_damage(pd_state *st, cudaStream_t s) {
    k_stencil_reset<<<blocks_of(st->st_len * st->B), 256, 0, s>>>(st->st_len, st->B, st->st_tmpl, (float *)st->dmg);
    PD_CHECK_LAUNCH();
    return PD_OK;
}

int stencil_map_damage(const pd_state *st, double *csr, bool to_state, cudaStream_t s) {
    const long long NB = st->N * st->B;
    if (to_state)
        k_stencil_map<true><<<blocks_of(NB), 256, 0, s>>>(st->row_ptr, st->col_csr, st->coord, st->N, st->B, st->nb,
                                                          st->g.nx, st->g.ny, st->by, st->bz, st->nbx, st->nby,
                                                          st->st_wpb, st->st_dim == 3 ? Sten<3>::kRounds : Sten<2>::kRounds,
                                                          st->st_len, st->st_box, (float *)st->dmg, csr);
    else
        k_stencil_map<false><<<blocks_of(NB), 256, 0, s>>>(st->row_ptr, st->col_csr, st->coord, st->N, st->B, st->nb,
                                                           st->g.nx, st->g.ny, st->by, st->bz, st->nbx, st->nby,
                                                           st->st_wpb, st->st_dim == 3 ? Sten<3>::kRounds : Sten<2>::kRounds,
                                                          st->st_len, st->st_box, (float *)st->dmg, csr);
    PD_CHECK_LAUNCH();
    return PD_OK;
}

int stencil_launch(const pd_state *st, const StepArgs &a, bool force_only, cudaStream_t s) {
    StencilKernel k = pick_stencil(st->st_dim, st->st_q, st->mat.law, st->has_kappa, force_only);
    const unsigned grid = (unsigned)st->n_bricks * (unsigned)st->B;
    k<<<grid, 32 * st->st_wpb * st->st_q, st->smem_bytes, s>>>(a);
    PD_CHECK_LAUNCH();
    return PD_OK;
}

}  // namespace pdi
