// pd_stencil.cu -- the mixed-precision step for the 122-offset horizon
// (|k|^2 <= 9 in cell units: m in [3, sqrt(10)), which covers m = 3.01, 3.14
// and pi of the workloads), with the stencil fixed at compile time.
//
// Every node keeps one damage slot for each of the 122 stencil offsets. A slot
// whose neighbour does not exist (outside the body, or across the notch) is a
// permanently broken bond (d = 1): its force (1 - d) c s is exactly zero, so
// the node sums equal those over the neighbour list alone, and the bond loop
// has no ids and no neighbour list. Two sub-lanes share a node: sub-lane 0
// takes the 61 offsets +k of the positive half-stencil, sub-lane 1 the mirrored
// offsets -k, in the same code with a sign table, so the two directed copies of
// a bond are computed by identical instruction sequences on exactly negated
// operands (bitwise-symmetric stretch and damage).
//
// Layout per sample: [brick][warp][64 rounds][32 lanes] damage words (the 61
// offsets padded to 64); lane L = 16 t + 8 r + c serves node (x0 + c, brick
// row 2 w + r) and sub-lane t. A block (one brick of 8 x BY x BZ nodes, one
// sample, or a pair of samples on the paired FP32 instructions) stages the
// brick's gather records and a 3-cell halo in shared memory, row-blocked so
// that gathers are free of bank conflicts (cells outside the grid read as zero
// displacement); all gathers are shared-memory loads.
//
// A step's reaction is reduced in its own launch, or, for launches of a single
// wave, by every block of the next launch before it steps (no serial tail at
// the end of each step; the run bookkeeping is double-buffered by parity).
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
constexpr int kChunkB = kWx * 16;    // bytes of one 16-byte chunk of a staged row's cells

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

// ---- lane arithmetic. A lane carries one sample (float) or a pair of samples
// (float2, on the paired FP32 instructions, which issue once for both). Every
// operation rounds once as written (no contraction), so the paired kernel
// gives each sample of the pair the same bits as the one-sample kernel.
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <class V>
__device__ __forceinline__ V splat(float x);
template <>
__device__ __forceinline__ float splat<float>(float x) { return x; }
template <>
__device__ __forceinline__ float2 splat<float2>(float x) { return make_float2(x, x); }

// a - b, rounded once (the fma -1 * b + a is exact before its rounding)
template <class V>
__device__ __forceinline__ V vsub(V a, V b) { return vfma(b, splat<V>(-1.0f), a); }

__device__ __forceinline__ float neg(float a) { return -a; }
__device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }

// PTX approximate reciprocal square root and reciprocal (the special-function
// unit; relative error a few ulp, ample for a stretch of order 1e-4..1e-2)
__device__ __forceinline__ float rsqrt_ap(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_ap(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float vrsqrt(float x) { return rsqrt_ap(x); }
__device__ __forceinline__ float2 vrsqrt(float2 x) { return make_float2(rsqrt_ap(x.x), rsqrt_ap(x.y)); }
__device__ __forceinline__ float vrcp(float x) { return rcp_ap(x); }
__device__ __forceinline__ float2 vrcp(float2 x) { return make_float2(rcp_ap(x.x), rcp_ap(x.y)); }

__device__ __forceinline__ float el(float v, int) { return v; }
__device__ __forceinline__ float el(float2 v, int s) { return s ? v.y : v.x; }

__device__ __forceinline__ float shfl16(float v) { return __shfl_xor_sync(0xffffffffu, v, 16); }
__device__ __forceinline__ float2 shfl16(float2 v) { return make_float2(shfl16(v.x), shfl16(v.y)); }

// s + x accumulated with the rounding error carried in c (Knuth's TwoSum)
template <class V>
__device__ __forceinline__ void two_sum_acc_v(V &s, V &c, V x) {
    const V t = vadd(s, x);
    const V z = vsub(t, s);
    const V e = vadd(vsub(s, vsub(t, z)), vsub(x, z));
    s = t;
    c = vadd(c, e);
}

template <int NS>
struct Lane;
template <>
struct Lane<1> {
    using V = float;
};
template <>
struct Lane<2> {
    using V = float2;
};

// A staged gather record. One sample: float4 hi (u_hi xyz, s0) and float4 lo
// (u_lo xyz, kappa). A pair: the same eight values interleaved by sample
// ({x0, x1, y0, y1}, ...) in four float4 chunks, with s0 halved at staging.
// Shared memory holds the records row-blocked: for every (y, z) row of the
// staged box, chunk k of its 14 cells is contiguous (kChunkB bytes), so the 8
// x-consecutive lanes of a gather read 128 contiguous bytes (no bank
// conflicts) and every chunk is an immediate offset from the first.
template <class V>
struct Rec {
    V hx, hy, hz, hw, lx, ly, lz, lw;
};

template <int NS>
__device__ __forceinline__ Rec<typename Lane<NS>::V> load_rec(const char *p) {
    if constexpr (NS == 1) {
        const float4 h = *(const float4 *)p, l = *(const float4 *)(p + kChunkB);
        return {h.x, h.y, h.z, h.w, l.x, l.y, l.z, l.w};
    } else {
        const float4 A = *(const float4 *)p, B = *(const float4 *)(p + kChunkB);
        const float4 C = *(const float4 *)(p + 2 * kChunkB), D = *(const float4 *)(p + 3 * kChunkB);
        return {make_float2(A.x, A.y), make_float2(A.z, A.w), make_float2(B.x, B.y), make_float2(B.z, B.w),
                make_float2(C.x, C.y), make_float2(C.z, C.w), make_float2(D.x, D.y), make_float2(D.z, D.w)};
    }
}

// Bond elastic limit s0_ij = (s0_i + s0_j) / 2. A pair stages s0 / 2 (an
// exact scaling), so its plain sum has the same bits as the halved sum.
__device__ __forceinline__ float bond_s0(float a, float b) { return vmul(0.5f, vadd(a, b)); }
__device__ __forceinline__ float2 bond_s0(float2 a, float2 b) { return vadd(a, b); }

struct LawC {
    float sr, kf, af, i1, i2, gfa;
};

// Damage of one sample's bond: d = max(d, D(s)) once s passes s0.
template <int LAW>
__device__ __forceinline__ void law_update(float s, float s0, float &d, float *slot, bool wr, const LawC &lc) {
    if (s > s0) {
        const float dl = law_damage<float>(LAW, s, s0, crit_stretch(s0, lc.sr, lc.gfa), lc.kf, lc.af, lc.i1, lc.i2);
        if (dl > d) {
            d = dl;
            if (wr) *slot = dl;
        }
    }
}

// Per-lane context of the bond loop: the sign tables, the lane's own staged
// record (displacements negated), its damage rows and the law constants.
template <int NS>
struct BondCtx {
    using V = typename Lane<NS>::V;
    const float4 *tab;  // per round: {kx, ky, kz, |k|} (one sample) or {kx, kx, ky, ky}, {kz, kz, |k|, |k|} (pair)
    const V *kw2;       // per round: |k|^2
    const int *offb;    // per round: byte offset of the neighbour's staged record
    const char *own;
    V nhx, nhy, nhz, hw, nlx, nly, nlz, kap;
    float *dm0, *dm1;   // damage rows of the lane's samples (stride 32 per round)
    bool w0, w1;        // damage writes enabled per sample
    LawC lc;
};

// One bond of the lane (round m), for its one or two samples: stretch
// s = (|xi+eta| - |xi|)/|xi| = eta.(xi+eta+xi) / (|xi| (|xi+eta| + |xi|)), the
// law, and the force (1 - d) s (xi+eta)/|xi+eta| (micromodulus and volume are
// applied to the node sum).
template <int NS, int LAW, bool KAPPA>
__device__ __forceinline__ void stencil_bond(int m, typename Lane<NS>::V &d, const BondCtx<NS> &cx,
                                             typename Lane<NS>::V &px, typename Lane<NS>::V &py,
                                             typename Lane<NS>::V &pz) {
    using V = typename Lane<NS>::V;
    V KX, KY, KZ, KW;
    if constexpr (NS == 1) {
        const float4 k = cx.tab[m];
        KX = k.x;
        KY = k.y;
        KZ = k.z;
        KW = k.w;
    } else {
        const float4 k0 = cx.tab[2 * m], k1 = cx.tab[2 * m + 1];
        KX = make_float2(k0.x, k0.y);
        KY = make_float2(k0.z, k0.w);
        KZ = make_float2(k1.x, k1.y);
        KW = make_float2(k1.z, k1.w);
    }
    const V KW2 = cx.kw2[m];
    const Rec<V> r = load_rec<NS>(cx.own + cx.offb[m]);
    const V ex = vadd(vadd(r.hx, cx.nhx), vadd(r.lx, cx.nlx));
    const V ey = vadd(vadd(r.hy, cx.nhy), vadd(r.ly, cx.nly));
    const V ez = vadd(vadd(r.hz, cx.nhz), vadd(r.lz, cx.nlz));
    const V yx = vadd(KX, ex), yy = vadd(KY, ey), yz = vadd(KZ, ez);
    const V wx = vadd(yx, KX), wy = vadd(yy, KY), wz = vadd(yz, KZ);
    const V y2 = vfma(yz, yz, vfma(yy, yy, vmul(yx, yx)));
    const V num = vfma(ez, wz, vfma(ey, wy, vmul(ex, wx)));
    const V rL = vrsqrt(y2);
    const V L = vmul(y2, rL);
    const V s = vmul(num, vrcp(vfma(KW, L, KW2)));
    const V s0 = bond_s0(cx.hw, r.hw);
    if constexpr (NS == 1) {
        law_update<LAW>(s, s0, d, cx.dm0 + 32 * m, true, cx.lc);
    } else {
        if (s.x > s0.x || s.y > s0.y) {
            law_update<LAW>(s.x, s0.x, d.x, cx.dm0 + 32 * m, cx.w0, cx.lc);
            law_update<LAW>(s.y, s0.y, d.y, cx.dm1 + 32 * m, cx.w1, cx.lc);
        }
    }
    V g = vmul(vmul(vfma(d, splat<V>(-1.0f), splat<V>(1.0f)), s), rL);
    if (KAPPA) g = vmul(g, vadd(cx.kap, r.lw));
    px = vfma(g, yx, px);
    py = vfma(g, yy, py);
    pz = vfma(g, yz, pz);
}

template <int NS, int U>
__device__ __forceinline__ void load_damage(typename Lane<NS>::V (&d)[U], int m, const BondCtx<NS> &cx) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if constexpr (NS == 1)
            d[u] = cx.dm0[32 * (m + u)];
        else
            d[u] = make_float2(cx.dm0[32 * (m + u)], cx.dm1[32 * (m + u)]);
    }
}

// Bonds [m0, m0 + 8 NG) of the padded half-stencil for one lane, in groups of
// 8: the FP32 sum of a group is added to the compensated (TwoSum)
// accumulator. Damage words are requested one unit (8 bonds for one sample, 4
// for a pair) ahead, in two register sets used in turn.
template <int NS, int NG, int LAW, bool KAPPA>
__device__ __forceinline__ void bond_span(int m0, const BondCtx<NS> &cx, typename Lane<NS>::V *acc) {
    using V = typename Lane<NS>::V;
    static_assert(NG % 2 == 0, "even number of groups");
    constexpr int U = NS == 1 ? 8 : 4, NU = 8 / U, J = 2 * NU;
    V da[U], db[U];
    load_damage<NS, U>(da, m0, cx);
    V px = splat<V>(0.f), py = px, pz = px;
#pragma unroll 1
    for (int g = 0; g < NG; g += 2) {
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int mu = m0 + 8 * g + U * j;
            const bool more = j + 1 < J || g + 2 < NG;
            if (j % 2 == 0) {
                if (more) load_damage<NS, U>(db, mu + U, cx);
#pragma unroll
                for (int u = 0; u < U; ++u) stencil_bond<NS, LAW, KAPPA>(mu + u, da[u], cx, px, py, pz);
            } else {
                if (more) load_damage<NS, U>(da, mu + U, cx);
#pragma unroll
                for (int u = 0; u < U; ++u) stencil_bond<NS, LAW, KAPPA>(mu + u, db[u], cx, px, py, pz);
            }
            if ((j + 1) % NU == 0) {
                two_sum_acc_v(acc[0], acc[3], px);
                two_sum_acc_v(acc[1], acc[4], py);
                two_sum_acc_v(acc[2], acc[5], pz);
                px = py = pz = splat<V>(0.f);
            }
        }
    }
}

// Warps of a block: wpb row pairs x Q parts of the half-stencil, for NS
// samples (one, or a pair on the paired FP32 instructions). Part 0's warp of
// a row pair adds the other parts' sums (fixed order) and integrates.
template <int DIM, int NS, int Q, int LAW, bool KAPPA, bool FORCE_ONLY>
__global__ void __launch_bounds__(512, NS == 1 ? 2 : 1) k_step_stencil(const StepArgs a) {
    using V = typename Lane<NS>::V;
    using S = Sten<DIM>;
    constexpr int kHalf = S::kHalf, kRounds = S::kRounds, kHaloZ = S::kHaloZ;
    constexpr int kRowB = 2 * NS * kChunkB;  // bytes of a staged (y, z) row of records
    extern __shared__ float4 s_rec[];
    __shared__ float2 red[NS][16];
    __shared__ float s_pre[NS][4];  // U(n+1) and the prescribed velocity, double-float
    __shared__ unsigned s_cnt[NS];
    __shared__ RunView s_rv[NS];               // run bookkeeping per sample, with the pending reaction added
    __shared__ int s_n[NS];                    // step index per sample
    __shared__ int s_ridx;                     // the brick's index among the reaction bricks, or -1
    __shared__ float4 s_tab[2][NS * kRounds];  // per sub-lane sign
    __shared__ V s_kw2[kRounds];
    __shared__ int s_offb[2][kRounds];          // per sign: byte offset of the neighbour's staged record

    const int nwarps = blockDim.x >> 5;
    const int wpb = a.st_wpb;
    const int ngrp = (a.B + NS - 1) / NS;
    const int grp = blockIdx.x % ngrp;
    const int brick = blockIdx.x / ngrp;
    // per-block scalars that the end of the kernel needs live in shared
    // memory or are recomputed there (fewer registers held across the bond loop)
    const auto sample_of = [&](int s) {
        const int b = NS * grp + s;
        return b < a.B ? b : NS * grp;  // the second member of the last pair of an odd batch is a copy
    };
    int ns[NS];
    bool live[NS];
    bool any = false;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const bool real = NS * grp + s < a.B;
        const int b = sample_of(s);
        ns[s] = a.step[a.par * a.B + b];
        const bool dn = FORCE_ONLY ? false : (a.done[a.par * a.B + b] != 0);
        live[s] = real && !dn;
        if (!FORCE_ONLY && real && dn && brick == 0 && threadIdx.x == 0) carry_done(a, b);
        any = any || live[s];
    }
    if (!any) return;  // block-uniform
    if (threadIdx.x == 0) s_ridx = FORCE_ONLY ? -1 : a.brick_ridx[brick];
    if (threadIdx.x < NS) s_n[threadIdx.x] = ns[threadIdx.x];
    // the run view (with the previous launch's reaction, if it left it
    // pending) is built by warp s for sample s while the staging copies fly
    const auto build_views = [&]() {
        if (FORCE_ONLY || !a.pendable) return;
        const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
        for (int s = w; s < NS; s += nwarps) {
            RunView rv;
            if (live[s]) {
                rv = run_view(a, sample_of(s), l);
            } else {
                rv.n = ns[s];
                rv.dn = 1;
                rv.Q = 0.0;
                rv.np = 0;
                rv.Rp = 0.0;
                rv.have = 0;
            }
            if (l == 0) s_rv[s] = rv;
        }
    };
    if (threadIdx.x < 16 * NS) (&red[0][0])[threadIdx.x] = make_float2(0.f, 0.f);
    if (threadIdx.x < NS) {
        df U1, vp;
        prescribed(a, ns[threadIdx.x], U1, vp);
        s_pre[threadIdx.x][0] = U1.hi;
        s_pre[threadIdx.x][1] = U1.lo;
        s_pre[threadIdx.x][2] = vp.hi;
        s_pre[threadIdx.x][3] = vp.lo;
        s_cnt[threadIdx.x] = 0u;
    }
    const int bx = brick % a.nbx, by = (brick / a.nbx) % a.nby, bz = brick / (a.nbx * a.nby);
    const int x0 = kSlice * bx, y0 = a.BY * by, z0 = a.BZ * bz;
    const size_t BN = (size_t)a.B * a.N;
    const int Wy = a.BY + 2 * kHalo, Wz = a.BZ + 2 * kHaloZ;
    const int Wtot = kWx * Wy * Wz;
    float *s_part = (float *)((char *)s_rec + (size_t)kRowB * Wy * Wz);  // [Q-1][wpb][16][6 NS]
    for (int m = threadIdx.x; m < kRounds; m += blockDim.x) {
        float4 k;
        int lo_ = 0;
        if (m < kHalf) {  // else padding: the node itself (zero stretch, zero force)
            k = a.half_tab[m];
            lo_ = 16 * a.half_off[0][m] + kRowB * (a.half_off[1][m] + Wy * a.half_off[2][m]);
        } else {
            k = make_float4(a.dxf, 0.f, 0.f, a.dxf);
        }
        if constexpr (NS == 1) {
            s_tab[0][m] = k;
            s_tab[1][m] = make_float4(-k.x, -k.y, -k.z, k.w);
        } else {
            s_tab[0][2 * m] = make_float4(k.x, k.x, k.y, k.y);
            s_tab[0][2 * m + 1] = make_float4(k.z, k.z, k.w, k.w);
            s_tab[1][2 * m] = make_float4(-k.x, -k.x, -k.y, -k.y);
            s_tab[1][2 * m + 1] = make_float4(-k.z, -k.z, k.w, k.w);
        }
        s_kw2[m] = splat<V>(k.w * k.w);
        s_offb[0][m] = lo_;
        s_offb[1][m] = -lo_;
    }
    // stage the brick and its halo (cells outside the grid read as zero)
    if constexpr (NS == 1) {
        const float4 *rhi = (const float4 *)((ns[0] & 1) ? a.rec1 : a.rec0) + (size_t)sample_of(0) * a.N;
        const float4 *rlo = rhi + BN;
        for (int q = threadIdx.x; q < Wtot; q += blockDim.x) {  // asynchronous copies, all requested at once
            const int lx = q % kWx, ly = (q / kWx) % Wy, lz = q / (kWx * Wy);
            const int gx = x0 - kHalo + lx, gy = y0 - kHalo + ly, gz = z0 - kHaloZ + lz;
            const bool in = gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz;
            const int gi = in ? gx + a.nx * (gy + a.ny * gz) : 0;
            char *dst = (char *)s_rec + (size_t)kRowB * (ly + Wy * lz) + 16 * lx;
            cp_async16(dst, rhi + gi, in ? 16 : 0);
            cp_async16(dst + kChunkB, rlo + gi, in ? 16 : 0);
        }
        build_views();
        cp_async_wait_all();
    } else {
        const float4 *rh0 = (const float4 *)((ns[0] & 1) ? a.rec1 : a.rec0) + (size_t)sample_of(0) * a.N;
        const float4 *rh1 = (const float4 *)((ns[NS - 1] & 1) ? a.rec1 : a.rec0) + (size_t)sample_of(NS - 1) * a.N;
        for (int q = threadIdx.x; q < Wtot; q += blockDim.x) {  // interleave the pair through registers
            const int lx = q % kWx, ly = (q / kWx) % Wy, lz = q / (kWx * Wy);
            const int gx = x0 - kHalo + lx, gy = y0 - kHalo + ly, gz = z0 - kHaloZ + lz;
            const bool in = gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz;
            float4 h0 = make_float4(0.f, 0.f, 0.f, 0.f), h1 = h0, l0 = h0, l1 = h0;
            if (in) {
                const int gi = gx + a.nx * (gy + a.ny * gz);
                h0 = rh0[gi];
                h1 = rh1[gi];
                l0 = rh0[BN + gi];
                l1 = rh1[BN + gi];
            }
            char *dst = (char *)s_rec + (size_t)kRowB * (ly + Wy * lz) + 16 * lx;
            *(float4 *)dst = make_float4(h0.x, h1.x, h0.y, h1.y);
            *(float4 *)(dst + kChunkB) = make_float4(h0.z, h1.z, 0.5f * h0.w, 0.5f * h1.w);
            *(float4 *)(dst + 2 * kChunkB) = make_float4(l0.x, l1.x, l0.y, l1.y);
            *(float4 *)(dst + 3 * kChunkB) = make_float4(l0.z, l1.z, l0.w, l1.w);
        }
        build_views();
    }
    __syncthreads();
    if (!FORCE_ONLY && a.pendable) {
        // samples that the reduced reaction stops are not stepped (every
        // block reaches the same decision); brick 0 records them
        bool anyl = false;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const bool stop = live[s] && s_rv[s].dn;
            if (stop && brick == 0 && threadIdx.x == 0) write_done(a, sample_of(s), s_rv[s]);
            live[s] = live[s] && !stop;
            anyl = anyl || live[s];
        }
        if (!anyl) return;  // block-uniform
    }

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rp = warp % wpb, part = warp / wpb;
    const int t = lane >> 4, r = (lane >> 3) & 1, c = lane & 7;
    df Rloc[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) Rloc[s] = df{0.f, 0.f};
    const int row = 2 * rp + r;
    const int ly = row % a.BY, lz = row / a.BY;
    const int gx = x0 + c, gy = y0 + ly, gz = z0 + lz;
    const bool own = gx < a.nx && gy < a.ny && gz < a.nz;
    const int ii = gx + a.nx * (gy + a.ny * gz);
    const char *ownp = (const char *)s_rec + (size_t)kRowB * ((kHalo + ly) + Wy * (kHaloZ + lz)) + 16 * (kHalo + c);
    V acc[6];  // sx, sy, sz, cx, cy, cz
#pragma unroll
    for (int q = 0; q < 6; ++q) acc[q] = splat<V>(0.f);
    if (own) {
        constexpr int R = kRounds / Q;
        const Rec<V> me = load_rec<NS>(ownp);
        BondCtx<NS> cx;
        cx.tab = s_tab[t];
        cx.kw2 = s_kw2;
        cx.offb = s_offb[t];
        cx.own = ownp;
        cx.nhx = neg(me.hx);
        cx.nhy = neg(me.hy);
        cx.nhz = neg(me.hz);
        cx.hw = me.hw;
        cx.nlx = neg(me.lx);
        cx.nly = neg(me.ly);
        cx.nlz = neg(me.lz);
        cx.kap = me.lw;
        cx.dm0 = (float *)a.dmg + (size_t)sample_of(0) * a.sell_len + ((size_t)brick * wpb + rp) * (kRounds * 32) + lane;
        cx.dm1 = cx.dm0 + (size_t)(sample_of(NS - 1) - sample_of(0)) * a.sell_len;
        cx.w0 = live[0];
        cx.w1 = live[NS - 1];
        cx.lc = LawC{a.s_ratio_f, a.k_f, a.alpha_f, a.inv_1mek_f, a.inv_1pa_f, a.gfA_f};
        bond_span<NS, R / 8, LAW, KAPPA>(part * R, cx, acc);
    }
    // add the two sub-lane partials in double-float (TwoSum is exact, so both
    // sub-lanes end with the same total)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const V p = shfl16(acc[q]);
        const V pc = shfl16(acc[3 + q]);
        V sq = acc[q], cq = splat<V>(0.f);
        two_sum_acc_v(sq, cq, p);
        acc[q] = sq;
        acc[3 + q] = vadd(cq, vadd(acc[3 + q], pc));
    }
    if (Q > 1) {
        if (part > 0 && t == 0) {
            float *dst = s_part + (((size_t)(part - 1) * wpb + rp) * 16 + (lane & 15)) * (6 * NS);
#pragma unroll
            for (int q = 0; q < 6; ++q)
#pragma unroll
                for (int s = 0; s < NS; ++s) dst[NS * q + s] = el(acc[q], s);
        }
        __syncthreads();
        if (part == 0) {
            for (int pp = 1; pp < Q; ++pp) {
                const float *src = s_part + (((size_t)(pp - 1) * wpb + rp) * 16 + (lane & 15)) * (6 * NS);
                V w[6];
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    if constexpr (NS == 1)
                        w[q] = src[q];
                    else
                        w[q] = make_float2(src[2 * q], src[2 * q + 1]);
                }
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    V sq = acc[q], cq = splat<V>(0.f);
                    two_sum_acc_v(sq, cq, w[q]);
                    acc[q] = sq;
                    acc[3 + q] = vadd(cq, vadd(acc[3 + q], w[3 + q]));
                }
            }
        }
    }
    if (own && part == 0) {
        const df cVd = KAPPA ? a.cVh_df : a.cV_df;
        const Rec<V> me = load_rec<NS>(ownp);  // the node's own displacement (re-read: fewer live registers)
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            if (FORCE_ONLY ? (NS * grp + s >= a.B) : !live[s]) continue;
            const size_t node = (size_t)sample_of(s) * a.N + ii;
            for (int q = t; q < 3; q += 2) {
                const float sq = el(q == 0 ? acc[0] : (q == 1 ? acc[1] : acc[2]), s);
                const float cq = el(q == 0 ? acc[3] : (q == 1 ? acc[4] : acc[5]), s);
                const df F = df_mul(two_sum(sq, cq), cVd);
                if (FORCE_ONLY) {
                    a.F_out[3 * node + q] = (double)F.hi + (double)F.lo;
                    continue;
                }
                const uint8_t code = a.codes[3 * (size_t)ii + q];
                df u = {el(q == 0 ? me.hx : (q == 1 ? me.hy : me.hz), s), el(q == 0 ? me.lx : (q == 1 ? me.ly : me.lz), s)};
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
                    Rloc[s] = df_add(Rloc[s], df{-sg * F.hi, -sg * F.lo});
                    v = df{sg * s_pre[s][2], sg * s_pre[s][3]};
                    u = df{sg * s_pre[s][0], sg * s_pre[s][1]};
                }
                vh[q] = v.hi;
                vl[q] = v.lo;
                float *oh = (float *)((float4 *)((s_n[s] & 1) ? a.rec0 : a.rec1) + node);
                float *ol = (float *)((float4 *)((s_n[s] & 1) ? a.rec0 : a.rec1) + BN + node);
                oh[q] = u.hi;
                ol[q] = u.lo;
            }
        }
    }
    if (FORCE_ONLY) return;

#pragma unroll
    for (int s = 0; s < NS; ++s) {
        if (!live[s]) continue;  // block-uniform
        RunView rv;
        if (a.pendable) {
            rv = s_rv[s];
        } else {  // nothing is ever pending: the finishing block reads the peak itself
            rv.n = s_n[s];
            rv.dn = 0;
            rv.Q = 0.0;
            rv.np = 0;
            rv.Rp = 0.0;
            rv.have = 0;
        }
        const int ridx = s_ridx;
        if (a.defer) {
            if (brick == 0 && threadIdx.x == 0) write_deferred(a, sample_of(s), rv);
            if (ridx >= 0) reaction_defer(a, Rloc[s], sample_of(s), ridx, warp, lane, nwarps, red[s]);
        } else if (ridx >= 0) {
            reaction_finish(a, Rloc[s], sample_of(s), ridx, warp, lane, nwarps, red[s], &s_cnt[s], rv);
        }
    }
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

// Slot, in one sample's damage array, of every CSR bond (every CSR neighbour
// is a stencil offset: checked when the template is built).
__global__ void k_stencil_slots(const int32_t *row_ptr, const int32_t *col, const int32_t *coord, long long N,
                                int nx, int ny, int BY, int BZ, int nbx, int nby, int wpb, int rounds,
                                const int16_t *box, int32_t *slot) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
        const int code = code_of(coord, (int)i, col[p], box);
        slot[p] = code < 0 ? 0 : (int32_t)slot_of((int)i, code, nx, ny, BY, BZ, nbx, nby, wpb, rounds);
    }
}

typedef void (*StencilKernel)(const StepArgs);

template <int DIM, int NS, int Q>
StencilKernel pick_q(int law, bool kappa, bool fo) {
    if constexpr (NS == 2) fo = false;  // force-only evaluations run one sample per block
    if (law == PD_LAW_BILINEAR) {
        if (fo) return kappa ? k_step_stencil<DIM, 1, Q, 0, true, true> : k_step_stencil<DIM, 1, Q, 0, false, true>;
        return kappa ? k_step_stencil<DIM, NS, Q, 0, true, false> : k_step_stencil<DIM, NS, Q, 0, false, false>;
    }
    if (fo) return kappa ? k_step_stencil<DIM, 1, Q, 1, true, true> : k_step_stencil<DIM, 1, Q, 1, false, true>;
    return kappa ? k_step_stencil<DIM, NS, Q, 1, true, false> : k_step_stencil<DIM, NS, Q, 1, false, false>;
}

template <int NS>
StencilKernel pick_ns(int dim, int q, int law, bool kappa, bool fo) {
    if (dim == 2) return pick_q<2, NS, 1>(law, kappa, fo);  // 16 rounds: two groups of 8 at Q = 1 only
    if (q == 4) return pick_q<3, NS, 4>(law, kappa, fo);
    if (q == 2) return pick_q<3, NS, 2>(law, kappa, fo);
    return pick_q<3, NS, 1>(law, kappa, fo);
}

// Force-only evaluations always take the one-sample kernel (same bits).
StencilKernel pick_stencil(int dim, int ns, int q, int law, bool kappa, bool fo) {
    return ns == 2 && !fo ? pick_ns<2>(dim, q, law, kappa, fo) : pick_ns<1>(dim, q, law, kappa, fo);
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
        for (int ns = 1; ns <= 2; ++ns)
            for (int q = 1; q <= 4; q *= 2)
                for (int law = 0; law < 2; ++law)
                    for (int kap = 0; kap < 2; ++kap)
                        for (int fo = 0; fo < 2; ++fo)
                            PD_CHECK_CUDA(cudaFuncSetAttribute((const void *)pick_stencil(dim, ns, q, law, kap, fo),
                                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                               (int)smem));
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
    // samples per block: one (measured on GB300, a pair per block is slower at
    // 122 registers a thread, 16 warps per SM); pairs on request
    st->st_ns = st->ns_req ? st->ns_req : 1;
    // staged records of the brick and its halo: float4 hi and lo per node and sample
    const size_t cells = (size_t)kWx * (st->by + 2 * kHalo) * (st->bz + 2 * haloz);
    // split the half-stencil over Q warps when the mesh gives too few warps per SM
    // (measured on GB300: Q = 2 for single samples of the 28k-node beam, 1 for batches)
    const long long warps1 = st->n_bricks * ((st->B + st->st_ns - 1) / st->st_ns) * st->st_wpb;
    st->st_q = warps1 >= 152ll * 24 ? 1 : 2;
    if (st->q_req) st->st_q = st->q_req;
    if (st->st_dim == 2) st->st_q = 1;
    while (st->st_q > 1 && 32 * st->st_wpb * st->st_q > 512) st->st_q /= 2;
    // Deferring the reaction to the next launch pays when a launch is a
    // single wave of a few blocks per SM, whose reduction tail would
    // otherwise stand alone at the end (measured on GB300: 28k-node beam,
    // one sample, 19.3 -> 18 us per step); with many waves the tail overlaps
    // other blocks and the deferred read only adds to each block's start.
    {
        int dev = 0, sms = 0;
        PD_CHECK_CUDA(cudaGetDevice(&dev));
        PD_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        st->st_defer = st->n_bricks * ((st->B + st->st_ns - 1) / st->st_ns) <= 4ll * sms;
        if (st->reduce_req) st->st_defer = st->reduce_req == 2;
    }
    // the one-sample kernel (force-only evaluations) needs no more than this
    st->smem_bytes = 2 * sizeof(float4) * st->st_ns * cells +
                     (size_t)(st->st_q - 1) * st->st_wpb * 16 * 6 * st->st_ns * sizeof(float);
    PD_REQUIRE(st->smem_bytes <= 227 * 1024, "stencil brick 8x%dx%d for %d samples needs %zu bytes of shared memory",
               st->by, st->bz, st->st_ns, st->smem_bytes);
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

int stencil_slot_table(const pd_state *st, int32_t *slot, cudaStream_t s) {
    k_stencil_slots<<<blocks_of(st->N), 256, 0, s>>>(st->row_ptr, st->col_csr, st->coord, st->N, st->g.nx, st->g.ny,
                                                     st->by, st->bz, st->nbx, st->nby, st->st_wpb,
                                                     st->st_dim == 3 ? Sten<3>::kRounds : Sten<2>::kRounds,
                                                     st->st_box, slot);
    PD_CHECK_LAUNCH();
    return PD_OK;
}

int stencil_launch(const pd_state *st, const StepArgs &a, bool force_only, cudaStream_t s) {
    const int ns = force_only ? 1 : st->st_ns;
    StencilKernel k = pick_stencil(st->st_dim, ns, st->st_q, st->mat.law, st->has_kappa, force_only);
    const unsigned grid = (unsigned)st->n_bricks * (unsigned)((st->B + ns - 1) / ns);
    k<<<grid, 32 * st->st_wpb * st->st_q, st->smem_bytes, s>>>(a);
    PD_CHECK_LAUNCH();
    return PD_OK;
}

}  // namespace pdi
