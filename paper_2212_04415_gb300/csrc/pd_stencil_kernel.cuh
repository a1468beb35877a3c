// pd_stencil_kernel.cuh -- device code of the compile-time stencil step,
// included by the translation units that instantiate its variants
// (pd_stencil_d3q1.cu, pd_stencil_d3q2.cu, pd_stencil_d3q4.cu, pd_stencil_d2.cu)
// and, for its layout constants, by pd_stencil.cu.
//
// The mixed-precision step for the 122-offset horizon
// (|k|^2 <= 9 in cell units: m in [3, sqrt(10)), which covers m = 3.01, 3.14
// and pi of the workloads), with the stencil fixed at compile time.
//
// Every node keeps one damage slot for each of the 122 stencil offsets. A slot
// whose neighbour does not exist (outside the body, or across the notch) is a
// permanently broken bond (d = 1): its force (1 - d) c s is exactly zero, so
// the node sums equal those over the neighbour list alone, and the bond loop
// has no ids and no neighbour list.
//
// Two sub-lanes share a node. Round m of the half-stencil has the offset k_m
// (k_m in the positive half): sub-lane 0 of node i evaluates the bond
// (i, i + k_m), sub-lane 1 of node j the bond (j - k_m, j), so every sub-lane
// evaluates a bond of offset +k_m from its lower end to its upper end. The two
// directed copies of a bond therefore run the same instructions on the same
// operands (bitwise-equal stretch and damage), and the lane's force is +f for
// sub-lane 0 and -f for sub-lane 1. Sub-lane 1 gathers from a point-reflected
// copy of the staged box, in which node j - k sits at (j's position) + k, so
// both sub-lanes address their neighbour as own + offset(k) with the same
// compile-time offset: the rounds are unrolled, the offsets, |k| and |k|^2 are
// immediates and no table is read per bond.
//
// Gather records are the displacements in cell units (u / dx) rounded to FP32,
// with s0 / 2 (the bond's elastic limit is the plain sum of the two halves):
// bond kinematics and forces are FP32 on FP32 positions (the stretch is
// scale-free, and the force direction is a unit vector). The state itself
// (u and v) stays double-float and is integrated per node.
//
// Layout per sample: [brick][warp][16 quads][32 lanes][4 rounds] damage words
// (the 61 offsets padded to 64; one 128-bit load per lane covers four rounds);
// lane L = 16 t + 8 r + c serves node (x0 + c, brick row 2 w + r) and sub-lane
// t. A block (one brick of 8 x BY x BZ nodes, one sample, or a pair of samples
// on the paired FP32 instructions) stages the brick's gather records and a
// 3-cell halo in shared memory: the upper part (the brick's layers and the 3
// above) as is for sub-lane 0, the lower part (the 3 below and the brick's
// layers) point-reflected for sub-lane 1. Rows are blocked so that the 8
// x-consecutive lanes of a gather read 128 contiguous bytes (no bank
// conflicts); cells outside the grid read as zero displacement.
//
// Most damage words never change: an intact bond stays at 0 until its
// stretch passes the elastic limit, an absent one stays at 1. Every lane
// keeps one bit per group of 8 rounds (per part of the half-stencil, so that
// parts never write the same byte), set when a fix-up first grows a damage
// word of the group. A group whose bit is clear still equals the template
// (the initial damage of every slot, shared by all samples of the state), so
// it is read from the template, which stays in L2, instead of from the
// sample's own words: the values are the same, and the DRAM stream of a
// launch shrinks to the groups that are softening or broken. Reset clears the
// bits; loading damage marks the groups whose loaded damage is not all zero.
//
// A step's reaction is reduced in its own launch, or, for launches of a single
// wave, by every block of the next launch before it steps (no serial tail at
// the end of each step; the run bookkeeping is double-buffered by parity).
//
// A one-layer grid (nz = 1, the plane models) has only the 28 in-plane
// offsets: the same kernel is compiled for that shape (14 offsets per sign,
// padded to 16 rounds, no z-halo), so a plane node costs 14 rounds, not 61.
#pragma once

#include <utility>

#include "pd_device.cuh"

namespace pdi {

namespace {

constexpr int kHalo = 3;           // largest offset component (x and y)
constexpr int kWx = kSlice + 2 * kHalo;
constexpr int kRowC = kWx * 16;    // bytes of one 16-byte chunk across a staged row's cells
constexpr int kRowK = kWx * 4;     // bytes of one staged row of kappa values (one sample)

// Stencil shape by dimension: the positive half of the horizon (61 of the 122
// offsets in 3D; 14 of the 28 offsets of a one-layer grid, where no bond
// leaves the layer), padded to a multiple of 16 rounds in the damage layout,
// and the z-halo staged in shared memory.
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

// |k| for |k|^2 = q (cell units; 7 is not a sum of three squares)
__host__ __device__ constexpr float knorm(int q) {
    return q == 1   ? 1.0f
           : q == 2 ? 1.41421356237309505f
           : q == 3 ? 1.73205080756887729f
           : q == 4 ? 2.0f
           : q == 5 ? 2.23606797749978970f
           : q == 6 ? 2.44948974278317810f
           : q == 8 ? 2.82842712474619010f
                    : 3.0f;
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

__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float2 vmax(float2 a, float2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
constexpr float kMinY2 = 1e-12f;

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

// The staged box (dynamic shared memory of the step kernel).
extern __shared__ float4 g_box[];

// ---- TMA staging of the box (one-sample blocks). One thread arms an
// mbarrier with the bytes of both record copies and issues two tiled copies
// of a 5D box (4 floats x 14 cells x rows x layers x 1 sample); cells outside
// the grid arrive as zeros. Waits are bounded: after kStageSpin polls the
// caller flags the sample and gives up.
constexpr uint32_t kStageSpin = 1u << 22;

__device__ __forceinline__ uint32_t sm_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void stage_bar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void stage_bar_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sm_addr(bar)), "r"(bytes) : "memory");
}

// true once phase 0 of the barrier has completed; false after kStageSpin polls
__device__ __forceinline__ bool stage_bar_wait(uint64_t *bar) {
    const uint32_t b = sm_addr(bar);
    for (uint32_t it = 0; it < kStageSpin; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(b)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// box of the records map at cell (x, y, z) of sample b, into shared memory at dst
__device__ __forceinline__ void stage_box(void *dst, const CUtensorMap *tm, int x, int y, int z, int b, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], "
        "[%7];" ::"r"(sm_addr(dst)),
        "l"((uint64_t)tm), "r"(0), "r"(x), "r"(y), "r"(z), "r"(b), "r"(sm_addr(bar))
        : "memory");
}

// A staged gather record: u / dx (x, y, z) and s0 / 2. One sample: one float4
// per cell. A pair: the two samples' values interleaved ({x0, x1, y0, y1},
// {z0, z1, h0, h1}) in two chunks, kRowC bytes apart (row-blocked).
template <class V>
struct Rec {
    V x, y, z, h;
};

template <int NS>
__device__ __forceinline__ Rec<typename Lane<NS>::V> load_rec(int off) {
    const char *p = (const char *)g_box + off;
    if constexpr (NS == 1) {
        const float4 v = *(const float4 *)p;
        return {v.x, v.y, v.z, v.w};
    } else {
        const float4 A = *(const float4 *)p, B = *(const float4 *)(p + kRowC);
        return {make_float2(A.x, A.y), make_float2(A.z, A.w), make_float2(B.x, B.y), make_float2(B.z, B.w)};
    }
}

template <int NS>
__device__ __forceinline__ typename Lane<NS>::V load_kap(int off) {
    const char *p = (const char *)g_box + off;
    if constexpr (NS == 1)
        return *(const float *)p;
    else
        return *(const float2 *)p;
}

struct LawC {
    float sr, kf, af, i1, i2, gfa;
};

// The law of a bond past its elastic limit. It is evaluated only in the
// fix-up of flagged bonds (below), never in the unrolled bond loop: the law
// (divisions, an exponential) inlined at each of the 61 rounds multiplied the
// loop's code until the instruction cache starved the warps.
template <int LAW>
__device__ __forceinline__ float law_cold(float s, float s0, LawC lc) {
    return law_damage<float>(LAW, s, s0, crit_stretch(s0, lc.sr, lc.gfa), lc.kf, lc.af, lc.i1, lc.i2);
}

// Per-lane context of the bond loop.
template <int NS>
struct BondCtx {
    using V = typename Lane<NS>::V;
    int rb, lb;        // byte offset (in the staged box) of the lane's own record; bytes per layer
    int kb, lk;        // the same for the staged kappa values
    V sg;              // +1 (sub-lane 0) or -1 (sub-lane 1)
    V cx, cy, cz;      // -sg x the lane's own displacement (cell units)
    V h, kap;          // own s0 / 2 and kappa
    float4 *dq0, *dq1; // damage quads of the lane's samples ([quad][32 lanes] float4)
    const float4 *tq;  // the same quads of the template (initial damage, shared by all samples)
    unsigned dw;       // groups of 8 rounds read from dq0 (bits 0-7) and dq1 (bits 8-15), else from tq
    bool w0, w1;       // damage writes enabled per sample
    LawC lc;
};

// Damage words of one prefetched group of rounds: two quads (8 rounds) of
// the one sample, or one quad (4 rounds) of each sample of a pair (half the
// words in flight, so that the pair kernel fits fewer registers).
template <int NS>
struct DQ;
template <>
struct DQ<1> {
    float4 a0, a1;
};
template <>
struct DQ<2> {
    float4 a0, b0;
};
template <int NS>
constexpr int kGroupRounds = NS == 1 ? 8 : 4;

// A group whose damage no bond has changed since the reset equals the
// template, which all samples of the launch share (it stays in L2): its words
// are read from there, and only groups that some fix-up has written come
// from the sample's own words (the same values either way).
template <int NS>
__device__ __forceinline__ DQ<NS> load_dq(const BondCtx<NS> &cx, int g) {
    DQ<NS> q;
    if constexpr (NS == 1) {
        const float4 *p = (cx.dw >> g) & 1u ? cx.dq0 : cx.tq;
        q.a0 = p[32 * (2 * g)];
        q.a1 = p[32 * (2 * g + 1)];
    } else {
        const float4 *p0 = (cx.dw >> (g / 2)) & 1u ? cx.dq0 : cx.tq;
        const float4 *p1 = (cx.dw >> (8 + g / 2)) & 1u ? cx.dq1 : cx.tq;
        q.a0 = p0[32 * g];
        q.b0 = p1[32 * g];
    }
    return q;
}

template <int J>
__device__ __forceinline__ float quad_el(const float4 &a0, const float4 &a1) {
    const float4 &v = J < 4 ? a0 : a1;
    constexpr int e = J % 4;
    return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}

// Damage of round J of the group, per sample of the lane.
template <int NS, int J>
__device__ __forceinline__ typename Lane<NS>::V dmg_el(const DQ<NS> &q) {
    if constexpr (NS == 1)
        return quad_el<J>(q.a0, q.a1);
    else
        return make_float2(quad_el<J>(q.a0, q.a0), quad_el<J>(q.b0, q.b0));
}

// Kinematics of one bond with offset k (cell units) from the staged record r
// of its neighbour: the lower end's displacement is subtracted from the upper
// end's (sg carries the sub-lane's role), eta = u_upper - u_lower, y = k +
// eta, and the stretch s = (|y| - |k|)/|k| = eta.(2k + eta) / (|k| (|y| + |k|))
// with |y|^2 = |k|^2 + eta.(2k + eta); zero components of k add nothing. The
// unrolled loop (k known at compile time) and the fix-up of bonds past their
// elastic limit (k from a table) run these same operations, so both see the
// same bits.
template <class V, class Ctx>
__device__ __forceinline__ void bond_kin(const Ctx &cx, const Rec<V> &r, int kx, int ky, int kz, float KW, float KW2,
                                         V &yx, V &yy, V &yz, V &rL, V &s) {
    const V ex = vfma(cx.sg, r.x, cx.cx);
    const V ey = vfma(cx.sg, r.y, cx.cy);
    const V ez = vfma(cx.sg, r.z, cx.cz);
    yx = kx ? vadd(ex, splat<V>((float)kx)) : ex;
    yy = ky ? vadd(ey, splat<V>((float)ky)) : ey;
    yz = kz ? vadd(ez, splat<V>((float)kz)) : ez;
    const V wx = kx ? vadd(ex, splat<V>(2.0f * kx)) : ex;
    const V wy = ky ? vadd(ey, splat<V>(2.0f * ky)) : ey;
    const V wz = kz ? vadd(ez, splat<V>(2.0f * kz)) : ez;
    const V num = vfma(ez, wz, vfma(ey, wy, vmul(ex, wx)));
    // |y|^2, kept at or above 1e-12 (cell units): the floor only acts on a
    // bond shorter than a millionth of a cell. A broken bond compressed to
    // zero length under a crushing load can reach |y|^2 <= 0 in FP32, where
    // 1/|y| would be infinite and (1 - d) s / |y| = 0 x inf not a number;
    // with the floor its force is exactly zero, as a broken bond's must be.
    const V y2 = vmax(vadd(num, splat<V>(KW2)), splat<V>(kMinY2));
    rL = vrsqrt(y2);
    const V L = vmul(y2, rL);
    s = vmul(num, vrcp(vfma(L, splat<V>(KW), splat<V>(KW2))));
}

// Force factor (1 - d) s / |y| of a bond (times kappa_i + kappa_j with a
// stiffness field; micromodulus and volume are applied to the node sum).
template <class V>
__device__ __forceinline__ V bond_g(V d, V s, V rL) {
    return vmul(vfma(neg(d), s, s), rL);
}

// Offsets of the rounds of the positive half-stencil, for the fix-up path:
// kx, ky, kz and |k|^2 in the bytes of one word (padding rounds: zero), and
// |k| (the float the unrolled loop uses for the same round). The lanes of a
// warp fix up different rounds, so the table is read through the read-only
// data cache, which serves divergent addresses of one line together (the
// constant bank serves them one address at a time).
struct __align__(8) HalfEnt {
    int k;
    float kw;
};
struct HalfTab {
    HalfEnt e[64];
};
template <int DIM>
__host__ __device__ constexpr HalfTab half_table() {
    HalfTab t{};
    for (int m = 0; m < 64; ++m) {
        const I3 k = m < Sten<DIM>::kHalf ? half_off<DIM>(m) : I3{0, 0, 0};
        const int q = k.x * k.x + k.y * k.y + k.z * k.z;
        t.e[m].k = (int)((unsigned)(k.x & 0xFF) | ((unsigned)(k.y & 0xFF) << 8) | ((unsigned)(k.z & 0xFF) << 16) |
                         ((unsigned)q << 24));
        t.e[m].kw = knorm(q);
    }
    return t;
}
__device__ const HalfTab g_half[2] = {half_table<2>(), half_table<3>()};

// The fix-up of one bond (round m) whose stretch passed its elastic limit
// this step: recompute it (the same operations as the unrolled loop, so the
// same bits), apply the law, store the damage where it grew (only when act),
// and return the correction of the force factor -- the unrolled loop formed
// the lane's sums with the previous damage dold, which the caller loads --
// with the bond's direction (zero where nothing grew). The two directed
// copies of a bond run the same correction.
template <class V>
struct FixOut {
    V dg, yx, yy, yz;
};

// Previous damage of round m, per sample of the lane (the sample's own words:
// a group read from the template holds the same values).
template <int NS>
__device__ __forceinline__ typename Lane<NS>::V load_dold(int m, const BondCtx<NS> &cx) {
    const float *slot0 = (const float *)(cx.dq0 + 32 * (m / 4)) + (m % 4);
    if constexpr (NS == 1) {
        return *slot0;
    } else {
        const float *slot1 = (const float *)(cx.dq1 + 32 * (m / 4)) + (m % 4);
        return make_float2(*slot0, *slot1);
    }
}

template <int DIM, int NS, int LAW, bool KAPPA>
__device__ __forceinline__ FixOut<typename Lane<NS>::V> fix_one(int m, bool act, const BondCtx<NS> &cx, unsigned &dwn,
                                                                typename Lane<NS>::V dold) {
    using V = typename Lane<NS>::V;
    const int2 e = __ldg(reinterpret_cast<const int2 *>(&g_half[DIM - 2].e[m]));
    const int kx = (int)((unsigned)e.x << 24) >> 24, ky = (int)((unsigned)e.x << 16) >> 24;
    const int kz = (int)((unsigned)e.x << 8) >> 24, q = (int)((unsigned)e.x >> 24);
    const Rec<V> r = load_rec<NS>(cx.rb + cx.lb * kz + 16 * kx + NS * kRowC * ky);
    FixOut<V> o;
    V rL, s;
    bond_kin<V>(cx, r, kx, ky, kz, __int_as_float(e.y), (float)q, o.yx, o.yy, o.yz, rL, s);
    const V s0 = vadd(cx.h, r.h);
    float *slot0 = (float *)(cx.dq0 + 32 * (m / 4)) + (m % 4);
    V dnew;
    if constexpr (NS == 1) {
        const float dl = s > s0 ? law_cold<LAW>(s, s0, cx.lc) : 0.f;
        const bool grow = act && dl > dold;
        dnew = grow ? dl : dold;
        if (grow) {
            *slot0 = dl;
            dwn |= 1u << (16 + m / 8);
        }
    } else {
        float *slot1 = (float *)(cx.dq1 + 32 * (m / 4)) + (m % 4);
        const float dlx = s.x > s0.x ? law_cold<LAW>(s.x, s0.x, cx.lc) : 0.f;
        const float dly = s.y > s0.y ? law_cold<LAW>(s.y, s0.y, cx.lc) : 0.f;
        const bool gx = act && dlx > dold.x, gy = act && dly > dold.y;
        dnew = make_float2(gx ? dlx : dold.x, gy ? dly : dold.y);
        if (gx && cx.w0) {
            *slot0 = dlx;
            dwn |= 1u << (16 + m / 8);
        }
        if (gy && cx.w1) {
            *slot1 = dly;
            dwn |= 1u << (24 + m / 8);
        }
    }
    o.dg = vsub(bond_g(dnew, s, rL), bond_g(dold, s, rL));
    if constexpr (KAPPA) {
        o.dg = vmul(o.dg, vadd(cx.kap, load_kap<NS>(cx.kb + cx.lk * kz + 4 * NS * kx + NS * kRowK * ky)));
    }
    return o;
}

// Bonds of rounds m0 + j (bit j of mask) whose stretch passed their elastic
// limit this step: fixed up two at a time (independent instruction streams,
// so that their latencies overlap in the few warps at a growing crack), the
// corrections added to the lane's sums in ascending round order.
template <int DIM, int NS, int LAW, bool KAPPA>
__device__ __forceinline__ void fix_bonds(unsigned mask, int m0, const BondCtx<NS> &cx, unsigned &dwn,
                                          typename Lane<NS>::V &px,
                                       typename Lane<NS>::V &py, typename Lane<NS>::V &pz) {
    using V = typename Lane<NS>::V;
    while (mask) {
        const int j1 = __ffs(mask) - 1;
        mask &= mask - 1;
        const bool two = mask != 0u;
        const int j2 = two ? __ffs(mask) - 1 : j1;  // without a second bond: the first again, with no effect
        if (two) mask &= mask - 1;
        // both damage words are read before either bond stores (the rounds
        // differ, or the second bond changes nothing), so the two reads share
        // one memory latency
        const V da = load_dold<NS>(m0 + j1, cx), db = load_dold<NS>(m0 + j2, cx);
        const FixOut<V> a = fix_one<DIM, NS, LAW, KAPPA>(m0 + j1, true, cx, dwn, da);
        const FixOut<V> b = fix_one<DIM, NS, LAW, KAPPA>(m0 + j2, two, cx, dwn, db);
        px = vfma(a.dg, a.yx, px);
        py = vfma(a.dg, a.yy, py);
        pz = vfma(a.dg, a.yz, pz);
        px = vfma(b.dg, b.yx, px);
        py = vfma(b.dg, b.yy, py);
        pz = vfma(b.dg, b.yz, pz);
    }
}

// One bond of the lane (round M, offset k = k_M) with the previous damage d,
// for its one or two samples; a stretch past the elastic limit of a bond not
// yet broken sets bit J of the group's mask (the law runs in fix_bonds).
template <int DIM, int NS, bool KAPPA, int M, int J>
__device__ __forceinline__ void stencil_bond(typename Lane<NS>::V d, const BondCtx<NS> &cx, typename Lane<NS>::V &px,
                                             typename Lane<NS>::V &py, typename Lane<NS>::V &pz, unsigned &mask) {
    using V = typename Lane<NS>::V;
    constexpr I3 k = half_off<DIM>(M);
    constexpr int q = k.x * k.x + k.y * k.y + k.z * k.z;
    const Rec<V> r = load_rec<NS>(cx.rb + cx.lb * k.z + 16 * k.x + NS * kRowC * k.y);
    V yx, yy, yz, rL, s;
    bond_kin<V>(cx, r, k.x, k.y, k.z, knorm(q), (float)q, yx, yy, yz, rL, s);
    const V s0 = vadd(cx.h, r.h);
    // a broken or absent bond (d = 1: cut by the notch, or a neighbour
    // outside the body, whose staged record reads as zero) has nothing left
    // to soften, whatever its stretch
    bool past;
    if constexpr (NS == 1)
        past = s > s0 && d < 1.0f;
    else
        past = (s.x > s0.x && d.x < 1.0f) || (s.y > s0.y && d.y < 1.0f);
    if (past) mask |= 1u << J;
    V g = bond_g(d, s, rL);
    if constexpr (KAPPA) g = vmul(g, vadd(cx.kap, load_kap<NS>(cx.kb + cx.lk * k.z + 4 * NS * k.x + NS * kRowK * k.y)));
    px = vfma(g, yx, px);
    py = vfma(g, yy, py);
    pz = vfma(g, yz, pz);
}

template <int DIM, int NS, bool KAPPA, int M, int J, int JG>
__device__ __forceinline__ void bond_if(const BondCtx<NS> &cx, const DQ<NS> &dq, typename Lane<NS>::V &px,
                                        typename Lane<NS>::V &py, typename Lane<NS>::V &pz, unsigned &mask) {
    if constexpr (M < Sten<DIM>::kHalf) {
        stencil_bond<DIM, NS, KAPPA, M, JG>(dmg_el<NS, J>(dq), cx, px, py, pz, mask);
    }
}

template <int DIM, int NS, bool KAPPA, int M0, int JG0, int... J>
__device__ __forceinline__ void bond_group(const BondCtx<NS> &cx, const DQ<NS> &dq, typename Lane<NS>::V &px,
                                           typename Lane<NS>::V &py, typename Lane<NS>::V &pz, unsigned &mask,
                                           std::integer_sequence<int, J...>) {
    (bond_if<DIM, NS, KAPPA, M0 + J, J, JG0 + J>(cx, dq, px, py, pz, mask), ...);
}

// The rounds are summed 16 at a time: the FP32 sum of 16 bonds is added to
// the compensated (TwoSum) accumulator after the bonds among them that passed
// their elastic limit have been fixed up. The sums do not depend on the
// prefetch group (8 or 4 rounds), so one-sample and paired lanes agree bit
// for bit.
constexpr int kSumRounds = 16;

// Groups [G, G1) of kGroupRounds rounds; the next group's damage words are
// requested before the current group is computed.
template <int DIM, int NS, int LAW, bool KAPPA, int G, int G1>
__device__ __forceinline__ void bond_groups(const BondCtx<NS> &cx, const DQ<NS> &cur, typename Lane<NS>::V *acc,
                                            typename Lane<NS>::V &px, typename Lane<NS>::V &py,
                                            typename Lane<NS>::V &pz, unsigned &mask, unsigned &dwn) {
    using V = typename Lane<NS>::V;
    constexpr int GR = kGroupRounds<NS>, GS = kSumRounds / GR;
    if constexpr (G < G1) {
        DQ<NS> nxt;
        if constexpr (G + 1 < G1) nxt = load_dq<NS>(cx, G + 1);
        constexpr int G0 = G - (G % GS);  // first group of the sum
        bond_group<DIM, NS, KAPPA, GR * G, GR * (G - G0)>(cx, cur, px, py, pz, mask,
                                                           std::make_integer_sequence<int, GR>{});
        if (G % GS == GS - 1 || G + 1 == G1) {
            if (__builtin_expect(mask != 0u, 0)) fix_bonds<DIM, NS, LAW, KAPPA>(mask, GR * G0, cx, dwn, px, py, pz);
            two_sum_acc_v(acc[0], acc[3], px);
            two_sum_acc_v(acc[1], acc[4], py);
            two_sum_acc_v(acc[2], acc[5], pz);
            px = py = pz = splat<V>(0.f);
            mask = 0u;
        }
        if constexpr (G + 1 < G1) bond_groups<DIM, NS, LAW, KAPPA, G + 1, G1>(cx, nxt, acc, px, py, pz, mask, dwn);
    }
}

// Rounds [R0, R1) of the half-stencil.
template <int DIM, int NS, int LAW, bool KAPPA, int R0, int R1>
__device__ __forceinline__ void bond_span(const BondCtx<NS> &cx, typename Lane<NS>::V *acc, unsigned &dwn) {
    static_assert(R0 % kSumRounds == 0, "spans start at a sum boundary");
    using V = typename Lane<NS>::V;
    constexpr int GR = kGroupRounds<NS>;
    const DQ<NS> first = load_dq<NS>(cx, R0 / GR);
    V px = splat<V>(0.f), py = px, pz = px;
    unsigned mask = 0u;
    bond_groups<DIM, NS, LAW, KAPPA, R0 / GR, R1 / GR>(cx, first, acc, px, py, pz, mask, dwn);
}

// Warps of a block: wpb row pairs x Q parts of the half-stencil, for NS
// samples (one, or a pair on the paired FP32 instructions). Part 0's warp of
// a row pair adds the other parts' sums (fixed order) and integrates.
template <int DIM, int NS, int Q, int LAW, bool KAPPA, bool FORCE_ONLY>
__device__ __forceinline__ void step_block(const StepArgs &a, const int blk, const StencilMaps *maps) {
    using V = typename Lane<NS>::V;
    using S = Sten<DIM>;
    constexpr int kRounds = S::kRounds, HZ = S::kHaloZ;
    constexpr int RB = NS * kRowC;  // bytes of a staged (y, z) row of records
    constexpr int RK = NS * kRowK;  // bytes of a staged row of kappa values
    __shared__ double red[NS][16];
    __shared__ float s_pre[NS][4];  // U(n+1) and the prescribed velocity, double-float
    __shared__ unsigned s_cnt[NS];
    __shared__ RunView s_rv[NS];    // run bookkeeping per sample, with the pending reaction added
    __shared__ int s_n[NS];         // step index per sample
    __shared__ int s_ridx;          // the brick's index among the reaction bricks, or -1
    __shared__ uint64_t s_bar;      // completion of the box's TMA copies (one-sample blocks)
    __shared__ int s_staged;

    const int nwarps = blockDim.x >> 5;
    const int wpb = a.st_wpb;
    const FastDiv fg = NS == 1 ? a.fd_grp1 : a.fd_grp2;  // (B + NS - 1) / NS sample groups
    const int brick = fdiv(blk, fg);
    const int grp = blk - fg.d * brick;
    const auto sample_of = [&](int s) {
        const int b = NS * grp + s;
        return b < a.B ? b : NS * grp;  // the second member of the last pair of an odd batch is a copy
    };
    // Launched as a programmatic dependent of the previous step: let the next
    // step's blocks be scheduled now, and wait here until the previous step
    // has completed and its writes are visible (both are no-ops otherwise).
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int bxy = fdiv(brick, a.fd_nbx), bz = fdiv(bxy, a.fd_nby);
    const int bx = brick - a.nbx * bxy, by = bxy - a.nby * bz;
    const int x0 = kSlice * bx, y0 = a.BY * by, z0 = a.BZ * bz;
    const size_t BN = (size_t)a.B * a.N;
    const int Wy = a.BY + 2 * kHalo;
    const int Zp = a.BZ + HZ;    // layers of each copy: upper (sub-lane 0) and reflected lower (sub-lane 1)
    const int LB = RB * Wy, LK = RK * Wy;
    // record copies on 128-byte boundaries (TMA destinations), then the kappa
    // copies (KAPPA) and the parts' partial sums (Q > 1)
    const int CP = (LB * Zp + 127) & ~127;
    const int pad = (int)((0u - sm_addr(g_box)) & 127u);
    const int oP = pad, oM = pad + CP;
    const int okP = pad + 2 * CP, okM = okP + LK * Zp;
    const int oPart = KAPPA ? okM + LK * Zp : okP;
    float *s_part = (float *)((char *)g_box + oPart);  // [Q-1][wpb][16][6 NS]
    // One-sample steps: every live sample of the state is at the step parity
    // a.par ^ a.rec_off (the launch parity and the offset set by the last
    // reset or load), which selects the record buffer to stage; the box's TMA
    // copies go out at once, before the per-sample bookkeeping is read (whose
    // step index is checked against it below). Force-only evaluations, which
    // include samples stopped at other steps, stage after reading it.
    constexpr bool kEarly = NS == 1 && !FORCE_ONLY;
    const int rpar = (a.par ^ a.rec_off) & 1;
    const auto issue_box = [&](int par0) {
        stage_bar_init(&s_bar);
        stage_bar_expect(&s_bar, 2u * (uint32_t)(LB * Zp));
        const int b0 = sample_of(0);
        stage_box((char *)g_box + oP, &maps->rec[par0], x0 - kHalo, y0 - kHalo, z0, b0, &s_bar);
        stage_box((char *)g_box + oM, &maps->ref[par0], a.nx - kSlice - kHalo - x0, a.ny - a.BY - kHalo - y0,
                  a.nz - a.BZ - z0, b0, &s_bar);
    };
    if constexpr (kEarly) {
        if (threadIdx.x == 0) issue_box(rpar);
    }
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
    if (!any) {  // block-uniform
        if (kEarly && threadIdx.x == 0) stage_bar_wait(&s_bar);  // the copies land before the block leaves
        return;
    }
    if (kEarly && threadIdx.x == 0 && (ns[0] & 1) != rpar) atomicOr(&a.status[sample_of(0)], 4);
    if (threadIdx.x == 0) s_ridx = FORCE_ONLY ? -1 : a.brick_ridx[brick];
    const int n_mine = (NS == 2 && threadIdx.x == 1) ? ns[NS - 1] : ns[0];  // the step of sample threadIdx.x
    if (threadIdx.x < NS) s_n[threadIdx.x] = n_mine;
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
    if (threadIdx.x < 16 * NS) (&red[0][0])[threadIdx.x] = 0.0;
    if (threadIdx.x < NS) {
        df U1, vp;
        prescribed(a, n_mine, U1, vp);
        s_pre[threadIdx.x][0] = U1.hi;
        s_pre[threadIdx.x][1] = U1.lo;
        s_pre[threadIdx.x][2] = vp.hi;
        s_pre[threadIdx.x][3] = vp.lo;
        s_cnt[threadIdx.x] = 0u;
    }

    // The dirty bits of this thread's lane and part (byte `part` of the lane's
    // word holds the part's groups of 8 rounds from bit 0), read before the
    // staging wait so that their latency overlaps it.
    constexpr int kGroups = kRounds / 8;
    const auto dirty_byte = [&](int s) {
        const size_t lane_slot = ((size_t)brick * wpb + (threadIdx.x >> 5) % wpb) * 32 + (threadIdx.x & 31);
        return a.dirty + ((size_t)sample_of(s) * (size_t)(a.sell_len / kRounds) + lane_slot) * 4 +
               (threadIdx.x >> 5) / wpb;
    };
    const unsigned dw0 = *dirty_byte(0), dw1 = NS == 2 ? (unsigned)*dirty_byte(NS - 1) : 0u;

    // stage the box (cells outside the grid read as zero): box layer lz holds
    // z0 - HZ + lz; the upper copy takes lz >= HZ, the reflected lower copy
    // lz < BZ + HZ at (Zp - 1 - lz, Wy - 1 - ly, kWx - 1 - lx). One sample:
    // both copies by TMA, the lower one from the point-reflected records (the
    // cell at (x, y, z) of the reflected grid is (nx-1-x, ny-1-y, nz-1-z)).
    {
        const int par0 = ns[0] & 1;
        if constexpr (NS == 1 && !kEarly) {
            if (threadIdx.x == 0) issue_box(par0);
        }
        if constexpr (NS == 2 || KAPPA) {
            const int nbox = kWx * Wy * (a.BZ + 2 * HZ);
            const float4 *gin0 = (par0 ? a.grec1 : a.grec0) + (size_t)sample_of(0) * a.N;
            const float4 *gin1 = ((ns[NS - 1] & 1) ? a.grec1 : a.grec0) + (size_t)sample_of(NS - 1) * a.N;
            const float *kin0 = KAPPA ? a.kappa + (size_t)sample_of(0) * a.N : nullptr;
            const float *kin1 = KAPPA ? a.kappa + (size_t)sample_of(NS - 1) * a.N : nullptr;
            // row / Wy as a multiply and shift: exact for rows below 2^20 / Wy
            // (the error of the rounded-up reciprocal stays below 1 / Wy); the
            // staged box has at most 38 x 22 rows
            const unsigned inv_wy = ((1u << 20) + (unsigned)Wy - 1u) / (unsigned)Wy;
            for (int qi = threadIdx.x; qi < nbox; qi += blockDim.x) {
                const int row = qi / kWx, lx = qi - kWx * row;
                const int lz = (int)(((unsigned)row * inv_wy) >> 20), ly = row - Wy * lz;
                const int gx = x0 - kHalo + lx, gy = y0 - kHalo + ly, gz = z0 - HZ + lz;
                const bool in = gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny && gz >= 0 && gz < a.nz;
                const int gi = in ? gx + a.nx * (gy + a.ny * gz) : 0;
                const bool toP = lz >= HZ, toM = lz < a.BZ + HZ;
                if constexpr (NS == 2) {
                    const int rP = LB * (lz - HZ) + RB * ly + 16 * lx;
                    const int rM = LB * (Zp - 1 - lz) + RB * (Wy - 1 - ly) + 16 * (kWx - 1 - lx);
                    float4 h0 = make_float4(0.f, 0.f, 0.f, 0.f), h1 = h0;
                    if (in) {
                        h0 = gin0[gi];
                        h1 = gin1[gi];
                    }
                    const float4 A = make_float4(h0.x, h1.x, h0.y, h1.y), C = make_float4(h0.z, h1.z, h0.w, h1.w);
                    if (toP) {
                        *(float4 *)((char *)g_box + oP + rP) = A;
                        *(float4 *)((char *)g_box + oP + rP + kRowC) = C;
                    }
                    if (toM) {
                        *(float4 *)((char *)g_box + oM + rM) = A;
                        *(float4 *)((char *)g_box + oM + rM + kRowC) = C;
                    }
                }
                if constexpr (KAPPA) {
                    const int kP = LK * (lz - HZ) + RK * ly + 4 * NS * lx;
                    const int kM = LK * (Zp - 1 - lz) + RK * (Wy - 1 - ly) + 4 * NS * (kWx - 1 - lx);
                    const float k0 = in ? kin0[gi] : 0.f;
                    if constexpr (NS == 1) {
                        if (toP) *(float *)((char *)g_box + okP + kP) = k0;
                        if (toM) *(float *)((char *)g_box + okM + kM) = k0;
                    } else {
                        const float2 kk = make_float2(k0, in ? kin1[gi] : 0.f);
                        if (toP) *(float2 *)((char *)g_box + okP + kP) = kk;
                        if (toM) *(float2 *)((char *)g_box + okM + kM) = kk;
                    }
                }
            }
        }
        build_views();
        if constexpr (NS == 1) {
            if (threadIdx.x == 0) s_staged = stage_bar_wait(&s_bar) ? 1 : 0;
        }
    }
    __syncthreads();
    if constexpr (NS == 1) {
        if (!s_staged) {  // block-uniform: the copies did not arrive within the limit
            if (threadIdx.x == 0) {
                atomicOr(&a.status[sample_of(0)], 2);
                stage_bar_wait(&s_bar);  // still in flight: wait once more (bounded) before leaving
            }
            return;
        }
        stage_bar_wait(&s_bar);  // completed: returns at once, and orders the box before this thread's reads
    }
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
    double Rloc[NS];  // this thread's share of each sample's reaction (FP64)
#pragma unroll
    for (int s = 0; s < NS; ++s) Rloc[s] = 0.0;
    const int row = 2 * rp + r;
    const int lz = fdiv(row, a.fd_by), ly = row - a.BY * lz;
    const int gx = x0 + c, gy = y0 + ly, gz = z0 + lz;
    const bool own = gx < a.nx && gy < a.ny && gz < a.nz;
    const int ii = gx + a.nx * (gy + a.ny * gz);
    V acc[6];  // sx, sy, sz, cx, cy, cz
#pragma unroll
    for (int q = 0; q < 6; ++q) acc[q] = splat<V>(0.f);
    if (own) {
        // own record: upper copy at (lz, kHalo + ly, kHalo + c) for sub-lane 0,
        // reflected copy at (Zp - 1 - HZ - lz, Wy - 1 - kHalo - ly, kWx - 1 - kHalo - c) for sub-lane 1
        const int rown = t == 0 ? oP + LB * lz + RB * (kHalo + ly) + 16 * (kHalo + c)
                                : oM + LB * (Zp - 1 - HZ - lz) + RB * (Wy - 1 - kHalo - ly) + 16 * (kWx - 1 - kHalo - c);
        const int kown = t == 0 ? okP + LK * lz + RK * (kHalo + ly) + 4 * NS * (kHalo + c)
                                : okM + LK * (Zp - 1 - HZ - lz) + RK * (Wy - 1 - kHalo - ly) +
                                      4 * NS * (kWx - 1 - kHalo - c);
        const Rec<V> me = load_rec<NS>(rown);
        BondCtx<NS> cx;
        cx.rb = rown;
        cx.lb = LB;
        cx.kb = kown;
        cx.lk = LK;
        cx.sg = splat<V>(t == 0 ? 1.0f : -1.0f);
        cx.cx = t == 0 ? neg(me.x) : me.x;
        cx.cy = t == 0 ? neg(me.y) : me.y;
        cx.cz = t == 0 ? neg(me.z) : me.z;
        cx.h = me.h;
        cx.kap = KAPPA ? load_kap<NS>(kown) : splat<V>(1.0f);
        cx.dq0 = (float4 *)a.dmg + (size_t)sample_of(0) * (a.sell_len / 4) +
                 ((size_t)brick * wpb + rp) * (kRounds / 4) * 32 + lane;
        cx.dq1 = cx.dq0 + (size_t)(sample_of(NS - 1) - sample_of(0)) * (a.sell_len / 4);
        cx.tq = (const float4 *)a.tmpl + ((size_t)brick * wpb + rp) * (kRounds / 4) * 32 + lane;
        const unsigned dbase = part * (kGroups / Q);  // the part's first group
        cx.dw = (dw0 << dbase) | (dw1 << (8 + dbase));
        cx.w0 = live[0];
        cx.w1 = live[NS - 1];
        cx.lc = LawC{a.s_ratio_f, a.k_f, a.alpha_f, a.inv_1mek_f, a.inv_1pa_f, a.gfA_f};
        constexpr int R = kRounds;
        unsigned dwn = 0u;  // groups whose damage a fix-up changed: bits 16-23 (sample 0), 24-31 (sample 1)
        if constexpr (Q == 1) {
            bond_span<DIM, NS, LAW, KAPPA, 0, R>(cx, acc, dwn);
        } else if constexpr (Q == 2) {
            if (part == 0)
                bond_span<DIM, NS, LAW, KAPPA, 0, R / 2>(cx, acc, dwn);
            else
                bond_span<DIM, NS, LAW, KAPPA, R / 2, R>(cx, acc, dwn);
        } else {
            static_assert(Q == 4 && R % (4 * kSumRounds) == 0, "four parts need a multiple of 64 rounds");
            if (part == 0)
                bond_span<DIM, NS, LAW, KAPPA, 0, R / 4>(cx, acc, dwn);
            else if (part == 1)
                bond_span<DIM, NS, LAW, KAPPA, R / 4, R / 2>(cx, acc, dwn);
            else if (part == 2)
                bond_span<DIM, NS, LAW, KAPPA, R / 2, 3 * R / 4>(cx, acc, dwn);
            else
                bond_span<DIM, NS, LAW, KAPPA, 3 * R / 4, R>(cx, acc, dwn);
        }
        if (__builtin_expect(dwn != 0u, 0)) {  // their words now differ from the template
            const unsigned db = part * (kGroups / Q), n0 = (dwn >> 16) & 0xFFu, n1 = dwn >> 24;
            if (n0) {
                uint8_t *p = dirty_byte(0);
                *p = (uint8_t)(*p | (n0 >> db));
            }
            if (NS == 2 && n1) {
                uint8_t *p = dirty_byte(NS - 1);
                *p = (uint8_t)(*p | (n1 >> db));
            }
        }
    }
    // The node's force is sub-lane 0's sum minus sub-lane 1's: negate on
    // sub-lane 1 (exact), then add the two partials in double-float (TwoSum is
    // exact and symmetric, so both sub-lanes end with the same total).
    if (t == 1) {
#pragma unroll
        for (int q = 0; q < 6; ++q) acc[q] = neg(acc[q]);
    }
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
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            if (FORCE_ONLY ? (NS * grp + s >= a.B) : !live[s]) continue;
            const size_t node = (size_t)sample_of(s) * a.N + ii;
            const bool odd = s_n[s] & 1;
            const float4 *rin = (const float4 *)(odd ? a.rec1 : a.rec0);
            float4 *rout = (float4 *)(odd ? a.rec0 : a.rec1);
            float4 *gout = odd ? a.grec0 : a.grec1;
            float4 *goutR = odd ? a.grecR0 : a.grecR1;
            const size_t nodeR = (size_t)sample_of(s) * a.N + (a.N - 1 - ii);  // its reflected cell
            // sub-lane 0 integrates components 0 and 2, sub-lane 1 component 1
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                const int q = t + 2 * it;
                if (q > 2) break;
                const float sq = el(it ? acc[2] : (t ? acc[1] : acc[0]), s);
                const float cq = el(it ? acc[5] : (t ? acc[4] : acc[3]), s);
                const df S = two_sum(sq, cq);  // the node's bond sum (F = cV S, or cV S / 2 with kappa)
                if (FORCE_ONLY) {
                    const df F = df_mul(S, cVd);
                    a.F_out[3 * node + q] = (double)F.hi + (double)F.lo;
                    continue;
                }
                const uint8_t code = a.codes[3 * (size_t)ii + q];
                df u = {__ldcs((const float *)(rin + node) + q), __ldcs((const float *)(rin + BN + node) + q)};
                float *vh = (float *)(a.vdf + node);
                float *vl = (float *)(a.vdf + BN + node);
                df v = {__ldcs(vh + q), __ldcs(vl + q)};
                if (code == 0) {
                    // v(n+1) = (ca v(n) + dtr F) icb with the constants folded on the host
                    v = df_add(df_mul(a.va_df, v), df_mul(KAPPA ? a.vfh_df : a.vf_df, S));
                    u = df_add(u, df_mul(a.dt_df, v));
                } else if (code == 1) {
                    u = {0.f, 0.f};
                    v = {0.f, 0.f};
                } else {
                    const df F = df_mul(S, cVd);
                    const float sg = code == 2 ? 1.0f : -1.0f;
                    Rloc[s] -= (double)sg * ((double)F.hi + (double)F.lo);
                    v = df{sg * s_pre[s][2], sg * s_pre[s][3]};
                    u = df{sg * s_pre[s][0], sg * s_pre[s][1]};
                }
                __stcs(vh + q, v.hi);
                __stcs(vl + q, v.lo);
                __stcs((float *)(rout + node) + q, u.hi);
                __stcs((float *)(rout + BN + node) + q, u.lo);
                const float gq = df_mul(u, a.idx_df).hi;
                ((float *)(gout + node))[q] = gq;
                ((float *)(goutR + nodeR))[q] = gq;
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

// One step of one state: blocks are (brick, sample group) pairs, sample fastest.
template <int DIM, int NS, int Q, int LAW, bool KAPPA, bool FORCE_ONLY>
// Register budgets: 64 registers at up to 512 threads (two blocks an SM),
// except the half-stencil split in two (Q = 2, the few-block launches of
// single samples): 80 registers at up to 256 threads, where 3 blocks an SM
// hold the whole grid; sample pairs take 128.
__global__ void __launch_bounds__(Q == 2 && NS == 1 ? 256 : 512, NS == 2 ? 1 : (Q == 2 ? 3 : 2))
    k_step_stencil(const StepArgs a, const __grid_constant__ StencilMaps t) {
    step_block<DIM, NS, Q, LAW, KAPPA, FORCE_ONLY>(a, blockIdx.x, &t);
}

// One step of two states in one launch (the fine and the coarse member of the
// coupled pairs of an MLMC level: meshes of different sizes with the same
// brick shape and law): the first nblk0 blocks step state 0, the others state
// 1, each exactly as its own launch would (same bits). The arguments stay in
// parameter space (grid constant), so selecting a state by block copies
// nothing.
template <int DIM, int Q, int LAW, bool KAPPA>
__global__ void __launch_bounds__(Q == 2 ? 256 : 512, Q == 2 ? 3 : 2) k_step_stencil_pair(const __grid_constant__ StepPair g) {
    const int i = (int)blockIdx.x >= g.nblk0 ? 1 : 0;
    step_block<DIM, 1, Q, LAW, KAPPA, false>(g.a[i], (int)blockIdx.x - (i ? g.nblk0 : 0), &g.t[i]);
}

typedef void (*StencilKernel)(const StepArgs, const StencilMaps);
typedef void (*StencilPairKernel)(const StepPair);

template <int DIM, int Q>
StencilPairKernel pick_pair_variant(int law, bool kappa) {
    if (law == PD_LAW_BILINEAR) return kappa ? k_step_stencil_pair<DIM, Q, 0, true> : k_step_stencil_pair<DIM, Q, 0, false>;
    return kappa ? k_step_stencil_pair<DIM, Q, 1, true> : k_step_stencil_pair<DIM, Q, 1, false>;
}

// The variant of one (dimension, parts) pair for samples per block, law,
// stiffness field and force-only mode; force-only evaluations always take the
// one-sample kernel (same bits).
template <int DIM, int Q>
StencilKernel pick_variant(int ns, int law, bool kappa, bool fo) {
    if (fo) {
        if (law == PD_LAW_BILINEAR)
            return kappa ? k_step_stencil<DIM, 1, Q, 0, true, true> : k_step_stencil<DIM, 1, Q, 0, false, true>;
        return kappa ? k_step_stencil<DIM, 1, Q, 1, true, true> : k_step_stencil<DIM, 1, Q, 1, false, true>;
    }
    if (ns == 2) {
        if (law == PD_LAW_BILINEAR)
            return kappa ? k_step_stencil<DIM, 2, Q, 0, true, false> : k_step_stencil<DIM, 2, Q, 0, false, false>;
        return kappa ? k_step_stencil<DIM, 2, Q, 1, true, false> : k_step_stencil<DIM, 2, Q, 1, false, false>;
    }
    if (law == PD_LAW_BILINEAR)
        return kappa ? k_step_stencil<DIM, 1, Q, 0, true, false> : k_step_stencil<DIM, 1, Q, 0, false, false>;
    return kappa ? k_step_stencil<DIM, 1, Q, 1, true, false> : k_step_stencil<DIM, 1, Q, 1, false, false>;
}

}  // namespace

// one per translation unit
typedef void (*StencilKernelFn)(const StepArgs, const StencilMaps);
typedef void (*StencilPairFn)(const StepPair);
StencilKernelFn stencil_pick_d3q1(int ns, int law, bool kappa, bool fo);
StencilKernelFn stencil_pick_d3q2(int ns, int law, bool kappa, bool fo);
StencilKernelFn stencil_pick_d3q4(int ns, int law, bool kappa, bool fo);
StencilKernelFn stencil_pick_d2(int ns, int law, bool kappa, bool fo);
StencilPairFn stencil_pair_d3q1(int law, bool kappa);
StencilPairFn stencil_pair_d3q2(int law, bool kappa);
StencilPairFn stencil_pair_d3q4(int law, bool kappa);
StencilPairFn stencil_pair_d2(int law, bool kappa);

}  // namespace pdi
