// pd_device.cuh -- device-side pieces shared by the step kernels: launch
// constants, the kernel argument block, double-float arithmetic and the bond
// laws.
#pragma once

#include <cmath>

#include "pd_internal.cuh"

namespace pdi {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kLanes = 4;   // sub-lanes per node (T)
constexpr int kSlice = 8;   // nodes per slice (C = 32 / T)
constexpr int kTab = 256;     // stencil table entries: ids 0..n_off-1, padding id 0xFF
constexpr int kPad = 0xFF;

struct df {
    float hi, lo;
};

// Division of 0 <= n < 2^31 by a launch constant d as a multiply and a shift:
// with c = ceil(log2 d), s = 31 + c and m = ceil(2^s / d) < 2^32,
// n m / 2^s = n / d + n (m d - 2^s) / (d 2^s), and the second term is below
// 2^-c <= 1/d, so it never carries the quotient past the next integer.
struct FastDiv {
    uint32_t m;
    int s;
    int d;
};

inline FastDiv fastdiv_make(int d) {
    int c = 0;
    while ((1ll << c) < (long long)d) ++c;
    const int s = 31 + c;
    const unsigned long long m = ((1ull << s) + (unsigned long long)d - 1ull) / (unsigned long long)d;
    return FastDiv{(uint32_t)m, s, d};
}

__device__ __forceinline__ int fdiv(int n, const FastDiv &f) {
    return (int)(((unsigned long long)(uint32_t)n * f.m) >> f.s);
}

struct StepArgs {
    long long N;
    long long n_slices;
    int nblk;  // bricks per sample
    int B;
    int nx, ny, nz, BY, BZ, nbx, nby, H, Wx, Wy, Wz;
    const long long *sell_off;
    const int32_t *sell_m;
    const int32_t *slice_i0;
    const int32_t *slice_nv;
    const uint8_t *ids;
    const float4 *xi_tab;
    const double4_32a *xid_tab;
    const int32_t *off_tab;
    int n_off;
    void *dmg;
    long long sell_len;
    double *u64;
    double *v64;
    void *rec0;
    void *rec1;
    const float *kappa;
    const uint8_t *codes;
    int32_t *step;         // [2][B]: step index, double-buffered by launch parity
    int32_t *done;         // [2][B]: stop flags, double-buffered the same way
    int32_t *pend;         // [2][B]: the launch that wrote this buffer left its reaction partials pending
    double *pk2;           // [2][B]: peak reaction so far, double-buffered the same way
    int32_t *ps2;          // [2][B]: its step
    int par;               // this launch reads buffer par and writes buffer 1 - par
    int rec_off;           // step parity of the live samples = par ^ rec_off (set by the last reset or load)
    int defer;             // stencil path: leave this step's reaction to the next launch
    int pendable;          // stencil path: some launch of this state may defer (blocks build run views)
    const int32_t *brick_ridx;  // [n_bricks]: index among the reaction bricks, or -1
    int32_t *status;
    double *peak;
    int32_t *peak_step;
    double *partial;       // [2][B][nblk] block partials (FP64), by launch parity
    unsigned int *ticket;
    double *reaction;
    int n_react;
    int k_local;
    double *F_out;
    double dt, rho, zeta, u_max;
    double ca, dtr, icb, idt;  // 1 - zeta dt/2, dt/rho, 1/(1 + zeta dt/2), 1/dt
    df du_df, dudt_df;         // u_max / n_ramp and u_max / (n_ramp dt)
    df ca_df, dtr_df, icb_df, dt_df;
    float4 *vdf;
    int n_ramp;
    int max_steps;
    int use_stop;
    int st_wpb;      // stencil path: row pairs per brick
    float dxf;       // dx in FP32
    float4 *grec0, *grec1;  // stencil path: gather records (u / dx in FP32, s0 / 2) by step parity
    float4 *grecR0, *grecR1;  // the same point-reflected (node i of a sample at N - 1 - i)
    const float *tmpl;        // stencil path: initial damage of every slot (0 real bond, 1 absent), shared by samples
    uint8_t *dirty;           // stencil path: per sample, lane and part, bit g = round group g differs from tmpl
    FastDiv fd_grp1, fd_grp2;   // stencil path: sample groups per brick with 1 and 2 samples per block
    FastDiv fd_nbx, fd_nby, fd_by;  // bricks along x, along y, brick rows along y
    df idx_df;              // stencil path: 1 / dx as double-float
    float L0q[10];   // sqrt(q) dx in FP32, q = |k|^2 (stencil path)
    double cV;  // micromodulus x node volume
    double V;
    double s_ratio, k, alpha, inv_1mek, inv_1pa;
    // the same constants rounded to FP32 on the host: a conversion from FP64
    // in the kernel would run on the FP64 pipe, which is narrow on this part
    float cVf, s_ratio_f, k_f, alpha_f, inv_1mek_f, inv_1pa_f;
    double gfA;   // > 0: s_crit = s0 + gfA / s0, else s_ratio s0
    float gfA_f;
    df cV_df, cVh_df;  // cV and cV / 2 as double-float (stencil path: applied to the node sums)
    // stencil path: v(n+1) = va v(n) + vf S for a free DOF with bond sum S,
    // va = ca icb and vf = dtr icb cV (vfh: cV / 2, with a stiffness field)
    df va_df, vf_df, vfh_df;
};

// The arguments of two states stepped in one launch (the first nblk0 blocks
// step a[0]).
struct StepPair {
    StepArgs a[2];
    int nblk0;
    StencilMaps t[2];
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---- double-float arithmetic (an unevaluated pair hi + lo of FP32 numbers;
// Dekker 1971, Knuth TAOCP vol. 2, 4.2.2): about 48 significant bits with
// FP32 instructions only.

// s + e = a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = a + b;
    const float z = s - a;
    const float e = (a - (s - z)) + (b - z);
    return {s, e};
}

// s + e = a + b exactly when |a| >= |b| (Dekker's FastTwoSum).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ df df_add(df x, df y) {
    const df s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}

__device__ __forceinline__ df df_mul(df x, df y) {
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return fast_two_sum(p, e);
}

__host__ __device__ __forceinline__ df df_split(double x) {
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}

// s + x with the rounding error carried in c (accumulation by TwoSum).
__device__ __forceinline__ void two_sum_acc(float &s, float &c, float x) {
    const df t = two_sum(s, x);
    s = t.hi;
    c += t.lo;
}

template <typename T>
__device__ __forceinline__ T law_damage(int law, T s, T s0, T sc, T k, T alpha, T inv_1mek, T inv_1pa);

template <>
__device__ __forceinline__ float law_damage<float>(int law, float s, float s0, float sc, float k, float alpha,
                                                   float inv_1mek, float inv_1pa) {
    if (s >= sc) return 1.0f;
    if (law == PD_LAW_BILINEAR) return 1.0f - s0 * (sc - s) / (s * (sc - s0));
    const float t = (s - s0) / (sc - s0);
    const float br = 1.0f - (1.0f - expf(-k * t)) * inv_1mek + alpha * (1.0f - t);
    return 1.0f - (s0 / s) * br * inv_1pa;
}

template <>
__device__ __forceinline__ double law_damage<double>(int law, double s, double s0, double sc, double k,
                                                     double alpha, double inv_1mek, double inv_1pa) {
    if (s >= sc) return 1.0;
    if (law == PD_LAW_BILINEAR) return 1.0 - s0 * (sc - s) / (s * (sc - s0));
    const double t = (s - s0) / (sc - s0);
    const double br = 1.0 - (1.0 - exp(-k * t)) * inv_1mek + alpha * (1.0 - t);
    return 1.0 - (s0 / s) * br * inv_1pa;
}

// Critical stretch of a bond with elastic limit s0: the fixed ratio, or the
// fracture-energy calibration s0 + A / s0.
__device__ __forceinline__ float crit_stretch(float s0, float ratio, float A) {
    return A > 0.f ? s0 + __fdividef(A, s0) : ratio * s0;
}
__device__ __forceinline__ double crit_stretch(double s0, double ratio, double A) {
    return A > 0.0 ? s0 + A / s0 : ratio * s0;
}

__device__ __forceinline__ double ramp(const StepArgs &a, int n) {
    const int m = n < a.n_ramp ? n : a.n_ramp;
    return a.u_max * (double)m / (double)a.n_ramp;
}

__device__ __forceinline__ float pick3(float a, float b, float c, int q) { return q == 0 ? a : (q == 1 ? b : c); }
__device__ __forceinline__ double pick3(double a, double b, double c, int q) { return q == 0 ? a : (q == 1 ? b : c); }


// 16-byte asynchronous global -> shared copy; src_bytes = 0 writes zeros.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }


// Prescribed displacement U(n+1) and the prescribed velocity
// (U(n+1) - U(n)) / dt of step n as double-float, from m = min(n, n_ramp)
// (FP32 only; m is exact in FP32 below 2^24).
__device__ __forceinline__ void prescribed(const StepArgs &a, int n, df &U1, df &vp) {
    const int m0 = n < a.n_ramp ? n : a.n_ramp, m1 = n + 1 < a.n_ramp ? n + 1 : a.n_ramp;
    U1 = df_mul(a.du_df, df{(float)m1, 0.f});
    vp = df_mul(a.dudt_df, df{(float)(m1 - m0), 0.f});
}

// Bookkeeping of a step launch. Blocks read step/done (and the peak so far)
// from buffer par and the launch writes buffer 1 - par, so no block has to
// wait for the others to have read them.
//
// The reaction of a step is reduced either in its own launch (the last
// reaction block to finish adds the block partials: a fence and a ticket,
// "finish") or, on the stencil path, in the next launch ("defer"): the step's
// reaction blocks store their partials with plain stores, and every block of
// the next launch adds them in the same fixed order before it does anything
// else, so all blocks reach the same peak and stop decision from the same
// bits; the kernel boundary orders the stores before those loads. The stop
// rule then applies at the same step either way. The last launch of every
// call (and of every captured chunk) finishes, so the host sees final values.

// Run bookkeeping of one sample as a launch sees it.
struct RunView {
    int n;      // the step this launch would compute
    int dn;     // the sample is done (this launch computes nothing for it)
    double Q;   // peak so far
    int np;     // its step
    double Rp;  // reaction of step n - 1, when this launch reduced it (have)
    int have;
};

// Read the bookkeeping of sample b, adding the pending reaction of the
// previous launch (one warp, all lanes; the view is complete in lane 0, the
// only lane that runs the FP64 part). The bookkeeping and the partials are
// all requested at once (one L2 round trip; the partials are read whether or
// not they are pending).
__device__ __forceinline__ RunView run_view(const StepArgs &a, int b, int lane) {
    const int i = a.par * a.B + b;
    const double *part = a.partial + ((size_t)(1 - a.par) * a.B + b) * a.nblk;
    RunView r;
    const int pe = a.pend[i];
    r.dn = a.done[i];
    r.n = a.step[i];
    r.Q = a.pk2[i];
    r.np = a.ps2[i];
    const double p0 = lane < a.nblk ? __ldcg(part + lane) : 0.0;
    r.Rp = 0.0;
    r.have = 0;
    if (r.dn || !pe) return r;
    double acc = p0;
    for (int q = lane + 32; q < a.nblk; q += 32) acc += __ldcg(part + q);
    acc = warp_sum(acc);
    r.have = 1;
    if (lane != 0) return r;
    const double R = a.V * acc;
    r.Rp = R;
    if (R > r.Q) {
        r.Q = R;
        r.np = r.n - 1;
    }
    r.dn = (a.use_stop && ((r.Q > 0.0 && (r.n - 1) - r.np >= 100 && R < 0.5 * r.Q) || r.n >= a.max_steps)) ||
                   !isfinite(R)
               ? 1
               : 0;
    return r;
}

// Outputs of the reaction this launch reduced for the previous step.
__device__ __forceinline__ void publish_pending(const StepArgs &a, int b, const RunView &r) {
    if (!r.have) return;
    a.peak[b] = r.Q;
    a.peak_step[b] = r.np;
    if (!isfinite(r.Rp)) a.status[b] |= 1;
    if (a.reaction && a.k_local >= 1) a.reaction[(size_t)b * a.n_react + a.k_local - 1] = r.Rp;
}

// Buffer 1 - par of a sample this launch does not step (done before, or done
// by the reaction it just reduced); brick 0 writes it.
__device__ __forceinline__ void write_done(const StepArgs &a, int b, const RunView &r) {
    const int o = (1 - a.par) * a.B + b;
    a.step[o] = r.n;
    a.done[o] = 1;
    a.pend[o] = 0;
    a.pk2[o] = r.Q;
    a.ps2[o] = r.np;
    publish_pending(a, b, r);
}

// Buffer 1 - par of a live sample whose reaction is left to the next launch.
__device__ __forceinline__ void write_deferred(const StepArgs &a, int b, const RunView &r) {
    const int o = (1 - a.par) * a.B + b;
    a.step[o] = r.n + 1;
    a.done[o] = 0;
    a.pend[o] = 1;
    a.pk2[o] = r.Q;
    a.ps2[o] = r.np;
    publish_pending(a, b, r);
}

// A sample that is already done is carried over by brick 0.
__device__ __forceinline__ void carry_done(const StepArgs &a, int b) {
    const int i = a.par * a.B + b;
    RunView r;
    r.n = a.step[i];
    r.Q = a.pk2[i];
    r.np = a.ps2[i];
    r.dn = 1;
    r.Rp = 0.0;
    r.have = 0;
    write_done(a, b, r);
}

// Deferred reaction: the block's partial (sum over its prescribed DOFs of
// -F sign, FP64, warp then the block's warps in order) is stored for the next
// launch. Called by every thread of a reaction block.
__device__ __forceinline__ void reaction_defer(const StepArgs &a, double Rloc, int b, int blk, int warp, int lane,
                                               int nwarps, double *red) {
    if (__any_sync(0xffffffffu, Rloc != 0.0)) Rloc = warp_sum(Rloc);
    if (lane == 0) red[warp] = Rloc;
    __syncthreads();
    if (warp == 0) {
        double v = lane < nwarps ? red[lane] : 0.0;
        if (__any_sync(0xffffffffu, v != 0.0)) v = warp_sum(v);
        if (lane == 0) a.partial[((size_t)a.par * a.B + b) * a.nblk + blk] = v;
    }
}

// End of a step kernel in a reaction brick (one holding prescribed DOFs, or
// brick 0), called by every warp of the block with all lanes active: the
// reaction sum (sum over prescribed DOFs of -F sign, FP64) is reduced in FP64
// along fixed trees -- warp, the block's warps in order (by the block's last
// warp to finish), the reaction bricks of the sample in order (by the
// sample's last reaction block) -- which then updates the run bookkeeping
// from the run view that every block of the launch holds (and publishes the
// previous step's reaction if this launch reduced it).
__device__ __forceinline__ void reaction_finish(const StepArgs &a, double Rloc, int b, int blk, int warp, int lane,
                                                int nwarps, double *red, unsigned *s_cnt, const RunView &rv) {
    if (__any_sync(0xffffffffu, Rloc != 0.0)) Rloc = warp_sum(Rloc);
    unsigned flag = 0u;
    if (lane == 0) {
        red[warp] = Rloc;
        __threadfence_block();
        flag = (atomicAdd(s_cnt, 1u) == (unsigned)(nwarps - 1));
    }
    flag = __shfl_sync(0xffffffffu, flag, 0);
    if (!flag) return;
    __threadfence_block();
    double v = 0.0;
    if (lane < nwarps) v = *(const volatile double *)(red + lane);
    // (shared-memory partials: one round trip)
    if (__any_sync(0xffffffffu, v != 0.0)) v = warp_sum(v);
    double *part = a.partial + ((size_t)a.par * a.B + b) * a.nblk;
    if (lane == 0) {
        part[blk] = v;
        __threadfence();
        flag = (atomicAdd(&a.ticket[b], 1u) == (unsigned)(a.nblk - 1));
    }
    flag = __shfl_sync(0xffffffffu, flag, 0);
    if (!flag) return;
    __threadfence();
    // the block partials are read with L2 loads issued eight at a time (a
    // dependent chain of volatile loads would cost one L2 round trip each),
    // in the order the deferred path adds them (lane, lane + 32, ...)
    double acc = 0.0;
    for (int q0 = lane; q0 < a.nblk; q0 += 256) {
        double pv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int q = q0 + 32 * u;
            pv[u] = q < a.nblk ? __ldcg(part + q) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (q0 + 32 * u < a.nblk) acc = (q0 + 32 * u == lane) ? pv[u] : acc + pv[u];
    }
    acc = warp_sum(acc);
    if (lane == 0) {
        const int n = rv.n;
        double Q = rv.have ? rv.Q : a.pk2[a.par * a.B + b];  // no view built: the buffer as read
        int np = rv.have ? rv.np : a.ps2[a.par * a.B + b];
        if (rv.have) {
            if (!isfinite(rv.Rp)) a.status[b] |= 1;
            if (a.reaction && a.k_local >= 1) a.reaction[(size_t)b * a.n_react + a.k_local - 1] = rv.Rp;
        }
        const double R = a.V * acc;
        if (!isfinite(R)) a.status[b] |= 1;
        if (a.reaction) a.reaction[(size_t)b * a.n_react + a.k_local] = R;
        if (R > Q) {
            Q = R;
            np = n;
        }
        a.peak[b] = Q;
        a.peak_step[b] = np;
        const int out = (1 - a.par) * a.B + b;
        a.pk2[out] = Q;
        a.ps2[out] = np;
        a.pend[out] = 0;
        a.step[out] = n + 1;
        a.done[out] = (a.use_stop && ((Q > 0.0 && n - np >= 100 && R < 0.5 * Q) || n + 1 >= a.max_steps)) ||
                              !isfinite(R)
                          ? 1
                          : 0;
        a.ticket[b] = 0u;
    }
}

// Kernels and host helpers of the compile-time 122-offset stencil path
// (pd_stencil.cu): the horizon |k|^2 <= 9 of m in [3, sqrt(10)).
bool stencil_applicable(const pd_state *st);
int stencil_build(pd_state *st, const int32_t *col);
int stencil_launch(const pd_state *st, const StepArgs &a, bool force_only, cudaStream_t s);
int stencil_reset_damage(pd_state *st, cudaStream_t s);
int stencil_map_damage(const pd_state *st, double *csr, bool to_state, cudaStream_t s);
// slot of every CSR bond in one sample's stencil damage array (the adjoint
// gathers its FP32 damage trajectory through it)
int stencil_slot_table(const pd_state *st, int32_t *slot, cudaStream_t s);
void stencil_fill_args(const pd_state *st, StepArgs &a);
// the stencil kernel's gather records (u / dx, s0 / 2), both parities, from the state's records
int stencil_refresh_grec(pd_state *st, cudaStream_t s);
size_t stencil_smem(const pd_state *st, int ns, bool kappa);
// two one-sample-per-block states with the same launch shape, law and kappa
// mode: one launch steps both (the fine and coarse members of MLMC pairs)
bool stencil_pairable(const pd_state *s0, const pd_state *s1);
int stencil_launch_pair(const pd_state *s0, const StepArgs &a0, const pd_state *s1, const StepArgs &a1,
                        cudaStream_t s);

}  // namespace pdi
