// pd_adjoint.cu -- discrete adjoint of the explicit step (Sections 2-3,
// Eq. PD_EOM_Dynamic, Eq. exp_scalar_force, Eq. exp_damage_parameter) and
// its chain rule back through the truncated-KL field (Section 5), giving
// dJ/dxi for J = sum_o w_o R^{n_o}.
//
// Reverse sweep with checkpoints: the forward run stores (u, v, d) every k
// steps; each segment is then recomputed step by step from its checkpoint
// (states u^n and damage d^n kept for the segment) and walked backwards:
//
//   integrator (per DOF), lv' = lamv^{n+1/2} + dt lamu^{n+1}:
//     free        lamF^n = dt lv' / (rho b),  lamv^{n-1/2} = a lv' / b,
//                 lamu^n = lamu^{n+1} + bond terms
//     prescribed  lamF^n = -sign V sum_{o: n_o = n} w_o  (u, v prescribed: no carry)
//     fixed       nothing
//   bonds (one warp per node, lanes over the node's bonds), y = xi + eta,
//   h = s / |y|, dlam = lamF_j - lamF_i, the branch of d_n = max(d_{n-1},
//   D(s_n)) taken forward kept (active when d_n > d_{n-1}):
//     lamd_tot = lamd + c_ij V h (y . dlam)
//     lamy     = -c_ij V (1 - d_n) [(y . dlam) dh/dy + h dlam]
//                + [active] lamd_tot D'(s) y / (|y| |xi|)
//     lamu_i  -= lamy;  grad_s0_i += [active] lamd_tot dD/ds0 / 2;
//     grad_kappa_i += c (-V (1 - d_n) h (y . dlam)) / 2;
//     lamd <- [not active] lamd_tot
//
// The undirected bond's damage adjoint is kept in both directed slots (both
// copies compute the same value), and the node sums are fixed xor trees, so
// the gradient is deterministic. For FP64-path states the arithmetic is FP64
// throughout. For mixed-path states the per-bond terms run in FP32
// (k_adj_bonds_f32) on an FP32 trajectory (node records u, s0 and, in
// sliced-ELL order, the damage of the bonds whose damage grows in the run;
// every other bond keeps its initial damage at every step), with the carried
// damage adjoint in double-float for growing bonds only and compensated FP32
// sums added to FP64 node sums. Both take their states from the state's own
// forward path.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pd_device.cuh"

namespace pdi {

struct AdjArgs {
    int B;
    long long N, nb;
    int nx, ny;
    double dx, c, V, dt, rho, a, b;
    double dt_rb, a_b;  // dt / (rho b) and a / b (no FP64 division per DOF)
    int law;
    double s_ratio, k, alpha, gfA;
    const int32_t *row_ptr, *col;
    const uint8_t *codes;
    const float *s0, *kappa;
    int n_obs;
    const int32_t *obs;  // [n_obs] local step of each observation
    const double *w;     // [B][n_obs]
    const int32_t *coord;  // packed grid coordinates per node
    // FP32 constants of the mixed path, rounded on the host (the FP64 pipe is
    // narrow on this part): c V, dx, and |xi| = sqrt(q) dx and its reciprocal
    // for q = |k|^2 < 64
    float cVf, dxf, s_ratio_f, gfA_f, k_f, alpha_f;
    float L0q[64], iL0q[64];
};

// dD/ds and the total dD/ds0 = dD/ds0|sc + (dsc/ds0) dD/dsc on (s0, sc),
// zero outside; sc = ratio s0 (dsc/ds0 = ratio) or s0 + A/s0 (1 - A/s0^2).
//   bilinear D = 1 - s0 (sc - s) / (s (sc - s0)):
//     dD/ds = s0 sc / (s^2 w), dD/ds0|sc = -(sc/s - 1) sc / w^2,
//     dD/dsc|s0 = -s0 (1 - s0/s) / w^2, w = sc - s0
//   exp-linear D = 1 - (s0/s) beta(t) / (1 + alpha), t = (s - s0) / w:
//     dt/ds = 1/w, dt/ds0 = (s - sc)/w^2, dt/dsc = -(s - s0)/w^2,
//     beta' = -k e^{-kt} / (1 - e^{-k}) - alpha
__device__ __forceinline__ void law_derivs(const AdjArgs &a, double s, double s0, double &dDds, double &dDds0) {
    const double sc = a.gfA > 0.0 ? s0 + a.gfA / s0 : a.s_ratio * s0;
    const double dsc = a.gfA > 0.0 ? 1.0 - a.gfA / (s0 * s0) : a.s_ratio;
    dDds = 0.0;
    dDds0 = 0.0;
    if (s <= s0 || s >= sc) return;
    const double w = sc - s0;
    if (a.law == PD_LAW_BILINEAR) {
        dDds = s0 * sc / (s * s * w);
        dDds0 = -(sc / s - 1.0) * sc / (w * w) + dsc * (-s0 * (1.0 - s0 / s) / (w * w));
        return;
    }
    const double t = (s - s0) / w;
    const double e = exp(-a.k * t), ek = 1.0 - exp(-a.k);
    const double beta = 1.0 - (1.0 - e) / ek + a.alpha * (1.0 - t);
    const double dbeta = -a.k * e / ek - a.alpha;
    const double dtds = 1.0 / w, dtds0 = (s - sc) / (w * w), dtdsc = -(s - s0) / (w * w);
    dDds = (s0 * beta / (s * s) - (s0 / s) * dbeta * dtds) / (1.0 + a.alpha);
    dDds0 = (-(beta / s + (s0 / s) * dbeta * dtds0) - dsc * (s0 / s) * dbeta * dtdsc) / (1.0 + a.alpha);
}

// Integrator adjoint of local step `ls`: lamF, lamv (in place) and the carried
// part of lamu^n (lun) from lamu^{n+1} (lu).
__global__ void k_adj_nodes(const AdjArgs a, int ls, const double *lu, double *lv, double *lF, double *lun) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // DOF of sample blockIdx.y
    if (q >= a.N * 3) return;
    const int b = blockIdx.y;
    const long long t = (long long)b * a.N * 3 + q;
    const uint8_t code = a.codes[q];
    if (code == 0) {
        const double lvp = lv[t] + a.dt * lu[t];
        lF[t] = a.dt_rb * lvp;
        lv[t] = a.a_b * lvp;
        lun[t] = lu[t];
    } else if (code == 1) {
        lF[t] = 0.0;
        lv[t] = 0.0;
        lun[t] = 0.0;
    } else {
        double wn = 0.0;
        for (int o = 0; o < a.n_obs; ++o)
            if (a.obs[o] == ls) wn += a.w[(size_t)b * a.n_obs + o];
        const double sg = code == 2 ? 1.0 : -1.0;
        lF[t] = -sg * a.V * wn;
        lv[t] = 0.0;
        lun[t] = 0.0;
    }
}

__device__ __forceinline__ double warp_sum_fixed(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Bond adjoint of one step: one warp per (sample, node).
__global__ void __launch_bounds__(256) k_adj_bonds(const AdjArgs a, const double *u, const double *dprev,
                                                   const double *dcur, const double *lF, double *ld, double *lun,
                                                   double *g_s0, double *g_k) {
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= (long long)a.B * a.N) return;  // warp-uniform
    const int b = (int)(gw / a.N);
    const long long i = gw % a.N;
    const int ix = (int)(i % a.nx), iy = (int)((i / a.nx) % a.ny), iz = (int)(i / ((long long)a.nx * a.ny));
    const double *ub = u + (size_t)b * a.N * 3;
    const double *lFb = lF + (size_t)b * a.N * 3;
    const float *s0b = a.s0 + (size_t)b * a.N;
    const float *kb = a.kappa ? a.kappa + (size_t)b * a.N : nullptr;
    const size_t db = (size_t)b * a.nb;
    const double ui[3] = {ub[3 * i], ub[3 * i + 1], ub[3 * i + 2]};
    const double li[3] = {lFb[3 * i], lFb[3 * i + 1], lFb[3 * i + 2]};
    const double s0i = (double)s0b[i], ki = kb ? (double)kb[i] : 1.0;
    double acc[3] = {0.0, 0.0, 0.0}, gs = 0.0, gk = 0.0;
    for (int q = a.row_ptr[i] + lane; q < a.row_ptr[i + 1]; q += 32) {
        const long long j = a.col[q];
        const int jx = (int)(j % a.nx), jy = (int)((j / a.nx) % a.ny), jz = (int)(j / ((long long)a.nx * a.ny));
        const double xi[3] = {(jx - ix) * a.dx, (jy - iy) * a.dx, (jz - iz) * a.dx};
        double y[3], dl[3], L0 = 0.0, L = 0.0, ydl = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            y[c] = xi[c] + (ub[3 * j + c] - ui[c]);
            dl[c] = lFb[3 * j + c] - li[c];
            L0 += xi[c] * xi[c];
            L += y[c] * y[c];
            ydl += y[c] * dl[c];
        }
        L0 = sqrt(L0);
        L = sqrt(L);
        const double s = (L - L0) / L0, h = s / L;
        const double s0 = 0.5 * (s0i + (double)s0b[j]);
        const double cij = kb ? a.c * 0.5 * (ki + (double)kb[j]) : a.c;
        const double dp = dprev[db + q], dc = dcur[db + q];
        const bool active = dc > dp;
        const double lamd = ld[db + q] + cij * a.V * h * ydl;
        double dDds = 0.0, dDds0 = 0.0;
        if (active) law_derivs(a, s, s0, dDds, dDds0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double dh = y[c] / (L * L * L0) - s * y[c] / (L * L * L);
            double lamy = -cij * a.V * (1.0 - dc) * (ydl * dh + h * dl[c]);
            if (active) lamy += lamd * dDds * y[c] / (L * L0);
            acc[c] -= lamy;
        }
        if (active) gs += 0.5 * lamd * dDds0;
        gk += 0.5 * a.c * (-a.V * (1.0 - dc) * h * ydl);
        ld[db + q] = active ? 0.0 : lamd;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c] = warp_sum_fixed(acc[c]);
    gs = warp_sum_fixed(gs);
    gk = warp_sum_fixed(gk);
    if (lane == 0) {
        double *lb = lun + (size_t)b * a.N * 3 + 3 * i;
        lb[0] += acc[0];
        lb[1] += acc[1];
        lb[2] += acc[2];
        g_s0[(size_t)b * a.N + i] += gs;
        if (g_k) g_k[(size_t)b * a.N + i] += gk;
    }
}

// FP32 variant for states of the mixed path (their trajectory is FP32-class
// already): the same terms per bond in FP32 on FP32 copies of u^n and lamF^n;
// per-lane partial sums in FP32 (a lane takes ~4 of a node's bonds), warp sums
// and the carried damage adjoint in FP64. GB300 runs FP64 at a small fraction
// of the FP32 rate, so this keeps the FP64 pipe to a few operations per bond.
__device__ __forceinline__ void law_derivs_f(const AdjArgs &a, float s, float s0, float &dDds, float &dDds0) {
    const float sc = a.gfA_f > 0.f ? s0 + a.gfA_f / s0 : a.s_ratio_f * s0;
    const float dsc = a.gfA_f > 0.f ? 1.0f - a.gfA_f / (s0 * s0) : a.s_ratio_f;
    dDds = 0.0f;
    dDds0 = 0.0f;
    if (s <= s0 || s >= sc) return;
    const float w = sc - s0;
    if (a.law == PD_LAW_BILINEAR) {
        dDds = s0 * sc / (s * s * w);
        dDds0 = -(sc / s - 1.0f) * sc / (w * w) + dsc * (-s0 * (1.0f - s0 / s) / (w * w));
        return;
    }
    const float k = a.k_f, al = a.alpha_f;
    const float t = (s - s0) / w;
    const float e = expf(-k * t), ek = 1.0f - expf(-k);
    const float beta = 1.0f - (1.0f - e) / ek + al * (1.0f - t);
    const float dbeta = -k * e / ek - al;
    const float dtds = 1.0f / w, dtds0 = (s - sc) / (w * w), dtdsc = -(s - s0) / (w * w);
    dDds = (s0 * beta / (s * s) - (s0 / s) * dbeta * dtds) / (1.0f + al);
    dDds0 = (-(beta / s + (s0 / s) * dbeta * dtds0) - dsc * (s0 / s) * dbeta * dtdsc) / (1.0f + al);
}


// Node records of the mixed path at one step: (u, s0) with u = u_hi + u_lo
// rounded to FP32, from the state's double-float gather records.
__global__ void k_rec_to_u4(long long BN, const float4 *rec, float4 *u4) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= BN) return;
    const float4 h = rec[t], l = rec[BN + t];
    u4[t] = make_float4(h.x + l.x, h.y + l.y, h.z + l.z, h.w);
}

// (lamF, kappa) per node in FP32 for the mixed path's bond adjoint.
__global__ void k_lF_to_f4(long long BN, const double *lF, const float *kappa, float4 *lF4) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= BN) return;
    lF4[t] = make_float4((float)lF[3 * t], (float)lF[3 * t + 1], (float)lF[3 * t + 2], kappa ? kappa[t] : 1.0f);
}

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

// Sliced ELL layout of the CSR bonds for the mixed path's bond adjoint:
// slices of 32 consecutive nodes, slot-major inside a slice (slot p of node
// 32 sl + lane at off[sl] + 32 p + lane), rows padded to the slice's longest.
// Rows are sorted, so at a slot the interior nodes of a slice take the same
// stencil offset and their neighbour gathers are contiguous. Per slot: the
// CSR position q_of, and the neighbour's grid offset k_of = (kx, ky, kz) as
// three signed bytes (the neighbour is i + kx + nx (ky + ny kz); |k| < 128
// cells, checked by the host), -1 for a padding slot.
__global__ void k_sell_fill(long long N, const int32_t *row_ptr, const int32_t *col, const int32_t *coord,
                            const long long *off, int32_t *q_of, int32_t *k_of) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const long long base = off[i >> 5] + (i & 31);
    const int ci = coord[i];
    for (int q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
        const long long x = base + 32ll * (q - row_ptr[i]);
        const int cj = coord[col[q]];
        const int kx = (cj & 2047) - (ci & 2047), ky = ((cj >> 11) & 2047) - ((ci >> 11) & 2047),
                  kz = (cj >> 22) - (ci >> 22);
        q_of[x] = q;
        k_of[x] = (kx & 0xff) | ((ky & 0xff) << 8) | ((kz & 0xff) << 16);
    }
}

// Damage of every sample in sliced-ELL order from the CSR-order slot table
// of the stencil damage array (padding slots read slot 0 and are unused).
__global__ void k_sell_slots(long long len, const int32_t *q_of, const int32_t *slot, int32_t *dslot) {
    const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= len) return;
    const int q = q_of[x];
    dslot[x] = q >= 0 ? slot[q] : 0;
}

// Damage history of a slot over an adjoint run (k_grows).
constexpr uint8_t kDmgZero = 0, kDmgGrows = 1, kDmgConst = 2;

// One block per slice of 32 nodes and sample, over all the slice's slots: the
// slice's damage words lie in a few kilobytes of the stencil array (two lanes
// of its nodes' warps), so they are read through L1 once instead of one
// partly used sector per slot from L2. Only slots whose damage grows in the
// run are gathered (code[] per sample and slot); the bond adjoint reads no
// other slot of the trajectory.
__global__ void k_gather_dmg(long long len, long long dlen, const long long *off, const int32_t *dslot,
                             const uint8_t *code, const float *dmg, float *out) {
    const long long a0 = off[blockIdx.x], a1 = off[blockIdx.x + 1];
    const int b = blockIdx.y;
    const float *src = dmg + (size_t)b * dlen;
    const uint8_t *cb = code + (size_t)b * len;
    float *dst = out + (size_t)b * len;
    // four slots per thread (a slice holds 32 W slots and starts on a multiple of 32)
    for (long long x = a0 + 4 * threadIdx.x; x < a1; x += 4 * blockDim.x) {
        const uchar4 c = *(const uchar4 *)(cb + x);
        if (c.x == kDmgGrows) dst[x] = __ldg(src + dslot[x]);
        if (c.y == kDmgGrows) dst[x + 1] = __ldg(src + dslot[x + 1]);
        if (c.z == kDmgGrows) dst[x + 2] = __ldg(src + dslot[x + 2]);
        if (c.w == kDmgGrows) dst[x + 3] = __ldg(src + dslot[x + 3]);
    }
}

// The same from an FP64 CSR-order array (the generic layout's store).
__global__ void k_gather_csr(long long len, long long nb, const int32_t *q_of, const double *csr, float *out) {
    const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= len) return;
    const int b = blockIdx.y;
    const int q = q_of[x];
    out[(size_t)b * len + x] = q >= 0 ? (float)csr[(size_t)b * nb + q] : 0.f;
}

// Damage history code of every slot (sliced-ELL order) over the run:
// kDmgGrows if its damage grows somewhere in the run, else kDmgZero or
// kDmgConst (its damage is the same at every step, zero or not). Damage
// never decreases, so a bond whose final damage equals its initial one never
// changes and is never active: its damage adjoint is never consumed, and its
// damage at any step is its initial value (a padding slot is kDmgZero).
__global__ void k_grows(long long len, long long nb, const int32_t *q_of, const double *d_first,
                        const double *d_last, uint8_t *code) {
    const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= len) return;
    const int b = blockIdx.y;
    const int q = q_of[x];
    uint8_t c = kDmgZero;
    if (q >= 0) {
        const double d0 = d_first[(size_t)b * nb + q], d1 = d_last[(size_t)b * nb + q];
        c = d1 > d0 ? kDmgGrows : (d0 != 0.0 ? kDmgConst : kDmgZero);
    }
    code[(size_t)b * len + x] = c;
}

// s + x accumulated with the rounding error carried in c (Knuth's TwoSum).
__device__ __forceinline__ void fold(float &s, float &c, float x) {
    const float t = s + x;
    const float z = t - s;
    c += (s - (t - z)) + (x - z);
    s = t;
}

// Bond adjoint of one step for mixed-path states: one thread per (sample,
// node), over its sliced-ELL row. Per bond: y = xi + eta, s = eta.(y + xi) /
// (|xi| (|y| + |xi|)), h = s / |y|, dh/dy = y (1/|xi| - s/|y|) / |y|^2 (|y|
// from the approximate reciprocal square root); the damage adjoint carried
// in double-float. The node's terms are summed in FP32 over 8 slots at a
// time and folded into compensated sums (fixed order), then added to the
// FP64 node sums. Capped at 64 registers (32 warps per SM; the kernel waits
// on its gathers): measured on GB300 2.11 against 2.24 ms per adjoint step
// with the compiler's 80.
__global__ void __launch_bounds__(256, 4) k_adj_bonds_f32(const AdjArgs a, long long sl_len,
                                                       const long long *__restrict__ off,
                                                       const int32_t *__restrict__ k_of,
                                                       const float4 *__restrict__ u4,
                                                       const float *__restrict__ dprev,
                                                       const float *__restrict__ dcur,
                                                       const float4 *__restrict__ lF4,
                                                       const uint8_t *__restrict__ dcode,
                                                       const int32_t *__restrict__ q_of,
                                                       const double *__restrict__ d_first, long long nb,
                                                       float2 *__restrict__ ld,
                                                       double *__restrict__ lun, double *__restrict__ g_s0,
                                                       double *__restrict__ g_k) {
    __shared__ float s_L0[64], s_iL0[64];
    if (threadIdx.x < 64) {
        s_L0[threadIdx.x] = a.L0q[threadIdx.x];
        s_iL0[threadIdx.x] = a.iL0q[threadIdx.x];
    }
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (i >= a.N) return;
    const float cV = a.cVf, dxf = a.dxf;
    const float4 *ub = u4 + (size_t)b * a.N;
    const float4 *lb4 = lF4 + (size_t)b * a.N;
    const size_t db = (size_t)b * sl_len;
    const float4 me = ub[i], ml = lb4[i];
    const long long base = off[i >> 5] + (i & 31);
    const int W = (int)((off[(i >> 5) + 1] - off[i >> 5]) >> 5);  // slots of the slice
    float S[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, Cc[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, P[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
    for (int p = 0; p < W; ++p) {
        const long long x = base + 32ll * p;
        const int kp = k_of[x];
        if (kp != -1) {
            const int kx = (int)(signed char)(kp & 0xff), ky = (int)(signed char)((kp >> 8) & 0xff),
                      kz = (int)(signed char)((kp >> 16) & 0xff);
            const int j = (int)i + kx + a.nx * (ky + a.ny * kz);
            const int q2 = kx * kx + ky * ky + kz * kz;
            const float L0 = q2 < 64 ? s_L0[q2] : sqrtf((float)q2) * dxf;
            const float iL0 = q2 < 64 ? s_iL0[q2] : 1.0f / L0;
            const float xi[3] = {(float)kx * dxf, (float)ky * dxf, (float)kz * dxf};
            const float4 nj = ub[j], lj = lb4[j];
            const float eta[3] = {nj.x - me.x, nj.y - me.y, nj.z - me.z};
            const float dl[3] = {lj.x - ml.x, lj.y - ml.y, lj.z - ml.z};
            float y[3], y2 = 0.f, num = 0.f, ydl = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                y[c] = xi[c] + eta[c];
                y2 = fmaf(y[c], y[c], y2);
                num = fmaf(eta[c], y[c] + xi[c], num);
                ydl = fmaf(y[c], dl[c], ydl);
            }
            const float rL = rsqrt_ap(y2);
            const float L = y2 * rL;
            const float s = num * rcp_ap(fmaf(L0, L, L0 * L0));
            const float h = s * rL;
            const float s0 = 0.5f * (me.w + nj.w);
            const float cijV = a.kappa ? cV * 0.5f * (ml.w + lj.w) : cV;
            // damage at this step and the next: from the trajectory for a bond
            // that grows in the run, else its constant value; the damage adjoint
            // of a bond that never grows is never used, so it is neither read
            // nor written (a bond is active only if it grows)
            const uint8_t cd = dcode[db + x];
            const bool gw = cd == kDmgGrows;
            float dp = 0.f, dc = 0.f;
            if (gw) {
                dp = dprev[db + x];
                dc = dcur[db + x];
            } else if (cd == kDmgConst) {
                dp = dc = (float)d_first[(size_t)b * nb + q_of[x]];
            }
            const bool active = dc > dp;
            df lamd = {0.f, 0.f};
            if (gw) {
                const float2 l0 = ld[db + x];
                lamd = df_add(df{l0.x, l0.y}, df{cijV * h * ydl, 0.f});
            }
            float dDds = 0.f, dDds0 = 0.f;
            if (active) law_derivs_f(a, s, s0, dDds, dDds0);
            const float lamdf = lamd.hi + lamd.lo;
            const float om = 1.0f - dc;
            const float dhk = rL * rL * (iL0 - s * rL);
            const float act = active ? lamdf * dDds * rL * iL0 : 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) P[c] += cijV * om * (ydl * dhk * y[c] + h * dl[c]) - act * y[c];
            if (active) P[3] += 0.5f * lamdf * dDds0;
            P[4] += 0.5f * cV * (-om * h * ydl);
            if (gw) ld[db + x] = active ? make_float2(0.f, 0.f) : make_float2(lamd.hi, lamd.lo);
        }
        if ((p & 7) == 7 || p + 1 == W) {
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                fold(S[v], Cc[v], P[v]);
                P[v] = 0.f;
            }
        }
    }
    double *lb = lun + (size_t)b * a.N * 3 + 3 * (size_t)i;
    lb[0] += (double)S[0] + (double)Cc[0];
    lb[1] += (double)S[1] + (double)Cc[1];
    lb[2] += (double)S[2] + (double)Cc[2];
    g_s0[(size_t)b * a.N + i] += (double)S[3] + (double)Cc[3];
    if (g_k) g_k[(size_t)b * a.N + i] += (double)S[4] + (double)Cc[4];
}

// R_obs[b][o] = reaction[b][m] for the observations inside a segment.
__global__ void k_gather_obs(int B, int len, int start, int n_obs, const int32_t *obs, const double *reaction,
                             double *R_obs) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * n_obs) return;
    const int b = t / n_obs, o = t % n_obs;
    const int m = obs[o] - start;
    if (m >= 0 && m < len) R_obs[t] = reaction[(size_t)b * len + m];
}

// ---- chain rule to the KL coefficients

constexpr int kFgNodes = 2048;  // nodes per partial
constexpr int kFgMaxK = 256;

// partial[b][chunk][k] = sum over the chunk's nodes of dJ/dg_i Psi_ik (FP64,
// fixed order: thread t takes nodes t, t + 256, ...; then a fixed tree).
__global__ void __launch_bounds__(256) k_field_grad_partial(long long N, int K, const float *psi, const double *xi,
                                                            const double *dJ_ds0, int marginal, double mu, double sig,
                                                            double wscale, double m_w, int nchunks, double *partial) {
    __shared__ double sxi[kFgMaxK];
    __shared__ double red[256];
    const int b = blockIdx.y, chunk = blockIdx.x;
    for (int k = threadIdx.x; k < K; k += 256) sxi[k] = xi[(size_t)b * K + k];
    __syncthreads();
    const long long i0 = (long long)chunk * kFgNodes;
    const long long i1 = min(N, i0 + kFgNodes);
    // dJ/dg per node for this thread's nodes, then one mode at a time
    double wts[kFgNodes / 256];
#pragma unroll
    for (int r = 0; r < kFgNodes / 256; ++r) {
        const long long i = i0 + threadIdx.x + 256 * r;
        double wg = 0.0;
        if (i < i1) {
            double g = 0.0;
            for (int k = 0; k < K; ++k) g += (double)psi[(size_t)i * K + k] * sxi[k];
            const double dj = dJ_ds0[(size_t)b * N + i];
            if (marginal == PD_MARG_LOGNORMAL) {
                wg = dj * sig * exp(mu + sig * g);
            } else {
                const double q = 0.5 * erfc(g / 1.4142135623730951);
                const double pdf = exp(-0.5 * g * g) / 2.5066282746310002;
                wg = dj * (wscale / m_w) * pow(-log(q), 1.0 / m_w - 1.0) * pdf / q;
            }
        }
        wts[r] = wg;
    }
    for (int k = 0; k < K; ++k) {
        double v = 0.0;
#pragma unroll
        for (int r = 0; r < kFgNodes / 256; ++r) {
            const long long i = i0 + threadIdx.x + 256 * r;
            if (i < i1) v += wts[r] * (double)psi[(size_t)i * K + k];
        }
        red[threadIdx.x] = v;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[((size_t)b * nchunks + chunk) * K + k] = red[0];
        __syncthreads();
    }
}

__global__ void k_field_grad_sum(int B, int K, int nchunks, const double *partial, double *out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * K) return;
    const int b = t / K, k = t % K;
    double v = 0.0;
    for (int c = 0; c < nchunks; ++c) v += partial[((size_t)b * nchunks + c) * K + k];
    out[t] = v;
}

template <class T>
struct DevBuf {
    T *p = nullptr;
    ~DevBuf() { cudaFree(p); }
};

}  // namespace pdi

using namespace pdi;

extern "C" int pd_adjoint(pd_state *st, int32_t n_steps, int32_t ckpt_every, int32_t n_obs, const int32_t *obs_steps,
                          const double *dJ_dR, const float *s0, const float *kappa, double *grad_s0,
                          double *grad_kappa, double *R_obs, pd_stream stream) {
    PD_REQUIRE(st != nullptr, "state is NULL");
    PD_REQUIRE(n_steps >= 1 && ckpt_every >= 1, "n_steps >= 1 and ckpt_every >= 1 required");
    PD_REQUIRE(n_obs >= 0 && (n_obs == 0 || (obs_steps && dJ_dR)), "obs_steps and dJ_dR are required");
    PD_REQUIRE(s0 && grad_s0, "s0 and grad_s0 are required");
    for (int o = 0; o < n_obs; ++o)
        PD_REQUIRE(obs_steps[o] >= 0 && obs_steps[o] < n_steps, "obs_steps[%d] = %d outside [0, %d)", o,
                   obs_steps[o], n_steps);
    cudaStream_t s = (cudaStream_t)stream;
    const int B = st->B;
    const long long N = st->N, nb = st->nb, U3 = (long long)B * N * 3, D1 = (long long)B * nb;
    const int k = std::min(ckpt_every, n_steps);
    const int nseg = (n_steps + k - 1) / k;
    int32_t n0 = 0;
    PD_CHECK_CUDA(cudaStreamSynchronize(s));
    PD_CHECK_CUDA(cudaMemcpy(&n0, st->step + st->bk_par * B, sizeof(int32_t), cudaMemcpyDeviceToHost));

    DevBuf<double> ck_u, ck_v, ck_d, tr_u, tr_d, lu, lun, lv, lF, ld, rbuf;
    // the mixed path's FP32 trajectory: node records (u, s0) per step, damage
    // in CSR order per step (+ the last), (lamF, kappa) per node, the damage
    // adjoint in double-float, and the CSR slot of every bond in the state's
    // stencil damage array
    DevBuf<float4> tr_u4, lF4;
    DevBuf<float> tr_d32;
    DevBuf<float2> ld2;
    DevBuf<int32_t> slot, q_of, k_of, dslot;
    DevBuf<long long> sl_off;
    DevBuf<uint8_t> grow8;  // mixed path: per sample and slot, the damage history code (k_grows)
    long long nsl = 0;  // slices of 32 nodes (mixed path)
    long long SL = 0;  // sliced-ELL slots per sample
    const bool f32 = st->mat.precision == PD_PREC_MIXED;
    const long long BN = (long long)B * N;
    DevBuf<int32_t> obs;
    PD_TRY(dalloc(&ck_u.p, (size_t)(nseg + 1) * U3));  // checkpoints + the final state
    PD_TRY(dalloc(&ck_v.p, (size_t)(nseg + 1) * U3));
    PD_TRY(dalloc(&ck_d.p, (size_t)(nseg + 1) * D1));
    PD_TRY(dalloc(&lu.p, U3));
    PD_TRY(dalloc(&lun.p, U3));
    PD_TRY(dalloc(&lv.p, U3));
    PD_TRY(dalloc(&lF.p, U3));
    PD_TRY(dalloc(&rbuf.p, (size_t)B * k));
    if (f32) {
        PD_REQUIRE(st->g.m_ratio < 127.0, "the mixed-path adjoint packs bond offsets in bytes: horizon below 127 cells");
        // sliced ELL of the CSR rows (slice widths on the host)
        std::vector<int32_t> hrow(N + 1);
        PD_CHECK_CUDA(cudaMemcpy(hrow.data(), st->row_ptr, (N + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
        nsl = (N + 31) / 32;
        std::vector<long long> hoff(nsl + 1, 0);
        for (long long sl = 0; sl < nsl; ++sl) {
            int w = 0;
            for (long long i = 32 * sl; i < std::min(N, 32 * sl + 32); ++i) w = std::max(w, hrow[i + 1] - hrow[i]);
            hoff[sl + 1] = hoff[sl] + 32ll * w;
        }
        SL = std::max(hoff[nsl], 1ll);
        PD_TRY(dalloc(&sl_off.p, nsl + 1));
        PD_CHECK_CUDA(cudaMemcpy(sl_off.p, hoff.data(), (nsl + 1) * sizeof(long long), cudaMemcpyHostToDevice));
        PD_TRY(dalloc(&q_of.p, SL));
        PD_TRY(dalloc(&k_of.p, SL));
        PD_CHECK_CUDA(cudaMemsetAsync(q_of.p, 0xff, SL * sizeof(int32_t), s));
        PD_CHECK_CUDA(cudaMemsetAsync(k_of.p, 0xff, SL * sizeof(int32_t), s));
        k_sell_fill<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(N, st->row_ptr, st->col_csr, st->coord, sl_off.p,
                                                                q_of.p, k_of.p);
        PD_CHECK_LAUNCH();
        PD_TRY(dalloc(&tr_u4.p, (size_t)k * BN));
        PD_TRY(dalloc(&tr_d32.p, (size_t)(k + 1) * B * SL));
        PD_TRY(dalloc(&lF4.p, BN));
        PD_TRY(dalloc(&ld2.p, (size_t)B * SL));
        PD_TRY(dalloc(&grow8.p, (size_t)B * SL));
        if (st->stencil) {
            PD_TRY(dalloc(&slot.p, nb));
            PD_TRY(stencil_slot_table(st, slot.p, s));
            PD_TRY(dalloc(&dslot.p, SL));
            k_sell_slots<<<(unsigned)((SL + 255) / 256), 256, 0, s>>>(SL, q_of.p, slot.p, dslot.p);
            PD_CHECK_LAUNCH();
        } else {
            PD_TRY(dalloc(&tr_d.p, D1));  // staging for the generic layout's FP64 store
        }
    } else {
        PD_TRY(dalloc(&tr_u.p, (size_t)k * U3));
        PD_TRY(dalloc(&tr_d.p, (size_t)(k + 1) * D1));
        PD_TRY(dalloc(&ld.p, D1));
    }
    PD_TRY(dalloc(&obs.p, std::max(n_obs, 1)));
    if (n_obs) PD_CHECK_CUDA(cudaMemcpyAsync(obs.p, obs_steps, n_obs * sizeof(int32_t), cudaMemcpyHostToDevice, s));

    // forward with checkpoints (the first load clears run bookkeeping, e.g. done flags)
    for (int g = 0; g < nseg; ++g) {
        const int start = g * k, len = std::min(k, n_steps - start);
        PD_TRY(pd_state_store(st, ck_u.p + (size_t)g * U3, ck_v.p + (size_t)g * U3, ck_d.p + (size_t)g * D1, stream));
        if (g == 0) PD_TRY(pd_state_load(st, ck_u.p, ck_v.p, ck_d.p, n0, stream));
        PD_TRY(pd_step(st, len, rbuf.p, stream));
        if (R_obs && n_obs) {
            k_gather_obs<<<(B * n_obs + 255) / 256, 256, 0, s>>>(B, len, start, n_obs, obs.p, rbuf.p, R_obs);
            PD_CHECK_LAUNCH();
        }
    }
    PD_TRY(pd_state_store(st, ck_u.p + (size_t)nseg * U3, ck_v.p + (size_t)nseg * U3, ck_d.p + (size_t)nseg * D1,
                          stream));
    if (f32) {
        k_grows<<<dim3((unsigned)((SL + 255) / 256), (unsigned)B), 256, 0, s>>>(SL, nb, q_of.p, ck_d.p,
                                                                             ck_d.p + (size_t)nseg * D1, grow8.p);
        PD_CHECK_LAUNCH();
    }

    AdjArgs a;
    a.B = B;
    a.N = N;
    a.nb = nb;
    a.nx = st->g.nx;
    a.ny = st->g.ny;
    a.dx = st->g.dx;
    a.c = st->c;
    a.V = st->V;
    a.dt = st->dt;
    a.rho = st->mat.rho;
    a.a = 1.0 - 0.5 * st->mat.zeta * st->dt;
    a.b = 1.0 + 0.5 * st->mat.zeta * st->dt;
    a.dt_rb = a.dt / (a.rho * a.b);
    a.a_b = a.a / a.b;
    a.law = st->mat.law;
    a.s_ratio = st->mat.s_ratio;
    a.k = st->mat.k;
    a.alpha = st->mat.alpha;
    a.gfA = st->gfA;
    a.row_ptr = st->row_ptr;
    a.col = st->col_csr;
    a.codes = st->codes;
    a.s0 = s0;
    a.kappa = kappa;
    a.n_obs = n_obs;
    a.obs = obs.p;
    a.w = dJ_dR;
    a.coord = st->coord;
    a.cVf = (float)(st->c * st->V);
    a.dxf = (float)st->g.dx;
    a.s_ratio_f = (float)st->mat.s_ratio;
    a.gfA_f = (float)st->gfA;
    a.k_f = (float)st->mat.k;
    a.alpha_f = (float)st->mat.alpha;
    for (int q = 0; q < 64; ++q) {
        const double L0 = std::sqrt((double)q) * st->g.dx;
        a.L0q[q] = (float)L0;
        a.iL0q[q] = q ? (float)(1.0 / L0) : 0.f;
    }
    PD_CHECK_CUDA(cudaMemsetAsync(lu.p, 0, U3 * sizeof(double), s));
    PD_CHECK_CUDA(cudaMemsetAsync(lv.p, 0, U3 * sizeof(double), s));
    if (f32)
        PD_CHECK_CUDA(cudaMemsetAsync(ld2.p, 0, (size_t)B * SL * sizeof(float2), s));
    else
        PD_CHECK_CUDA(cudaMemsetAsync(ld.p, 0, D1 * sizeof(double), s));
    PD_CHECK_CUDA(cudaMemsetAsync(grad_s0, 0, (size_t)B * N * sizeof(double), s));
    if (grad_kappa) PD_CHECK_CUDA(cudaMemsetAsync(grad_kappa, 0, (size_t)B * N * sizeof(double), s));
    const unsigned nblk_bond = (unsigned)(((long long)B * N * 32 + 255) / 256);
    const unsigned nblk_node = (unsigned)((BN + 255) / 256);
    PD_REQUIRE(B <= 65535, "at most 65535 samples per state");
    const dim3 grid_sl((unsigned)((SL + 255) / 256), (unsigned)B);
    const dim3 grid_nodes((unsigned)((N + 255) / 256), (unsigned)B);
    const dim3 grid_dof((unsigned)((3 * N + 255) / 256), (unsigned)B);
    // FP32 trajectory of the mixed path at the state's current step n: the
    // gather records of parity n and the damage in CSR order
    auto snap_f32 = [&](int n, float4 *u4, float *d32) -> int {
        if (u4) {
            k_rec_to_u4<<<nblk_node, 256, 0, s>>>(BN, (const float4 *)st->rec[n & 1], u4);
            PD_CHECK_LAUNCH();
        }
        if (st->stencil) {
            k_gather_dmg<<<dim3((unsigned)nsl, (unsigned)B), 256, 0, s>>>(SL, st->st_len, sl_off.p, dslot.p,
                                                                          grow8.p, (const float *)st->dmg, d32);
        } else {
            PD_TRY(pd_state_store(st, nullptr, nullptr, tr_d.p, stream));
            k_gather_csr<<<grid_sl, 256, 0, s>>>(SL, nb, q_of.p, tr_d.p, d32);
        }
        PD_CHECK_LAUNCH();
        return PD_OK;
    };
    double *plu = lu.p, *plun = lun.p;
    for (int g = nseg - 1; g >= 0; --g) {
        const int start = g * k, len = std::min(k, n_steps - start);
        PD_TRY(pd_state_load(st, ck_u.p + (size_t)g * U3, ck_v.p + (size_t)g * U3, ck_d.p + (size_t)g * D1,
                             n0 + start, stream));
        for (int m = 0; m < len; ++m) {
            if (f32)
                PD_TRY(snap_f32(n0 + start + m, tr_u4.p + (size_t)m * BN, tr_d32.p + (size_t)m * B * SL));
            else
                PD_TRY(pd_state_store(st, tr_u.p + (size_t)m * U3, nullptr, tr_d.p + (size_t)m * D1, stream));
            PD_TRY(pd_step(st, 1, nullptr, stream));
        }
        if (f32)
            PD_TRY(snap_f32(n0 + start + len, nullptr, tr_d32.p + (size_t)len * B * SL));
        else
            PD_TRY(pd_state_store(st, nullptr, nullptr, tr_d.p + (size_t)len * D1, stream));
        for (int m = len - 1; m >= 0; --m) {
            k_adj_nodes<<<grid_dof, 256, 0, s>>>(a, start + m, plu, lv.p, lF.p, plun);
            PD_CHECK_LAUNCH();
            if (f32) {
                k_lF_to_f4<<<nblk_node, 256, 0, s>>>(BN, lF.p, kappa, lF4.p);
                PD_CHECK_LAUNCH();
                k_adj_bonds_f32<<<grid_nodes, 256, 0, s>>>(a, SL, sl_off.p, k_of.p, tr_u4.p + (size_t)m * BN,
                                                           tr_d32.p + (size_t)m * B * SL,
                                                           tr_d32.p + (size_t)(m + 1) * B * SL, lF4.p, grow8.p,
                                                           q_of.p, ck_d.p, nb, ld2.p, plun, grad_s0, grad_kappa);
            } else {
                k_adj_bonds<<<nblk_bond, 256, 0, s>>>(a, tr_u.p + (size_t)m * U3, tr_d.p + (size_t)m * D1,
                                                      tr_d.p + (size_t)(m + 1) * D1, lF.p, ld.p, plun, grad_s0,
                                                      grad_kappa);
            }
            PD_CHECK_LAUNCH();
            std::swap(plu, plun);
        }
    }
    // leave the state where the forward run left it
    PD_TRY(pd_state_load(st, ck_u.p + (size_t)nseg * U3, ck_v.p + (size_t)nseg * U3, ck_d.p + (size_t)nseg * D1,
                         n0 + n_steps, stream));
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("adjoint failed: %s", cudaGetErrorString(cudaGetLastError()));
        return PD_ERR_CUDA;
    }
    return PD_OK;
}

// The field's basis and marginal parameters live in pd_field.cu.
int field_grad_inputs(const pd_field *f, int level, const float **psi, long long *N, int *K, int *marginal,
                      double *mu, double *sig, double *wscale, double *m_w);

extern "C" int pd_field_adjoint(const pd_field *f, int32_t level, const double *xi, int32_t B, const double *dJ_ds0,
                                double *dJ_dxi, pd_stream stream) {
    PD_REQUIRE(f && xi && dJ_ds0 && dJ_dxi, "field, xi, dJ_ds0 and dJ_dxi are required");
    PD_REQUIRE(B >= 0, "B must be >= 0");
    if (B == 0) return PD_OK;
    const float *psi;
    long long N;
    int K, marginal;
    double mu, sig, wscale, m_w;
    PD_TRY(field_grad_inputs(f, level, &psi, &N, &K, &marginal, &mu, &sig, &wscale, &m_w));
    PD_REQUIRE(K <= kFgMaxK, "n_modes above %d", kFgMaxK);
    cudaStream_t s = (cudaStream_t)stream;
    const int nchunks = (int)((N + kFgNodes - 1) / kFgNodes);
    DevBuf<double> part;
    PD_TRY(dalloc(&part.p, (size_t)B * nchunks * K));
    k_field_grad_partial<<<dim3(nchunks, B), 256, 0, s>>>(N, K, psi, xi, dJ_ds0, marginal, mu, sig, wscale, m_w,
                                                          nchunks, part.p);
    PD_CHECK_LAUNCH();
    k_field_grad_sum<<<(B * K + 255) / 256, 256, 0, s>>>(B, K, nchunks, part.p, dJ_dxi);
    PD_CHECK_LAUNCH();
    PD_CHECK_CUDA(cudaStreamSynchronize(s));  // the partials are freed on return
    return PD_OK;
}
