// pd_stencil.cu -- host side of the compile-time stencil step (the 122-offset
// horizon |k|^2 <= 9 of m in [3, sqrt(10)), and the 28-offset planar horizon
// of one-layer grids): the damage-slot layout and its maps to and from CSR
// order, the gather records, launch configuration and dispatch. The kernel
// itself is in pd_stencil_kernel.cuh.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <utility>
#include <vector>

#include "pd_stencil_kernel.cuh"

namespace pdi {

namespace {

// Slot of node i, stencil code (2 m + t), in the per-sample damage array:
// [brick][warp][quad m / 4][lane][m % 4].
__device__ __forceinline__ long long slot_of(int i, int code, int nx, int ny, int BY, int BZ, int nbx, int nby,
                                             int wpb, int rounds) {
    const int ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
    const long long brick = (ix / kSlice) + (long long)nbx * ((iy / BY) + (long long)nby * (iz / BZ));
    const int row = (iy % BY) + BY * (iz % BZ);
    const int w = row >> 1, rr = row & 1, c = ix % kSlice;
    const int m = code >> 1, t = code & 1;
    return (((brick * wpb + w) * (rounds / 4) + m / 4) * 32 + (16 * t + 8 * rr + c)) * 4 + (m % 4);
}

// Gather records of both parities from the state's double-float records:
// (u / dx rounded to FP32, s0 / 2), and the same point-reflected (node i of a
// sample at N - 1 - i).
__global__ void k_stencil_grec(long long N, long long NB, const float4 *rec0, const float4 *rec1, df idx, float4 *g0,
                               float4 *g1, float4 *r0, float4 *r1) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= NB) return;
    const long long b = t / N, i = t - b * N;
    for (int p = 0; p < 2; ++p) {
        const float4 *rc = p ? rec1 : rec0;
        const float4 h = rc[t], l = rc[NB + t];
        const float4 o = make_float4(df_mul(df{h.x, l.x}, idx).hi, df_mul(df{h.y, l.y}, idx).hi,
                                     df_mul(df{h.z, l.z}, idx).hi, 0.5f * h.w);
        (p ? g1 : g0)[t] = o;
        (p ? r1 : r0)[b * N + (N - 1 - i)] = o;
    }
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

// Damage between CSR order (FP64) and the stencil layout. Loading (TO_STATE)
// also sets the damage flags of the node's two lanes: a group of 8 rounds
// whose loaded damage is not all zero (the template value of a present bond)
// is marked, in the byte of the part of the half-stencil that owns it (q
// parts; byte part of the lane's word, bit group - first group of the part).
// A node's bonds lie in its own two lanes only, so each word has one writer.
template <bool TO_STATE>
__global__ void k_stencil_map(const int32_t *row_ptr, const int32_t *col, const int32_t *coord, long long N, int B,
                              long long nb, int nx, int ny, int BY, int BZ, int nbx, int nby, int wpb, int rounds,
                              long long len, const int16_t *box, float *dmg, double *csr, uint32_t *dirty,
                              int q) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * B) return;
    const int b = (int)(t / N);
    const int i = (int)(t % N);
    const int gpp = rounds / 8 / q;  // groups of 8 rounds per part
    uint32_t w[2] = {0u, 0u};        // flags of sub-lanes 0 and 1
    for (int p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
        const int code = code_of(coord, i, col[p], box);
        if (code < 0) continue;
        const long long e = (long long)b * len + slot_of(i, code, nx, ny, BY, BZ, nbx, nby, wpb, rounds);
        const long long qq = (long long)b * nb + p;
        if (TO_STATE) {
            const float d = (float)csr[qq];
            dmg[e] = d;
            if (d != 0.0f) {
                const int g = (code >> 1) / 8, part = g / gpp;
                w[code & 1] |= 1u << (8 * part + (g - part * gpp));
            }
        } else {
            csr[qq] = (double)dmg[e];
        }
    }
    if (TO_STATE) {
        const int ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
        const long long brick = (ix / kSlice) + (long long)nbx * ((iy / BY) + (long long)nby * (iz / BZ));
        const int row = (iy % BY) + BY * (iz % BZ);
        const long long lane0 = (brick * wpb + (row >> 1)) * 32 + 8 * (row & 1) + (ix % kSlice);
        const long long per_sample = len / rounds;  // lanes of a sample
        dirty[(size_t)b * per_sample + lane0] = w[0];
        dirty[(size_t)b * per_sample + lane0 + 16] = w[1];
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

StencilPairFn pick_pair(int dim, int q, int law, bool kappa) {
    if (dim == 2) return stencil_pair_d2(law, kappa);
    if (q == 4) return stencil_pair_d3q4(law, kappa);
    if (q == 2) return stencil_pair_d3q2(law, kappa);
    return stencil_pair_d3q1(law, kappa);
}

// The step kernel variant of a launch (force-only evaluations take the
// one-sample kernel).
StencilKernel pick_stencil(int dim, int ns, int q, int law, bool kappa, bool fo) {
    if (dim == 2) return stencil_pick_d2(ns, law, kappa, fo);  // 16 rounds: two groups of 8 at Q = 1 only
    if (q == 4) return stencil_pick_d3q4(ns, law, kappa, fo);
    if (q == 2) return stencil_pick_d3q2(ns, law, kappa, fo);
    return stencil_pick_d3q1(ns, law, kappa, fo);
}

unsigned blocks_of(long long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

// Dynamic shared memory of a launch: the upper and the reflected lower copy
// of the staged records (BZ + halo layers each), the same for kappa when a
// stiffness field is set, and the partial sums of Q > 1 parts.
// Dynamic shared memory of a launch: the two record copies, each rounded up to
// 128 bytes (TMA destinations), the kappa copies, the parts' partial sums,
// and 128 bytes to align the box.
size_t stencil_smem(const pd_state *st, int ns, bool kappa) {
    const int hz = st->st_dim == 3 ? Sten<3>::kHaloZ : Sten<2>::kHaloZ;
    const size_t rows = (size_t)(st->by + 2 * kHalo) * (st->bz + hz);
    size_t b = 2 * ((rows * ns * kRowC + 127) & ~(size_t)127) + 128;
    if (kappa) b += 2 * rows * ns * kRowK;
    return b + (size_t)(st->st_q - 1) * st->st_wpb * 16 * 6 * ns * sizeof(float);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn tiled_encoder() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// Map of a [B][nz][ny][nx] array of 4-float records, read in boxes of 14 cells
// x Wy rows x Zp layers of one sample; cells outside the grid read as zero.
static int encode_box_map(CUtensorMap *tm, float4 *base, const pd_state *st, int Wy, int Zp) {
    EncodeTiledFn enc = tiled_encoder();
    PD_REQUIRE(enc != nullptr, "cuTensorMapEncodeTiled is unavailable");
    const cuuint64_t nx = (cuuint64_t)st->g.nx, ny = (cuuint64_t)st->g.ny, nz = (cuuint64_t)st->g.nz;
    const cuuint64_t dims[5] = {4, nx, ny, nz, (cuuint64_t)st->B};
    const cuuint64_t strides[4] = {16, 16 * nx, 16 * nx * ny, 16 * nx * ny * nz};
    const cuuint32_t box[5] = {4, (cuuint32_t)kWx, (cuuint32_t)Wy, (cuuint32_t)Zp, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, base, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    PD_REQUIRE(r == CUDA_SUCCESS, "cuTensorMapEncodeTiled failed for the stencil box (%d)", (int)r);
    return PD_OK;
}

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
    for (int dim = 2; dim <= 3; ++dim)
        for (int q = 1; q <= 4; q *= 2)
            for (int law = 0; law < 2; ++law)
                for (int kap = 0; kap < 2; ++kap)
                    PD_CHECK_CUDA(cudaFuncSetAttribute((const void *)pick_pair(dim, q, law, kap),
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (dev >= 0 && dev < 64) limit[dev] = smem;
    return PD_OK;
}

int stencil_build(pd_state *st, const int32_t *col) {
    const long long N = st->N;
    st->st_wpb = st->by * st->bz / 2;
    st->st_dim = st->g.nz == 1 ? 2 : 3;  // a one-layer grid has only the planar offsets
    const int rounds = st->st_dim == 3 ? Sten<3>::kRounds : Sten<2>::kRounds;
    st->st_len = st->n_bricks * st->st_wpb * (long long)rounds * 32;
    // samples per block: one (measured on GB300, a pair per block is slower at
    // 122 registers a thread, 16 warps per SM); pairs on request
    st->st_ns = st->ns_req ? st->ns_req : 1;
    // split the half-stencil over Q warps when the mesh gives too few warps per SM
    // (measured on GB300: Q = 2 for single samples of the 28k-node beam, 1 for batches)
    const long long warps1 = st->n_bricks * ((st->B + st->st_ns - 1) / st->st_ns) * st->st_wpb;
    st->st_q = warps1 >= 152ll * 24 ? 1 : 2;
    if (st->q_req) st->st_q = st->q_req;
    if (st->st_dim == 2) st->st_q = 1;
    // threads a block: at most 512, or 256 for one sample at Q = 2 (its register budget)
    while (st->st_q > 1 && 32 * st->st_wpb * st->st_q > (st->st_q == 2 && st->st_ns == 1 ? 256 : 512)) st->st_q /= 2;
    // Deferring the reaction to the next launch pays when a launch is a
    // single wave of a few blocks per SM, whose reduction tail would
    // otherwise stand alone at the end (measured on GB300: 28k-node beam,
    // one sample, 19.3 -> 18 us per step); with many waves the tail overlaps
    // other blocks and the deferred read only adds to each block's start.
    {
        int dev = 0, sms = 0;
        PD_CHECK_CUDA(cudaGetDevice(&dev));
        PD_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        st->st_one_wave = st->n_bricks * ((st->B + st->st_ns - 1) / st->st_ns) <= 4ll * sms;
        st->st_defer = st->st_one_wave;
        if (st->reduce_req) st->st_defer = st->reduce_req == 2;
    }
    // the largest launch of this state (kappa staged; force-only evaluations
    // take the one-sample kernel, which needs no more)
    st->smem_bytes = stencil_smem(st, st->st_ns, true);
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
    PD_TRY(dalloc(&st->st_dirty, (size_t)st->B * (st->st_len / rounds) * 4));
    PD_CHECK_CUDA(cudaMemset(st->st_dirty, 0, (size_t)st->B * (st->st_len / rounds) * 4));
    PD_TRY(dalloc(&st->grec[0], (size_t)st->B * N));
    PD_TRY(dalloc(&st->grec[1], (size_t)st->B * N));
    PD_TRY(dalloc(&st->grecR[0], (size_t)st->B * N));
    PD_TRY(dalloc(&st->grecR[1], (size_t)st->B * N));
    {
        const int Wy = st->by + 2 * kHalo;
        const int Zp = st->bz + (st->st_dim == 3 ? Sten<3>::kHaloZ : Sten<2>::kHaloZ);
        for (int p = 0; p < 2; ++p) {
            PD_TRY(encode_box_map(&st->st_maps.rec[p], st->grec[p], st, Wy, Zp));
            PD_TRY(encode_box_map(&st->st_maps.ref[p], st->grecR[p], st, Wy, Zp));
        }
    }
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

int stencil_refresh_grec(pd_state *st, cudaStream_t s) {
    const long long NB = st->N * st->B;
    k_stencil_grec<<<blocks_of(NB), 256, 0, s>>>(st->N, NB, (const float4 *)st->rec[0], (const float4 *)st->rec[1],
                                                 df_split(1.0 / st->g.dx), st->grec[0], st->grec[1], st->grecR[0],
                                                 st->grecR[1]);
    PD_CHECK_LAUNCH();
    return PD_OK;
}

void stencil_fill_args(const pd_state *st, StepArgs &a) {
    a.grec0 = st->grec[0];
    a.grec1 = st->grec[1];
    a.grecR0 = st->grecR[0];
    a.grecR1 = st->grecR[1];
    a.idx_df = df_split(1.0 / st->g.dx);
    a.tmpl = st->st_tmpl;
    a.dirty = st->st_dirty;
    a.fd_grp1 = fastdiv_make(st->B);
    a.fd_grp2 = fastdiv_make((st->B + 1) / 2);
    a.fd_nbx = fastdiv_make(st->nbx);
    a.fd_nby = fastdiv_make(st->nby);
    a.fd_by = fastdiv_make(st->by);
}

int stencil_reset_damage(pd_state *st, cudaStream_t s) {
    k_stencil_reset<<<blocks_of(st->st_len * st->B), 256, 0, s>>>(st->st_len, st->B, st->st_tmpl, (float *)st->dmg);
    PD_CHECK_LAUNCH();
    // every group equals the template again
    const int rounds = st->st_dim == 3 ? Sten<3>::kRounds : Sten<2>::kRounds;
    PD_CHECK_CUDA(cudaMemsetAsync(st->st_dirty, 0, (size_t)st->B * (st->st_len / rounds) * 4, s));
    return PD_OK;
}

int stencil_map_damage(const pd_state *st, double *csr, bool to_state, cudaStream_t s) {
    const long long NB = st->N * st->B;
    const int rounds = st->st_dim == 3 ? Sten<3>::kRounds : Sten<2>::kRounds;
    if (to_state)  // loaded damage, with the damage flags of every node's lanes
        k_stencil_map<true><<<blocks_of(NB), 256, 0, s>>>(st->row_ptr, st->col_csr, st->coord, st->N, st->B, st->nb,
                                                          st->g.nx, st->g.ny, st->by, st->bz, st->nbx, st->nby,
                                                          st->st_wpb, rounds, st->st_len, st->st_box, (float *)st->dmg,
                                                          csr, (uint32_t *)st->st_dirty, st->st_q);
    else
        k_stencil_map<false><<<blocks_of(NB), 256, 0, s>>>(st->row_ptr, st->col_csr, st->coord, st->N, st->B, st->nb,
                                                           st->g.nx, st->g.ny, st->by, st->bz, st->nbx, st->nby,
                                                           st->st_wpb, rounds, st->st_len, st->st_box, (float *)st->dmg,
                                                           csr, nullptr, st->st_q);
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

bool stencil_pairable(const pd_state *s0, const pd_state *s1) {
    return s0->stencil && s1->stencil && s0->st_ns == 1 && s1->st_ns == 1 && s0->st_dim == s1->st_dim &&
           s0->st_q == s1->st_q && s0->st_wpb == s1->st_wpb && s0->mat.law == s1->mat.law &&
           s0->has_kappa == s1->has_kappa;
}

// A step launch of many waves may start while the previous kernel in the
// stream is finishing (programmatic dependent launch): the kernel waits for it
// (griddepcontrol.wait) before it reads anything, so only the launch and the
// scheduling of its blocks overlap the previous step's tail. Single-wave
// launches (one sample of a small mesh) are launched plainly: there the
// steps without softening gain (28k-node beam, one sample, GB300: 12.4 ->
// 10.8 us) but the steps with a growing crack lose more, and whole runs to
// the peak were slower (14.07 against 14.00 us per step).
static cudaLaunchConfig_t pdl_config(unsigned grid, int threads, size_t smem, cudaStream_t s, bool pdl) {
    static const cudaLaunchAttribute attr = [] {
        cudaLaunchAttribute x{};
        x.id = cudaLaunchAttributeProgrammaticStreamSerialization;
        x.val.programmaticStreamSerializationAllowed = 1;
        return x;
    }();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = const_cast<cudaLaunchAttribute *>(&attr);
    cfg.numAttrs = pdl ? 1 : 0;
    return cfg;
}

int stencil_launch_pair(const pd_state *s0, const StepArgs &a0, const pd_state *s1, const StepArgs &a1,
                        cudaStream_t s) {
    PD_REQUIRE(stencil_pairable(s0, s1), "the two states do not share a launch shape");
    StepPair g;
    g.a[0] = a0;
    g.a[1] = a1;
    g.nblk0 = (int)s0->n_bricks * s0->B;
    g.t[0] = s0->st_maps;
    g.t[1] = s1->st_maps;
    const unsigned grid = (unsigned)g.nblk0 + (unsigned)s1->n_bricks * (unsigned)s1->B;
    const size_t smem = std::max(stencil_smem(s0, 1, s0->has_kappa), stencil_smem(s1, 1, s1->has_kappa));
    cudaLaunchConfig_t cfg = pdl_config(grid, 32 * s0->st_wpb * s0->st_q, smem, s, !s0->st_one_wave || !s1->st_one_wave);
    PD_CHECK_CUDA(cudaLaunchKernelEx(&cfg, pick_pair(s0->st_dim, s0->st_q, s0->mat.law, s0->has_kappa), g));
    return PD_OK;
}

int stencil_launch(const pd_state *st, const StepArgs &a, bool force_only, cudaStream_t s) {
    const int ns = force_only ? 1 : st->st_ns;
    StencilKernel k = pick_stencil(st->st_dim, ns, st->st_q, st->mat.law, st->has_kappa, force_only);
    const unsigned grid = (unsigned)st->n_bricks * (unsigned)((st->B + ns - 1) / ns);
    cudaLaunchConfig_t cfg =
        pdl_config(grid, 32 * st->st_wpb * st->st_q, stencil_smem(st, ns, st->has_kappa), s, !st->st_one_wave);
    PD_CHECK_CUDA(cudaLaunchKernelEx(&cfg, k, a, st->st_maps));
    return PD_OK;
}

}  // namespace pdi
