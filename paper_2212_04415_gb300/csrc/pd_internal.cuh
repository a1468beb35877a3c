// pd_internal.cuh -- shared internals of the GB300 peridynamic library
// (error plumbing, small device helpers, the state layout).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/pd.h"

namespace pdi {

// Record the last error text for pd_last_error (thread-local).
void set_error(const char *fmt, ...);

#define PD_CHECK_CUDA(call)                                                           \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            pdi::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,                 \
                           cudaGetErrorString(e_));                                   \
            return PD_ERR_CUDA;                                                       \
        }                                                                             \
    } while (0)

#define PD_CHECK_LAUNCH() PD_CHECK_CUDA(cudaGetLastError())

#define PD_REQUIRE(cond, ...)                                                         \
    do {                                                                              \
        if (!(cond)) {                                                                \
            pdi::set_error(__VA_ARGS__);                                              \
            return PD_ERR_ARG;                                                        \
        }                                                                             \
    } while (0)

// Device allocation that reports PD_ERR_OOM through the caller.
template <typename T>
int dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
        *p = nullptr;
        return PD_ERR_OOM;
    }
    return PD_OK;
}

#define PD_TRY(expr)                \
    do {                            \
        int rc_ = (expr);           \
        if (rc_ != PD_OK) return rc_; \
    } while (0)

int validate_grid(const pd_grid *g);

// Exclusive-free inclusive scan of a[1..n] in place (a[0] untouched), int32
// with an int64 running sum; sets *overflow if the total exceeds INT32_MAX.
int scan_inplace_i32(int32_t *a, int64_t n, int32_t *overflow_flag_dev, cudaStream_t s);

// Packed grid coordinate of a node: ix | iy << 11 | iz << 22.
__host__ __device__ __forceinline__ int32_t pack_coord(int ix, int iy, int iz) {
    return ix | (iy << 11) | (iz << 22);
}

}  // namespace pdi

// Opaque handles (definitions shared between translation units).
// Tensor maps (TMA) of the stencil step's staged box, by step parity: the
// gather records [B][nz][ny][nx] x 4 floats and their point-reflected copy,
// in boxes of 4 x 14 x (by + 6) x (bz + z-halo) floats.
struct StencilMaps {
    CUtensorMap rec[2];
    CUtensorMap ref[2];
};

struct pd_state {
    pd_grid g;
    pd_material mat;
    pd_bc bc;
    int32_t B;
    int64_t N;
    int64_t nb;
    double dt, c, V;
    double gfA;             // > 0: s_crit = s0 + gfA / s0 (fracture-energy calibration)
    // neighbour list: CSR copy and a brick-ordered SELL-8 layout of stencil ids
    int32_t *row_ptr;
    int32_t by, bz;         // brick = 8 x by x bz nodes; one slice = 8 x-consecutive nodes
    int32_t nbx, nby, nbz;  // bricks per axis
    int32_t halo;           // largest stencil offset component
    int64_t n_bricks;
    int64_t n_slices;       // n_bricks * by * bz (rows outside the grid are empty slices)
    int64_t sell_len;
    long long *sell_off;    // [n_slices]: first element of each slice
    int32_t *sell_m;        // [n_slices]: 32-wide rounds per slice (slots / 4)
    int32_t *slice_i0;      // [n_slices]: node of lane 0
    int32_t *slice_nv;      // [n_slices]: valid lanes (0..8)
    uint8_t *ids;           // [sell_len]: stencil id of each slot, 0xFF = padding
    int32_t n_off;          // stencil size
    float4 *xi_tab;         // [256]: xi (x, y, z) and |xi| in FP32
    double4_32a *xid_tab;   // [256]: the same in FP64
    int32_t *off_tab;       // [256]: neighbour offset (fp64 path: global j - i; mixed: brick-local)
    size_t smem_bytes;      // staged brick records (mixed path)
    // compile-time 122-offset stencil path (mixed precision, m in [3, sqrt(10)))
    bool stencil;
    int32_t st_wpb;         // row pairs per brick (2 brick rows per warp)
    int32_t st_q;           // warps sharing a row pair (parts of the half-stencil)
    int32_t q_req;          // requested st_q (schedule), 0 = built-in choice
    int32_t st_dim;         // 3, or 2 for a one-layer grid (planar 28-offset stencil)
    int32_t st_ns;          // samples per block (1, or 2 on the paired FP32 instructions)
    int32_t st_defer;       // launches may leave their reaction to the next launch (few blocks per SM)
    int32_t st_one_wave;    // a launch is a single wave of at most 4 blocks per SM
    int32_t ns_req;         // requested st_ns (schedule), 0 = built-in choice
    int32_t reduce_req;     // requested reaction reduction (schedule): 0 built-in, 1 own launch, 2 deferred
    int64_t st_len;         // damage slots per sample
    float *st_tmpl;         // [st_len]: 0 for real bonds, 1 for absent (broken) slots
    uint8_t *st_dirty;      // [B][bricks][wpb][32 lanes][4 parts]: 8-round groups whose damage differs from st_tmpl
    float4 *grec[2];        // gather records by step parity, [B][N]: (u / dx rounded to FP32, s0 / 2)
    float4 *grecR[2];       // the same point-reflected: node i of a sample at N - 1 - i
    StencilMaps st_maps;    // TMA maps of the staged box over grec and grecR
    int16_t *st_box;        // [7^3]: stencil code 2 m + t of an offset, -1 outside
    int32_t *col_csr;       // CSR copy for damage load/store
    // per-sample state
    void *dmg;          // float or double [B][sell_len]
    double *u64;        // fp64 path: [B][N][3]
    double *v64;        // fp64 path: [B][N][3]
    float4 *vdf;        // mixed path: v as double-float, float4 hi[B][N] then float4 lo[B][N]
    void *rec[2];       // gather records, double-buffered by step parity:
                        // mixed: float4 hi[B][N] then float4 lo[B][N]; fp64: double4_32a [B][N]
    float *kappa;       // [B][N] or nullptr
    bool has_kappa;
    uint8_t *codes;     // [N][3]
    int32_t *coord;     // [N] packed grid coordinates
    // run bookkeeping (device)
    int32_t *step;      // [2][B], double-buffered by launch parity
    int32_t *done;      // [2][B]
    int32_t *pend;      // [2][B]: reaction partials left pending by the launch that wrote this buffer
    double *pk2;        // [2][B]: peak so far, double-buffered like step
    int32_t *ps2;       // [2][B]: its step
    int32_t bk_par;     // buffer holding the current step/done
    int32_t chunk_par;  // parity the captured chunk starts from
    int32_t rec_off;    // step parity of the live samples = bk_par ^ rec_off (reset: 0 at bk_par; load: step & 1)
    int32_t chunk_rec_off;  // rec_off the captured chunk was made with
    int32_t *brick_ridx;  // [n_bricks]: index among reaction bricks, or -1
    int32_t nrb;          // reaction bricks (bricks with prescribed DOFs, and brick 0)
    int32_t *status;    // [B] bit 0: non-finite reaction
    double *peak;       // [B]
    int32_t *peak_step; // [B]
    double *partial;    // [2][B][nblk]: reaction block partials (double-float), by launch parity
    uint32_t *ticket;   // [B]
    int32_t nblk;
    // run_to_peak chunk graph
    cudaGraphExec_t chunk_exec;
    int32_t chunk_steps;
    int32_t chunk_max_steps;
    int32_t *host_flag;     // pinned mapped [2]
    int32_t *host_flag_dev; // device alias
    cudaEvent_t ev[2];
};

// Tensor-core KL sampling (pd_kl.cu): the split TF32 operand Psi of one level
// with its TMA descriptors, and the sampling launch.
struct KlOperand;
int kl_operand_create(const float *phi, long long N, int K, KlOperand **out);
void kl_operand_destroy(KlOperand *op);
int kl_operand_error(const KlOperand *op);
int kl_sample_tc(KlOperand *op, const double *xi, int B, int marginal, double mu, double sig, double wscale,
                 double winvm, float *out, cudaStream_t s);
