// pd_kl.cu -- truncated-KL field sampling on the tensor cores (Section 3):
// g[b][i] = sum_k Psi[i][k] xi[b][k], Psi = Phi diag(sqrt(lambda)), followed by
// the marginal transform (lognormal, or the Weibull copula of Section 6),
// written as FP32 node fields [B][N].
//
// The contraction runs as tcgen05.mma kind::tf32 with FP32 accumulators in
// tensor memory. TF32 keeps 11 significant bits, so each operand is split
// into hi = tf32(x) and lo = tf32(x - hi) and the product is taken as
// hi*hi + hi*lo + lo*hi (three MMAs; the dropped lo*lo term is below
// 2^-22 relative), which gives FP32-class accuracy.
//
// The coefficients are split once per call (k_split_xi: FP64 -> TF32 hi /
// lo, [B][Kp], zero-padded modes). One CTA of 256 threads owns a tile of
// 128 nodes (the MMA's M) by NT samples (its N). Modes are consumed in chunks
// of 32 (one 128-byte swizzle atom of FP32): the Psi and xi chunks (hi and lo)
// arrive by TMA with the 128B swizzle and one thread issues the 4 x 3 MMAs of
// the chunk. The epilogue reads the accumulators with tcgen05.ld (warps w and
// w + 4 share TMEM lanes 32 (w mod 4) .. + 31 and split the columns), applies
// the marginal transform and writes the node fields, coalesced along nodes.
// Every wait on an mbarrier has an iteration limit; on expiry the CTA records
// an error, writes NaN into its tile and still waits (bounded) for its own
// copies and MMAs before it frees tensor memory.
#include <cuda.h>

#include <mutex>

#include "pd_internal.cuh"

namespace pdi {

constexpr int kKlM = 128;          // nodes per tile (MMA M)
constexpr int kKlChunk = 32;       // modes per chunk (128 B of FP32)
constexpr int kKlThreads = 256;
constexpr uint32_t kSpinLimit = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bounded wait for the phase with the given parity; false when the limit expired.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < kSpinLimit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"((uint64_t)tm), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzle: rows of 128 B, 8-row groups 1024 B apart (stride byte offset),
// descriptor version 1, swizzle mode 2 (128B).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
    d |= (uint64_t)1 << 46;            // descriptor version
    d |= (uint64_t)2 << 61;            // 128B swizzle
    return d;
}

// Instruction descriptor, kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, N = n, M = 128.
__host__ __device__ constexpr uint32_t tf32_idesc(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kKlM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// Psi_hi / Psi_lo [N][Kp] from Phi [N][K] (sqrt(lambda) folded in), zero-padded to Kp.
__global__ void k_split_psi(long long N, int K, int Kp, const float *phi, float *hi, float *lo) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * Kp) return;
    const long long i = t / Kp;
    const int k = (int)(t % Kp);
    const float x = k < K ? phi[i * K + k] : 0.0f;
    const float h = tf32_rna(x);
    hi[t] = h;
    lo[t] = tf32_rna(x - h);
}

// xi_hi / xi_lo [B][Kp] from xi [B][K] (FP64), zero-padded to Kp.
__global__ void k_split_xi(int B, int K, int Kp, const double *xi, float *hi, float *lo) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)B * Kp) return;
    const long long b = t / Kp;
    const int k = (int)(t % Kp);
    const float x = k < K ? (float)xi[b * K + k] : 0.0f;
    const float h = tf32_rna(x);
    hi[t] = h;
    lo[t] = tf32_rna(x - h);
}

struct KlArgs {
    long long N;
    int K, Kp, B, nt;
    int marginal;
    float mu, sig, wscale, winvm;
    float *out;  // [B][N]
    int *err;
};

__global__ void __launch_bounds__(kKlThreads) k_sample_tc(const __grid_constant__ CUtensorMap tm_hi,
                                                          const __grid_constant__ CUtensorMap tm_lo,
                                                          const __grid_constant__ CUtensorMap tx_hi,
                                                          const __grid_constant__ CUtensorMap tx_lo, const KlArgs a) {
    extern __shared__ __align__(1024) uint8_t kl_smem_raw[];
    __shared__ uint64_t bar_tma, bar_mma;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail, s_fail_chunk;
    uint8_t *sm = (uint8_t *)(((uintptr_t)kl_smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *sA_hi = sm;                       // 128 rows x 128 B
    uint8_t *sA_lo = sm + kKlM * 128;          // 128 rows x 128 B
    uint8_t *sB_hi = sm + 2 * kKlM * 128;      // nt rows x 128 B
    uint8_t *sB_lo = sB_hi + (size_t)a.nt * 128;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // tiles in a 1D grid, sample tile fastest: the CTAs that share a node
    // tile's Psi rows run together, so its second read comes from L2
    const int nbt = (a.B + a.nt - 1) / a.nt;
    const long long n0 = (long long)(blockIdx.x / (unsigned)nbt) * kKlM;
    const int b0 = (int)(blockIdx.x % (unsigned)nbt) * a.nt;
    const int ncols = a.nt < 32 ? 32 : a.nt;  // power of two by construction (host)

    if (tid == 0) {
        mbar_init(&bar_tma, 1);
        mbar_init(&bar_mma, 1);
        s_fail = 0;
        s_fail_chunk = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = tf32_idesc(a.nt);
    const int nchunks = a.Kp / kKlChunk;
    bool ok = true;

    for (int c = 0; c < nchunks; ++c) {
        if (tid == 0 && ok) {
            mbar_expect_tx(&bar_tma, 2u * kKlM * 128u + 2u * (uint32_t)a.nt * 128u);
            tma_load_2d(sA_hi, &tm_hi, c * kKlChunk, (int)n0, &bar_tma);
            tma_load_2d(sA_lo, &tm_lo, c * kKlChunk, (int)n0, &bar_tma);
            tma_load_2d(sB_hi, &tx_hi, c * kKlChunk, b0, &bar_tma);
            tma_load_2d(sB_lo, &tx_lo, c * kKlChunk, b0, &bar_tma);
        }
        if (tid == 0 && ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!mbar_wait(&bar_tma, (uint32_t)(c & 1))) {
                ok = false;
                s_fail = 1;
                s_fail_chunk = c;
            } else {
                const uint32_t aH = smem_u32(sA_hi), aL = smem_u32(sA_lo);
                const uint32_t bH = smem_u32(sB_hi), bL = smem_u32(sB_lo);
#pragma unroll
                for (int s = 0; s < kKlChunk / 8; ++s) {  // K = 8 per MMA: 32 B along the row
                    const uint32_t o = 32u * s;
                    const uint32_t acc0 = (c > 0 || s > 0) ? 1u : 0u;
                    mma_tf32(tmem, sw128_desc(aL + o), sw128_desc(bH + o), idesc, acc0);
                    mma_tf32(tmem, sw128_desc(aH + o), sw128_desc(bL + o), idesc, 1u);
                    mma_tf32(tmem, sw128_desc(aH + o), sw128_desc(bH + o), idesc, 1u);
                }
                mma_commit(&bar_mma);
            }
        }
        __syncthreads();
        if (s_fail) break;
        // every thread waits for the chunk's MMAs before the buffers are reused
        if (!mbar_wait(&bar_mma, (uint32_t)(c & 1))) {
            s_fail = 2;  // any thread that gave up; all write the same values
            s_fail_chunk = c;
        }
        __syncthreads();
        if (s_fail) break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    const int row = (warp & 3) * 32 + lane;
    const long long i = n0 + row;
    const int half = a.nt / 2;  // columns of this warp: [jb, jb + half)
    const int jb = (warp >> 2) * half;
    if (!s_fail) {
        const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        for (int j0 = jb; j0 < jb + half; j0 += 16) {
            float v[16];
            tmem_ld16(lane_base + (uint32_t)j0, v);
            if (i < a.N) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int b = b0 + j0 + q;
                    if (b < a.B) {
                        const float g = v[q];
                        float f;
                        if (a.marginal == PD_MARG_LOGNORMAL) {
                            f = expf(a.mu + a.sig * g);
                        } else {
                            const float q1 = 0.5f * erfcf(g * 0.70710678118654752f);  // 1 - Phi(g)
                            f = a.wscale * powf(-logf(q1), a.winvm);
                        }
                        a.out[(size_t)b * a.N + i] = f;
                    }
                }
            }
        }
    } else {
        if (tid == 0) atomicOr(a.err, s_fail);
        if (i < a.N)
            for (int j = jb; j < jb + half && b0 + j < a.B; ++j)
                a.out[(size_t)(b0 + j) * a.N + i] = __int_as_float(0x7fc00000);
        // outstanding copies or MMAs of this CTA: bounded waits before the memory is released
        if (tid == 0) {
            const uint32_t par = (uint32_t)(s_fail_chunk & 1);
            if (s_fail == 1) mbar_wait(&bar_tma, par);
            else mbar_wait(&bar_mma, par);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
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

// A [rows][Kp] FP32 operand, K-major, read in boxes of 32 modes x box_rows rows, 128B swizzle.
static int encode_kmajor(CUtensorMap *tm, float *base, long long rows, int Kp, int box_rows) {
    EncodeTiledFn enc = encode_fn();
    PD_REQUIRE(enc != nullptr, "cuTensorMapEncodeTiled is unavailable");
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kKlChunk, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    PD_REQUIRE(r == CUDA_SUCCESS, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return PD_OK;
}

static size_t kl_smem_bytes(int nt) { return 1024 + 2 * (size_t)kKlM * 128 + 2 * (size_t)nt * 128; }

}  // namespace pdi

using namespace pdi;

struct KlOperand {
    CUtensorMap tm_hi, tm_lo;  // 64-byte aligned by type
    float *hi = nullptr, *lo = nullptr;
    float *xs = nullptr;       // split coefficients: hi [cap][Kp] then lo [cap][Kp]
    int xs_cap = 0;
    int *err = nullptr;
    long long N = 0;
    int K = 0, Kp = 0;
};

int kl_operand_create(const float *phi, long long N, int K, KlOperand **out) {
    PD_REQUIRE(N >= 1 && K >= 1 && K <= 256, "1 <= K <= 256 and N >= 1 required");
    PD_REQUIRE(N < (1LL << 31), "N too large for the TMA coordinate");
    KlOperand *op = new KlOperand();
    op->N = N;
    op->K = K;
    op->Kp = (K + kKlChunk - 1) / kKlChunk * kKlChunk;
    int rc = dalloc(&op->hi, (size_t)N * op->Kp);
    if (rc == PD_OK) rc = dalloc(&op->lo, (size_t)N * op->Kp);
    if (rc == PD_OK) rc = dalloc(&op->err, 1);
    if (rc == PD_OK && cudaMemset(op->err, 0, sizeof(int)) != cudaSuccess) rc = PD_ERR_CUDA;
    if (rc == PD_OK) {
        const long long n = N * op->Kp;
        k_split_psi<<<(unsigned)((n + 255) / 256), 256>>>(N, K, op->Kp, phi, op->hi, op->lo);
        if (cudaGetLastError() != cudaSuccess) rc = PD_ERR_CUDA;
    }
    if (rc == PD_OK) rc = encode_kmajor(&op->tm_hi, op->hi, N, op->Kp, kKlM);
    if (rc == PD_OK) rc = encode_kmajor(&op->tm_lo, op->lo, N, op->Kp, kKlM);
    if (rc == PD_OK) {
        static std::once_flag attr;
        std::call_once(attr, [] {
            cudaFuncSetAttribute(k_sample_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kl_smem_bytes(256));
        });
        if (cudaGetLastError() != cudaSuccess) rc = PD_ERR_CUDA;
    }
    if (rc != PD_OK) {
        cudaFree(op->hi);
        cudaFree(op->lo);
        cudaFree(op->err);
        delete op;
        return rc;
    }
    *out = op;
    return PD_OK;
}

void kl_operand_destroy(KlOperand *op) {
    if (!op) return;
    cudaFree(op->xs);
    cudaFree(op->hi);
    cudaFree(op->lo);
    cudaFree(op->err);
    delete op;
}

int kl_operand_error(const KlOperand *op) {
    int h = 0;
    if (op && cudaMemcpy(&h, op->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    return h;
}

// Samples per tile: a power of two of at least 32 columns of tensor memory
// covering B, capped at 128. At the cap a CTA holds 67 KB of shared memory,
// so three CTAs share an SM and one's epilogue stores overlap another's loads
// and MMAs (measured on GB300, 224,000 nodes x 256 samples: 109 us per field
// sample at a cap of 256 with two CTAs per SM, 103 us at 128, 121 us at 64).
static int pick_nt(int B) {
    int nt = 32;
    while (nt < B && nt < 128) nt *= 2;
    return nt;
}

int kl_sample_tc(KlOperand *op, const double *xi, int B, int marginal, double mu, double sig, double wscale,
                 double winvm, float *out, cudaStream_t s) {
    if (B <= 0) return PD_OK;
    if (B > op->xs_cap) {  // grows only; cudaFree orders itself after work in flight
        cudaFree(op->xs);
        op->xs = nullptr;
        op->xs_cap = 0;
        PD_TRY(dalloc(&op->xs, 2 * (size_t)B * op->Kp));
        op->xs_cap = B;
    }
    float *xh = op->xs, *xl = op->xs + (size_t)op->xs_cap * op->Kp;
    KlArgs a;
    a.N = op->N;
    a.K = op->K;
    a.Kp = op->Kp;
    a.B = B;
    a.nt = pick_nt(B);
    a.marginal = marginal;
    a.mu = (float)mu;
    a.sig = (float)sig;
    a.wscale = (float)wscale;
    a.winvm = (float)winvm;
    a.out = out;
    a.err = op->err;
    alignas(64) CUtensorMap tx_hi, tx_lo;
    PD_TRY(encode_kmajor(&tx_hi, xh, B, op->Kp, a.nt));
    PD_TRY(encode_kmajor(&tx_lo, xl, B, op->Kp, a.nt));
    const long long n = (long long)B * op->Kp;
    k_split_xi<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(B, op->K, op->Kp, xi, xh, xl);
    PD_CHECK_LAUNCH();
    const long long n_tiles = (op->N + kKlM - 1) / kKlM * ((B + a.nt - 1) / a.nt);
    PD_REQUIRE(n_tiles < (1ll << 31), "too many KL tiles for one launch");
    const dim3 grid((unsigned)n_tiles);
    k_sample_tc<<<grid, kKlThreads, kl_smem_bytes(a.nt), s>>>(op->tm_hi, op->tm_lo, tx_hi, tx_lo, a);
    PD_CHECK_LAUNCH();
    return PD_OK;
}
