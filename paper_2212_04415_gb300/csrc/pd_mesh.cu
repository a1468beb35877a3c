// pd_mesh.cu -- neighbour list (horizon, Eq. PD_Horizon) and boundary sets.
//
// The grid is regular, so the horizon of a node is a fixed integer stencil
// |offset|^2 <= m^2 (in cell units) clipped by the body and by the notch
// plane. Each node's row is produced by one thread that walks its candidate
// box in ascending linear index order, so rows come out sorted and the list
// is a pure integer function of the grid (bit-exact, no atomics).
#include <stdarg.h>
#include <string.h>

#include <cmath>

#include "pd_internal.cuh"

namespace pdi {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int validate_grid(const pd_grid *g) {
    PD_REQUIRE(g != nullptr, "grid is NULL");
    PD_REQUIRE(g->nx > 0 && g->ny > 0 && g->nz > 0, "grid sizes must be positive");
    PD_REQUIRE(g->nx <= 2047 && g->ny <= 2047 && g->nz <= 1023,
               "grid too large for packed coordinates (nx, ny <= 2047, nz <= 1023)");
    PD_REQUIRE((int64_t)g->nx * g->ny * g->nz < (1ll << 31), "more than 2^31 nodes");
    PD_REQUIRE(g->dx > 0.0 && std::isfinite(g->dx), "dx must be positive");
    PD_REQUIRE(g->m_ratio > 0.0 && g->m_ratio <= 8.0, "m_ratio must be in (0, 8]");
    return PD_OK;
}

struct GridDev {
    int nx, ny, nz, r;
    double m2;
    int notch, X2, Y2;
};

// Strict crossing of the notch plane below the tip, in exact integers.
__device__ __forceinline__ bool notch_cut(const GridDev &g, int ix, int iy, int jx, int jy) {
    if (!g.notch) return false;
    const long long Xi = 2 * ix + 1, Xj = 2 * jx + 1;
    const long long Yi = 2 * iy + 1, Yj = 2 * jy + 1;
    const long long Xn = g.X2;
    if ((Xi - Xn) * (Xj - Xn) >= 0) return false;
    const long long dX = Xj - Xi;
    const long long lhs = Yi * dX + (Xn - Xi) * (Yj - Yi);
    const long long rhs = (long long)g.Y2 * dX;
    return dX > 0 ? (lhs < rhs) : (lhs > rhs);
}

template <bool FILL>
__global__ void k_rows(GridDev g, int32_t *__restrict__ row_ptr, int32_t *__restrict__ col) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int ix = (int)(i % g.nx);
    const int iy = (int)((i / g.nx) % g.ny);
    const int iz = (int)(i / ((long long)g.nx * g.ny));
    int cnt = 0;
    long long out = FILL ? (long long)row_ptr[i] : 0;
    for (int dz = -g.r; dz <= g.r; ++dz) {
        const int jz = iz + dz;
        if (jz < 0 || jz >= g.nz) continue;
        for (int dy = -g.r; dy <= g.r; ++dy) {
            const int jy = iy + dy;
            if (jy < 0 || jy >= g.ny) continue;
            for (int dxo = -g.r; dxo <= g.r; ++dxo) {
                const int jx = ix + dxo;
                if (jx < 0 || jx >= g.nx) continue;
                const int q = dxo * dxo + dy * dy + dz * dz;
                if (q == 0 || (double)q > g.m2) continue;
                if (notch_cut(g, ix, iy, jx, jy)) continue;
                if (FILL) {
                    col[out + cnt] = (int32_t)(jx + (long long)g.nx * (jy + (long long)g.ny * jz));
                }
                ++cnt;
            }
        }
    }
    if (!FILL) {
        row_ptr[i + 1] = cnt;
        if (i == 0) row_ptr[0] = 0;
    }
}

// Single-CTA inclusive scan of a[1..n] (a[0] is the zero start).
__global__ void __launch_bounds__(1024) k_scan(int32_t *a, long long n, int32_t *overflow) {
    __shared__ long long part[1024];
    const int t = threadIdx.x;
    const long long per = (n + 1023) / 1024;
    const long long lo = 1 + t * per;
    const long long hi = min(n + 1, lo + per);
    long long s = 0;
    for (long long k = lo; k < hi; ++k) s += a[k];
    part[t] = s;
    __syncthreads();
    // Hillis-Steele scan over 1024 partial sums
    for (int off = 1; off < 1024; off <<= 1) {
        long long v = (t >= off) ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    long long run = (t == 0) ? 0 : part[t - 1];
    for (long long k = lo; k < hi; ++k) {
        run += a[k];
        if (run > 2147483647ll) {
            *overflow = 1;
            run = 2147483647ll;
        }
        a[k] = (int32_t)run;
    }
}

int scan_inplace_i32(int32_t *a, int64_t n, int32_t *overflow_flag_dev, cudaStream_t s) {
    k_scan<<<1, 1024, 0, s>>>(a, (long long)n, overflow_flag_dev);
    PD_CHECK_LAUNCH();
    return PD_OK;
}

static GridDev make_dev(const pd_grid *g) {
    GridDev d;
    d.nx = g->nx;
    d.ny = g->ny;
    d.nz = g->nz;
    d.m2 = g->m_ratio * g->m_ratio;
    d.r = (int)std::ceil(g->m_ratio);
    d.notch = g->notch ? 1 : 0;
    d.X2 = g->notch_x2;
    d.Y2 = g->notch_y2;
    return d;
}

__global__ void k_bc(int nx, int ny, int nz, pd_bc bc, uint8_t *__restrict__ codes) {
    const long long n = (long long)nx * ny * nz;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int ix = (int)(i % nx), iy = (int)((i / nx) % ny);
    const int X = 2 * ix + 1;
    uint8_t c0 = 0, c1 = 0, c2 = 0;
    if (bc.type == PD_BC_BAR_TENSION) {
        if (ix < bc.grip_planes) {
            c0 = c1 = c2 = 1;
        } else if (ix >= nx - bc.grip_planes) {
            c0 = 2;
            c1 = c2 = 1;
        }
    } else {
        if (iy == 0) {
            const int d0 = X - bc.support_x2[0], d1 = X - bc.support_x2[1];
            if ((d0 >= -1 && d0 <= 1) || (d1 >= -1 && d1 <= 1)) c1 = 1;
        }
        if (iy == ny - 1) {
            const int d = X - bc.load_x2;
            if (d >= -1 && d <= 1) c1 = 3;
        }
    }
    codes[3 * i + 0] = c0;
    codes[3 * i + 1] = c1;
    codes[3 * i + 2] = c2;
}

}  // namespace pdi

using namespace pdi;

extern "C" int pd_last_error(char *buf, size_t len) {
    if (!buf || len == 0) return PD_ERR_ARG;
    strncpy(buf, g_err, len - 1);
    buf[len - 1] = 0;
    return PD_OK;
}

extern "C" const char *pd_version(void) { return "pd-gb300 0.1 (sm_103a)"; }

extern "C" int pd_build_neighbours(const pd_grid *g, int32_t *row_ptr, int32_t *col, int64_t cap,
                                   int64_t *n_bonds, pd_stream stream) {
    PD_TRY(validate_grid(g));
    PD_REQUIRE(row_ptr != nullptr && n_bonds != nullptr, "row_ptr and n_bonds are required");
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = (long long)g->nx * g->ny * g->nz;
    GridDev d = make_dev(g);
    int32_t *flag = nullptr;
    PD_TRY(dalloc(&flag, 1));
    int rc = PD_OK;
    do {
        if (cudaMemsetAsync(flag, 0, sizeof(int32_t), s) != cudaSuccess) { rc = PD_ERR_CUDA; break; }
        const int bs = 256;
        const unsigned nblk = (unsigned)((n + bs - 1) / bs);
        k_rows<false><<<nblk, bs, 0, s>>>(d, row_ptr, nullptr);
        if (cudaGetLastError() != cudaSuccess) { rc = PD_ERR_CUDA; break; }
        if ((rc = scan_inplace_i32(row_ptr, n, flag, s)) != PD_OK) break;
        int32_t total = 0, ovf = 0;
        if (cudaMemcpyAsync(&total, row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(&ovf, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            rc = PD_ERR_CUDA;
            break;
        }
        if (ovf) {
            set_error("more than 2^31-1 bonds");
            rc = PD_ERR_ARG;
            break;
        }
        *n_bonds = total;
        if (col == nullptr) break;
        if (cap < total) {
            set_error("col capacity %lld < %d bonds", (long long)cap, total);
            rc = PD_ERR_CAP;
            break;
        }
        k_rows<true><<<nblk, bs, 0, s>>>(d, row_ptr, col);
        if (cudaGetLastError() != cudaSuccess) { rc = PD_ERR_CUDA; break; }
    } while (0);
    if (rc == PD_ERR_CUDA) set_error("CUDA failure in pd_build_neighbours: %s", cudaGetErrorString(cudaGetLastError()));
    cudaFree(flag);
    return rc;
}

extern "C" int pd_bc_codes(const pd_grid *g, const pd_bc *bc, uint8_t *codes, pd_stream stream) {
    PD_TRY(validate_grid(g));
    PD_REQUIRE(bc != nullptr && codes != nullptr, "bc and codes are required");
    PD_REQUIRE(bc->type == PD_BC_BAR_TENSION || bc->type == PD_BC_BEAM_3PT, "unknown bc type %d", bc->type);
    const long long n = (long long)g->nx * g->ny * g->nz;
    k_bc<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(g->nx, g->ny, g->nz, *bc, codes);
    PD_CHECK_LAUNCH();
    return PD_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of pd_build_neighbours.
//
// The build needs one word of device scratch beyond its inputs and outputs:
// the overflow flag of the row-pointer scan. pd_build_neighbours takes it from
// cudaMalloc on every call; this variant keeps it in a file-scope device array
// instead, for callers that cannot allocate device memory. Its address is
// looked up on every call with the current device (cudaGetSymbolAddress), so a
// context torn down by cudaDeviceReset leaves no stale pointer behind.
static __device__ __align__(256) int32_t g_noalloc_scratch[64];  // 256 bytes; word 0 = scan overflow flag

static int noalloc_scratch(int32_t **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
        set_error("cudaGetSymbolAddress of the neighbour-build scratch failed: %s", cudaGetErrorString(e));
        return PD_ERR_CUDA;
    }
    *out = (int32_t *)p;
    return PD_OK;
}

extern "C" int pd_build_neighbours_noalloc(const pd_grid *g, int32_t *row_ptr, int32_t *col, int64_t cap,
                                           int64_t *n_bonds, pd_stream stream) {
    PD_TRY(validate_grid(g));
    PD_REQUIRE(row_ptr != nullptr && n_bonds != nullptr, "row_ptr and n_bonds are required");
    const long long n = (long long)g->nx * g->ny * g->nz;
    PD_REQUIRE(n + 1 <= 2147483647ll, "at most 2^31 - 2 nodes");
    cudaStream_t s = (cudaStream_t)stream;
    if (s != nullptr) {  // the scratch address is the current device's: the stream must run there
        int cur = 0, sdev = 0;
        PD_CHECK_CUDA(cudaGetDevice(&cur));
        PD_CHECK_CUDA(cudaStreamGetDevice(s, &sdev));
        PD_REQUIRE(sdev == cur, "the stream belongs to device %d, not the current device %d", sdev, cur);
    }
    int32_t *flag = nullptr;
    PD_TRY(noalloc_scratch(&flag));
    GridDev d = make_dev(g);
    PD_CHECK_CUDA(cudaMemsetAsync(flag, 0, sizeof(int32_t), s));  // the array keeps the previous call's value
    const int bs = 256;
    const unsigned nblk = (unsigned)((n + bs - 1) / bs);
    k_rows<false><<<nblk, bs, 0, s>>>(d, row_ptr, nullptr);
    PD_CHECK_LAUNCH();
    PD_TRY(scan_inplace_i32(row_ptr, n, flag, s));
    int32_t total = 0, ovf = 0;
    PD_CHECK_CUDA(cudaMemcpyAsync(&total, row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PD_CHECK_CUDA(cudaMemcpyAsync(&ovf, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PD_CHECK_CUDA(cudaStreamSynchronize(s));
    PD_REQUIRE(!ovf, "more than 2^31-1 bonds");
    *n_bonds = total;
    if (col == nullptr) return PD_OK;
    if (cap < total) {
        set_error("col capacity %lld < %d bonds", (long long)cap, total);
        return PD_ERR_CAP;
    }
    k_rows<true><<<nblk, bs, 0, s>>>(d, row_ptr, col);
    PD_CHECK_LAUNCH();
    return PD_OK;
}
