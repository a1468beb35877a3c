// pd_cdf.cu -- multilevel estimate of the peak-load distribution (Section 7):
// the inverse CDF F_L^-1(u) = R_0^[N_0 u] + sum_{l >= 1} (R_l^[N_l u] -
// R~_{l-1}^[N_l u]), where R_l are the fine and R~_{l-1} the coarse members of
// level l's pairs, each sorted ascending, and R^[k] is the k-th smallest.
// Readings: the index [N u] is ceil(N u), 1-based, clamped to [1, N]; the
// coarse term of level l uses the level's own pair count N_l (with N_{l-1},
// as printed, the sum would telescope to the finest level alone). The CDF at
// x is the fraction of the points F_L^-1((i + 1/2) / n), i < n, that are <= x.
//
// Every level's members are ordered by an exact rank count (element j goes to
// position #{i : x_i < x_j, or x_i = x_j and i < j}), one thread per element
// over shared-memory tiles: O(N^2) comparisons, deterministic, and cheap at
// MLMC sample counts.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pd_internal.cuh"

namespace pdi {

constexpr int kCdfTile = 256;

__global__ void __launch_bounds__(kCdfTile) k_rank_sort(long long n, const double *x, double *sorted) {
    __shared__ double tile[kCdfTile];
    const long long j = (long long)blockIdx.x * kCdfTile + threadIdx.x;
    const double xj = j < n ? x[j] : 0.0;
    long long rank = 0;
    for (long long t0 = 0; t0 < n; t0 += kCdfTile) {
        const long long i = t0 + threadIdx.x;
        tile[threadIdx.x] = i < n ? x[i] : 0.0;
        __syncthreads();
        const int m = (int)min((long long)kCdfTile, n - t0);
        for (int k = 0; k < m; ++k) {
            const double xi = tile[k];
            rank += (xi < xj || (xi == xj && t0 + k < j)) ? 1 : 0;
        }
        __syncthreads();
    }
    if (j < n) sorted[rank] = xj;
}

struct CdfLevels {
    int n_levels;
    long long n[PD_MAX_LEVELS];
    long long off[PD_MAX_LEVELS];
};

__device__ __forceinline__ long long order_index(long long N, double u) {
    long long k = (long long)ceil((double)N * u);
    k = k < 1 ? 1 : (k > N ? N : k);
    return k - 1;
}

__device__ __forceinline__ double ml_inverse(const CdfLevels &L, const double *sf, const double *sc, double u) {
    double v = sf[L.off[0] + order_index(L.n[0], u)];
    for (int l = 1; l < L.n_levels; ++l) {
        const long long k = order_index(L.n[l], u);
        v += sf[L.off[l] + k] - sc[L.off[l] + k];
    }
    return v;
}

__global__ void k_ml_inverse(CdfLevels L, const double *sf, const double *sc, int n_u, const double *u,
                             double *out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_u) out[t] = ml_inverse(L, sf, sc, u[t]);
}

__global__ void k_ml_points(CdfLevels L, const double *sf, const double *sc, int n_u, double *X) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_u) X[t] = ml_inverse(L, sf, sc, ((double)t + 0.5) / (double)n_u);
}

__global__ void k_cdf_count(int n_u, const double *X, int n_x, const double *x, double *F) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_x) return;
    long long c = 0;
    for (int i = 0; i < n_u; ++i) c += X[i] <= x[t] ? 1 : 0;
    F[t] = (double)c / (double)n_u;
}

template <class T>
struct CdfBuf {
    T *p = nullptr;
    ~CdfBuf() { cudaFree(p); }
};

// Sorted fine and coarse members of every level (level-major, as given).
static int sort_levels(int n_levels, const int64_t *n_per_level, const double *q_fine, const double *q_coarse,
                       CdfLevels &L, CdfBuf<double> &sf, CdfBuf<double> &sc, cudaStream_t s) {
    PD_REQUIRE(n_levels >= 1 && n_levels <= PD_MAX_LEVELS, "n_levels out of range");
    PD_REQUIRE(n_per_level && q_fine, "n_per_level and q_fine are required");
    PD_REQUIRE(n_levels == 1 || q_coarse, "q_coarse is required with more than one level");
    long long tot = 0;
    L.n_levels = n_levels;
    for (int l = 0; l < n_levels; ++l) {
        PD_REQUIRE(n_per_level[l] >= 1, "every level needs at least one sample");
        L.n[l] = n_per_level[l];
        L.off[l] = tot;
        tot += n_per_level[l];
    }
    PD_TRY(dalloc(&sf.p, tot));
    PD_TRY(dalloc(&sc.p, tot));
    for (int l = 0; l < n_levels; ++l) {
        const unsigned g = (unsigned)((L.n[l] + kCdfTile - 1) / kCdfTile);
        k_rank_sort<<<g, kCdfTile, 0, s>>>(L.n[l], q_fine + L.off[l], sf.p + L.off[l]);
        PD_CHECK_LAUNCH();
        if (l > 0) {
            k_rank_sort<<<g, kCdfTile, 0, s>>>(L.n[l], q_coarse + L.off[l], sc.p + L.off[l]);
            PD_CHECK_LAUNCH();
        }
    }
    return PD_OK;
}

}  // namespace pdi

using namespace pdi;

extern "C" int pd_ml_inverse_cdf(int32_t n_levels, const int64_t *n_per_level, const double *q_fine,
                                 const double *q_coarse, int32_t n_u, const double *u, double *out,
                                 pd_stream stream) {
    PD_REQUIRE(n_u >= 0 && (n_u == 0 || (u && out)), "u and out are required");
    cudaStream_t s = (cudaStream_t)stream;
    CdfLevels L;
    CdfBuf<double> sf, sc;
    PD_TRY(sort_levels(n_levels, n_per_level, q_fine, q_coarse, L, sf, sc, s));
    if (n_u) {
        k_ml_inverse<<<(n_u + 255) / 256, 256, 0, s>>>(L, sf.p, sc.p, n_u, u, out);
        PD_CHECK_LAUNCH();
    }
    PD_CHECK_CUDA(cudaStreamSynchronize(s));  // the sorted copies are freed on return
    return PD_OK;
}

extern "C" int pd_ml_cdf(int32_t n_levels, const int64_t *n_per_level, const double *q_fine,
                         const double *q_coarse, int32_t n_u, int32_t n_x, const double *x, double *F,
                         pd_stream stream) {
    PD_REQUIRE(n_u >= 1, "n_u must be >= 1");
    PD_REQUIRE(n_x >= 0 && (n_x == 0 || (x && F)), "x and F are required");
    cudaStream_t s = (cudaStream_t)stream;
    CdfLevels L;
    CdfBuf<double> sf, sc, X;
    PD_TRY(sort_levels(n_levels, n_per_level, q_fine, q_coarse, L, sf, sc, s));
    PD_TRY(dalloc(&X.p, n_u));
    k_ml_points<<<(n_u + 255) / 256, 256, 0, s>>>(L, sf.p, sc.p, n_u, X.p);
    PD_CHECK_LAUNCH();
    if (n_x) {
        k_cdf_count<<<(n_x + 255) / 256, 256, 0, s>>>(n_u, X.p, n_x, x, F);
        PD_CHECK_LAUNCH();
    }
    PD_CHECK_CUDA(cudaStreamSynchronize(s));
    return PD_OK;
}
