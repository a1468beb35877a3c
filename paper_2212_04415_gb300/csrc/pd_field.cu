// pd_field.cu -- spatially correlated random fields (Section 5): Philox
// KL coefficients, truncated Karhunen-Loeve basis, field sampling with the
// marginal (copula) transform, and the fine-to-coarse coupling of MLMC pairs
// (Section 4.2).
//
// Basis construction (once per hierarchy, host-synchronous):
//   * squared-exponential kernel exp(-r^2/l^2) on a regular grid factorises
//     into three 1D covariance matrices; their eigenpairs come from a cyclic
//     Jacobi eigensolver (Golub & Van Loan, "Matrix Computations", 8.5) in
//     FP64 on the host, the 3D modes are products of 1D eigenvectors, and the
//     K largest products are kept;
//   * sign rule: each eigenvector's largest-magnitude entry is positive
//     (lowest index among entries within 1e-9 relative of the largest);
//   * order rule: products sorted descending; runs whose products lie
//     within 1e-10 relative of the run's first product are re-ordered by
//     (a, b, c) ascending;
//   * Phi_L[i][k] = sqrt(lambda_k) phi_k(x_i) is assembled on the GPU in
//     FP64 and stored as FP32; every coarser level's basis is the 2x2x2 mean
//     of the next finer one, so a coarse field equals the coarsened fine
//     field of the same coefficients.
// Sampling: g = Phi_l xi as a tensor-core GEMM (split TF32, FP32
// accumulation; pd_kl.cu), then the marginal transform, written as FP32
// node fields.
#include <algorithm>
#include <cmath>
#include <vector>

#include "pd_internal.cuh"

struct pd_field {
    pd_field_cfg cfg;
    int32_t n_levels;
    pd_grid grid[PD_MAX_LEVELS];
    int32_t K;
    std::vector<double> lambda;
    float *phi[PD_MAX_LEVELS];  // [N_l][K], sqrt(lambda) folded in
    KlOperand *kl[PD_MAX_LEVELS];  // the same, split into TF32 hi / lo, with TMA descriptors
};

namespace pdi {

// ------------------------------------------------------------- Philox

__device__ __forceinline__ void philox_round(uint32_t c[4], uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
    const uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
    c[0] = n0;
    c[1] = n1;
    c[2] = n2;
    c[3] = n3;
}

// Philox4x32-10 (Salmon et al., SC'11): ten rounds, Weyl key schedule.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += W0;
            k1 += W1;
        }
        philox_round(c, k0, k1);
    }
}

__global__ void k_draw_xi(uint64_t seed, int level, const uint64_t *ids, int B, int K, double *xi) {
    const int nblk = (K + 1) / 2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)B * nblk) return;
    const int b = (int)(t / nblk), j = (int)(t % nblk);
    const uint64_t sid = ids[b];
    uint32_t c[4] = {(uint32_t)j, (uint32_t)(sid & 0xffffffffu), (uint32_t)(sid >> 32), (uint32_t)level};
    philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
    const uint64_t a = ((((uint64_t)c[0]) << 32) | c[1]) >> 11;
    const uint64_t bb = ((((uint64_t)c[2]) << 32) | c[3]) >> 11;
    const double u1 = ((double)a + 0.5) * 0x1p-53;
    const double u2 = ((double)bb + 0.5) * 0x1p-53;
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    xi[(size_t)b * K + 2 * j] = r * cs;
    if (2 * j + 1 < K) xi[(size_t)b * K + 2 * j + 1] = r * sn;
}

// ----------------------------------------------------- host eigensolver

// Cyclic Jacobi: A (n x n, row-major, symmetric) is diagonalised in place;
// V receives the eigenvectors as columns, w the eigenvalues.
static void jacobi_eig(int n, std::vector<double> &A, std::vector<double> &w, std::vector<double> &V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    double fro = 0.0;
    for (double x : A) fro += x * x;
    fro = std::sqrt(fro);
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
        if (std::sqrt(2.0 * off) <= 1e-15 * fro) break;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)p * n + q];
                if (std::fabs(apq) <= 1e-300) continue;
                const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                const double tau = (aqq - app) / (2.0 * apq);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < n; ++k) {  // A <- A J
                    const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // A <- J^T A
                    const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                A[(size_t)p * n + q] = A[(size_t)q * n + p] = 0.0;
                for (int k = 0; k < n; ++k) {  // V <- V J
                    const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

// Eigenpairs sorted by descending eigenvalue, sign-normalised; vectors
// returned column-major: vec[k * n + i] = phi_k(i).
static void eig_sorted(int n, std::vector<double> A, std::vector<double> &lam, std::vector<double> &vec) {
    std::vector<double> w, V;
    jacobi_eig(n, A, w, V);
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return w[x] > w[y]; });
    lam.resize(n);
    vec.resize((size_t)n * n);
    for (int k = 0; k < n; ++k) {
        const int c = idx[k];
        lam[k] = w[c];
        double top = 0.0;
        for (int i = 0; i < n; ++i) top = std::max(top, std::fabs(V[(size_t)i * n + c]));
        int first = 0;
        for (int i = 0; i < n; ++i)
            if (std::fabs(V[(size_t)i * n + c]) >= top * (1.0 - 1e-9)) {
                first = i;
                break;
            }
        const double sg = V[(size_t)first * n + c] < 0 ? -1.0 : 1.0;
        for (int i = 0; i < n; ++i) vec[(size_t)k * n + i] = sg * V[(size_t)i * n + c];
    }
}

static std::vector<double> cov1d(int n, double dx, double l) {
    std::vector<double> C((size_t)n * n);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b) {
            const double r = std::fabs(((a + 0.5) - (b + 0.5)) * dx);
            C[(size_t)a * n + b] = std::exp(-(r * r) / (l * l));
        }
    return C;
}

struct Cand {
    double p;
    int a, b, c;
};

// The K largest products with the run/tie rule described at the top.
static std::vector<Cand> select_modes(const std::vector<double> &lx, const std::vector<double> &ly,
                                      const std::vector<double> &lz, int kx, int ky, int kz, int K) {
    std::vector<Cand> v;
    v.reserve((size_t)kx * ky * kz);
    for (int a = 0; a < kx; ++a)
        for (int b = 0; b < ky; ++b)
            for (int c = 0; c < kz; ++c) v.push_back({lx[a] * ly[b] * lz[c], a, b, c});
    auto lex = [](const Cand &x, const Cand &y) {
        if (x.a != y.a) return x.a < y.a;
        if (x.b != y.b) return x.b < y.b;
        return x.c < y.c;
    };
    std::sort(v.begin(), v.end(), [&](const Cand &x, const Cand &y) {
        if (x.p != y.p) return x.p > y.p;
        return lex(x, y);
    });
    size_t g0 = 0;
    while (g0 < v.size()) {
        size_t g1 = g0 + 1;
        while (g1 < v.size() && v[g0].p - v[g1].p <= 1e-10 * std::fabs(v[g0].p)) ++g1;
        std::sort(v.begin() + g0, v.begin() + g1, lex);
        g0 = g1;
    }
    v.resize(std::min<size_t>(v.size(), (size_t)K));
    return v;
}

// Phi[i][k] = sqrt(lambda_k) vx[a_k](ix) vy[b_k](iy) vz[c_k](iz) in FP64, stored FP32.
__global__ void k_assemble(int nx, int ny, int nz, int K, const double *vx, const double *vy,
                           const double *vz, const int *ia, const int *ib, const int *ic,
                           const double *sq, float *phi) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long N = (long long)nx * ny * nz;
    if (t >= N * K) return;
    const long long i = t / K;
    const int k = (int)(t % K);
    const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((long long)nx * ny));
    phi[t] = (float)(sq[k] * vx[(size_t)ia[k] * nx + ix] * vy[(size_t)ib[k] * ny + iy] *
                     vz[(size_t)ic[k] * nz + iz]);
}

// Dense (non-separable) covariance basis for small meshes: Phi = V sqrt(lambda).
__global__ void k_assemble_dense(long long N, int K, const double *vec, const double *sq, float *phi) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * K) return;
    const long long i = t / K;
    const int k = (int)(t % K);
    phi[t] = (float)(sq[k] * vec[(size_t)k * N + i]);
}

// Coarse basis = mean over the 2x2x2 fine children (fixed order: x, y, z pairs).
// Coarse basis = mean over the fine children: 2x2x2 in 3D, 2x2 in a planar
// hierarchy (one-layer grids, planar = 1), summed x pairs, then y, then z.
__global__ void k_restrict_basis(int cnx, int cny, int cnz, int K, int planar, const float *fine, float *coarse) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long Nc = (long long)cnx * cny * cnz;
    if (t >= Nc * K) return;
    const long long I = t / K;
    const int k = (int)(t % K);
    const int X = (int)(I % cnx), Y = (int)((I / cnx) % cny), Z = (int)(I / ((long long)cnx * cny));
    const int fnx = 2 * cnx, fny = 2 * cny;
    float s[2][2];
    for (int dz = 0; dz < (planar ? 1 : 2); ++dz)
        for (int dy = 0; dy < 2; ++dy) {
            const long long f = (2 * X) + (long long)fnx * ((2 * Y + dy) + (long long)fny * (2 * Z + dz));
            s[dz][dy] = fine[f * K + k] + fine[(f + 1) * K + k];
        }
    if (planar) {
        coarse[t] = (s[0][0] + s[0][1]) * 0.25f;
        return;
    }
    const float yz0 = s[0][0] + s[0][1], yz1 = s[1][0] + s[1][1];
    coarse[t] = (yz0 + yz1) * 0.125f;
}

constexpr int kMaxK = 256;

}  // namespace pdi

using namespace pdi;

extern "C" int pd_draw_xi(uint64_t seed, int32_t level, const uint64_t *sample_ids, int32_t B,
                          int32_t n_modes, double *xi, pd_stream stream) {
    PD_REQUIRE(sample_ids && xi, "sample_ids and xi are required");
    PD_REQUIRE(B >= 0 && n_modes >= 1 && n_modes <= kMaxK, "B >= 0 and 1 <= n_modes <= 256");
    if (B == 0) return PD_OK;
    const long long n = (long long)B * ((n_modes + 1) / 2);
    k_draw_xi<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(seed, level, sample_ids, B,
                                                                              n_modes, xi);
    PD_CHECK_LAUNCH();
    return PD_OK;
}

static void free_field(pd_field *f) {
    if (!f) return;
    for (int l = 0; l < PD_MAX_LEVELS; ++l) {
        cudaFree(f->phi[l]);
        kl_operand_destroy(f->kl[l]);
    }
    delete f;
}

static int build_field(pd_field *f) {
    const pd_grid &g = f->grid[f->n_levels - 1];
    const int K = f->cfg.n_modes;
    const long long N = (long long)g.nx * g.ny * g.nz;
    std::vector<double> sq;
    if (f->cfg.kernel == PD_COV_SQEXP) {
        std::vector<double> lx, vx, ly, vy, lz, vz;
        eig_sorted(g.nx, cov1d(g.nx, g.dx, f->cfg.length), lx, vx);
        eig_sorted(g.ny, cov1d(g.ny, g.dx, f->cfg.length), ly, vy);
        eig_sorted(g.nz, cov1d(g.nz, g.dx, f->cfg.length), lz, vz);
        const int kx = std::min(g.nx, K), ky = std::min(g.ny, K), kz = std::min(g.nz, K);
        std::vector<Cand> sel = select_modes(lx, ly, lz, kx, ky, kz, K);
        PD_REQUIRE((int)sel.size() == K, "grid has fewer than K = %d modes", K);
        std::vector<int> ia(K), ib(K), ic(K);
        f->lambda.resize(K);
        sq.resize(K);
        for (int k = 0; k < K; ++k) {
            ia[k] = sel[k].a;
            ib[k] = sel[k].b;
            ic[k] = sel[k].c;
            f->lambda[k] = sel[k].p;
            sq[k] = std::sqrt(std::max(0.0, sel[k].p));
        }
        double *dvx = nullptr, *dvy = nullptr, *dvz = nullptr, *dsq = nullptr;
        int *dia = nullptr, *dib = nullptr, *dic = nullptr;
        int rc = PD_OK;
        do {
            if ((rc = dalloc(&dvx, vx.size())) || (rc = dalloc(&dvy, vy.size())) || (rc = dalloc(&dvz, vz.size())) ||
                (rc = dalloc(&dsq, K)) || (rc = dalloc(&dia, K)) || (rc = dalloc(&dib, K)) || (rc = dalloc(&dic, K)) ||
                (rc = dalloc(&f->phi[f->n_levels - 1], (size_t)N * K)))
                break;
            cudaMemcpy(dvx, vx.data(), vx.size() * 8, cudaMemcpyHostToDevice);
            cudaMemcpy(dvy, vy.data(), vy.size() * 8, cudaMemcpyHostToDevice);
            cudaMemcpy(dvz, vz.data(), vz.size() * 8, cudaMemcpyHostToDevice);
            cudaMemcpy(dsq, sq.data(), K * 8, cudaMemcpyHostToDevice);
            cudaMemcpy(dia, ia.data(), K * 4, cudaMemcpyHostToDevice);
            cudaMemcpy(dib, ib.data(), K * 4, cudaMemcpyHostToDevice);
            cudaMemcpy(dic, ic.data(), K * 4, cudaMemcpyHostToDevice);
            k_assemble<<<(unsigned)((N * K + 255) / 256), 256>>>(g.nx, g.ny, g.nz, K, dvx, dvy, dvz, dia, dib,
                                                                 dic, dsq, f->phi[f->n_levels - 1]);
            if (cudaDeviceSynchronize() != cudaSuccess) {
                set_error("basis assembly failed: %s", cudaGetErrorString(cudaGetLastError()));
                rc = PD_ERR_CUDA;
            }
        } while (0);
        cudaFree(dvx);
        cudaFree(dvy);
        cudaFree(dvz);
        cudaFree(dsq);
        cudaFree(dia);
        cudaFree(dib);
        cudaFree(dic);
        PD_TRY(rc);
    } else {
        PD_REQUIRE(N <= 4096, "the exponential kernel needs a dense eigensolve (finest N <= 4096)");
        std::vector<double> C((size_t)N * N);
        for (long long i = 0; i < N; ++i)
            for (long long j = 0; j < N; ++j) {
                const double xi_[3] = {(i % g.nx + 0.5) * g.dx, ((i / g.nx) % g.ny + 0.5) * g.dx,
                                       (i / ((long long)g.nx * g.ny) + 0.5) * g.dx};
                const double xj[3] = {(j % g.nx + 0.5) * g.dx, ((j / g.nx) % g.ny + 0.5) * g.dx,
                                      (j / ((long long)g.nx * g.ny) + 0.5) * g.dx};
                const double r = std::sqrt((xi_[0] - xj[0]) * (xi_[0] - xj[0]) + (xi_[1] - xj[1]) * (xi_[1] - xj[1]) +
                                           (xi_[2] - xj[2]) * (xi_[2] - xj[2]));
                C[(size_t)i * N + j] = std::exp(-r / f->cfg.length);
            }
        std::vector<double> lam, vec;
        eig_sorted((int)N, C, lam, vec);
        PD_REQUIRE(K <= N, "K larger than the number of nodes");
        f->lambda.assign(lam.begin(), lam.begin() + K);
        sq.resize(K);
        for (int k = 0; k < K; ++k) sq[k] = std::sqrt(std::max(0.0, lam[k]));
        double *dvec = nullptr, *dsq = nullptr;
        int rc = PD_OK;
        do {
            if ((rc = dalloc(&dvec, (size_t)K * N)) || (rc = dalloc(&dsq, K)) ||
                (rc = dalloc(&f->phi[f->n_levels - 1], (size_t)N * K)))
                break;
            cudaMemcpy(dvec, vec.data(), (size_t)K * N * 8, cudaMemcpyHostToDevice);
            cudaMemcpy(dsq, sq.data(), K * 8, cudaMemcpyHostToDevice);
            k_assemble_dense<<<(unsigned)((N * K + 255) / 256), 256>>>(N, K, dvec, dsq, f->phi[f->n_levels - 1]);
            if (cudaDeviceSynchronize() != cudaSuccess) rc = PD_ERR_CUDA;
        } while (0);
        cudaFree(dvec);
        cudaFree(dsq);
        PD_TRY(rc);
    }
    for (int l = f->n_levels - 2; l >= 0; --l) {
        const pd_grid &c = f->grid[l];
        const long long Nc = (long long)c.nx * c.ny * c.nz;
        PD_TRY(dalloc(&f->phi[l], (size_t)Nc * K));
        k_restrict_basis<<<(unsigned)((Nc * K + 255) / 256), 256>>>(c.nx, c.ny, c.nz, K, f->grid[l + 1].nz == 1 ? 1 : 0,
                                                                    f->phi[l + 1], f->phi[l]);
        PD_CHECK_LAUNCH();
    }
    for (int l = 0; l < f->n_levels; ++l) {
        const pd_grid &c = f->grid[l];
        PD_TRY(kl_operand_create(f->phi[l], (long long)c.nx * c.ny * c.nz, K, &f->kl[l]));
    }
    PD_CHECK_CUDA(cudaDeviceSynchronize());
    return PD_OK;
}

extern "C" int pd_field_create(const pd_grid *finest, int32_t n_levels, const pd_field_cfg *cfg,
                               pd_field **out) {
    PD_REQUIRE(out != nullptr, "out is NULL");
    *out = nullptr;
    PD_TRY(validate_grid(finest));
    PD_REQUIRE(cfg != nullptr, "cfg is NULL");
    PD_REQUIRE(n_levels >= 1 && n_levels <= PD_MAX_LEVELS, "n_levels must be in [1, %d]", PD_MAX_LEVELS);
    PD_REQUIRE(cfg->n_modes >= 1 && cfg->n_modes <= kMaxK, "n_modes must be in [1, 256]");
    PD_REQUIRE(cfg->kernel == PD_COV_SQEXP || cfg->kernel == PD_COV_EXP, "unknown kernel");
    PD_REQUIRE(cfg->marginal == PD_MARG_LOGNORMAL || cfg->marginal == PD_MARG_WEIBULL, "unknown marginal");
    PD_REQUIRE(cfg->length > 0 && cfg->mean > 0, "length and mean must be positive");
    PD_REQUIRE(cfg->marginal != PD_MARG_WEIBULL || cfg->weibull_m > 0, "weibull_m must be positive");
    pd_field *f = new pd_field();
    f->cfg = *cfg;
    f->n_levels = n_levels;
    f->K = cfg->n_modes;
    for (int l = 0; l < PD_MAX_LEVELS; ++l) {
        f->phi[l] = nullptr;
        f->kl[l] = nullptr;
    }
    f->grid[n_levels - 1] = *finest;
    for (int l = n_levels - 2; l >= 0; --l) {
        pd_grid c = f->grid[l + 1];
        const bool planar = c.nz == 1;  // one-layer hierarchy: halve in plane only
        if (c.nx % 2 || c.ny % 2 || (!planar && c.nz % 2)) {
            delete f;
            set_error("grid of level %d cannot be halved (%d x %d x %d)", l + 1, c.nx, c.ny, c.nz);
            return PD_ERR_ARG;
        }
        c.nx /= 2;
        c.ny /= 2;
        if (!planar) c.nz /= 2;
        c.dx *= 2.0;
        f->grid[l] = c;
    }
    const int rc = build_field(f);
    if (rc != PD_OK) {
        free_field(f);
        return rc;
    }
    *out = f;
    return PD_OK;
}

extern "C" int pd_field_destroy(pd_field *f) {
    int rc = PD_OK;
    if (f) {
        cudaDeviceSynchronize();
        for (int l = 0; l < f->n_levels; ++l)
            if (f->kl[l] && kl_operand_error(f->kl[l]) != 0) {
                set_error("a field sampling tile gave up waiting for its copies or MMAs (level %d)", l);
                rc = PD_ERR_TIMEOUT;
            }
        free_field(f);
    }
    return rc;
}

extern "C" int pd_field_info(const pd_field *f, int32_t *n_modes, double *lambda) {
    PD_REQUIRE(f != nullptr, "field is NULL");
    if (n_modes) *n_modes = f->K;
    if (lambda)
        for (int k = 0; k < f->K; ++k) lambda[k] = f->lambda[k];
    return PD_OK;
}

// Inputs of the coefficient gradient (pd_adjoint.cu): the level's basis with
// sqrt(lambda) folded in and the marginal's parameters.
int field_grad_inputs(const pd_field *f, int level, const float **psi, long long *N, int *K, int *marginal,
                      double *mu, double *sig, double *wscale, double *m_w) {
    PD_REQUIRE(level >= 0 && level < f->n_levels, "level out of range");
    const pd_grid &g = f->grid[level];
    const pd_field_cfg &c = f->cfg;
    *psi = f->phi[level];
    *N = (long long)g.nx * g.ny * g.nz;
    *K = f->K;
    *marginal = c.marginal;
    *mu = *sig = *wscale = *m_w = 0.0;
    if (c.marginal == PD_MARG_LOGNORMAL) {
        const double s2 = std::log(1.0 + c.cov * c.cov);
        *mu = std::log(c.mean) - 0.5 * s2;
        *sig = std::sqrt(s2);
    } else {
        *wscale = c.mean / std::tgamma(1.0 + 1.0 / c.weibull_m);
        *m_w = c.weibull_m;
    }
    return PD_OK;
}

static int sample_level(const pd_field *f, int level, const double *xi, int B, float *out, cudaStream_t s) {
    const pd_field_cfg &c = f->cfg;
    double mu = 0, sig = 0, wscale = 0, winvm = 0;
    if (c.marginal == PD_MARG_LOGNORMAL) {
        const double s2 = std::log(1.0 + c.cov * c.cov);
        mu = std::log(c.mean) - 0.5 * s2;
        sig = std::sqrt(s2);
    } else {
        wscale = c.mean / std::tgamma(1.0 + 1.0 / c.weibull_m);
        winvm = 1.0 / c.weibull_m;
    }
    return kl_sample_tc(f->kl[level], xi, B, c.marginal, mu, sig, wscale, winvm, out, s);
}

extern "C" int pd_sample_field(pd_field *f, int32_t level, const double *xi, int32_t B, float *node_field,
                               float *coarse_field, pd_stream stream) {
    PD_REQUIRE(f != nullptr && xi != nullptr && node_field != nullptr, "field, xi and node_field are required");
    PD_REQUIRE(level >= 0 && level < f->n_levels, "level out of range");
    PD_REQUIRE(B >= 0, "B must be >= 0");
    PD_REQUIRE(coarse_field == nullptr || level > 0, "coarse_field needs level > 0");
    if (B == 0) return PD_OK;
    cudaStream_t s = (cudaStream_t)stream;
    PD_TRY(sample_level(f, level, xi, B, node_field, s));
    if (coarse_field) PD_TRY(sample_level(f, level - 1, xi, B, coarse_field, s));
    return PD_OK;
}
