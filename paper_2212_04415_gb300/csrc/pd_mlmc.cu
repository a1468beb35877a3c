// pd_mlmc.cu -- multilevel Monte Carlo driver (Section 4): coupled fine /
// coarse samples on nested grids sharing one KL realisation, FP64 level
// sums on the GPU, the estimator Q_ML = sum_l Y_hat_l (Eq. MLMC_estimator),
// the sample variance of Eq. sample_variance and the optimal allocation of
// Eq. sample_allocation.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "pd_internal.cuh"

namespace pdi {

// Y = Qf - Qc and the FP64 sums of Y and Y^2 over one batch, in a fixed order
// (thread t sums t, t + 256, ...; then a fixed tree), one CTA.
__global__ void k_level_sums(int n, const double *qf, const double *qc, double *y, double *out2) {
    __shared__ double s1[256], s2[256];
    double a = 0.0, b = 0.0;
    for (int t = threadIdx.x; t < n; t += 256) {
        const double v = qf[t] - (qc ? qc[t] : 0.0);
        y[t] = v;
        a += v;
        b += v * v;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s1[threadIdx.x] += s1[threadIdx.x + o];
            s2[threadIdx.x] += s2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out2[0] = s1[0];
        out2[1] = s2[0];
    }
}

__global__ void k_iota(uint64_t start, int n, uint64_t *ids) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) ids[t] = start + (uint64_t)t;
}

struct Mesh {
    int32_t *row = nullptr, *col = nullptr;
    int64_t nb = 0;
    ~Mesh() {
        cudaFree(row);
        cudaFree(col);
    }
};

static int make_mesh(const pd_grid &g, Mesh &m, cudaStream_t s) {
    const long long N = (long long)g.nx * g.ny * g.nz;
    PD_TRY(dalloc(&m.row, N + 1));
    PD_TRY(pd_build_neighbours(&g, m.row, nullptr, 0, &m.nb, (pd_stream)s));
    PD_TRY(dalloc(&m.col, m.nb));
    PD_TRY(pd_build_neighbours(&g, m.row, m.col, m.nb, &m.nb, (pd_stream)s));
    return PD_OK;
}

struct Buffers {
    uint64_t *ids = nullptr;
    double *xi = nullptr, *qf = nullptr, *qc = nullptr, *y = nullptr, *sums = nullptr;
    float *ff = nullptr, *fc = nullptr;
    int32_t *ps = nullptr, *psc = nullptr, *nd = nullptr, *ndc = nullptr;
    ~Buffers() {
        cudaFree(ids);
        cudaFree(xi);
        cudaFree(qf);
        cudaFree(qc);
        cudaFree(y);
        cudaFree(sums);
        cudaFree(ff);
        cudaFree(fc);
        cudaFree(ps);
        cudaFree(psc);
        cudaFree(nd);
        cudaFree(ndc);
    }
};

// Sample mean Y_hat = sum_y / n and variance s^2 = sum_y2 / n - Y_hat^2 (Eq.
// sample_variance, the paper's 1/n form) with the unbiased n/(n-1) form.
static void level_stats(pd_mlmc_level *lv) {
    if (lv->n <= 0) {
        lv->mean = lv->var = lv->var_unbiased = 0.0;
        return;
    }
    lv->mean = lv->sum_y / (double)lv->n;
    lv->var = lv->sum_y2 / (double)lv->n - lv->mean * lv->mean;
    lv->var_unbiased = lv->n > 1 ? lv->var * (double)lv->n / (double)(lv->n - 1) : 0.0;
}

// Q_hat^ML = sum_l Y_hat_l (Eq. MLMC_estimator) and its sampling variance
// sum_l s_l^2 / n_l (Eq. MLMC_error), over the levels that have samples.
static void estimator(pd_mlmc_result *r) {
    r->q_ml = r->var_ml = 0.0;
    for (int l = 0; l < r->n_levels; ++l) {
        if (r->level[l].n > 0) {
            r->q_ml += r->level[l].mean;
            r->var_ml += r->level[l].var / (double)r->level[l].n;
        }
    }
}

static int run_level(const pd_mlmc_cfg *cfg, pd_field *field, int l, pd_mlmc_level *lv, double *q_fine,
                     double *q_coarse, double *batch_sums, cudaStream_t s) {
    const int64_t n_total = cfg->n_samples[l];
    lv->n = 0;
    lv->sum_y = lv->sum_y2 = 0.0;
    lv->cost_s = 0.0;
    lv->steps = 0;
    lv->bond_updates = 0;
    if (n_total <= 0) return PD_OK;
    const int K = cfg->field.n_modes;
    const int Bmax = (int)std::min<int64_t>(cfg->batch, n_total);
    Mesh mf, mc;
    PD_TRY(make_mesh(cfg->grid[l], mf, s));
    if (l > 0) PD_TRY(make_mesh(cfg->grid[l - 1], mc, s));
    const long long Nf = (long long)cfg->grid[l].nx * cfg->grid[l].ny * cfg->grid[l].nz;
    const long long Nc = l > 0 ? (long long)cfg->grid[l - 1].nx * cfg->grid[l - 1].ny * cfg->grid[l - 1].nz : 0;
    Buffers bf;
    PD_TRY(dalloc(&bf.ids, Bmax));
    PD_TRY(dalloc(&bf.xi, (size_t)Bmax * K));
    PD_TRY(dalloc(&bf.qf, Bmax));
    PD_TRY(dalloc(&bf.qc, Bmax));
    PD_TRY(dalloc(&bf.y, Bmax));
    PD_TRY(dalloc(&bf.sums, 2));
    PD_TRY(dalloc(&bf.ff, (size_t)Bmax * Nf));
    if (l > 0) PD_TRY(dalloc(&bf.fc, (size_t)Bmax * Nc));
    PD_TRY(dalloc(&bf.ps, Bmax));
    PD_TRY(dalloc(&bf.psc, Bmax));
    PD_TRY(dalloc(&bf.nd, Bmax));
    PD_TRY(dalloc(&bf.ndc, Bmax));
    pd_state *sf = nullptr, *sc = nullptr;
    int cur_b = 0;
    int rc = PD_OK;
    std::vector<double> hq(Bmax), hqc(Bmax);
    std::vector<int32_t> hnd(Bmax), hndc(Bmax);
    for (int64_t first = 0; first < n_total && rc == PD_OK; first += Bmax) {
        const int b = (int)std::min<int64_t>(Bmax, n_total - first);
        if (b != cur_b) {
            pd_state_destroy(sf);
            pd_state_destroy(sc);
            sf = sc = nullptr;
            pd_schedule shf{0, 0, 0};
            if (cfg->tune_steps > 0 &&
                (rc = pd_autotune(&cfg->grid[l], mf.row, mf.col, mf.nb, &cfg->mat, &cfg->bc[l], b, cfg->tune_steps,
                                  &shf, nullptr)))
                break;
            if ((rc = pd_state_create_sched(&cfg->grid[l], mf.row, mf.col, mf.nb, &cfg->mat, &cfg->bc[l], b,
                                            cfg->tune_steps > 0 ? &shf : nullptr, &sf)))
                break;
            // the coarse member takes the fine member's launch shape (a brick
            // of the same rows, the same warp split, one sample per block), so
            // that one launch per step covers the pair (pd_run_to_peak_multi)
            pd_schedule shc{sf->by, sf->bz, sf->st_q, sf->st_ns, 0};
            if (l > 0 && (rc = pd_state_create_sched(&cfg->grid[l - 1], mc.row, mc.col, mc.nb, &cfg->mat,
                                                     &cfg->bc[l - 1], b, sf->stencil ? &shc : nullptr, &sc)))
                break;
            cur_b = b;
        }
        cudaStreamSynchronize(s);
        const auto t0 = std::chrono::steady_clock::now();
        const int64_t id0 = (cfg->first_sample ? cfg->first_sample[l] : 0) + first;
        k_iota<<<(b + 255) / 256, 256, 0, s>>>((uint64_t)id0, b, bf.ids);
        if ((rc = pd_draw_xi(cfg->seed, l, bf.ids, b, K, bf.xi, (pd_stream)s))) break;
        if ((rc = pd_sample_field(field, l, bf.xi, b, bf.ff, l > 0 ? bf.fc : nullptr, (pd_stream)s))) break;
        if ((rc = pd_state_reset(sf, bf.ff, nullptr, (pd_stream)s))) break;
        if (l == 0) {
            if ((rc = pd_run_to_peak(sf, cfg->max_steps[l], bf.qf, bf.ps, bf.nd, (pd_stream)s))) break;
        } else {
            // the pair's fine and coarse members run together (one chunk graph, two branches)
            if ((rc = pd_state_reset(sc, bf.fc, nullptr, (pd_stream)s))) break;
            pd_state *both[2] = {sf, sc};
            const int32_t ms[2] = {cfg->max_steps[l], cfg->max_steps[l - 1]};
            double *pk[2] = {bf.qf, bf.qc};
            int32_t *ps2[2] = {bf.ps, bf.psc};
            int32_t *nd[2] = {bf.nd, bf.ndc};
            if ((rc = pd_run_to_peak_multi(both, 2, ms, pk, ps2, nd, (pd_stream)s))) break;
        }
        k_level_sums<<<1, 256, 0, s>>>(b, bf.qf, l > 0 ? bf.qc : nullptr, bf.y, bf.sums);
        double sums[2];
        cudaMemcpyAsync(sums, bf.sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(hq.data(), bf.qf, b * sizeof(double), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(hnd.data(), bf.nd, b * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (l > 0) {
            cudaMemcpyAsync(hqc.data(), bf.qc, b * sizeof(double), cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(hndc.data(), bf.ndc, b * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            set_error("MLMC batch failed: %s", cudaGetErrorString(cudaGetLastError()));
            rc = PD_ERR_CUDA;
            break;
        }
        const auto t1 = std::chrono::steady_clock::now();
        lv->cost_s += std::chrono::duration<double>(t1 - t0).count();
        lv->sum_y += sums[0];
        lv->sum_y2 += sums[1];
        lv->n += b;
        if (batch_sums) {
            const int64_t q = first / Bmax;
            batch_sums[3 * q + 0] = (double)b;
            batch_sums[3 * q + 1] = sums[0];
            batch_sums[3 * q + 2] = sums[1];
        }
        for (int q = 0; q < b; ++q) {
            lv->steps += hnd[q];
            lv->bond_updates += (int64_t)hnd[q] * mf.nb;
            if (l > 0) {
                lv->steps += hndc[q];
                lv->bond_updates += (int64_t)hndc[q] * mc.nb;
            }
            if (q_fine) q_fine[first + q] = hq[q];
            if (q_coarse) q_coarse[first + q] = l > 0 ? hqc[q] : 0.0;
        }
    }
    pd_state_destroy(sf);
    pd_state_destroy(sc);
    if (rc != PD_OK) return rc;
    level_stats(lv);
    return PD_OK;
}

}  // namespace pdi

using namespace pdi;

extern "C" int pd_mlmc_allocation(int32_t n_levels, const double *V, const double *C, double eps_s, int64_t *N) {
    PD_REQUIRE(n_levels >= 1 && V && C && N, "n_levels >= 1 and V, C, N are required");
    PD_REQUIRE(eps_s > 0, "eps_s must be positive");
    double S = 0.0;
    for (int l = 0; l < n_levels; ++l) {
        PD_REQUIRE(V[l] >= 0 && C[l] > 0, "V >= 0 and C > 0 required");
        S += std::sqrt(V[l] * C[l]);
    }
    for (int l = 0; l < n_levels; ++l) N[l] = (int64_t)std::floor(S * std::sqrt(V[l] / C[l]) / (eps_s * eps_s));
    return PD_OK;
}

extern "C" int mlmc_estimate(const pd_mlmc_cfg *cfg, pd_mlmc_result *out, double *q_fine, double *q_coarse,
                             double *batch_sums, pd_stream stream) {
    PD_REQUIRE(cfg && out, "cfg and out are required");
    PD_REQUIRE(cfg->n_levels >= 1 && cfg->n_levels <= PD_MAX_LEVELS, "n_levels out of range");
    PD_REQUIRE(cfg->grid && cfg->bc && cfg->max_steps && cfg->n_samples, "per-level arrays are required");
    PD_REQUIRE(cfg->batch >= 1 && cfg->batch <= 4096, "batch must be in [1, 4096]");
    for (int l = 0; l < cfg->n_levels; ++l) {
        PD_REQUIRE(cfg->n_samples[l] >= 0, "n_samples[%d] is negative", l);
        PD_REQUIRE(!cfg->first_sample || cfg->first_sample[l] >= 0, "first_sample[%d] is negative", l);
    }
    for (int l = 1; l < cfg->n_levels; ++l) {
        const pd_grid &f = cfg->grid[l], &c = cfg->grid[l - 1];
        PD_REQUIRE(f.nx == 2 * c.nx && f.ny == 2 * c.ny && (f.nz == 2 * c.nz || (f.nz == 1 && c.nz == 1)) &&
                       std::fabs(f.dx * 2.0 - c.dx) <= 1e-12 * c.dx,
                   "grid %d is not the 2x refinement of grid %d", l, l - 1);
    }
    cudaStream_t s = (cudaStream_t)stream;
    pd_field *field = nullptr;
    PD_TRY(pd_field_create(&cfg->grid[cfg->n_levels - 1], cfg->n_levels, &cfg->field, &field));
    pd_mlmc_result r;
    memset(&r, 0, sizeof(r));
    r.n_levels = cfg->n_levels;
    int rc = PD_OK;
    int64_t off = 0, boff = 0;
    for (int l = 0; l < cfg->n_levels && rc == PD_OK; ++l) {
        rc = run_level(cfg, field, l, &r.level[l], q_fine ? q_fine + off : nullptr,
                       q_coarse ? q_coarse + off : nullptr, batch_sums ? batch_sums + 3 * boff : nullptr, s);
        off += cfg->n_samples[l];
        const int64_t bl = std::min<int64_t>(cfg->batch, std::max<int64_t>(cfg->n_samples[l], 1));
        boff += (cfg->n_samples[l] + bl - 1) / bl;
    }
    pd_field_destroy(field);
    if (rc != PD_OK) return rc;
    estimator(&r);
    *out = r;
    return PD_OK;
}

extern "C" int mlmc_merge(int32_t n_levels, const int64_t *n_batches, const double *batch_sums, pd_mlmc_result *out) {
    PD_REQUIRE(n_levels >= 1 && n_levels <= PD_MAX_LEVELS, "n_levels out of range");
    PD_REQUIRE(n_batches && out, "n_batches and out are required");
    int64_t tot = 0;
    for (int l = 0; l < n_levels; ++l) {
        PD_REQUIRE(n_batches[l] >= 0, "n_batches[%d] is negative", l);
        tot += n_batches[l];
    }
    PD_REQUIRE(tot == 0 || batch_sums, "batch_sums is required");
    pd_mlmc_result r;
    memset(&r, 0, sizeof(r));
    r.n_levels = n_levels;
    int64_t q = 0;
    for (int l = 0; l < n_levels; ++l) {
        pd_mlmc_level &lv = r.level[l];
        for (int64_t k = 0; k < n_batches[l]; ++k, ++q) {
            const double nb = batch_sums[3 * q];
            PD_REQUIRE(nb >= 0.0 && nb == std::floor(nb), "batch %lld of level %d has a non-integer count",
                       (long long)k, l);
            lv.n += (int64_t)nb;
            lv.sum_y += batch_sums[3 * q + 1];
            lv.sum_y2 += batch_sums[3 * q + 2];
        }
        level_stats(&lv);
    }
    estimator(&r);
    *out = r;
    return PD_OK;
}

// Adaptive MLMC (Algorithm MLMC). Level l's samples are taken in id order
// across rounds (warm-up, then top-ups), each round one call of run_level.
extern "C" int mlmc_adaptive(const pd_mlmc_cfg *cfg, const pd_mlmc_adaptive_cfg *ad, pd_mlmc_result *out,
                             int32_t *L_used, double *bias, double *q_fine, double *q_coarse, int64_t cap,
                             pd_stream stream) {
    PD_REQUIRE(cfg && ad && out, "cfg, ad and out are required");
    PD_REQUIRE(cfg->n_levels >= 1 && cfg->n_levels <= PD_MAX_LEVELS, "n_levels out of range");
    PD_REQUIRE(cfg->grid && cfg->bc && cfg->max_steps, "per-level grids, bcs and max_steps are required");
    PD_REQUIRE(cfg->batch >= 1 && cfg->batch <= 4096, "batch must be in [1, 4096]");
    PD_REQUIRE(ad->eps_s > 0 && ad->eps_b > 0, "eps_s and eps_b must be positive");
    PD_REQUIRE(ad->m_dof > 1 && ad->alpha > 0, "m_dof > 1 and alpha > 0 required");
    PD_REQUIRE(ad->n_star >= 2, "n_star must be >= 2");
    for (int l = 1; l < cfg->n_levels; ++l) {
        const pd_grid &f = cfg->grid[l], &c = cfg->grid[l - 1];
        PD_REQUIRE(f.nx == 2 * c.nx && f.ny == 2 * c.ny && (f.nz == 2 * c.nz || (f.nz == 1 && c.nz == 1)) &&
                       std::fabs(f.dx * 2.0 - c.dx) <= 1e-12 * c.dx,
                   "grid %d is not the 2x refinement of grid %d", l, l - 1);
    }
    if (ad->cost_model)
        for (int l = 0; l < cfg->n_levels; ++l) PD_REQUIRE(ad->cost_model[l] > 0, "cost_model must be positive");
    cudaStream_t s = (cudaStream_t)stream;
    pd_field *field = nullptr;
    PD_TRY(pd_field_create(&cfg->grid[cfg->n_levels - 1], cfg->n_levels, &cfg->field, &field));

    const int Lmax = cfg->n_levels - 1;
    pd_mlmc_level acc[PD_MAX_LEVELS];
    memset(acc, 0, sizeof(acc));
    std::vector<double> qf[PD_MAX_LEVELS], qc[PD_MAX_LEVELS];
    int64_t ns[PD_MAX_LEVELS] = {0}, fs[PD_MAX_LEVELS] = {0};
    pd_mlmc_cfg c2 = *cfg;
    c2.n_samples = ns;
    c2.first_sample = fs;
    // take n more samples on level l (ids continue from the samples already taken)
    auto take = [&](int l, int64_t n) -> int {
        for (int k = 0; k <= Lmax; ++k) ns[k] = 0;
        ns[l] = n;
        fs[l] = (cfg->first_sample ? cfg->first_sample[l] : 0) + acc[l].n;
        pd_mlmc_level lv;
        std::vector<double> f(n), c(n);
        PD_TRY(run_level(&c2, field, l, &lv, f.data(), c.data(), nullptr, s));
        acc[l].n += lv.n;
        acc[l].sum_y += lv.sum_y;
        acc[l].sum_y2 += lv.sum_y2;
        acc[l].cost_s += lv.cost_s;
        acc[l].steps += lv.steps;
        acc[l].bond_updates += lv.bond_updates;
        qf[l].insert(qf[l].end(), f.begin(), f.end());
        qc[l].insert(qc[l].end(), c.begin(), c.end());
        return PD_OK;
    };
    auto mean_of = [&](int l) { return acc[l].n ? acc[l].sum_y / (double)acc[l].n : 0.0; };
    auto var_of = [&](int l) {
        const double m = mean_of(l);
        return acc[l].n ? acc[l].sum_y2 / (double)acc[l].n - m * m : 0.0;
    };
    int rc = PD_OK;
    int L = 0;
    double eb = 0.0;
    while (rc == PD_OK) {
        if ((rc = take(L, ad->n_star))) break;
        std::vector<double> V(L + 1), C(L + 1);
        std::vector<int64_t> Nh(L + 1);
        for (int l = 0; l <= L; ++l) {
            V[l] = std::max(var_of(l), 0.0);
            C[l] = ad->cost_model ? ad->cost_model[l] : std::max(acc[l].cost_s / (double)acc[l].n, 1e-12);
        }
        if ((rc = pd_mlmc_allocation(L + 1, V.data(), C.data(), ad->eps_s, Nh.data()))) break;
        for (int l = 0; l <= L && rc == PD_OK; ++l)
            if (Nh[l] > acc[l].n) rc = take(l, Nh[l] - acc[l].n);
        if (rc) break;
        eb = std::fabs(mean_of(L)) / (std::pow(ad->m_dof, ad->alpha) - 1.0);
        if (eb < ad->eps_b || L >= Lmax) break;
        ++L;
    }
    pd_field_destroy(field);
    if (rc != PD_OK) return rc;
    pd_mlmc_result r;
    memset(&r, 0, sizeof(r));
    r.n_levels = L + 1;
    int64_t total = 0;
    for (int l = 0; l <= L; ++l) {
        pd_mlmc_level &lv = acc[l];
        lv.mean = mean_of(l);
        lv.var = var_of(l);
        lv.var_unbiased = lv.n > 1 ? lv.var * (double)lv.n / (double)(lv.n - 1) : 0.0;
        r.level[l] = lv;
        r.q_ml += lv.mean;
        r.var_ml += lv.var / (double)lv.n;
        total += lv.n;
    }
    *out = r;
    if (L_used) *L_used = L;
    if (bias) *bias = eb;
    if (q_fine || q_coarse) {
        if (total > cap) {
            set_error("the run took %lld samples, more than cap = %lld", (long long)total, (long long)cap);
            return PD_ERR_CAP;
        }
        int64_t o = 0;
        for (int l = 0; l <= L; ++l)
            for (size_t k = 0; k < qf[l].size(); ++k, ++o) {
                if (q_fine) q_fine[o] = qf[l][k];
                if (q_coarse) q_coarse[o] = qc[l][k];
            }
    }
    return PD_OK;
}
