// pd_tune.cu -- launch-schedule autotuner for the step kernels: times every
// candidate (brick rows by x bz, warps q sharing a row pair's half-stencil)
// of a mesh and batch size on the GPU and keeps the fastest. A schedule only
// regroups the same arithmetic (results agree to rounding), so the choice is
// purely one of speed: bricks that fit the grid waste fewer slots on ragged
// edges, larger bricks stage fewer halo records per node, and q trades
// occupancy for per-warp work.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pd_internal.cuh"

namespace pdi {

struct TuneEntry {
    pd_schedule s;
    double us;
};

static std::mutex g_tune_mu;
static std::map<std::string, TuneEntry> g_tune_cache;

static std::string tune_key(const pd_grid *g, const pd_material *mat, int batch, int dev) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%d|%d %d %d|%.17g %.17g|%d %d %d|%d|%d %d", dev, g->nx, g->ny, g->nz, g->dx,
             g->m_ratio, g->notch, g->notch_x2, g->notch_y2, batch, mat->law, mat->precision);
    return buf;
}

// Slots of the brick layout per grid node (ragged bricks at the grid's edges).
static double slot_ratio(const pd_grid *g, int by, int bz) {
    const double slots = (double)((g->nx + 7) / 8 * 8) * ((g->ny + by - 1) / by * by) * ((g->nz + bz - 1) / bz * bz);
    return slots / ((double)g->nx * g->ny * g->nz);
}

// Candidates: the five bricks with the least ragged-edge waste (larger bricks
// first among equals: they stage fewer halo records per node), each with
// every warp split that fits a block and, for batches on the stencil path,
// one or two samples per block.
static std::vector<pd_schedule> candidates(const pd_grid *g, const pd_material *mat, int batch) {
    std::vector<pd_schedule> out;
    const double m2 = g->m_ratio * g->m_ratio;
    const bool stencil = mat->precision == PD_PREC_MIXED && m2 >= 9.0 && m2 < 10.0;
    std::vector<std::pair<double, std::pair<int, int>>> bricks;
    if (stencil) {
        static const int list[][2] = {{2, 2},  {4, 2}, {2, 4},  {4, 4}, {8, 2},  {2, 8}, {8, 4},  {4, 8},
                                      {6, 2},  {2, 6}, {6, 4},  {4, 6}, {10, 2}, {2, 10}, {12, 2}, {2, 12},
                                      {16, 2}, {2, 16}, {8, 1}, {4, 1}, {2, 1},  {6, 1}};
        for (const auto &b : list) {
            if ((size_t)14 * (b[0] + 6) * (b[1] + 6) * 32 > 160 * 1024) continue;
            bricks.push_back({slot_ratio(g, b[0], b[1]), {b[0], b[1]}});
        }
    } else {
        static const int list[][2] = {{8, 8}, {8, 4}, {4, 4}, {4, 2}, {2, 2}, {2, 1}, {1, 1}};
        for (const auto &b : list) bricks.push_back({slot_ratio(g, b[0], b[1]), {b[0], b[1]}});
    }
    std::stable_sort(bricks.begin(), bricks.end(), [](const auto &x, const auto &y) {
        if (x.first != y.first) return x.first < y.first;
        return x.second.first * x.second.second > y.second.first * y.second.second;
    });
    int kept = 0;
    for (const auto &b : bricks) {
        if (kept == 5) break;
        ++kept;
        const int by = b.second.first, bz = b.second.second;
        if (!stencil) {
            out.push_back(pd_schedule{by, bz, 0, 0, 0});
            continue;
        }
        const int wpb = by * bz / 2;
        const int zhalo = g->nz == 1 ? 0 : 6;
        for (int ns = batch >= 2 ? 2 : 1; ns >= 1; --ns) {
            if ((size_t)14 * (by + 6) * (bz + zhalo) * 32 * ns > 200 * 1024) continue;
            for (int q = 1; q <= (g->nz == 1 ? 1 : 4); q *= 2)  // the planar stencil runs at q = 1
                if (32 * wpb * q <= (q == 2 && ns == 1 ? 256 : 512)) out.push_back(pd_schedule{by, bz, q, ns, 0});
        }
    }
    return out;
}

}  // namespace pdi

using namespace pdi;

extern "C" int pd_autotune(const pd_grid *g, const int32_t *row_ptr, const int32_t *col, int64_t n_bonds,
                           const pd_material *mat, const pd_bc *bc, int32_t batch, int32_t trial_steps,
                           pd_schedule *best, double *best_us) {
    PD_REQUIRE(g && row_ptr && col && mat && bc && best, "grid, CSR, material, bc and best are required");
    PD_REQUIRE(trial_steps >= 1 && trial_steps <= 10000, "trial_steps must be in [1, 10000]");
    int dev = 0;
    PD_CHECK_CUDA(cudaGetDevice(&dev));
    const std::string key = tune_key(g, mat, batch, dev);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *best = it->second.s;
            if (best_us) *best_us = it->second.us;
            return PD_OK;
        }
    }
    const std::vector<pd_schedule> cand = candidates(g, mat, batch);
    PD_REQUIRE(!cand.empty(), "no candidate schedule for this grid");
    cudaStream_t s;
    PD_CHECK_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    TuneEntry win{{0, 0, 0, 0, 0}, INFINITY};
    for (const pd_schedule &c : cand) {
        pd_state *st = nullptr;
        if (pd_state_create_sched(g, row_ptr, col, n_bonds, mat, bc, batch, &c, &st) != PD_OK) continue;
        float ms = 0.f;
        bool ok = pd_state_reset(st, nullptr, nullptr, (pd_stream)s) == PD_OK &&
                  pd_step(st, 2, nullptr, (pd_stream)s) == PD_OK && cudaEventRecord(e0, s) == cudaSuccess &&
                  pd_step(st, trial_steps, nullptr, (pd_stream)s) == PD_OK && cudaEventRecord(e1, s) == cudaSuccess &&
                  cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        pd_state_destroy(st);
        if (!ok) {
            cudaGetLastError();  // a candidate that cannot run (resources) is skipped
            continue;
        }
        const double us = 1e3 * ms / trial_steps;
        if (us < win.us) win = TuneEntry{c, us};
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    PD_REQUIRE(std::isfinite(win.us), "no candidate schedule could run");
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = win;
    }
    *best = win.s;
    if (best_us) *best_us = win.us;
    return PD_OK;
}
