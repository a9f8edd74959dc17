// batch.cu -- many independent star fields in one persistent launch (Section 2.2:
// a grid of simulations over (<M*>, gamma, kappa_*, kappa_c), each its own map),
// replayed as a CUDA graph, with an autotuner for the launch shape.
//
// The work queue holds one item per (field, ray tile); fields are ordered by the
// cost of one tile (stars x rays per tile), heaviest first, so the last items
// handed out are the cheapest and CTAs finish together (longest-processing-time
// ordering).  The graph holds the map clears, the counter clears and the
// persistent kernel; it is captured once per launch shape on a private stream
// and launched on the caller's stream.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "mlens_internal.h"

using namespace mlens;

struct mlens_batch {
    int device = -1;
    int nfields = 0;
    uint32_t flags = 0;
    std::vector<ShootArgs> h_fields;      // per field (stats/counts pointers filled)
    std::vector<mlens_grid> rays, srcs;
    std::vector<uint32_t *> counts;
    std::vector<int64_t> n_pad;
    ShootArgs *d_fields = nullptr;
    int *d_order = nullptr;
    int64_t *d_begin = nullptr;
    unsigned long long *d_counter = nullptr;
    unsigned long long *d_stats = nullptr;  // 3 per field
    int pairs_per_thread = 4;
    int star_stage = 256;
    int fma_pairs = kDefaultFmaPairs;
    int64_t total = 0;
    int grid = 0;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

int bfail(int code, const std::string &m)
{
    set_last_error(m);
    return code;
}

int bcuda(cudaError_t e, const char *what)
{
    set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
    clear_pending_error();
    return e == cudaErrorMemoryAllocation ? MLENS_ERR_NOMEM : MLENS_ERR_CUDA;
}

#define BCUDA(call, what)                               \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return bcuda(e_, what);  \
    } while (0)

bool grid_ok(const mlens_grid &g, bool rays)
{
    if (!(std::isfinite(g.x0) && std::isfinite(g.x1) && std::isfinite(g.y0) && std::isfinite(g.y1))) return false;
    if (!(g.x1 > g.x0 && g.y1 > g.y0) || g.nx < 1 || g.ny < 1) return false;
    if (rays) return g.nx <= (1 << 20) && g.ny <= (1 << 20);
    return (int64_t)g.nx * g.ny <= (int64_t(1) << 30);
}

void drop_graph(mlens_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Work-queue tables for the current launch shape: LPT order and item offsets.
int build_tables(mlens_batch *b)
{
    const int nf = b->nfields;
    std::vector<int64_t> tiles(nf), cost(nf);
    for (int f = 0; f < nf; ++f) {
        tiles[f] = tiles_of(b->h_fields[f].rays, b->pairs_per_thread);
        cost[f] = std::max<int64_t>(b->n_pad[f], 1);
    }
    std::vector<int> order(nf);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<int64_t> begin(nf + 1, 0);
    for (int k = 0; k < nf; ++k) begin[k + 1] = begin[k] + tiles[order[k]];
    b->total = begin[nf];
    BCUDA(cudaMemcpy(b->d_order, order.data(), sizeof(int) * nf, cudaMemcpyHostToDevice), "cudaMemcpy(order)");
    BCUDA(cudaMemcpy(b->d_begin, begin.data(), sizeof(int64_t) * (nf + 1), cudaMemcpyHostToDevice),
          "cudaMemcpy(begin)");
    BCUDA(batch_grid_size(b->pairs_per_thread, b->star_stage, &b->grid, b->fma_pairs), "occupancy query");
    return MLENS_OK;
}

int capture(mlens_batch *b)
{
    drop_graph(b);
    BatchLaunch L;
    L.grid = b->grid;
    L.fields = b->d_fields;
    L.order = b->d_order;
    L.begin = b->d_begin;
    L.nfields = b->nfields;
    L.total = b->total;
    L.counter = b->d_counter;
    BCUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    cudaError_t e = cudaSuccess;
    if (!(b->flags & MLENS_ACCUMULATE))
        for (int f = 0; f < b->nfields && e == cudaSuccess; ++f)
            e = cudaMemsetAsync(b->counts[f], 0, (size_t)b->srcs[f].nx * b->srcs[f].ny * sizeof(uint32_t), b->cap);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_stats, 0, sizeof(unsigned long long) * 3 * b->nfields, b->cap);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), b->cap);
    if (e == cudaSuccess) e = launch_shoot_batch(L, b->pairs_per_thread, b->star_stage, b->cap, b->fma_pairs);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda(e, "batch graph capture");
    }
    if (e2 != cudaSuccess) return bcuda(e2, "cudaStreamEndCapture");
    b->graph = g;
    BCUDA(cudaGraphInstantiate(&b->exec, b->graph, 0), "cudaGraphInstantiate");
    return MLENS_OK;
}

int set_shape(mlens_batch *b, int rpt, int stage, int fma)
{
    if (rpt != 4 && rpt != 8) return bfail(MLENS_ERR_ARG, "rays_per_thread must be 4 or 8");
    if (stage != 128 && stage != 256 && stage != 512) return bfail(MLENS_ERR_ARG, "star_stage must be 128, 256 or 512");
    if (fma != 0 && fma != 1) return bfail(MLENS_ERR_ARG, "fma_pairs must be 0 or 1");
    if (b->pairs_per_thread == rpt / 2 && b->star_stage == stage && b->fma_pairs == fma && b->exec) return MLENS_OK;
    // the tables are rewritten below: no launch of the old shape may still read them
    BCUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    b->pairs_per_thread = rpt / 2;
    b->star_stage = stage;
    b->fma_pairs = fma;
    drop_graph(b);
    return build_tables(b);
}

// process-wide cache of tuned shapes, keyed by device and workload signature;
// also read from / appended to the file named by MLENS_TUNE_CACHE, if set
std::mutex g_tune_mu;
struct Shape {
    int rpt, stage, fma;
};
std::map<std::string, Shape> g_tune;
bool g_tune_file_read = false;

std::string signature(const mlens_batch *b)
{
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, b->device);
    // bucket the star counts by powers of two and the ray counts exactly
    std::map<int, int> hist;
    for (int f = 0; f < b->nfields; ++f) hist[(int)std::ceil(std::log2((double)std::max<int64_t>(b->n_pad[f], 1)))]++;
    std::string s = std::string(p.name) + "|sm" + std::to_string(p.multiProcessorCount) + "|nf" +
                    std::to_string(b->nfields) + "|r" + std::to_string(b->rays[0].nx) + "x" + std::to_string(b->rays[0].ny);
    for (auto &kv : hist) s += "|" + std::to_string(kv.first) + ":" + std::to_string(kv.second);
    for (char &c : s)
        if (c == ' ') c = '_';
    return s;
}

void read_tune_file()
{
    if (g_tune_file_read) return;
    g_tune_file_read = true;
    const char *path = getenv("MLENS_TUNE_CACHE");
    if (!path) return;
    FILE *fh = fopen(path, "r");
    if (!fh) return;
    char key[1024];
    int rpt, st, fm;
    double ms;
    while (fscanf(fh, "%1023s %d %d %d %lf", key, &rpt, &st, &fm, &ms) == 5) g_tune[key] = {rpt, st, fm};
    fclose(fh);
}

void append_tune_file(const std::string &key, int rpt, int st, int fm, double ms)
{
    const char *path = getenv("MLENS_TUNE_CACHE");
    if (!path) return;
    FILE *fh = fopen(path, "a");
    if (!fh) return;
    fprintf(fh, "%s %d %d %d %.6f\n", key.c_str(), rpt, st, fm, ms);
    fclose(fh);
}

}  // namespace

extern "C" {

int mlens_batch_create(mlens_batch **out, mlens_ctx *const *ctxs, int32_t nfields, const mlens_grid *rays,
                       const mlens_grid *srcs, uint32_t *const *counts_dev, uint32_t flags)
{
    if (!out) return bfail(MLENS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nfields < 1 || nfields > (1 << 20)) return bfail(MLENS_ERR_ARG, "nfields must be in [1, 2^20]");
    if (!ctxs || !rays || !srcs || !counts_dev) return bfail(MLENS_ERR_ARG, "ctxs, rays, srcs, counts_dev must be non-NULL");
    if (flags & ~MLENS_ACCUMULATE) return bfail(MLENS_ERR_ARG, "unknown flag bits");
    for (int f = 0; f < nfields; ++f) {
        if (!ctxs[f]) return bfail(MLENS_ERR_ARG, "field " + std::to_string(f) + ": context is NULL");
        if (!grid_ok(rays[f], true)) return bfail(MLENS_ERR_ARG, "field " + std::to_string(f) + ": bad rays grid");
        if (!grid_ok(srcs[f], false)) return bfail(MLENS_ERR_ARG, "field " + std::to_string(f) + ": bad source grid");
        if (!counts_dev[f] || ((uintptr_t)counts_dev[f] & 3u))
            return bfail(MLENS_ERR_ARG, "field " + std::to_string(f) + ": counts must be non-NULL, 4-byte aligned");
        if (tiles_of(make_ray_grid(rays[f]), 2) > (int64_t(1) << 40))
            return bfail(MLENS_ERR_ARG, "field " + std::to_string(f) + ": too many rays");
    }
    int dev = -1;
    BCUDA(cudaGetDevice(&dev), "cudaGetDevice");
    for (int f = 0; f < nfields; ++f)
        if (ctxs[f]->device != dev)
            return bfail(MLENS_ERR_STATE, "field " + std::to_string(f) + ": context lives on another device");
    mlens_batch *b = new mlens_batch();
    b->device = dev;
    b->nfields = nfields;
    b->flags = flags;
    b->rays.assign(rays, rays + nfields);
    b->srcs.assign(srcs, srcs + nfields);
    b->counts.assign(counts_dev, counts_dev + nfields);
    b->h_fields.resize(nfields);
    b->n_pad.resize(nfields);
    cudaError_t e = dmalloc(&b->d_fields, sizeof(ShootArgs) * nfields);
    if (e == cudaSuccess) e = dmalloc(&b->d_order, sizeof(int) * nfields);
    if (e == cudaSuccess) e = dmalloc(&b->d_begin, sizeof(int64_t) * (nfields + 1));
    if (e == cudaSuccess) e = dmalloc(&b->d_counter, sizeof(unsigned long long));
    if (e == cudaSuccess) e = dmalloc(&b->d_stats, sizeof(unsigned long long) * 3 * nfields);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        int rc = bcuda(e, "mlens_batch_create device setup");
        mlens_batch_destroy(b);
        return rc;
    }
    for (int f = 0; f < nfields; ++f) {
        ShootArgs a{};
        a.stars = ctxs[f]->d_stars;
        a.nstars = ctxs[f]->n_pad;
        a.rays = make_ray_grid(rays[f]);
        a.bin = make_bin_grid(srcs[f]);
        a.lens = ctxs[f]->lens;
        a.counts = counts_dev[f];
        a.stats = b->d_stats + 3 * f;
        a.beta_out = nullptr;
        b->h_fields[f] = a;
        b->n_pad[f] = ctxs[f]->n_pad;
    }
    e = cudaMemcpy(b->d_fields, b->h_fields.data(), sizeof(ShootArgs) * nfields, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        int rc = bcuda(e, "cudaMemcpy(field descriptors)");
        mlens_batch_destroy(b);
        return rc;
    }
    int rc = build_tables(b);
    if (rc != MLENS_OK) {
        mlens_batch_destroy(b);
        return rc;
    }
    *out = b;
    return MLENS_OK;
}

int mlens_batch_set_tuning(mlens_batch *b, int32_t rays_per_thread, int32_t star_stage, int32_t fma_pairs)
{
    if (!b) return bfail(MLENS_ERR_ARG, "batch is NULL");
    return set_shape(b, rays_per_thread, star_stage ? star_stage : 256, fma_pairs);
}

int mlens_batch_run(mlens_batch *b, mlens_stats *stats_host, void *stream)
{
    if (!b) return bfail(MLENS_ERR_ARG, "batch is NULL");
    int dev = -1;
    BCUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != b->device) return bfail(MLENS_ERR_STATE, "the batch belongs to another CUDA device than the current one");
    if (!b->exec) {
        int rc = capture(b);
        if (rc != MLENS_OK) return rc;
    }
    cudaStream_t s = (cudaStream_t)stream;
    BCUDA(cudaGraphLaunch(b->exec, s), "cudaGraphLaunch");
    if (stats_host) {
        std::vector<unsigned long long> h(3 * (size_t)b->nfields);
        BCUDA(cudaMemcpyAsync(h.data(), b->d_stats, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost, s),
              "cudaMemcpyAsync(batch stats)");
        BCUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
        for (int f = 0; f < b->nfields; ++f) {
            stats_host[f].rays_total = (uint64_t)b->rays[f].nx * (uint64_t)b->rays[f].ny;
            stats_host[f].rays_binned = h[3 * f];
            stats_host[f].rays_out = h[3 * f + 1];
            stats_host[f].rays_nan = h[3 * f + 2];
        }
    }
    return MLENS_OK;
}

int mlens_batch_tune(mlens_batch *b, void *stream, int32_t *rays_per_thread, int32_t *star_stage, int32_t *fma_pairs,
                     double *best_ms)
{
    if (!b) return bfail(MLENS_ERR_ARG, "batch is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    const std::string key = signature(b);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        read_tune_file();
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            int rc = set_shape(b, it->second.rpt, it->second.stage, it->second.fma);
            if (rc != MLENS_OK) return rc;
            if (rays_per_thread) *rays_per_thread = it->second.rpt;
            if (star_stage) *star_stage = it->second.stage;
            if (fma_pairs) *fma_pairs = it->second.fma;
            if (best_ms) *best_ms = -1.0;  // taken from the cache, not timed now
            return MLENS_OK;
        }
    }
    const int cand_rpt[2] = {8, 4};
    const int cand_st[2] = {256, 512};
    cudaEvent_t e0, e1;
    BCUDA(cudaEventCreate(&e0), "cudaEventCreate");
    BCUDA(cudaEventCreate(&e1), "cudaEventCreate");
    double best = 1e300;
    int brpt = 8, bst = 256, bfm = 0;
    int rc = MLENS_OK;
    for (int c = 0; c < 8 && rc == MLENS_OK; ++c) {
        const int i = (c / 2) % 2, j = c % 2, fm = c / 4;
        {
            if ((rc = set_shape(b, cand_rpt[i], cand_st[j], fm)) != MLENS_OK) break;
            if ((rc = mlens_batch_run(b, nullptr, stream)) != MLENS_OK) break;  // warm-up + capture
            double tmin = 1e300;
            for (int r = 0; r < 2; ++r) {
                cudaEventRecord(e0, s);
                if ((rc = mlens_batch_run(b, nullptr, stream)) != MLENS_OK) break;
                cudaEventRecord(e1, s);
                cudaError_t e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) {
                    rc = bcuda(e, "cudaEventSynchronize");
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                tmin = std::min(tmin, (double)ms);
            }
            if (rc == MLENS_OK && tmin < best) {
                best = tmin;
                brpt = cand_rpt[i];
                bst = cand_st[j];
                bfm = fm;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != MLENS_OK) return rc;
    if ((rc = set_shape(b, brpt, bst, bfm)) != MLENS_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = {brpt, bst, bfm};
        append_tune_file(key, brpt, bst, bfm, best);
    }
    if (rays_per_thread) *rays_per_thread = brpt;
    if (star_stage) *star_stage = bst;
    if (fma_pairs) *fma_pairs = bfm;
    if (best_ms) *best_ms = best;
    return MLENS_OK;
}

void mlens_batch_destroy(mlens_batch *b)
{
    if (!b) return;
    if (b->d_fields || b->cap) cudaDeviceSynchronize();
    drop_graph(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    dfree(b->d_fields);
    dfree(b->d_order);
    dfree(b->d_begin);
    dfree(b->d_counter);
    dfree(b->d_stats);
    delete b;
}

int mlens_shoot_batch(mlens_ctx *const *ctxs, int32_t nfields, const mlens_grid *rays, const mlens_grid *srcs,
                      uint32_t *const *counts_dev, uint32_t flags, mlens_stats *stats_host, void *stream)
{
    mlens_batch *b = nullptr;
    int rc = mlens_batch_create(&b, ctxs, nfields, rays, srcs, counts_dev, flags);
    if (rc != MLENS_OK) return rc;
    rc = mlens_batch_run(b, stats_host, stream);
    if (rc == MLENS_OK && !stats_host) {
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);  // the batch's tables must outlive the launch
        if (e != cudaSuccess) rc = bcuda(e, "cudaStreamSynchronize");
    }
    mlens_batch_destroy(b);
    return rc;
}

}  // extern "C"
