// Kernel shapes and the autotuner.
//
// The paper fixes no kernel shape (Sec. 3.1.1 tiles the data points through shared memory for a
// block of queries and leaves the sizes open), so the FP32 kernels take theirs from an
// aidw_tune_config: phase-2 queries per thread (the query-block size), phase-2 tile depth, the
// k-list register length, and for batches the points per phase-2 work unit and the persistent
// CTAs per SM. The autotuner times candidates on the caller's own workload by coordinate search
// (one field at a time, from the current shape, keeping a change only if it is faster by more
// than the noise margin) and records winners in a process-wide cache keyed by device and
// workload size class, which can be saved to and loaded from a JSON-lines file.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "aidw_runtime.h"

namespace aidw {

aidw_tune_config tune_default()
{
    aidw_tune_config c{};
    c.queries_per_thread = 2;
    c.tile_points = 512;
    c.knn_list = 0;
    c.split_points = 65536;
    c.ctas_per_sm = 0;
    c.knn_queries_per_thread = 2;
    c.unit_order = 0;
    return c;
}

bool tune_valid(const aidw_tune_config &c)
{
    const bool qw = c.queries_per_thread == 2 || c.queries_per_thread == 4 ||
                    c.queries_per_thread == 8;
    const bool tw = c.tile_points == 256 || c.tile_points == 512;
    const bool kl = c.knn_list == 0 || c.knn_list == 16 || c.knn_list == 32;
    const bool sp = c.split_points >= kPadPoints && c.split_points <= (1 << 22) &&
                    c.split_points % kPadPoints == 0;
    const bool ct = c.ctas_per_sm >= 0 && c.ctas_per_sm <= 32;
    const bool kq = c.knn_queries_per_thread == 0 || c.knn_queries_per_thread == 2 ||
                    c.knn_queries_per_thread == 4;
    const bool uo = c.unit_order == 0 || c.unit_order == 1;
    return qw && tw && kl && sp && ct && kq && uo && c.reserved == 0;
}

namespace {

bool same(const aidw_tune_config &a, const aidw_tune_config &b)
{
    return a.queries_per_thread == b.queries_per_thread && a.tile_points == b.tile_points &&
           a.knn_list == b.knn_list && a.split_points == b.split_points &&
           a.ctas_per_sm == b.ctas_per_sm &&
           a.knn_queries_per_thread == b.knn_queries_per_thread &&
           a.unit_order == b.unit_order;
}

// ---- process-wide cache ----------------------------------------------------------------------

struct CacheEntry {
    aidw_tune_config cfg;
    double ms;
};

std::mutex g_cache_mu;
std::map<std::string, CacheEntry> g_cache;

bool key_valid(const char *key)
{
    if (!key)
        return false;
    const size_t n = std::strlen(key);
    if (n == 0 || n > 255)
        return false;
    for (size_t i = 0; i < n; ++i) {
        const unsigned char ch = static_cast<unsigned char>(key[i]);
        if (ch < 0x20 || ch > 0x7e || ch == '"' || ch == '\\')
            return false;
    }
    return true;
}

// Parses one line written by aidw_tune_cache_save (whitespace between tokens is free).
bool parse_line(const char *line, std::string *key, CacheEntry *e)
{
    char kbuf[256];
    aidw_tune_config c{};
    double ms = 0.0;
    int used = -1;
    const int got = std::sscanf(
        line,
        " { \"key\" : \"%255[^\"]\" , \"queries_per_thread\" : %d , \"tile_points\" : %d , "
        "\"knn_list\" : %d , \"split_points\" : %d , \"ctas_per_sm\" : %d , "
        "\"knn_queries_per_thread\" : %d , \"unit_order\" : %d , \"ms\" : %lf } %n",
        kbuf, &c.queries_per_thread, &c.tile_points, &c.knn_list, &c.split_points,
        &c.ctas_per_sm, &c.knn_queries_per_thread, &c.unit_order, &ms, &used);
    if (got != 9 || used < 0 || line[used] != '\0')
        return false;
    if (!key_valid(kbuf) || !tune_valid(c) || !std::isfinite(ms))
        return false;
    *key = kbuf;
    e->cfg = c;
    e->ms = ms;
    return true;
}

bool blank(const char *s)
{
    for (; *s; ++s)
        if (*s != ' ' && *s != '\t' && *s != '\r' && *s != '\n')
            return false;
    return true;
}

// ---- workload keys ---------------------------------------------------------------------------

int log2_round(double v)
{
    return v >= 1.0 ? static_cast<int>(std::lround(std::log2(v))) : 0;
}

std::string device_tag(aidw_ctx *ctx)
{
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, ctx_device(ctx));
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, ctx_device(ctx));
    char b[64];
    std::snprintf(b, sizeof(b), "dev=sm_%d%d x%d", major, minor, ctx_sm_count(ctx));
    return b;
}

// ---- timing ----------------------------------------------------------------------------------

struct Timer {
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    bool ok = false;
    Timer()
    {
        ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    }
    ~Timer()
    {
        if (e0)
            cudaEventDestroy(e0);
        if (e1)
            cudaEventDestroy(e1);
        if (st)
            cudaStreamDestroy(st);
    }
};

// Coordinate search: for each field in turn, try its other values on the current best shape and
// keep a value only if it is faster by more than kMargin.
constexpr double kMargin = 0.005;

struct Field {
    int32_t aidw_tune_config::*member;
    std::vector<int32_t> values;
};

template <typename Measure, typename Skip>
int coordinate_search(const std::vector<Field> &fields, aidw_tune_config *best, double *best_ms,
                      Measure measure, Skip skip)
{
    double t0 = 0.0;
    int rc = measure(*best, &t0);
    if (rc)
        return rc;
    for (const Field &f : fields) {
        const aidw_tune_config start = *best;
        for (int32_t v : f.values) {
            aidw_tune_config c = start;
            c.*f.member = v;
            if (same(c, start) || same(c, *best) || skip(c, *best))
                continue;
            double t = 0.0;
            rc = measure(c, &t);
            if (rc)
                return rc;
            if (t < t0 * (1.0 - kMargin)) {
                *best = c;
                t0 = t;
            }
        }
    }
    *best_ms = t0;
    return AIDW_OK;
}

}  // namespace
}  // namespace aidw

using namespace aidw;

extern "C" {

int aidw_tune_config_default(aidw_tune_config *out)
{
    if (!out)
        return AIDW_ERR_INVALID_ARG;
    *out = tune_default();
    return AIDW_OK;
}

int aidw_tune_config_check(const aidw_tune_config *cfg)
{
    return cfg && tune_valid(*cfg) ? AIDW_OK : AIDW_ERR_INVALID_ARG;
}

int aidw_set_tune_config(aidw_ctx *ctx, const aidw_tune_config *cfg)
{
    if (!ctx || !cfg || !tune_valid(*cfg))
        return AIDW_ERR_INVALID_ARG;
    ctx_set_tune(ctx, *cfg);
    return AIDW_OK;
}

int aidw_get_tune_config(aidw_ctx *ctx, aidw_tune_config *out)
{
    if (!ctx || !out)
        return AIDW_ERR_INVALID_ARG;
    *out = ctx_tune(ctx);
    return AIDW_OK;
}

int aidw_tune_cache_put(const char *key, const aidw_tune_config *cfg, double ms)
{
    if (!key_valid(key) || !cfg || !tune_valid(*cfg) || !std::isfinite(ms))
        return AIDW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(g_cache_mu);
    g_cache[key] = CacheEntry{*cfg, ms};
    return AIDW_OK;
}

int aidw_tune_cache_get(const char *key, aidw_tune_config *out, double *ms)
{
    if (!key_valid(key) || !out)
        return AIDW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(g_cache_mu);
    auto it = g_cache.find(key);
    if (it == g_cache.end())
        return AIDW_ERR_NOT_FOUND;
    *out = it->second.cfg;
    if (ms)
        *ms = it->second.ms;
    return AIDW_OK;
}

int aidw_tune_cache_clear(void)
{
    std::lock_guard<std::mutex> g(g_cache_mu);
    g_cache.clear();
    return AIDW_OK;
}

int aidw_tune_cache_size(void)
{
    std::lock_guard<std::mutex> g(g_cache_mu);
    return static_cast<int>(g_cache.size());
}

int aidw_tune_cache_save(const char *path)
{
    if (!path || !*path)
        return AIDW_ERR_INVALID_ARG;
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f)
        return AIDW_ERR_NOT_FOUND;
    bool ok = true;
    {
        std::lock_guard<std::mutex> g(g_cache_mu);
        for (const auto &kv : g_cache) {
            const aidw_tune_config &c = kv.second.cfg;
            ok &= std::fprintf(f,
                               "{\"key\": \"%s\", \"queries_per_thread\": %d, \"tile_points\": "
                               "%d, \"knn_list\": %d, \"split_points\": %d, \"ctas_per_sm\": %d, "
                               "\"knn_queries_per_thread\": %d, \"unit_order\": %d, "
                               "\"ms\": %.6f}\n",
                               kv.first.c_str(), c.queries_per_thread, c.tile_points,
                               c.knn_list, c.split_points, c.ctas_per_sm,
                               c.knn_queries_per_thread, c.unit_order, kv.second.ms) > 0;
        }
    }
    ok &= std::fclose(f) == 0;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return AIDW_ERR_INVALID_ARG;
    }
    return AIDW_OK;
}

int aidw_tune_cache_load(const char *path)
{
    if (!path || !*path)
        return AIDW_ERR_INVALID_ARG;
    FILE *f = std::fopen(path, "r");
    if (!f)
        return AIDW_ERR_NOT_FOUND;
    std::map<std::string, CacheEntry> got;
    char line[1024];
    bool ok = true;
    while (std::fgets(line, sizeof(line), f)) {
        const size_t n = std::strlen(line);
        if (n == sizeof(line) - 1 && line[n - 1] != '\n') {
            ok = false;  // longer than any line the cache writes
            break;
        }
        if (blank(line))
            continue;
        std::string key;
        CacheEntry e;
        if (!parse_line(line, &key, &e)) {
            ok = false;
            break;
        }
        got[key] = e;
    }
    std::fclose(f);
    if (!ok)
        return AIDW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(g_cache_mu);
    for (const auto &kv : got)
        g_cache[kv.first] = kv.second;
    return AIDW_OK;
}

int aidw_autotune_interpolate(aidw_ctx *ctx, aidw_dataset ds, const void *qx, const void *qy,
                              int64_t m, const aidw_params *p, void *out, int32_t reps,
                              uint32_t flags, aidw_tune_config *best, double *best_ms)
{
    if (!ctx || !p || !best || !best_ms || reps < 1 || m < 1 || p->precision != AIDW_F32C)
        return AIDW_ERR_INVALID_ARG;
    DatasetDev dev;
    double r_exp;
    if (!dataset_lookup(ctx, ds, &dev, &r_exp))
        return AIDW_ERR_NOT_FOUND;
    int rc = validate_params(p, dev.n);
    if (rc)
        return rc;
    const int device = ctx_device(ctx);
    if (pointer_kind(qx, device) != 1 || pointer_kind(qy, device) != 1 ||
        pointer_kind(out, device) != 1)
        return AIDW_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess)
        return AIDW_ERR_CUDA;
    char kb[192];
    std::snprintf(kb, sizeof(kb), "interpolate %s n=2^%d m=2^%d k=%d", device_tag(ctx).c_str(),
                  log2_round(static_cast<double>(dev.n)), log2_round(static_cast<double>(m)),
                  p->k);
    Timer tm;
    if (!tm.ok)
        return AIDW_ERR_CUDA;
    auto run = [&](const aidw_tune_config &c) {
        return interpolate_impl(ctx, ds, qx, qy, m, p, out, nullptr, nullptr, tm.st, 0, 0, &c);
    };
    aidw_tune_config cfg = ctx_tune(ctx);
    double ms = -1.0;
    if ((flags & AIDW_TUNE_CACHE) && aidw_tune_cache_get(kb, &cfg, nullptr) == AIDW_OK) {
        rc = run(cfg);
        if (rc == AIDW_OK && cudaStreamSynchronize(tm.st) != cudaSuccess)
            rc = AIDW_ERR_CUDA;
        if (rc == AIDW_OK)
            rc = consume_device_error(ctx, tm.st);
    } else {
        auto measure = [&](const aidw_tune_config &c, double *t) {
            int r = run(c);  // warm-up
            float best_run = 1e30f;
            for (int i = 0; i < reps && r == AIDW_OK; ++i) {
                cudaEventRecord(tm.e0, tm.st);
                r = run(c);
                cudaEventRecord(tm.e1, tm.st);
                float e = 0.0f;
                if (r == AIDW_OK && (cudaEventSynchronize(tm.e1) != cudaSuccess ||
                                     cudaEventElapsedTime(&e, tm.e0, tm.e1) != cudaSuccess))
                    r = AIDW_ERR_CUDA;
                best_run = e < best_run ? e : best_run;
            }
            if (r == AIDW_OK)
                r = consume_device_error(ctx, tm.st);
            *t = best_run;
            return r;
        };
        const int k = p->k;
        auto skip = [&](const aidw_tune_config &c, const aidw_tune_config &b) {
            // The same kernels as the shape already timed: nothing to time.
            const int kc = f32_list_length(k, c.knn_list), kb = f32_list_length(k, b.knn_list);
            return kc == kb &&
                   cull_queries_per_thread(kc, c.knn_queries_per_thread) ==
                       cull_queries_per_thread(kb, b.knn_queries_per_thread) &&
                   c.queries_per_thread == b.queries_per_thread &&
                   c.tile_points == b.tile_points && c.split_points == b.split_points &&
                   c.ctas_per_sm == b.ctas_per_sm;
        };
        const std::vector<Field> fields = {
            {&aidw_tune_config::queries_per_thread, {2, 4, 8}},
            {&aidw_tune_config::tile_points, {256, 512}},
            {&aidw_tune_config::knn_list, {0, 16, 32}},
            {&aidw_tune_config::knn_queries_per_thread, {0, 2, 4}},
        };
        rc = coordinate_search(fields, &cfg, &ms, measure, skip);
        if (rc == AIDW_OK && (flags & AIDW_TUNE_CACHE))
            aidw_tune_cache_put(kb, &cfg, ms);
        // Leave `out` holding the winner's results.
        if (rc == AIDW_OK)
            rc = run(cfg);
        if (rc == AIDW_OK && cudaStreamSynchronize(tm.st) != cudaSuccess)
            rc = AIDW_ERR_CUDA;
    }
    if (rc)
        return rc;
    if (flags & AIDW_TUNE_APPLY)
        ctx_set_tune(ctx, cfg);
    *best = cfg;
    *best_ms = ms;
    return AIDW_OK;
}

int aidw_batch_autotune(aidw_ctx *ctx, aidw_batch *b, int32_t reps, uint32_t flags,
                        aidw_tune_config *best, double *best_ms)
{
    if (!ctx || !b || !best || !best_ms || reps < 1)
        return AIDW_ERR_INVALID_ARG;
    if (cudaSetDevice(ctx_device(ctx)) != cudaSuccess)
        return AIDW_ERR_CUDA;
    // Workload key: item count, total queries and total pairs (size classes), largest k.
    double pairs = 0.0, queries = 0.0;
    int kmax = 0;
    for (const aidw_batch_item &it : b->items) {
        DatasetDev dev;
        double r_exp;
        if (!dataset_lookup(ctx, it.ds, &dev, &r_exp))
            return AIDW_ERR_NOT_FOUND;
        pairs += static_cast<double>(it.m) * static_cast<double>(dev.n);
        queries += static_cast<double>(it.m);
        kmax = it.params.k > kmax ? it.params.k : kmax;
    }
    char kb[192];
    std::snprintf(kb, sizeof(kb), "batch %s items=%zu q=2^%d pairs=2^%d kmax=%d",
                  device_tag(ctx).c_str(), b->items.size(), log2_round(queries),
                  log2_round(pairs), kmax);
    Timer tm;
    if (!tm.ok)
        return AIDW_ERR_CUDA;
    aidw_tune_config cfg = b->st.cfg;
    double ms = -1.0;
    int rc = AIDW_OK;
    if ((flags & AIDW_TUNE_CACHE) && aidw_tune_cache_get(kb, &cfg, nullptr) == AIDW_OK) {
        if (!same(cfg, b->st.cfg))
            rc = batch_prepare(ctx, b, cfg);
    } else {
        // CTAs per SM: the values below the occupancy limit of the current shape.
        const int occ = b->st.grid / (ctx_sm_count(ctx) > 0 ? ctx_sm_count(ctx) : 1);
        std::vector<int32_t> ctas = {0};
        for (int c = occ - 1; c >= 2 && c >= occ - 2; --c)
            ctas.push_back(c);
        auto measure = [&](const aidw_tune_config &c, double *t) {
            int r = same(c, b->st.cfg) ? AIDW_OK : batch_prepare(ctx, b, c);
            if (r)
                return r;
            if (b->st.n_units == 0) {
                *t = 0.0;
                return AIDW_OK;
            }
            r = cudaGraphLaunch(b->st.graph, tm.st) == cudaSuccess ? AIDW_OK : AIDW_ERR_CUDA;
            float best_run = 1e30f;
            for (int i = 0; i < reps && r == AIDW_OK; ++i) {
                cudaEventRecord(tm.e0, tm.st);
                if (cudaGraphLaunch(b->st.graph, tm.st) != cudaSuccess)
                    r = AIDW_ERR_CUDA;
                cudaEventRecord(tm.e1, tm.st);
                float e = 0.0f;
                if (r == AIDW_OK && (cudaEventSynchronize(tm.e1) != cudaSuccess ||
                                     cudaEventElapsedTime(&e, tm.e0, tm.e1) != cudaSuccess))
                    r = AIDW_ERR_CUDA;
                best_run = e < best_run ? e : best_run;
            }
            if (r == AIDW_OK)
                r = consume_device_error(ctx, tm.st);
            *t = best_run;
            return r;
        };
        auto skip = [&](const aidw_tune_config &c, const aidw_tune_config &bb) {
            // The same kernels for every item as the shape already timed: nothing to time.
            if (c.queries_per_thread != bb.queries_per_thread ||
                c.tile_points != bb.tile_points || c.split_points != bb.split_points ||
                c.ctas_per_sm != bb.ctas_per_sm || c.unit_order != bb.unit_order)
                return false;
            for (const aidw_batch_item &it : b->items) {
                const int kc = f32_list_length(it.params.k, c.knn_list);
                const int kb = f32_list_length(it.params.k, bb.knn_list);
                if (kc != kb || cull_queries_per_thread(kc, c.knn_queries_per_thread) !=
                                    cull_queries_per_thread(kb, bb.knn_queries_per_thread))
                    return false;
            }
            return true;
        };
        const std::vector<Field> fields = {
            {&aidw_tune_config::queries_per_thread, {2, 4, 8}},
            {&aidw_tune_config::tile_points, {256, 512}},
            {&aidw_tune_config::knn_list, {0, 16, 32}},
            {&aidw_tune_config::knn_queries_per_thread, {0, 2, 4}},
            {&aidw_tune_config::unit_order, {0, 1}},
            {&aidw_tune_config::split_points, {16384, 32768, 65536, 131072, 262144}},
            {&aidw_tune_config::ctas_per_sm, ctas},
        };
        rc = coordinate_search(fields, &cfg, &ms, measure, skip);
        if (rc == AIDW_OK && !same(cfg, b->st.cfg)) {
            // Rebuild with the winner and run it once, so the outputs are the winner's.
            rc = batch_prepare(ctx, b, cfg);
            if (rc == AIDW_OK && b->st.n_units > 0 &&
                (cudaGraphLaunch(b->st.graph, tm.st) != cudaSuccess ||
                 cudaStreamSynchronize(tm.st) != cudaSuccess))
                rc = AIDW_ERR_CUDA;
        }
        if (rc == AIDW_OK && (flags & AIDW_TUNE_CACHE))
            aidw_tune_cache_put(kb, &cfg, ms);
    }
    if (rc)
        return rc;
    *best = cfg;
    *best_ms = ms;
    return AIDW_OK;
}

}  // extern "C"
