// Tuning table and the exhaustive autotuner.
//
// The paper finds the best configuration for every size by exhaustive
// search over its generated variants (Sec. 5.1; Sec. 7 names a performance
// model as the faster alternative).  Here tsm_tune() times every compiled
// variant that supports the shape, at several grid sizes, with CUDA events
// on the caller's buffers, and records the fastest in an in-memory table
// keyed by (product, dtype, M, N, floor(log2 K)).  The table stores variant
// NAMES, so a file written by one build stays valid for another build whose
// variant order differs.  Files are plain text, one entry per line:
//   kind dtype M N kbucket variant_name grid milliseconds
// TSM_TUNE_FILE names a file loaded on first lookup.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "tsm_internal.h"
#include "tsm_tune.h"
#include "tune.h"

namespace tsm {
namespace {

struct Entry {
    std::string name;
    int grid;
    float ms;
    int index = -2;  // the variant's table index, resolved on first lookup (-1: no such variant)
};
typedef std::tuple<int, int, int, int, int> Key;

std::mutex g_mu;
std::map<Key, Entry> g_table;
bool g_env_loaded = false;

int find_variant(int kind, const std::string& name) {
    const int n = tsm_variant_count((tsm_kind)kind);
    for (int i = 0; i < n; ++i) {
        const Variant* v = variant_at((tsm_kind)kind, i);
        if (v && name == v->info.name) return i;
    }
    return -1;
}

tsm_status load_file(const char* path) {
    FILE* f = fopen(path, "r");
    if (!f) return TSM_ERR_INVALID_VALUE;
    char line[512];
    while (fgets(line, sizeof(line), f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        int kind, dtype, M, N, kb, grid;
        char name[128];
        float ms;
        if (sscanf(line, "%d %d %d %d %d %127s %d %f", &kind, &dtype, &M, &N, &kb, name, &grid, &ms) == 8)
            g_table[Key(kind, dtype, M, N, kb)] = Entry{name, grid, ms};
    }
    fclose(f);
    return TSM_OK;
}

}  // namespace

int k_bucket(int64_t K) {
    int b = 0;
    while (K >= 2) {
        K >>= 1;
        ++b;
    }
    return b;
}

tsm_status tune_lookup(int kind, int dtype, int M, int N, int64_t K, int* variant, int* grid) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_env_loaded) {
        g_env_loaded = true;
        const char* p = getenv("TSM_TUNE_FILE");
        if (p && *p) load_file(p);
    }
    // exact K bucket first, then the nearest bucket tuned for this shape
    const int kb = k_bucket(K);
    Entry* best = nullptr;
    int best_d = 1 << 30;
    for (auto it = g_table.lower_bound(Key(kind, dtype, M, N, 0));
         it != g_table.end() && std::get<0>(it->first) == kind && std::get<1>(it->first) == dtype &&
         std::get<2>(it->first) == M && std::get<3>(it->first) == N;
         ++it) {
        const int d = std::abs(std::get<4>(it->first) - kb);
        if (d < best_d) {
            best_d = d;
            best = &it->second;
        }
    }
    if (!best) return TSM_ERR_NOT_SUPPORTED;
    // the name is resolved once per entry: a scan of a few hundred variant
    // names per call would cost microseconds of host time
    if (best->index == -2) best->index = find_variant(kind, best->name);
    const int v = best->index;
    if (v < 0) return TSM_ERR_NOT_SUPPORTED;
    *variant = v;
    *grid = best->grid;
    return TSM_OK;
}

}  // namespace tsm

using namespace tsm;

extern "C" {

tsm_status tsm_load_tuning(const char* path) {
    if (!path) return TSM_ERR_INVALID_VALUE;
    std::lock_guard<std::mutex> lock(g_mu);
    g_env_loaded = true;
    return load_file(path);
}

tsm_status tsm_save_tuning(const char* path) {
    if (!path) return TSM_ERR_INVALID_VALUE;
    std::lock_guard<std::mutex> lock(g_mu);
    FILE* f = fopen(path, "w");
    if (!f) return TSM_ERR_INVALID_VALUE;
    fprintf(f, "# kind dtype M N kbucket variant grid ms\n");
    for (auto& kv : g_table)
        fprintf(f, "%d %d %d %d %d %s %d %.6f\n", std::get<0>(kv.first), std::get<1>(kv.first),
                std::get<2>(kv.first), std::get<3>(kv.first), std::get<4>(kv.first), kv.second.name.c_str(),
                kv.second.grid, kv.second.ms);
    fclose(f);
    return TSM_OK;
}

tsm_status tsm_clear_tuning(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_table.clear();
    g_env_loaded = true;
    return TSM_OK;
}

tsm_status tsm_set_tuning(tsm_kind kind, tsm_dtype dtype, int M, int N, int64_t K, int variant, int grid) {
    const Variant* v = variant_at(kind, variant);
    if (!v || !supports(kind, variant, dtype, M, N) || grid < 0) return TSM_ERR_INVALID_VALUE;
    std::lock_guard<std::mutex> lock(g_mu);
    g_env_loaded = true;
    g_table[Key(kind, dtype, M, N, k_bucket(K))] = Entry{v->info.name, grid, -1.0f};
    return TSM_OK;
}

tsm_status tsm_set_tuning_timed(tsm_kind kind, tsm_dtype dtype, int M, int N, int64_t K, int variant, int grid,
                                float ms) {
    const Variant* v = variant_at(kind, variant);
    if (!v || !supports(kind, variant, dtype, M, N) || grid < 0) return TSM_ERR_INVALID_VALUE;
    std::lock_guard<std::mutex> lock(g_mu);
    g_env_loaded = true;
    g_table[Key(kind, dtype, M, N, k_bucket(K))] = Entry{v->info.name, grid, ms};
    return TSM_OK;
}

tsm_status tsm_tune_grids(tsm_kind kind, int variant, tsm_dtype dtype, int M, int N, int* grids, int max,
                          int* count) {
    if (!grids || !count || max < 0) return TSM_ERR_INVALID_VALUE;
    *count = 0;
    if (!supports(kind, variant, dtype, M, N)) return TSM_OK;
    const Variant* var = variant_at(kind, variant);
    const int occ = var->occupancy ? var->occupancy(M, N) : 1;
    if (occ <= 0) return TSM_OK;
    const int sm = device_info().sm_count;
    // one CTA per SM, two, full occupancy, two waves
    const int cand[4] = {sm, sm * 2, sm * occ, sm * occ * 2};
    int n = 0;
    for (int i = 0; i < 4; ++i) {
        if (i < 2 && cand[i] > sm * occ) continue;
        bool dup = false;
        for (int j = 0; j < n; ++j) dup |= grids[j] == cand[i];
        if (dup || n >= max) continue;
        grids[n++] = cand[i];
    }
    *count = n;
    return TSM_OK;
}

tsm_status tsm_time_variant(tsm_kind kind, tsm_dtype dtype, int M, int N, int64_t K, const void* X,
                            int64_t ldx, const void* Y, int64_t ldy, void* Z, int64_t ldz, int variant,
                            int grid, int reps, float* ms, tsm_stream_t stream) {
    if (!ms || reps < 1) return TSM_ERR_INVALID_VALUE;
    if (!supports(kind, variant, dtype, M, N)) return TSM_ERR_NOT_SUPPORTED;
    const double one[2] = {1.0, 0.0}, zero[2] = {0.0, 0.0};
    cudaStream_t s = (cudaStream_t)stream;
    // TSM_KIND_TSMM_BETA: the TSMM variants with beta = 1 (B is read too)
    const double* beta = kind == TSM_KIND_TSMM_BETA ? one : zero;
    auto run = [&]() -> tsm_status {
        if (kind == TSM_KIND_TSMTTSM)
            return run_tsmttsm(TSM_OP_T, dtype, M, N, K, one, X, ldx, Y, ldy, zero, Z, ldz, variant, grid, s);
        return run_tsmm(TSM_OP_N, dtype, M, N, K, one, X, ldx, Y, ldy, beta, Z, ldz, variant, grid, s);
    };
    tsm_status st = run();  // warm-up (also grows the workspace)
    if (st != TSM_OK) return st;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return TSM_ERR_LAUNCH;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return TSM_ERR_LAUNCH;
    }
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && st == TSM_OK; ++r) st = run();
    cudaEventRecord(e1, s);
    float t = 0.f;
    if (st == TSM_OK) {
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
            st = TSM_ERR_LAUNCH;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = t / reps;
    return st;
}

tsm_status tsm_tune(tsm_kind kind, tsm_dtype dtype, int M, int N, int64_t K, const void* X, int64_t ldx,
                    const void* Y, int64_t ldy, void* Z, int64_t ldz, int reps, tsm_tune_sample* samples,
                    int max_samples, int* n_samples, tsm_stream_t stream) {
    const int nv = tsm_variant_count(kind);
    if (nv < 0 || reps < 1) return TSM_ERR_INVALID_VALUE;
    if (M < 1 || N < 1 || M > 64 || N > 64) return TSM_ERR_NOT_SUPPORTED;
    const int sm = device_info().sm_count;
    int count = 0;
    float best_ms = 1e30f;
    int best_v = -1, best_g = 0;
    for (int v = 0; v < nv; ++v) {
        if (!supports(kind, v, dtype, M, N)) continue;
        int grids[4], ng = 0;
        if (tsm_tune_grids(kind, v, dtype, M, N, grids, 4, &ng) != TSM_OK) continue;
        for (int gi = 0; gi < ng; ++gi) {
            const int g = grids[gi];
            float ms = 0.f;
            tsm_status st = tsm_time_variant(kind, dtype, M, N, K, X, ldx, Y, ldy, Z, ldz, v, g, reps, &ms, stream);
            if (st != TSM_OK) return st;
            if (samples && count < max_samples) samples[count] = tsm_tune_sample{v, g, ms};
            ++count;
            if (ms < best_ms) {
                best_ms = ms;
                best_v = v;
                best_g = g;
            }
        }
    }
    if (n_samples) *n_samples = count;
    if (best_v < 0) return TSM_ERR_NOT_SUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    g_env_loaded = true;
    g_table[Key(kind, dtype, M, N, k_bucket(K))] = Entry{variant_at(kind, best_v)->info.name, best_g, best_ms};
    return TSM_OK;
}

}  // extern "C"
