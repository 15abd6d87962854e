// Autotuner for the inter-task kernel variant (rows per strip x warps per block): times
// each variant on a probe search and keeps the fastest, with an optional on-disk cache.
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/swgb.h"
#include "db_view.h"
#include "runtime_internal.h"
#include "swgb_device.cuh"

using namespace swgb;

namespace {

std::string cache_key(const sw_db* db, const int32_t* lens, int32_t nq) {
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, db->device);
    int64_t total = 0;
    for (int q = 0; q < nq; ++q) total += lens[q];
    // Probe length class: powers of two of the mean query length.
    int64_t mean = nq > 0 ? total / nq : 0, cls = 1;
    while (cls < mean) cls <<= 1;
    int64_t lmax = 8;
    while (lmax < db->layout.max_group_len) lmax <<= 1;
    std::ostringstream k;
    k << prop.name << "|sm" << db->sms << "|A" << db->A << "|G" << (db->layout.num_groups > 4096 ? "big" : "small")
      << "|L" << lmax << "|m" << cls;
    std::string s = k.str();
    for (auto& c : s)
        if (c == ' ') c = '_';
    return s;
}

int cache_lookup(const char* path, const std::string& key) {
    std::ifstream f(path);
    std::string k;
    int v;
    int found = -1;
    while (f >> k >> v)
        if (k == key) found = v;
    return found;
}

void cache_store(const char* path, const std::string& key, int variant) {
    std::vector<std::pair<std::string, int>> rows;
    {
        std::ifstream f(path);
        std::string k;
        int v;
        while (f >> k >> v)
            if (k != key) rows.emplace_back(k, v);
    }
    rows.emplace_back(key, variant);
    const std::string tmp = std::string(path) + ".tmp";
    {
        std::ofstream o(tmp);
        for (auto& r : rows) o << r.first << " " << r.second << "\n";
    }
    std::rename(tmp.c_str(), path);
}

}  // namespace

extern "C" sw_status sw_db_set_variant(sw_db* db, int32_t variant) {
    if (!db) return set_last_error(SW_ERR_ARG, "db is null");
    std::lock_guard<std::mutex> lock(db->mu);
    if (variant < 0) variant = 0;
    if (variant >= inter_num_variants() || db->inter_occ[variant] <= 0)
        return set_last_error(SW_ERR_ARG, "variant not available on this device");
    db->variant = variant;
    return SW_OK;
}

extern "C" sw_status sw_db_tune(sw_db* db, const uint8_t* const* queries, const int32_t* query_lens,
                                int32_t num_queries, const int8_t* matrix, int32_t gap_open,
                                int32_t gap_extend, const char* cache_path, int32_t force,
                                sw_tune_result* out) {
    if (!db || !out) return set_last_error(SW_ERR_ARG, "null pointer");
    if (num_queries <= 0 || !queries || !query_lens)
        return set_last_error(SW_ERR_ARG, "the probe needs at least one query");
    std::memset(out, 0, sizeof(*out));
    out->num_variants = std::min(inter_num_variants(), 8);
    const std::string key = cache_key(db, query_lens, num_queries);
    if (cache_path && !force) {
        const int v = cache_lookup(cache_path, key);
        if (v >= 0 && v < inter_num_variants() && db->inter_occ[v] > 0) {
            sw_status s = sw_db_set_variant(db, v);
            if (s != SW_OK) return s;
            out->variant = v;
            out->rows_per_strip = inter_variant_rows(v);
            out->warps_per_block = inter_variant_warps(v);
            out->from_cache = 1;
            return SW_OK;
        }
    }
    const int64_t N = db->layout.num_seqs;
    if (N == 0 || db->layout.num_groups == 0) {
        out->variant = db->variant;
        out->rows_per_strip = inter_variant_rows(db->variant);
        out->warps_per_block = inter_variant_warps(db->variant);
        return SW_OK;
    }
    std::vector<int32_t> scores(static_cast<size_t>(N) * num_queries);
    struct NoRoute {   // time the inter-task variants on every group, whatever the database size
        sw_db* db;
        explicit NoRoute(sw_db* d) : db(d) { db->no_route = true; }
        ~NoRoute() { db->no_route = false; }
    } no_route(db);
    int best = -1;
    float best_gcups = 0.f;
    for (int v = 0; v < out->num_variants; ++v) {
        if (db->inter_occ[v] <= 0) continue;
        sw_status s = sw_db_set_variant(db, v);
        if (s != SW_OK) return s;
        float gcups = 0.f;
        for (int rep = 0; rep < 2; ++rep) {   // warm-up, then the timed run
            s = sw_search_batch(db, queries, query_lens, num_queries, matrix, gap_open, gap_extend,
                                scores.data());
            if (s != SW_OK) return s;
            sw_stats st{};
            s = sw_get_stats(db, &st);
            if (s != SW_OK) return s;
            if (st.inter_ms > 0) gcups = static_cast<float>(st.inter_cells / (st.inter_ms * 1e6));
        }
        out->gcups[v] = gcups;
        if (gcups > best_gcups) {
            best_gcups = gcups;
            best = v;
        }
    }
    if (best < 0) best = 0;
    sw_status s = sw_db_set_variant(db, best);
    if (s != SW_OK) return s;
    out->variant = best;
    out->rows_per_strip = inter_variant_rows(best);
    out->warps_per_block = inter_variant_warps(best);
    if (cache_path) cache_store(cache_path, key, best);
    return SW_OK;
}
