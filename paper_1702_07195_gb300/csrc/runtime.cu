// Host runtime of libswgb: the device-resident database, the search orchestration (query
// profiles, persistent inter-task launch, intra-task launch for long subjects, int32 rescore
// of saturated lanes, CUDA-graph replay) and the C ABI declared in include/swgb.h.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/swgb.h"
#include "db_view.h"
#include "layout.h"
#include "swgb_device.cuh"

using namespace swgb;

namespace {

thread_local std::string g_err;
std::atomic<int64_t> g_launches{0};

sw_status fail(sw_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

sw_status cuda_fail(cudaError_t e, const char* what) {
    const sw_status st = (e == cudaErrorMemoryAllocation) ? SW_ERR_OOM : SW_ERR_CUDA;
    return fail(st, "%s: %s", what, cudaGetErrorString(e));
}

#define CU(call)                                                      \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);           \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

template <class T>
struct DevBuf {
    T* ptr = nullptr;
    size_t cap = 0;   // elements
    cudaError_t ensure(size_t n) {
        if (n <= cap && ptr) return cudaSuccess;
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        cap = 0;
        const size_t want = std::max<size_t>(n, 1);
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&ptr), want * sizeof(T));
        if (e == cudaSuccess) cap = want;
        return e;
    }
    void release() {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        cap = 0;
    }
};

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

// A captured launch sequence, replayed when shapes and pointers repeat.
struct GraphEntry {
    std::vector<int64_t> key;
    cudaGraphExec_t exec = nullptr;
};

struct sw_db {
    int device = 0;
    int sms = 0;
    int32_t A = 0;
    int32_t long_cutoff = 0;
    int32_t flag_cap = 1 << 20;
    Layout layout;
    int64_t num_residues = 0;
    // device database
    DevBuf<uint8_t> inter;
    DevBuf<int64_t> group_off;
    DevBuf<int32_t> group_len;
    DevBuf<int32_t> perm;
    DevBuf<uint8_t> plain;
    DevBuf<int64_t> plain_off;
    DevBuf<int32_t> long_ids;
    // workspace
    DevBuf<int16_t> qp;
    DevBuf<QueryDesc> descs;
    DevBuf<InterItem> items;
    DevBuf<int64_t> qp_off;
    DevBuf<int32_t> mpad;
    DevBuf<int64_t> qoff;
    DevBuf<int32_t> query_order;
    DevBuf<int8_t> matrix;
    DevBuf<Control> ctrl;
    DevBuf<FlagEntry> flags;
    DevBuf<uint4> bnd;
    DevBuf<int2> spill;
    DevBuf<uint8_t> h_queries;   // device copy of host queries (host-buffer API)
    DevBuf<int32_t> h_scores;    // device scores (host-buffer API)
    cudaStream_t stream = nullptr;   // internal stream for the host-buffer API
    cudaEvent_t ev[5] = {};
    std::vector<GraphEntry> graphs;
    // last search
    sw_stats stats{};
    bool stats_pending = false;
    std::mutex mu;
    int inter_occ = 0, intra_occ = 0;
};

namespace {

void destroy_graphs(sw_db* db) {
    for (auto& g : db->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    db->graphs.clear();
}

sw_status validate_matrix(const int8_t* matrix, int32_t A, int* max_s) {
    if (!matrix) return fail(SW_ERR_ARG, "matrix is null");
    int mx = 0;
    for (int i = 0; i < A * A; ++i) mx = std::max<int>(mx, matrix[i]);
    *max_s = mx;
    return SW_OK;
}

// The whole search on device-resident queries.  `h_qoff` is host memory.
sw_status search_device(sw_db* db, const uint8_t* d_queries, const int64_t* h_qoff, int32_t nq,
                        const int8_t* h_matrix, int32_t gap_open, int32_t gap_extend,
                        int32_t* d_scores, cudaStream_t st) {
    if (nq < 0) return fail(SW_ERR_ARG, "num_queries < 0");
    if (gap_open < 0 || gap_extend < 0 || gap_open > 1000000 || gap_extend > 1000000)
        return fail(SW_ERR_ARG, "gap costs must be in [0, 1000000]");
    if (nq == 0) return SW_OK;
    if (!h_qoff || !d_scores || (!d_queries && h_qoff[nq] > 0))
        return fail(SW_ERR_ARG, "null query/offset/score pointer");
    const int32_t A = db->A;
    int max_s = 0;
    sw_status vs = validate_matrix(h_matrix, A, &max_s);
    if (vs != SW_OK) return vs;
    if (h_qoff[0] != 0) return fail(SW_ERR_ARG, "query_offsets[0] must be 0");
    std::vector<int32_t> m(static_cast<size_t>(nq));
    int64_t max_m = 0;
    for (int q = 0; q < nq; ++q) {
        const int64_t len = h_qoff[q + 1] - h_qoff[q];
        if (len < 0 || len > (int64_t{1} << 28))
            return fail(SW_ERR_ARG, "query %d: bad length %lld", q, static_cast<long long>(len));
        m[static_cast<size_t>(q)] = static_cast<int32_t>(len);
        max_m = std::max(max_m, len);
    }
    if (static_cast<double>(std::min<int64_t>(max_m, db->layout.max_len)) * max_s > 2147483647.0)
        return fail(SW_ERR_ARG, "scores could exceed the int32 range");
    const int64_t N = db->layout.num_seqs;
    const int32_t goe = gap_open, ge = gap_extend, gep = std::min(goe, ge);
    const bool int16_ok = goe <= 16383 && ge <= 16383;
    const int32_t qp_bias = (goe + 128 <= 32767) ? goe : 0;   // profile entries stay in int16

    // ---- plan: profiles, descriptors, items
    std::vector<int64_t> qp_off(static_cast<size_t>(nq));
    std::vector<int32_t> mpad(static_cast<size_t>(nq));
    int64_t total_qp = 0, max_mpad = 0;
    for (int q = 0; q < nq; ++q) {
        const int64_t mp = round_up(std::max<int64_t>(m[static_cast<size_t>(q)], 1), kQpRows);
        mpad[static_cast<size_t>(q)] = static_cast<int32_t>(mp);
        qp_off[static_cast<size_t>(q)] = total_qp;
        total_qp += mp * (A + 1);
        max_mpad = std::max(max_mpad, mp);
    }
    std::vector<int32_t> order(static_cast<size_t>(nq));
    for (int q = 0; q < nq; ++q) order[static_cast<size_t>(q)] = q;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return m[static_cast<size_t>(a)] > m[static_cast<size_t>(b)]; });

    const int W = inter_block_threads() / kWarp;
    std::vector<InterItem> items;
    const int64_t G = db->layout.num_groups;
    if (int16_ok && G > 0) {
        const int64_t chunks = (G + W - 1) / W;
        items.reserve(static_cast<size_t>(chunks * nq));
        // queries longest first, groups longest first: big items start early, the tail is short
        for (int32_t q : order) {
            if (m[static_cast<size_t>(q)] == 0) continue;
            for (int64_t c = chunks - 1; c >= 0; --c) {
                const int64_t g0 = c * W;
                const int32_t ng = static_cast<int32_t>(std::min<int64_t>(W, G - g0));
                items.push_back(InterItem{q, static_cast<int32_t>(g0), ng, 0});
            }
        }
        std::vector<int64_t> cost(items.size());
        for (size_t i = 0; i < items.size(); ++i) {
            const InterItem& it = items[i];
            const int64_t L = db->layout.group_len[static_cast<size_t>(it.group + it.ngroups - 1)];
            cost[i] = static_cast<int64_t>(m[static_cast<size_t>(it.query)]) * L;
        }
        std::vector<int32_t> idx(items.size());
        for (size_t i = 0; i < idx.size(); ++i) idx[i] = static_cast<int32_t>(i);
        std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
        std::vector<InterItem> sorted(items.size());
        for (size_t i = 0; i < idx.size(); ++i) sorted[i] = items[static_cast<size_t>(idx[i])];
        items.swap(sorted);
    }

    // ---- workspace
    const int inter_grid = db->sms * std::max(1, db->inter_occ);
    const int intra_grid = db->sms * std::max(1, db->intra_occ);
    const int64_t inter_slots = static_cast<int64_t>(inter_grid) * W;
    const int64_t intra_slots = static_cast<int64_t>(intra_grid) * (intra_block_threads() / kWarp);
    const int64_t bnd_stride = std::max<int64_t>(1, db->layout.max_group_len / 2 * kWarp);
    const int64_t spill_stride = std::max<int64_t>(1, round_up(db->layout.max_len, 32) + 64);
    const uint32_t flag_cap =
        static_cast<uint32_t>(std::min<int64_t>(std::max<int64_t>(N * nq, 1), db->flag_cap));
    CU(db->qp.ensure(static_cast<size_t>(total_qp)));
    CU(db->descs.ensure(static_cast<size_t>(nq)));
    CU(db->items.ensure(std::max<size_t>(items.size(), 1)));
    CU(db->qp_off.ensure(static_cast<size_t>(nq)));
    CU(db->mpad.ensure(static_cast<size_t>(nq)));
    CU(db->qoff.ensure(static_cast<size_t>(nq) + 1));
    CU(db->query_order.ensure(static_cast<size_t>(nq)));
    CU(db->matrix.ensure(static_cast<size_t>(A * A)));
    CU(db->ctrl.ensure(1));
    CU(db->flags.ensure(flag_cap));
    if (!items.empty()) CU(db->bnd.ensure(static_cast<size_t>(inter_slots * bnd_stride)));
    CU(db->spill.ensure(static_cast<size_t>(intra_slots * spill_stride)));

    std::vector<QueryDesc> descs(static_cast<size_t>(nq));
    for (int q = 0; q < nq; ++q)
        descs[static_cast<size_t>(q)] = QueryDesc{db->qp.ptr + qp_off[static_cast<size_t>(q)],
                                                  d_scores + static_cast<int64_t>(q) * N,
                                                  m[static_cast<size_t>(q)], mpad[static_cast<size_t>(q)]};
    CU(cudaMemcpyAsync(db->descs.ptr, descs.data(), sizeof(QueryDesc) * nq, cudaMemcpyHostToDevice, st));
    if (!items.empty())
        CU(cudaMemcpyAsync(db->items.ptr, items.data(), sizeof(InterItem) * items.size(),
                           cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(db->qp_off.ptr, qp_off.data(), sizeof(int64_t) * nq, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(db->mpad.ptr, mpad.data(), sizeof(int32_t) * nq, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(db->qoff.ptr, h_qoff, sizeof(int64_t) * (nq + 1), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(db->query_order.ptr, order.data(), sizeof(int32_t) * nq, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(db->matrix.ptr, h_matrix, static_cast<size_t>(A * A), cudaMemcpyHostToDevice, st));

    // ---- launch sequence
    int64_t launches = 0;
    CU(cudaEventRecord(db->ev[0], st));
    CU(cudaMemsetAsync(db->ctrl.ptr, 0, sizeof(Control), st));
    for (int q = 0; q < nq; ++q)   // empty queries score 0 everywhere
        if (m[static_cast<size_t>(q)] == 0 && N > 0)
            CU(cudaMemsetAsync(d_scores + static_cast<int64_t>(q) * N, 0, sizeof(int32_t) * N, st));
    CU(launch_build_qp(d_queries, db->qoff.ptr, nq, db->matrix.ptr, A, qp_bias, db->qp_off.ptr,
                       db->mpad.ptr, db->qp.ptr, max_mpad, db->ctrl.ptr, st));
    ++launches;
    CU(cudaEventRecord(db->ev[1], st));
    const Gaps gaps{goe, ge, gep};
    if (!items.empty()) {
        InterParams p{};
        p.inter = db->inter.ptr;
        p.group_off = db->group_off.ptr;
        p.group_len = db->group_len.ptr;
        p.perm = db->perm.ptr;
        p.queries = db->descs.ptr;
        p.items = db->items.ptr;
        p.num_items = static_cast<int32_t>(items.size());
        p.alphabet1 = A + 1;
        p.ctrl = db->ctrl.ptr;
        p.flags = db->flags.ptr;
        p.flag_cap = flag_cap;
        p.thresh = 32767 - std::max(0, max_s);
        p.bnd = db->bnd.ptr;
        p.bnd_stride = bnd_stride;
        p.gaps = gaps;
        CU(launch_inter(p, inter_grid, inter_block_threads(), st));
        ++launches;
    }
    CU(cudaEventRecord(db->ev[2], st));
    IntraParams ip{};
    ip.plain = db->plain.ptr;
    ip.plain_off = db->plain_off.ptr;
    ip.queries = db->descs.ptr;
    ip.num_queries = nq;
    ip.long_ids = db->long_ids.ptr;
    ip.num_long = static_cast<int64_t>(db->layout.long_ids.size());
    ip.query_order = db->query_order.ptr;
    ip.num_seqs = N;
    ip.flags = db->flags.ptr;
    ip.flag_cap = flag_cap;
    ip.alphabet1 = A + 1;
    ip.ctrl = db->ctrl.ptr;
    ip.spill = db->spill.ptr;
    ip.spill_stride = spill_stride;
    ip.gaps = gaps;
    ip.qp_add = goe - qp_bias;
    if (!int16_ok) {
        ip.mode = kIntraAll;
        if (N > 0) {
            CU(launch_intra(ip, intra_grid, intra_block_threads(), st));
            ++launches;
        }
    } else if (ip.num_long > 0) {
        ip.mode = kIntraLong;
        CU(launch_intra(ip, intra_grid, intra_block_threads(), st));
        ++launches;
    }
    CU(cudaEventRecord(db->ev[3], st));
    if (int16_ok && !items.empty()) {
        ip.mode = kIntraRescore;
        CU(launch_intra(ip, intra_grid, intra_block_threads(), st));
        ++launches;
    }
    CU(cudaEventRecord(db->ev[4], st));
    g_launches += launches;

    int64_t cells = 0, inter_cells = 0;
    for (int q = 0; q < nq; ++q) {
        cells += static_cast<int64_t>(m[static_cast<size_t>(q)]) * db->num_residues;
        if (int16_ok) inter_cells += static_cast<int64_t>(m[static_cast<size_t>(q)]) * db->layout.short_residues;
    }
    db->stats = sw_stats{};
    db->stats.cells = cells;
    db->stats.inter_cells = inter_cells;
    db->stats.launches = launches;
    db->stats.inter_grid = inter_grid;
    db->stats.inter_block = inter_block_threads();
    db->stats_pending = true;
    return SW_OK;
}

sw_status finish_stats(sw_db* db) {
    if (!db->stats_pending) return SW_OK;
    CU(cudaEventSynchronize(db->ev[4]));
    float t = 0;
    CU(cudaEventElapsedTime(&t, db->ev[1], db->ev[2]));
    db->stats.inter_ms = t;
    CU(cudaEventElapsedTime(&t, db->ev[2], db->ev[3]));
    db->stats.intra_ms = t;
    CU(cudaEventElapsedTime(&t, db->ev[3], db->ev[4]));
    db->stats.rescore_ms = t;
    CU(cudaEventElapsedTime(&t, db->ev[0], db->ev[4]));
    db->stats.total_ms = t;
    Control c{};
    CU(cudaMemcpy(&c, db->ctrl.ptr, sizeof(Control), cudaMemcpyDeviceToHost));
    db->stats.flagged = c.flag_count;
    db->stats_pending = false;
    if (c.status & 1u) return fail(SW_ERR_CODE, "a query residue code was >= alphabet_size");
    return SW_OK;
}

}  // namespace

// ================================================================= C ABI

extern "C" {

const char* sw_last_error(void) { return g_err.c_str(); }
const char* sw_version(void) { return "swgb 0.1 (sm_103a)"; }
int64_t sw_launch_count(void) { return g_launches.load(); }

sw_status sw_layout_sizes(const int64_t* offsets, int64_t num_seqs, int32_t long_cutoff,
                          int64_t* num_groups, int64_t* inter_bytes, int64_t* num_long) {
    if (!num_groups || !inter_bytes || !num_long) return fail(SW_ERR_ARG, "null output pointer");
    Layout L;
    const std::string err = plan_layout(offsets, num_seqs, long_cutoff, L);
    if (!err.empty()) return fail(SW_ERR_ARG, "%s", err.c_str());
    *num_groups = L.num_groups;
    *inter_bytes = L.inter_bytes;
    *num_long = static_cast<int64_t>(L.long_ids.size());
    return SW_OK;
}

sw_status sw_layout_build(const uint8_t* residues, const int64_t* offsets, int64_t num_seqs,
                          int32_t alphabet_size, int32_t long_cutoff, int64_t* group_off,
                          int32_t* group_len, int32_t* perm, uint8_t* inter, int32_t* long_ids) {
    if (alphabet_size < 1 || alphabet_size > kMaxAlphabet)
        return fail(SW_ERR_ARG, "alphabet_size must be in [1, 32]");
    Layout L;
    const std::string err = plan_layout(offsets, num_seqs, long_cutoff, L);
    if (!err.empty()) return fail(SW_ERR_ARG, "%s", err.c_str());
    const int64_t R = num_seqs > 0 ? offsets[num_seqs] : 0;
    if (R > 0 && !residues) return fail(SW_ERR_ARG, "residues is null");
    const int64_t bad = find_bad_code(residues, R, alphabet_size);
    if (bad >= 0) return fail(SW_ERR_CODE, "residue %lld has code %d >= alphabet_size %d",
                              static_cast<long long>(bad), residues[bad], alphabet_size);
    if (L.num_groups > 0 && (!group_off || !group_len || !perm || !inter))
        return fail(SW_ERR_ARG, "null output buffer");
    if (!L.long_ids.empty() && !long_ids) return fail(SW_ERR_ARG, "long_ids is null");
    std::copy(L.group_off.begin(), L.group_off.end(), group_off);
    std::copy(L.group_len.begin(), L.group_len.end(), group_len);
    std::copy(L.perm.begin(), L.perm.end(), perm);
    std::copy(L.long_ids.begin(), L.long_ids.end(), long_ids);
    if (L.num_groups > 0) fill_inter(residues, offsets, alphabet_size, L, inter);
    return SW_OK;
}

sw_status sw_db_load_ex(const uint8_t* residues, const int64_t* offsets, int64_t num_seqs,
                        int32_t alphabet_size, const sw_db_options* opts, sw_db** out) {
    if (!out) return fail(SW_ERR_ARG, "out is null");
    *out = nullptr;
    if (alphabet_size < 1 || alphabet_size > kMaxAlphabet)
        return fail(SW_ERR_ARG, "alphabet_size must be in [1, 32]");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    int32_t cutoff = 3072;
    if (opts) {
        if (opts->device > 0) dev = opts->device;
        if (opts->long_cutoff > 0) cutoff = opts->long_cutoff;
        if (opts->flag_cap < 0) return fail(SW_ERR_ARG, "flag_cap < 0");
    }
    std::unique_ptr<sw_db> db(new sw_db());
    db->device = dev;
    db->A = alphabet_size;
    db->long_cutoff = cutoff;
    if (opts && opts->flag_cap > 0) db->flag_cap = opts->flag_cap;
    const std::string err = plan_layout(offsets, num_seqs, cutoff, db->layout);
    if (!err.empty()) return fail(SW_ERR_ARG, "%s", err.c_str());
    const int64_t R = num_seqs > 0 ? offsets[num_seqs] : 0;
    if (R > 0 && !residues) return fail(SW_ERR_ARG, "residues is null");
    const int64_t bad = find_bad_code(residues, R, alphabet_size);
    if (bad >= 0) return fail(SW_ERR_CODE, "residue %lld has code %d >= alphabet_size %d",
                              static_cast<long long>(bad), residues[bad], alphabet_size);
    db->num_residues = R;
    DeviceGuard guard(dev);
    CU(cudaDeviceGetAttribute(&db->sms, cudaDevAttrMultiProcessorCount, dev));
    db->inter_occ = inter_occupancy(alphabet_size + 1);
    db->intra_occ = intra_occupancy(alphabet_size + 1);
    if (db->inter_occ <= 0 || db->intra_occ <= 0)
        return fail(SW_ERR_CUDA, "kernels cannot be resident on device %d", dev);
    CU(cudaStreamCreateWithFlags(&db->stream, cudaStreamNonBlocking));
    for (auto& e : db->ev) CU(cudaEventCreate(&e));
    const Layout& L = db->layout;
    std::vector<uint8_t> inter(static_cast<size_t>(std::max<int64_t>(L.inter_bytes, 1)));
    if (L.num_groups > 0) fill_inter(residues, offsets, alphabet_size, L, inter.data());
    CU(db->inter.ensure(inter.size()));
    CU(cudaMemcpy(db->inter.ptr, inter.data(), inter.size(), cudaMemcpyHostToDevice));
    CU(db->group_off.ensure(L.group_off.size()));
    CU(db->group_len.ensure(L.group_len.size()));
    CU(db->perm.ensure(L.perm.size()));
    if (!L.group_off.empty()) {
        CU(cudaMemcpy(db->group_off.ptr, L.group_off.data(), sizeof(int64_t) * L.group_off.size(), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(db->group_len.ptr, L.group_len.data(), sizeof(int32_t) * L.group_len.size(), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(db->perm.ptr, L.perm.data(), sizeof(int32_t) * L.perm.size(), cudaMemcpyHostToDevice));
    }
    CU(db->plain.ensure(static_cast<size_t>(std::max<int64_t>(R, 16))));
    if (R > 0) CU(cudaMemcpy(db->plain.ptr, residues, static_cast<size_t>(R), cudaMemcpyHostToDevice));
    CU(db->plain_off.ensure(static_cast<size_t>(num_seqs) + 1));
    CU(cudaMemcpy(db->plain_off.ptr, offsets, sizeof(int64_t) * (num_seqs + 1), cudaMemcpyHostToDevice));
    CU(db->long_ids.ensure(std::max<size_t>(L.long_ids.size(), 1)));
    if (!L.long_ids.empty())
        CU(cudaMemcpy(db->long_ids.ptr, L.long_ids.data(), sizeof(int32_t) * L.long_ids.size(), cudaMemcpyHostToDevice));
    *out = db.release();
    return SW_OK;
}

sw_status sw_db_load(const uint8_t* residues, const int64_t* offsets, int64_t num_seqs,
                     int32_t alphabet_size, sw_db** out) {
    return sw_db_load_ex(residues, offsets, num_seqs, alphabet_size, nullptr, out);
}

void sw_db_free(sw_db* db) {
    if (!db) return;
    {
        DeviceGuard guard(db->device);
        if (db->stream) cudaStreamSynchronize(db->stream);
        destroy_graphs(db);
        DevBuf<uint8_t>* u8s[] = {&db->inter, &db->plain, &db->h_queries};
        for (auto* b : u8s) b->release();
        db->group_off.release();
        db->group_len.release();
        db->perm.release();
        db->plain_off.release();
        db->long_ids.release();
        db->qp.release();
        db->descs.release();
        db->items.release();
        db->qp_off.release();
        db->mpad.release();
        db->qoff.release();
        db->query_order.release();
        db->matrix.release();
        db->ctrl.release();
        db->flags.release();
        db->bnd.release();
        db->spill.release();
        db->h_scores.release();
        for (auto& e : db->ev)
            if (e) cudaEventDestroy(e);
        if (db->stream) cudaStreamDestroy(db->stream);
    }
    delete db;
}

int64_t sw_db_num_seqs(const sw_db* db) { return db ? db->layout.num_seqs : -1; }
int64_t sw_db_num_residues(const sw_db* db) { return db ? db->num_residues : -1; }

sw_status sw_search_batch_device(const sw_db* cdb, const uint8_t* d_queries,
                                 const int64_t* query_offsets, int32_t num_queries,
                                 const int8_t* matrix, int32_t gap_open, int32_t gap_extend,
                                 int32_t* d_scores, void* stream) {
    if (!cdb) return fail(SW_ERR_ARG, "db is null");
    sw_db* db = const_cast<sw_db*>(cdb);
    std::lock_guard<std::mutex> lock(db->mu);
    DeviceGuard guard(db->device);
    return search_device(db, d_queries, query_offsets, num_queries, matrix, gap_open, gap_extend,
                         d_scores, static_cast<cudaStream_t>(stream));
}

sw_status sw_search_batch(const sw_db* cdb, const uint8_t* const* queries, const int32_t* query_lens,
                          int32_t num_queries, const int8_t* matrix, int32_t gap_open,
                          int32_t gap_extend, int32_t* scores) {
    if (!cdb) return fail(SW_ERR_ARG, "db is null");
    if (num_queries < 0) return fail(SW_ERR_ARG, "num_queries < 0");
    if (num_queries > 0 && (!queries || !query_lens || !scores))
        return fail(SW_ERR_ARG, "null query/length/score pointer");
    sw_db* db = const_cast<sw_db*>(cdb);
    std::lock_guard<std::mutex> lock(db->mu);
    DeviceGuard guard(db->device);
    const int64_t N = db->layout.num_seqs;
    std::vector<int64_t> qoff(static_cast<size_t>(num_queries) + 1, 0);
    for (int q = 0; q < num_queries; ++q) {
        if (query_lens[q] < 0) return fail(SW_ERR_ARG, "query %d: negative length", q);
        if (query_lens[q] > 0 && !queries[q]) return fail(SW_ERR_ARG, "query %d is null", q);
        qoff[static_cast<size_t>(q) + 1] = qoff[static_cast<size_t>(q)] + query_lens[q];
    }
    std::vector<uint8_t> cat(static_cast<size_t>(std::max<int64_t>(qoff.back(), 1)));
    for (int q = 0; q < num_queries; ++q) {
        if (query_lens[q] > 0) std::memcpy(cat.data() + qoff[static_cast<size_t>(q)], queries[q], static_cast<size_t>(query_lens[q]));
    }
    for (int64_t i = 0; i < qoff.back(); ++i)
        if (cat[static_cast<size_t>(i)] >= db->A)
            return fail(SW_ERR_CODE, "query residue %lld has code %d >= alphabet_size %d",
                        static_cast<long long>(i), cat[static_cast<size_t>(i)], db->A);
    if (num_queries == 0 || N == 0) return SW_OK;
    CU(db->h_queries.ensure(cat.size()));
    CU(db->h_scores.ensure(static_cast<size_t>(N * num_queries)));
    CU(cudaMemcpyAsync(db->h_queries.ptr, cat.data(), cat.size(), cudaMemcpyHostToDevice, db->stream));
    sw_status s = search_device(db, db->h_queries.ptr, qoff.data(), num_queries, matrix, gap_open,
                                gap_extend, db->h_scores.ptr, db->stream);
    if (s != SW_OK) return s;
    CU(cudaMemcpyAsync(scores, db->h_scores.ptr, sizeof(int32_t) * N * num_queries,
                       cudaMemcpyDeviceToHost, db->stream));
    CU(cudaStreamSynchronize(db->stream));
    return SW_OK;
}

sw_status sw_search(const sw_db* db, const uint8_t* query, int32_t query_len, const int8_t* matrix,
                    int32_t gap_open, int32_t gap_extend, int32_t* scores) {
    const uint8_t* qs[1] = {query};
    const int32_t lens[1] = {query_len};
    return sw_search_batch(db, qs, lens, 1, matrix, gap_open, gap_extend, scores);
}

sw_status sw_get_stats(const sw_db* cdb, sw_stats* out) {
    if (!cdb || !out) return fail(SW_ERR_ARG, "null pointer");
    sw_db* db = const_cast<sw_db*>(cdb);
    std::lock_guard<std::mutex> lock(db->mu);
    DeviceGuard guard(db->device);
    sw_status s = finish_stats(db);
    if (s != SW_OK) return s;
    *out = db->stats;
    return SW_OK;
}

}  // extern "C"

// ================================================================= internal accessors
// Read-only view of a loaded database for other translation units of the library.

namespace swgb {

bool db_view(const sw_db* db, DbView* v) {
    if (!db || !v) return false;
    v->device = db->device;
    v->sms = db->sms;
    v->alphabet = db->A;
    v->num_seqs = db->layout.num_seqs;
    v->num_residues = db->num_residues;
    v->short_residues = db->layout.short_residues;
    v->num_groups = db->layout.num_groups;
    v->max_group_len = db->layout.max_group_len;
    v->max_len = db->layout.max_len;
    v->num_long = static_cast<int64_t>(db->layout.long_ids.size());
    v->flag_cap = db->flag_cap;
    v->inter_occ = db->inter_occ;
    v->intra_occ = db->intra_occ;
    v->inter = db->inter.ptr;
    v->group_off = db->group_off.ptr;
    v->group_len = db->group_len.ptr;
    v->perm = db->perm.ptr;
    v->plain = db->plain.ptr;
    v->plain_off = db->plain_off.ptr;
    v->long_ids = db->long_ids.ptr;
    return true;
}

sw_status set_last_error(sw_status st, const char* msg) { return fail(st, "%s", msg); }

void add_launches(int64_t n) { g_launches += n; }

}  // namespace swgb
