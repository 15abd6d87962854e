// Host runtime of libswgb: the device-resident database, the search orchestration (query
// profiles, persistent inter-task launch, intra-task launch for long subjects, int32 rescore
// of saturated lanes), cached launch plans replayed as CUDA graphs, and the C ABI declared in
// include/swgb.h.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/swgb.h"
#include "db_view.h"
#include "layout.h"
#include "runtime_internal.h"
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

#define CU(call)                                            \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

bool graphs_enabled() {
    const char* v = std::getenv("SWGB_GRAPHS");
    return !(v && v[0] == '0');
}

int64_t forced_split() {
    const char* v = std::getenv("SWGB_GROUP_SPLIT");
    return v ? std::atoll(v) : -1;
}

bool mq_enabled() {
    const char* v = std::getenv("SWGB_MQ");
    return !(v && v[0] == '0');
}

// Score profile instead of query profile in the single-query inter-task kernel.
bool score_profile_enabled() {
    const char* v = std::getenv("SWGB_SCORE_PROFILE");
    return v && v[0] == '1';
}

// Packed int16x2 wavefront kernel for the long subjects of multi-query searches (default on).
bool wave_enabled() {
    const char* v = std::getenv("SWGB_WAVE");
    return !(v && v[0] == '0');
}

// Packed int16x2 two-subject wavefront kernel for the routed groups of one-query searches
// (default on).
bool pair_enabled() {
    const char* v = std::getenv("SWGB_PAIR");
    return !(v && v[0] == '0');
}

// Two 16-lane wavefronts per warp for the shorter pairs of the two-subject kernel's bulk: 0
// never (default: measured slower, the two-pair items lengthen the end of the search), 1 for
// the whole bulk whenever they fit, -1 the plan's split where the cost model prefers it.
int pair_half_mode() {
    const char* v = std::getenv("SWGB_PAIR_HALF");
    if (!v || !v[0]) return 0;
    return v[0] == '0' ? 0 : v[0] == 'a' ? -1 : 1;
}

// Blocks per SM of the block int32 kernel (0: as many as fit).
int forced_intra_blocks_per_sm() {
    const char* v = std::getenv("SWGB_INTRA_BLOCKS_PER_SM");
    return v ? std::max(0, std::atoi(v)) : 0;
}

}  // namespace

namespace swgb {

DeviceGuard::DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
}

DeviceGuard::~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
}

sw_status set_last_error(sw_status st, const char* msg) { return fail(st, "%s", msg); }
void add_launches(int64_t n) { g_launches += n; }

void destroy_plans(sw_db* db) {
    for (auto& p : db->plans) {
        if (p->exec) cudaGraphExecDestroy(p->exec);
        p->exec = nullptr;
    }
    db->plans.clear();
}

// Two streams of T-row strips for the kernels that pair two queries per register: queries
// (longest first) go whole, strip by strip, to the stream with fewer strips; step k pairs strip
// k of stream a with strip k of stream b.  Absent lanes and first strips are flagged "first"
// (they start from the zero boundary), last strips "last" (their half's score is emitted).
std::vector<MqStep> build_streams(const std::vector<int32_t>& m, const std::vector<int32_t>& order,
                                  int T) {
    std::vector<int32_t> stream[2];
    int64_t len[2] = {0, 0};
    for (int32_t q : order) {
        const int32_t mq = m[static_cast<size_t>(q)];
        if (mq == 0) continue;
        const int x = len[0] <= len[1] ? 0 : 1;
        stream[x].push_back(q);
        len[x] += (mq + T - 1) / T;
    }
    const int64_t num_steps = std::max(len[0], len[1]);
    std::vector<MqStep> steps(static_cast<size_t>(num_steps), MqStep{-1, -1, 0, 0, kMqFirstA | kMqFirstB, 0});
    for (int x = 0; x < 2; ++x) {
        int64_t k = 0;
        for (int32_t q : stream[x]) {
            const int32_t S = (m[static_cast<size_t>(q)] + T - 1) / T;
            for (int32_t sidx = 0; sidx < S; ++sidx, ++k) {
                MqStep& st = steps[static_cast<size_t>(k)];
                uint32_t fl = st.flags & (x == 0 ? (kMqFirstB | kMqLastB) : (kMqFirstA | kMqLastA));
                if (sidx == 0) fl |= (x == 0 ? kMqFirstA : kMqFirstB);
                if (sidx == S - 1) fl |= (x == 0 ? kMqLastA : kMqLastB);
                st.flags = fl;
                if (x == 0) {
                    st.qa = q;
                    st.sa = sidx;
                } else {
                    st.qb = q;
                    st.sb = sidx;
                }
            }
        }
    }
    return steps;
}

// Two streams of lanes for the two-query wavefront: a query of m rows takes ceil(m / kTB)
// lanes; queries (longest first) go to the stream with fewer lanes, and each stream is cut into
// passes of 32 lanes, so a pass can hold the end of one query and the start of the next.
std::vector<WavePass> build_wave_passes(const std::vector<int32_t>& m, const std::vector<int32_t>& order,
                                        int kTB) {
    std::vector<int32_t> stream[2];
    int64_t lanes[2] = {0, 0};
    for (int32_t q : order) {
        const int32_t mq = m[static_cast<size_t>(q)];
        if (mq == 0) continue;
        const int x = lanes[0] <= lanes[1] ? 0 : 1;
        stream[x].push_back(q);
        lanes[x] += (mq + kTB - 1) / kTB;
    }
    const int64_t num_passes = (std::max(lanes[0], lanes[1]) + kWarp - 1) / kWarp;
    WavePass none{};
    for (int x = 0; x < 2; ++x) {
        none.first[x] = 0xFFFFFFFFu;
        none.last[x] = 0u;
        for (int l = 0; l < kWarp; ++l) {
            none.q[x][l] = -1;
            none.row0[x][l] = 0;
        }
    }
    std::vector<WavePass> passes(static_cast<size_t>(num_passes), none);
    for (int x = 0; x < 2; ++x) {
        int64_t g = 0;
        for (int32_t q : stream[x]) {
            const int32_t L = (m[static_cast<size_t>(q)] + kTB - 1) / kTB;
            for (int32_t i = 0; i < L; ++i, ++g) {
                WavePass& wp = passes[static_cast<size_t>(g / kWarp)];
                const int l = static_cast<int>(g % kWarp);
                const uint32_t bit = 1u << l;
                wp.q[x][l] = q;
                wp.row0[x][l] = i * kTB;
                if (i == 0)
                    wp.first[x] |= bit;
                else
                    wp.first[x] &= ~bit;
                if (i == L - 1) wp.last[x] |= bit;
            }
        }
    }
    return passes;
}

// Grows the shared scratch (control block, saturation list, boundary buffers).  Cached plans
// bake these pointers into their graphs, so a reallocation drops them.
sw_status ensure_scratch(sw_db* db, size_t flag_cap, size_t bnd_elems, size_t spill_elems) {
    const bool grow = !db->ctrl.ptr || flag_cap > db->flags.cap || bnd_elems > db->bnd.cap ||
                      spill_elems > db->spill.cap;
    if (!grow) return SW_OK;
    if (db->stream) cudaStreamSynchronize(db->stream);
    if (db->done_recorded) cudaEventSynchronize(db->ev[4]);
    destroy_plans(db);
    CU(db->ctrl.ensure(1));
    CU(db->flags.ensure(std::max(flag_cap, db->flags.cap)));
    CU(db->bnd.ensure(std::max(bnd_elems, db->bnd.cap)));
    CU(db->spill.ensure(std::max(spill_elems, db->spill.cap)));
    return SW_OK;
}

int64_t max_m_of(const Plan& P) {
    int64_t mx = 0;
    for (int32_t m : P.m) mx = std::max<int64_t>(mx, m);
    return mx;
}

// Builds the launch plan of one search shape: host tables, device copies, kernel parameters.
sw_status build_plan(sw_db* db, const int64_t* h_qoff, int32_t nq, const int8_t* h_matrix,
                     int max_s, int32_t goe, int32_t ge, int32_t* d_scores,
                     std::vector<int64_t> key, Plan** out) {
    const int32_t A = db->A;
    const int64_t N = db->layout.num_seqs;
    auto plan = std::make_unique<Plan>();
    Plan& P = *plan;
    P.key = std::move(key);
    P.nq = nq;
    P.d_scores = d_scores;
    P.int16_ok = goe <= 16383 && ge <= 16383;
    P.qp_bias = (goe + 128 <= 32767) ? goe : 0;   // profile entries stay in int16
    P.variant = db->variant;
    P.m.resize(static_cast<size_t>(nq));
    for (int q = 0; q < nq; ++q)
        P.m[static_cast<size_t>(q)] = static_cast<int32_t>(h_qoff[q + 1] - h_qoff[q]);

    std::vector<int64_t> qp_off(static_cast<size_t>(nq));
    std::vector<int32_t> mpad(static_cast<size_t>(nq));
    int64_t total_qp = 0;
    for (int q = 0; q < nq; ++q) {
        const int64_t mp = round_up(std::max<int64_t>(P.m[static_cast<size_t>(q)], 1), kQpRows);
        mpad[static_cast<size_t>(q)] = static_cast<int32_t>(mp);
        qp_off[static_cast<size_t>(q)] = total_qp;
        total_qp += mp * (A + 1);
        P.max_mpad = std::max(P.max_mpad, mp);
    }
    std::vector<int32_t> order(static_cast<size_t>(nq));
    for (int q = 0; q < nq; ++q) order[static_cast<size_t>(q)] = q;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return P.m[static_cast<size_t>(a)] > P.m[static_cast<size_t>(b)];
    });

    int nonempty = 0;
    for (int q = 0; q < nq; ++q) nonempty += P.m[static_cast<size_t>(q)] > 0;
    // Score-profile kernel (single-query launches only; 32 rows per strip, 4 warps per block).
    P.sp = score_profile_enabled() && P.int16_ok && !(mq_enabled() && nonempty >= 2) &&
           db->inter_sp_occ > 0;
    if (P.sp) P.variant = 0;

    // Work items of the inter-task kernel: (query, W consecutive groups), largest first.
    const int W = P.sp ? inter_sp_warps() : inter_variant_warps(P.variant);
    std::vector<InterItem> items;
    const int64_t G = db->layout.num_groups;
    if (P.int16_ok && G > 0) {
        const int64_t chunks = (G + W - 1) / W;
        std::vector<int64_t> cost;
        items.reserve(static_cast<size_t>(chunks * nq));
        cost.reserve(static_cast<size_t>(chunks * nq));
        for (int32_t q : order) {
            if (P.m[static_cast<size_t>(q)] == 0) continue;
            for (int64_t c = chunks - 1; c >= 0; --c) {
                const int64_t g0 = c * W;
                const int32_t ng = static_cast<int32_t>(std::min<int64_t>(W, G - g0));
                items.push_back(InterItem{q, static_cast<int32_t>(g0), ng, 0});
                cost.push_back(static_cast<int64_t>(P.m[static_cast<size_t>(q)]) *
                               db->layout.group_len[static_cast<size_t>(g0 + ng - 1)]);
            }
        }
        std::vector<int32_t> idx(items.size());
        for (size_t i = 0; i < idx.size(); ++i) idx[i] = static_cast<int32_t>(i);
        std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
        std::vector<InterItem> sorted(items.size());
        for (size_t i = 0; i < idx.size(); ++i) sorted[i] = items[static_cast<size_t>(idx[i])];
        items.swap(sorted);
    }
    P.num_items = static_cast<int64_t>(items.size());
    if (P.num_items > INT32_MAX) return fail(SW_ERR_ARG, "too many work items");

    // Two or more queries: pair them two per register (multi-query kernel).  Queries go, strip
    // by strip, into two streams balanced by strip count, longest first.
    std::vector<MqStep> steps;
    const int mqT = inter_mq_variant_rows(P.variant);
    P.mq = mq_enabled() && P.int16_ok && G > 0 && nonempty >= 2 &&
           db->inter_mq_occ[P.variant] > 0;
    if (P.mq) {
        steps = build_streams(P.m, order, mqT);
        P.num_steps = static_cast<int32_t>(steps.size());
        P.rows_pad = round_up(static_cast<int64_t>(P.num_steps) * mqT, kQpRows);
    }

    // Long subjects of a search with two or more queries: the packed wavefront kernel pairs two
    // queries per register against one subject (passes of 32 x 8, 12 or 16 rows).
    std::vector<WavePass> wpasses;
    P.wave = wave_enabled() && P.int16_ok && nonempty >= 2 && !db->layout.long_ids.empty() &&
             db->wave_occ[0] > 0 && db->wave_occ[1] > 0 && db->wave_occ[2] > 0;
    if (P.wave) {
        // the pass height with the fewest computed rows (both streams, padding included),
        // charging about 10 operations of per-step overhead per lane
        double best_cost = 1e300;
        for (int v = 0; v < 3; ++v) {
            const int T = 32 * kWaveRows[v];
            const double passes_v = static_cast<double>(build_wave_passes(P.m, order, kWaveRows[v]).size());
            const double cost = passes_v * 2.0 * T * (5.5 + 10.0 / kWaveRows[v]);
            if (cost < best_cost * 0.999) {
                best_cost = cost;
                P.wave_rows = kWaveRows[v];
            }
        }
        const char* wr = std::getenv("SWGB_WAVE_ROWS");
        if (wr && (std::atoi(wr) == 8 || std::atoi(wr) == 12 || std::atoi(wr) == 16)) P.wave_rows = std::atoi(wr);
        const int T = 32 * P.wave_rows;
        wpasses = build_wave_passes(P.m, order, P.wave_rows);
        P.num_wpasses = static_cast<int32_t>(wpasses.size());
        P.wrows_pad = round_up(static_cast<int64_t>(P.num_wpasses) * T, kQpRows);
        const int occ = db->wave_occ[P.wave_rows == 8 ? 0 : P.wave_rows == 12 ? 1 : 2];
        const int64_t items = (static_cast<int64_t>(db->layout.long_ids.size()) + wave_warps() - 1) / wave_warps();
        P.wave_grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(items, static_cast<int64_t>(db->sms) * occ)));
    }

    // Groups whose single-warp work would outlast the rest of the search run on the int32
    // intra-task kernel instead (one warp per pair): pick the split that minimises
    // max(inter work / rate, longest inter item) + routed work / intra rate.
    int64_t max_m_q = 0;
    for (int q = 0; q < nq; ++q) max_m_q = std::max<int64_t>(max_m_q, P.m[static_cast<size_t>(q)]);
    {
        const double scale = db->sms / 152.0;
        // the int32 kernel computes whole passes of 32 x (5, 8 or 16) rows: charge it for the
        // padded rows and the per-step overhead, relative to 16 rows per lane
        double padded = 0.0, real = 0.0;
        for (int q = 0; q < nq; ++q) {
            const double mq = P.m[static_cast<size_t>(q)];
            real += mq;
            double c = 1e300;
            for (int v = 0; v < 3; ++v) {
                const double tb = kIntraBlockRows[v], rows = 32.0 * tb;
                c = std::min(c, std::ceil(mq / rows) * rows * (5.5 + 10.0 / tb) / (5.5 + 10.0 / 16));
            }
            padded += c;
        }
        const double r_inter = (P.mq ? 6.5e12 : 5.4e12) * scale;
        // a one-query search routes its groups to the packed two-subject wavefront kernel
        const bool pair_route = pair_enabled() && P.int16_ok && nonempty == 1 &&
                                wave_ss_fits(5, A + 1, static_cast<int>(std::max<int64_t>(1, max_m_q)),
                                             db->layout.max_group_len, db->max_smem, false);
        const double r_intra = (pair_route ? 4.0e12 : 3.0e12) * scale * (padded > 0 ? real / padded : 1.0);
        const int64_t warps = static_cast<int64_t>(db->sms) *
                              std::max(1, P.mq ? db->inter_mq_occ[P.variant] : db->inter_occ[P.variant]) * W;
        double sum_m = 0, max_m = 0;
        for (int q = 0; q < nq; ++q) {
            sum_m += P.m[static_cast<size_t>(q)];
            max_m = std::max<double>(max_m, P.m[static_cast<size_t>(q)]);
        }
        const double per_item_rows = P.mq ? sum_m * 32.0 : max_m * 64.0;
        int64_t best_s = G;
        if (P.int16_ok && G > 0) {
            std::vector<double> pre(static_cast<size_t>(G) + 1, 0.0);
            for (int64_t g = 0; g < G; ++g)
                pre[static_cast<size_t>(g) + 1] = pre[static_cast<size_t>(g)] + db->layout.group_res[static_cast<size_t>(g)];
            double best_t = 1e300;
            for (int64_t s = G; s >= 0; --s) {
                const double w_in = sum_m * pre[static_cast<size_t>(s)];
                const double w_out = sum_m * (pre[static_cast<size_t>(G)] - pre[static_cast<size_t>(s)]);
                const double crit = s > 0 ? per_item_rows * db->layout.group_len[static_cast<size_t>(s - 1)] * warps / r_inter : 0.0;
                const double t = std::max(w_in / r_inter, crit) + w_out / r_intra;
                if (t < best_t * 0.999) {
                    best_t = t;
                    best_s = s;
                }
            }
        }
        const int64_t f = forced_split();
        if (f >= 0) best_s = std::min<int64_t>(f, G);
        if (db->no_route) best_s = G;
        P.g_split = best_s;
    }
    if (P.g_split < G && !items.empty()) {   // drop the routed groups from the inter items
        std::vector<InterItem> kept;
        kept.reserve(items.size());
        for (const InterItem& it : items) {
            if (it.group >= P.g_split) continue;
            InterItem k2 = it;
            k2.ngroups = static_cast<int32_t>(std::min<int64_t>(it.ngroups, P.g_split - it.group));
            kept.push_back(k2);
        }
        items.swap(kept);
        P.num_items = static_cast<int64_t>(items.size());
    }
    if (P.g_split == 0) P.mq = false;
    // One query with routed groups: the packed two-subject wavefront kernel, if its whole
    // profile fits in shared memory: 32-lane wavefronts with passes of 160 or 256 rows (the
    // cheaper padded height), and, for the bulk's shorter pairs, two 16-lane wavefronts of
    // 144-row passes per warp (a 15-step fill per slot pair instead of 31) when they fit and
    // cost less.
    P.pair = false;
    P.pair_half = false;
    if (pair_enabled() && P.int16_ok && nonempty == 1 && P.g_split < G) {
        const int mq = static_cast<int>(max_m_q);
        const int mgl = db->layout.max_group_len;
        double best_cost = 1e300;
        for (int v = 0; v < 2; ++v) {
            const int rows_l = kWaveSsRows[v];
            if (!wave_ss_fits(rows_l, A + 1, mq, mgl, db->max_smem, false)) continue;
            const double rows = 32.0 * rows_l;
            const double cost = std::ceil(max_m_q / rows) * rows * (6.5 + 12.0 / rows_l);
            if (cost < best_cost * 0.999) {
                best_cost = cost;
                P.pair_rows = rows_l;
                P.pair = true;
            }
        }
        if (P.pair && (pair_half_mode() != 0 || std::getenv("SWGB_PAIR_HALF_FROM") != nullptr) &&
            wave_ss_fits(P.pair_rows, A + 1, mq, mgl, db->max_smem, true)) {
            double n_avg = 0.0;
            for (int64_t g = P.g_split; g < G; ++g) n_avg += db->layout.group_len[static_cast<size_t>(g)];
            n_avg /= static_cast<double>(G - P.g_split);
            auto bulk_cost = [&](int tb, int lanes) {
                const double rows = static_cast<double>(lanes) * tb;
                return std::ceil(max_m_q / rows) * rows * (n_avg + lanes - 1) * (6.5 + 12.0 / tb);
            };
            P.pair_half = pair_half_mode() == 1 || std::getenv("SWGB_PAIR_HALF_FROM") != nullptr ||
                          bulk_cost(wave_ss_bulk_rows(), wave_ss_bulk_lanes()) < 0.999 * bulk_cost(P.pair_rows, kWarp);
        }
    }
    P.g_pair_end = P.pair ? G : P.g_split;
    if (P.pair) {
        P.pair_grid = db->sms * wave_ss_blocks_per_sm();
        // Work split (slot pairs longest first: a first phase, 32-lane items, 16-lane items).
        // Model in ALU-pipe clocks (a warp issues half an instruction per clock): a 32-lane step
        // of kTB rows costs c_l = 2 (kTB x 6.5 + 8), a 16-lane step (two pairs) c_b =
        // 2 (9 x 6.5 + 8).  The bulk spreads over every sub-partition at ~70 % of the pipe and
        // takes t_bulk (estimated for the whole routed work on 32-lane wavefronts); there four
        // warps share a sub-partition, so an item lasts four times its issue time.  Groups whose
        // 32-lane items would outlast t_bulk go to the first phase (one warp alone per
        // sub-partition); the groups whose 16-lane items would not outlast t_bulk either run
        // two pairs per item (they start last).
        const int rows_l = P.pair_rows;
        const double c_l = 2.0 * (rows_l * 6.5 + 8.0);
        const double passes_l = std::ceil(static_cast<double>(max_m_q) / (32.0 * rows_l));
        const double c_b = 2.0 * (wave_ss_bulk_rows() * 6.5 + 8.0);
        const double passes_b = std::ceil(static_cast<double>(max_m_q) /
                                          (static_cast<double>(wave_ss_bulk_lanes()) * wave_ss_bulk_rows()));
        auto item_l = [&](int64_t g) {   // issue clocks of one pair on a 32-lane wavefront
            return (db->layout.group_len[static_cast<size_t>(g)] + 31.0) * passes_l * c_l;
        };
        auto item_b = [&](int64_t g) {   // issue clocks of two pairs on 16-lane wavefronts
            return (db->layout.group_len[static_cast<size_t>(g)] + 15.0) * passes_b * c_b;
        };
        const int64_t routed = G - P.g_split;
        double clocks = 0.0;   // the whole routed work on 32-lane wavefronts
        for (int64_t g = P.g_split; g < G; ++g) clocks += (kGroupSeqs / 2) * item_l(g);
        const double t_bulk = clocks / (4.0 * db->sms) / 0.7;
        int64_t long_groups = 0, half_groups = 0;
        for (int64_t g = G - 1; g >= P.g_split && 4.0 * item_l(g) / 0.7 > t_bulk; --g) ++long_groups;
        if (P.pair_half)
            for (int64_t g = P.g_split; g < G - long_groups && 4.0 * item_b(g) / 0.7 <= t_bulk; ++g)
                ++half_groups;
        const char* ev = std::getenv("SWGB_LONG_PAIRS");
        int64_t long_pairs = long_groups * (kGroupSeqs / 2);
        if (ev) long_pairs = std::max<int64_t>(0, std::atoll(ev));
        P.pair_long_pairs = long_pairs;
        P.pair_long_blocks = static_cast<int>(std::min<int64_t>(
            db->sms / 2, (long_pairs + wave_ss_long_warps() - 1) / wave_ss_long_warps()));
        const char* eb = std::getenv("SWGB_LONG_BLOCKS");
        if (eb) P.pair_long_blocks = std::max(0, std::min(db->sms, std::atoi(eb)));
        // 16-lane items from pair half_from on (pair 0 = the longest)
        P.pair_half_from = (routed - half_groups) * (kGroupSeqs / 2);
        if (pair_half_mode() == 1) P.pair_half_from = 0;
        const char* eh = std::getenv("SWGB_PAIR_HALF_FROM");
        if (eh && P.pair_half) P.pair_half_from = std::max<int64_t>(0, std::atoll(eh));
        if (!P.pair_half) P.pair_half_from = routed * (kGroupSeqs / 2);
    }

    // Scratch shared by all plans of this database.
    P.inter_grid = db->sms * std::max(1, P.mq ? db->inter_mq_occ[P.variant]
                                              : P.sp ? db->inter_sp_occ : db->inter_occ[P.variant]);
    P.intra_grid = db->sms * std::max(1, db->intra_occ);
    // Rows per lane of the block int32 kernel: the fewer padded rows (with a per-step overhead
    // of about 10 operations per lane against 5.5 per cell) the better.
    int tb_index = 2;
    {
        double best_cost = 1e300;
        for (int v = 0; v < 3; ++v) {
            double cost = 0.0;
            for (int q = 0; q < nq; ++q) {
                const double rows = 32.0 * kIntraBlockRows[v];
                cost += std::ceil(P.m[static_cast<size_t>(q)] / rows) * rows * (5.5 + 10.0 / kIntraBlockRows[v]);
            }
            if (db->intra_block_occ[v] > 0 && cost < best_cost * 0.999) {
                best_cost = cost;
                tb_index = v;
            }
        }
        P.intra_rows_per_lane = kIntraBlockRows[tb_index];
    }
    // the block variant shares the per-warp pass buffers: never more blocks than the generic grid
    {
        // With few block items (a small database searched by a short query), the search ends
        // with the longest subjects' warps, each sharing its SM sub-partition with the other
        // resident warps; at most three 4-warp blocks per SM (three warps per sub-partition)
        // shortens that tail more than it costs in latency hiding (measured: 144 residues vs
        // 10,000 sequences 0.38 -> 0.33 ms).  The 8-warp blocks of long queries keep every block
        // that fits (one per SM ran 1,000 residues vs 10,000 long subjects 12 % slower).
        int per_sm = db->intra_block_occ[tb_index];
        const int bw = intra_block_warps(P.intra_rows_per_lane);
        const int64_t n_subjects = static_cast<int64_t>(db->layout.long_ids.size()) +
                                   static_cast<int64_t>(G - P.g_pair_end) * kGroupSeqs;
        const int64_t block_items = (n_subjects + bw - 1) / bw * nq;
        if (bw == 4 && block_items < 8LL * db->sms * per_sm) per_sm = std::min(per_sm, 3);
        const int forced = forced_intra_blocks_per_sm();
        if (forced > 0) per_sm = std::min(db->intra_block_occ[tb_index], forced);
        P.intra_block_grid = db->sms * per_sm;
        P.intra_block_warps = bw;
    }
    const int64_t inter_slots = static_cast<int64_t>(P.inter_grid) * W;
    // per-warp pass buffers, shared by the generic and the block kernel
    const int64_t intra_slots = std::max<int64_t>(
        std::max<int64_t>(static_cast<int64_t>(P.intra_grid) * (intra_block_threads() / kWarp),
                          static_cast<int64_t>(P.intra_block_grid) * P.intra_block_warps),
        std::max<int64_t>(static_cast<int64_t>(P.wave_grid) * wave_warps(),
                          static_cast<int64_t>(P.pair_grid) * wave_ss_warps() * 2));
    const int64_t bnd_stride = std::max<int64_t>(1, db->layout.max_group_len / 2 * kWarp);
    const int64_t spill_stride = std::max<int64_t>(1, round_up(db->layout.max_len, 32) + 64);
    P.flag_cap = static_cast<uint32_t>(std::min<int64_t>(std::max<int64_t>(N * nq, 1), db->flag_cap));
    sw_status s = ensure_scratch(db, P.flag_cap, static_cast<size_t>(inter_slots * bnd_stride),
                                 static_cast<size_t>(intra_slots * spill_stride));
    if (s != SW_OK) return s;

    // Plan-owned device tables (uploaded once, synchronously, on the database's own stream).
    CU(P.qp.ensure(static_cast<size_t>(total_qp)));
    CU(P.descs.ensure(static_cast<size_t>(nq)));
    CU(P.items.ensure(std::max<size_t>(items.size(), 1)));
    CU(P.qp_off.ensure(static_cast<size_t>(nq)));
    CU(P.mpad.ensure(static_cast<size_t>(nq)));
    CU(P.qoff.ensure(static_cast<size_t>(nq) + 1));
    CU(P.order.ensure(static_cast<size_t>(nq)));
    CU(P.matrix.ensure(static_cast<size_t>(A * A)));
    std::vector<int16_t> mt;
    if (P.sp) {   // transposed biased matrix: mt[s][a] = SM(a, s) + bias, the dummy letter scores 0
        const int ms = inter_sp_mt_stride();
        mt.assign(static_cast<size_t>((A + 1) * ms), static_cast<int16_t>(P.qp_bias));
        for (int sl = 0; sl < A; ++sl)
            for (int a = 0; a < A; ++a)
                mt[static_cast<size_t>(sl * ms + a)] = static_cast<int16_t>(h_matrix[a * A + sl] + P.qp_bias);
        CU(P.mt.ensure(mt.size()));
    }
    if (P.mq) {
        CU(P.steps.ensure(steps.size()));
        CU(P.pp.ensure(static_cast<size_t>((A + 1) * P.rows_pad)));
    }
    if (P.wave) {
        CU(P.wpasses.ensure(wpasses.size()));
        CU(P.wpp.ensure(static_cast<size_t>((A + 1) * P.wrows_pad)));
    }
    std::vector<QueryDesc> descs(static_cast<size_t>(nq));
    for (int q = 0; q < nq; ++q)
        descs[static_cast<size_t>(q)] = QueryDesc{P.qp.ptr + qp_off[static_cast<size_t>(q)],
                                                  d_scores + static_cast<int64_t>(q) * N,
                                                  P.m[static_cast<size_t>(q)], mpad[static_cast<size_t>(q)]};
    cudaStream_t us = db->stream;
    CU(cudaMemcpyAsync(P.descs.ptr, descs.data(), sizeof(QueryDesc) * nq, cudaMemcpyHostToDevice, us));
    if (!items.empty())
        CU(cudaMemcpyAsync(P.items.ptr, items.data(), sizeof(InterItem) * items.size(),
                           cudaMemcpyHostToDevice, us));
    CU(cudaMemcpyAsync(P.qp_off.ptr, qp_off.data(), sizeof(int64_t) * nq, cudaMemcpyHostToDevice, us));
    CU(cudaMemcpyAsync(P.mpad.ptr, mpad.data(), sizeof(int32_t) * nq, cudaMemcpyHostToDevice, us));
    CU(cudaMemcpyAsync(P.qoff.ptr, h_qoff, sizeof(int64_t) * (nq + 1), cudaMemcpyHostToDevice, us));
    CU(cudaMemcpyAsync(P.order.ptr, order.data(), sizeof(int32_t) * nq, cudaMemcpyHostToDevice, us));
    CU(cudaMemcpyAsync(P.matrix.ptr, h_matrix, static_cast<size_t>(A * A), cudaMemcpyHostToDevice, us));
    if (P.mq)
        CU(cudaMemcpyAsync(P.steps.ptr, steps.data(), sizeof(MqStep) * steps.size(),
                           cudaMemcpyHostToDevice, us));
    if (P.sp)
        CU(cudaMemcpyAsync(P.mt.ptr, mt.data(), sizeof(int16_t) * mt.size(), cudaMemcpyHostToDevice, us));
    if (P.wave)
        CU(cudaMemcpyAsync(P.wpasses.ptr, wpasses.data(), sizeof(WavePass) * wpasses.size(),
                           cudaMemcpyHostToDevice, us));
    CU(cudaStreamSynchronize(us));

    const Gaps gaps{goe, ge, std::min(goe, ge)};
    InterParams& ip = P.inter;
    ip.inter = db->inter_ptr;
    ip.group_off = db->group_off.ptr;
    ip.group_len = db->group_len.ptr;
    ip.group_cols = db->group_cols.ptr;
    ip.perm = db->perm.ptr;
    ip.queries = P.descs.ptr;
    ip.items = P.items.ptr;
    ip.num_items = static_cast<int32_t>(P.num_items);
    ip.alphabet1 = A + 1;
    ip.ctrl = db->ctrl.ptr;
    ip.flags = db->flags.ptr;
    ip.flag_cap = P.flag_cap;
    ip.thresh = 32767 - std::max(0, max_s);
    ip.bnd = db->bnd.ptr;
    ip.bnd_stride = bnd_stride;
    ip.gaps = gaps;
    ip.qres_off = P.qoff.ptr;
    ip.mt = P.sp ? P.mt.ptr : nullptr;
    if (P.mq) {
        InterMqParams& mp = P.inter_mq;
        mp.inter = db->inter_ptr;
        mp.group_off = db->group_off.ptr;
        mp.group_len = db->group_len.ptr;
        mp.group_cols = db->group_cols.ptr;
        mp.perm = db->perm.ptr;
        mp.queries = P.descs.ptr;
        mp.pp = P.pp.ptr;
        mp.rows_pad = P.rows_pad;
        mp.steps = P.steps.ptr;
        mp.num_steps = P.num_steps;
        mp.num_half_groups = static_cast<int32_t>(2 * P.g_split);
        mp.alphabet1 = A + 1;
        mp.ctrl = db->ctrl.ptr;
        mp.flags = db->flags.ptr;
        mp.flag_cap = P.flag_cap;
        mp.thresh = ip.thresh;
        mp.bnd = db->bnd.ptr;
        mp.bnd_stride = bnd_stride;
        mp.gaps = gaps;
        mp.tick = nullptr;
    }
    if (P.wave) {
        WaveParams& wp = P.wave_p;
        wp.plain = db->plain_ptr;
        wp.plain_off = db->plain_off.ptr;
        wp.subjects = db->long_ids.ptr;
        wp.num_subjects = static_cast<int64_t>(db->layout.long_ids.size());
        wp.queries = P.descs.ptr;
        wp.pp = P.wpp.ptr;
        wp.rows_pad = P.wrows_pad;
        wp.passes = P.wpasses.ptr;
        wp.num_passes = P.num_wpasses;
        wp.alphabet1 = A + 1;
        wp.ctrl = db->ctrl.ptr;
        wp.flags = db->flags.ptr;
        wp.flag_cap = P.flag_cap;
        wp.thresh = ip.thresh;
        wp.spill = db->spill.ptr;
        wp.spill_stride = spill_stride;
        wp.gaps = gaps;
    }
    if (P.pair) {
        WaveParams& wp = P.pair_p;
        wp.plain_off = db->plain_off.ptr;
        wp.queries = P.descs.ptr;
        for (int q = 0; q < nq; ++q)
            if (P.m[static_cast<size_t>(q)] > 0) wp.query = q;
        wp.inter = db->inter_ptr;
        wp.group_off = db->group_off.ptr;
        wp.group_len = db->group_len.ptr;
        wp.perm = db->perm.ptr;
        wp.group_begin = P.g_split;
        wp.group_end = P.g_pair_end;
        wp.long_pairs = P.pair_long_pairs;
        wp.half_from = P.pair_half_from;
        wp.prefix_f = static_cast<int64_t>(goe) + static_cast<int64_t>(P.pair_rows) * std::min(goe, ge) <= 32767 ? 1 : 0;
        wp.max_group_len = db->layout.max_group_len;
        wp.qres_off = P.qoff.ptr;
        wp.matrix = P.matrix.ptr;
        wp.long_blocks = P.pair_long_blocks;
        wp.alphabet1 = A + 1;
        wp.ctrl = db->ctrl.ptr;
        wp.flags = db->flags.ptr;
        wp.flag_cap = P.flag_cap;
        wp.thresh = ip.thresh;
        wp.spill = db->spill.ptr;
        wp.spill_stride = spill_stride;
        wp.gaps = gaps;
        wp.qp_out = P.qp.ptr + qp_off[static_cast<size_t>(wp.query)];
        wp.qp_mpad = mpad[static_cast<size_t>(wp.query)];
        wp.qp_bias = P.qp_bias;
    }
    IntraParams& jp = P.intra;
    jp.plain = db->plain_ptr;
    jp.plain_off = db->plain_off.ptr;
    jp.queries = P.descs.ptr;
    jp.num_queries = nq;
    jp.long_ids = db->long_ids.ptr;
    jp.num_long = static_cast<int64_t>(db->layout.long_ids.size());
    jp.query_order = P.order.ptr;
    jp.num_seqs = N;
    jp.flags = db->flags.ptr;
    jp.flag_cap = P.flag_cap;
    jp.alphabet1 = A + 1;
    jp.ctrl = db->ctrl.ptr;
    jp.spill = db->spill.ptr;
    jp.spill_stride = spill_stride;
    jp.gaps = gaps;
    jp.qp_add = goe - P.qp_bias;
    jp.perm = db->perm.ptr;
    jp.slot_begin = P.g_pair_end * kGroupSeqs;
    jp.slot_end = G * kGroupSeqs;

    for (int q = 0; q < nq; ++q) {
        P.cells += static_cast<int64_t>(P.m[static_cast<size_t>(q)]) * db->num_residues;
        if (P.int16_ok) {
            int64_t res_in = 0;
            for (int64_t g = 0; g < P.g_split; ++g) res_in += db->layout.group_res[static_cast<size_t>(g)];
            P.inter_cells += static_cast<int64_t>(P.m[static_cast<size_t>(q)]) * res_in;
        }
    }
    if (db->plans.size() >= 32) {
        if (db->done_recorded) cudaEventSynchronize(db->ev[4]);   // its graph may still run
        if (db->plans.front()->exec) cudaGraphExecDestroy(db->plans.front()->exec);
        db->plans.erase(db->plans.begin());
    }
    db->plans.push_back(std::move(plan));
    *out = db->plans.back().get();
    return SW_OK;
}

// Event records become external event nodes when captured, so the timing events (and ev[4],
// which orders the next search) stay usable after a graph replay.
cudaError_t record(cudaEvent_t ev, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) cs = cudaStreamCaptureStatusNone;
    return cs == cudaStreamCaptureStatusActive
               ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal)
               : cudaEventRecord(ev, st);
}

// A one-query search whose every group runs on the two-subject wavefront kernel.
bool pair_only_plan(const sw_db* db, const Plan& P) {
    return P.pair && P.int16_ok && P.num_items == 0 && !P.mq && db->layout.long_ids.empty() &&
           P.g_pair_end == db->layout.num_groups && !P.wave;
}

// Enqueues the launch sequence of a plan on `st` (captured into a graph or run directly).
sw_status enqueue_plan(sw_db* db, Plan& P, const uint8_t* d_queries, cudaStream_t st) {
    const int64_t N = db->layout.num_seqs;
    int64_t launches = 0;
    CU(record(db->ev[0], st));
    CU(cudaMemsetAsync(db->ctrl.ptr, 0, sizeof(Control), st));
    for (int q = 0; q < P.nq; ++q)   // empty queries score 0 everywhere
        if (P.m[static_cast<size_t>(q)] == 0 && N > 0)
            CU(cudaMemsetAsync(P.d_scores + static_cast<int64_t>(q) * N, 0, sizeof(int32_t) * N, st));
    // A one-query search that runs only the two-subject wavefront kernel (which builds its own
    // profile) needs the int16 query profile for the rescore alone: that kernel writes it too,
    // and the rescore follows as its programmatic dependent (launched while it runs, waiting
    // for its completion), with no event node between them.
    const bool pair_only = pair_only_plan(db, P);
    if (!pair_only) {
        CU(launch_build_qp(d_queries, P.qoff.ptr, P.nq, P.matrix.ptr, db->A, P.qp_bias, P.qp_off.ptr,
                           P.mpad.ptr, P.qp.ptr, P.max_mpad, db->ctrl.ptr, st));
        ++launches;
    }
    if (P.wave) {
        CU(launch_build_pp_wave(d_queries, P.qoff.ptr, P.wpasses.ptr, P.num_wpasses, P.wave_rows,
                                P.matrix.ptr, db->A, P.qp_bias, P.wpp.ptr, P.wrows_pad,
                                db->ctrl.ptr, st));
        ++launches;
    }
    // An event node costs about two microseconds of a replay: the inter-task stage is bracketed
    // only when the plan has one.
    const bool inter_stage = P.mq || P.num_items > 0;
    if (inter_stage) CU(record(db->ev[1], st));
    if (P.mq) {
        CU(launch_build_pp(d_queries, P.qoff.ptr, nullptr, P.steps.ptr, P.num_steps, nullptr,
                           inter_mq_variant_rows(P.variant), P.matrix.ptr, db->A, P.qp_bias,
                           P.pp.ptr, P.rows_pad, db->ctrl.ptr, st));
        CU(launch_inter_mq(P.inter_mq, P.variant, P.inter_grid, st));
        launches += 2;
    } else if (P.num_items > 0) {
        if (P.sp) {
            InterParams ip = P.inter;
            ip.qres = d_queries;
            CU(launch_inter_sp(ip, P.inter_grid, st));
        } else {
            CU(launch_inter(P.inter, P.variant, P.inter_grid, st));
        }
        ++launches;
    }
    CU(record(db->ev[2], st));
    IntraParams jp = P.intra;
    if (!P.int16_ok) {
        jp.mode = kIntraAll;
        if (N > 0) {
            CU(launch_intra(jp, P.intra_grid, intra_block_threads(), st));
            ++launches;
        }
    } else {
        if (jp.num_long > 0) {
            jp.mode = kIntraLong;
            if (P.wave)
                CU(launch_wave_mq(P.wave_p, P.wave_rows, P.wave_grid, st));
            else
                CU(P.intra_block_grid > 0 ? launch_intra_block(jp, P.intra_rows_per_lane, P.intra_block_grid, st)
                                          : launch_intra(jp, P.intra_grid, intra_block_threads(), st));
            ++launches;
        }
        if (P.pair) {
            WaveParams pp = P.pair_p;
            pp.qres = d_queries;
            if (!pair_only) pp.qp_out = nullptr;
            CU(launch_wave_ss(pp, P.pair_rows, P.pair_half, static_cast<int>(max_m_of(P)), P.pair_grid, st));
            ++launches;
        }
        if (P.g_pair_end < db->layout.num_groups) {
            jp.mode = kIntraGroups;
            CU(P.intra_block_grid > 0 ? launch_intra_block(jp, P.intra_rows_per_lane, P.intra_block_grid, st)
                                      : launch_intra(jp, P.intra_grid, intra_block_threads(), st));
            ++launches;
        }
    }
    if (!pair_only) CU(record(db->ev[3], st));
    if (P.int16_ok && (P.num_items > 0 || P.mq || P.wave || P.pair)) {
        // one block per SM: saturated lanes are rare (the list is usually empty, and a launch
        // of blocks that find it empty costs in proportion to their number)
        jp.mode = kIntraRescore;
        CU(pair_only ? launch_intra_dependent(jp, std::min(P.intra_grid, db->sms), intra_block_threads(), st)
                     : launch_intra(jp, std::min(P.intra_grid, db->sms), intra_block_threads(), st));
        ++launches;
    }
    CU(record(db->ev[4], st));
    P.launches = launches;
    return SW_OK;
}

sw_status search_device(sw_db* db, const uint8_t* d_queries, const int64_t* h_qoff, int32_t nq,
                        const int8_t* h_matrix, int32_t gap_open, int32_t gap_extend,
                        int32_t* d_scores, cudaStream_t st) {
    if (nq < 0) return fail(SW_ERR_ARG, "num_queries < 0");
    if (gap_open < 0 || gap_extend < 0 || gap_open > 1000000 || gap_extend > 1000000)
        return fail(SW_ERR_ARG, "gap costs must be in [0, 1000000]");
    if (nq == 0) return SW_OK;
    if (!h_qoff || !d_scores || (!d_queries && h_qoff[nq] > 0))
        return fail(SW_ERR_ARG, "null query/offset/score pointer");
    if (!h_matrix) return fail(SW_ERR_ARG, "matrix is null");
    const int32_t A = db->A;
    int max_s = 0;
    for (int i = 0; i < A * A; ++i) max_s = std::max<int>(max_s, h_matrix[i]);
    if (h_qoff[0] != 0) return fail(SW_ERR_ARG, "query_offsets[0] must be 0");
    int64_t max_m = 0;
    for (int q = 0; q < nq; ++q) {
        const int64_t len = h_qoff[q + 1] - h_qoff[q];
        if (len < 0 || len > (int64_t{1} << 28))
            return fail(SW_ERR_ARG, "query %d: bad length %lld", q, static_cast<long long>(len));
        max_m = std::max(max_m, len);
    }
    if (static_cast<double>(std::min<int64_t>(max_m, db->layout.max_len)) * max_s > 2147483647.0)
        return fail(SW_ERR_ARG, "scores could exceed the int32 range");
    if (db->layout.num_seqs == 0) return SW_OK;

    // Identity of this search shape: pointers, lengths, costs, matrix, kernel variant.
    std::vector<int64_t> key;
    key.reserve(static_cast<size_t>(nq) + 8 + static_cast<size_t>(A * A));
    key.push_back(reinterpret_cast<int64_t>(d_queries));
    key.push_back(reinterpret_cast<int64_t>(d_scores));
    key.push_back(nq);
    key.push_back(gap_open);
    key.push_back(gap_extend);
    key.push_back(db->variant);
    key.push_back(mq_enabled() ? 1 : 0);
    key.push_back(forced_split());
    key.push_back(db->no_route ? 1 : 0);
    key.push_back(forced_intra_blocks_per_sm());
    key.push_back(score_profile_enabled() ? 1 : 0);
    key.push_back(wave_enabled() ? 1 : 0);
    key.push_back(pair_enabled() ? 1 : 0);
    key.push_back(pair_half_mode());
    {
        const char* ev = std::getenv("SWGB_LONG_PAIRS");
        key.push_back(ev ? std::atoll(ev) : -1);
        const char* eb = std::getenv("SWGB_LONG_BLOCKS");
        key.push_back(eb ? std::atoll(eb) : -1);
        const char* wr = std::getenv("SWGB_WAVE_ROWS");
        key.push_back(wr ? std::atoll(wr) : -1);
        const char* eh = std::getenv("SWGB_PAIR_HALF_FROM");
        key.push_back(eh ? std::atoll(eh) : -1);
    }
    for (int q = 0; q <= nq; ++q) key.push_back(h_qoff[q]);
    for (int i = 0; i < A * A; ++i) key.push_back(h_matrix[i]);

    Plan* plan = nullptr;
    for (auto& p : db->plans)
        if (p->key == key) plan = p.get();
    if (!plan) {
        sw_status s = build_plan(db, h_qoff, nq, h_matrix, max_s, gap_open, gap_extend, d_scores,
                                 key, &plan);
        if (s != SW_OK) return s;
    }
    // Searches on one database share scratch: order this one after the previous one,
    // whatever stream that ran on.
    if (db->done_recorded) CU(cudaStreamWaitEvent(st, db->ev[4], 0));
    bool replay = false;
    if (graphs_enabled()) {
        if (!plan->exec) {
            cudaGraph_t graph = nullptr;
            CU(cudaStreamBeginCapture(db->capture_stream, cudaStreamCaptureModeThreadLocal));
            sw_status s = enqueue_plan(db, *plan, d_queries, db->capture_stream);
            cudaError_t ec = cudaStreamEndCapture(db->capture_stream, &graph);
            if (s != SW_OK) {
                if (graph) cudaGraphDestroy(graph);
                return s;
            }
            if (ec != cudaSuccess) return cuda_fail(ec, "cudaStreamEndCapture");
            ec = cudaGraphInstantiate(&plan->exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ec != cudaSuccess) {
                plan->exec = nullptr;
                return cuda_fail(ec, "cudaGraphInstantiate");
            }
        } else {
            replay = true;
        }
        CU(cudaGraphLaunch(plan->exec, st));
    } else {
        sw_status s = enqueue_plan(db, *plan, d_queries, st);
        if (s != SW_OK) return s;
    }
    db->done_recorded = true;
    g_launches += plan->launches;
    db->stats = sw_stats{};
    db->stats.cells = plan->cells;
    db->stats.inter_cells = plan->inter_cells;
    db->stats.launches = plan->launches;
    db->stats.inter_grid = plan->inter_grid;
    db->stats.inter_block = inter_variant_warps(plan->variant) * kWarp;
    db->stats.multi_query = plan->mq ? 1 : 0;
    db->stats.score_profile = plan->sp && plan->num_items > 0 ? 1 : 0;
    db->stats.intra_packed = plan->wave ? 1 : plan->pair ? 2 : 0;
    const bool half_items = plan->pair && plan->pair_half &&
                            plan->pair_half_from < (db->layout.num_groups - plan->g_split) * (kGroupSeqs / 2);
    db->stats.wave_lanes = plan->wave ? kWarp : plan->pair ? (half_items ? wave_ss_bulk_lanes() : kWarp) : 0;
    db->stats.graph_replay = replay ? 1 : 0;
    db->stats.variant = plan->variant;
    db->stats_inter = plan->mq || plan->num_items > 0;
    db->stats_pair_only = pair_only_plan(db, *plan);
    db->stats_pending = true;
    return SW_OK;
}

sw_status finish_stats(sw_db* db) {
    if (!db->stats_pending) return SW_OK;
    CU(cudaEventSynchronize(db->ev[4]));
    float t = 0;
    if (db->stats_inter) CU(cudaEventElapsedTime(&t, db->ev[1], db->ev[2]));
    db->stats.inter_ms = t;
    if (db->stats_pair_only) {   // no event between the wavefront kernel and its dependent rescore
        CU(cudaEventElapsedTime(&t, db->ev[2], db->ev[4]));
        db->stats.intra_ms = t;
        db->stats.rescore_ms = 0;
    } else {
        CU(cudaEventElapsedTime(&t, db->ev[2], db->ev[3]));
        db->stats.intra_ms = t;
        CU(cudaEventElapsedTime(&t, db->ev[3], db->ev[4]));
        db->stats.rescore_ms = t;
    }
    CU(cudaEventElapsedTime(&t, db->ev[0], db->ev[4]));
    db->stats.total_ms = t;
    Control c{};
    CU(cudaMemcpy(&c, db->ctrl.ptr, sizeof(Control), cudaMemcpyDeviceToHost));
    db->stats.flagged = c.flag_count;
    db->stats_pending = false;
    if (c.status & 1u) return fail(SW_ERR_CODE, "a query residue code was >= alphabet_size");
    return SW_OK;
}

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
    v->inter_occ = db->inter_occ[0];
    v->intra_occ = db->intra_occ;
    v->inter = db->inter_ptr;
    v->group_off = db->group_off.ptr;
    v->group_len = db->group_len.ptr;
    v->group_cols = db->group_cols.ptr;
    v->perm = db->perm.ptr;
    v->plain = db->plain_ptr;
    v->plain_off = db->plain_off.ptr;
    v->long_ids = db->long_ids.ptr;
    return true;
}

}  // namespace swgb

// ================================================================= C ABI

extern "C" {

const char* sw_last_error(void) { return g_err.c_str(); }
const char* sw_version(void) { return "swgb 0.3 (sm_103a)"; }
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
        if (opts->placement != SW_PLACE_DEVICE && opts->placement != SW_PLACE_HOST)
            return fail(SW_ERR_ARG, "placement must be SW_PLACE_DEVICE or SW_PLACE_HOST");
    }
    std::unique_ptr<sw_db> db(new sw_db());
    db->device = dev;
    db->A = alphabet_size;
    db->long_cutoff = cutoff;
    if (opts && opts->flag_cap > 0) db->flag_cap = opts->flag_cap;
    if (opts) db->placement = opts->placement;
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
    for (int v = 0; v < inter_num_variants() && v < kMaxVariants; ++v)
        db->inter_occ[v] = inter_occupancy(v, alphabet_size + 1);
    for (int v = 0; v < inter_mq_num_variants() && v < kMaxVariants; ++v)
        db->inter_mq_occ[v] = inter_mq_occupancy(v, alphabet_size + 1);
    db->intra_occ = intra_occupancy(alphabet_size + 1);
    db->inter_sp_occ = inter_sp_occupancy(alphabet_size + 1);
    const bool block_off = std::getenv("SWGB_INTRA_BLOCK") && std::getenv("SWGB_INTRA_BLOCK")[0] == '0';
    for (int v = 0; v < 3; ++v)
        db->intra_block_occ[v] = block_off ? 0 : intra_block_occupancy(kIntraBlockRows[v], alphabet_size + 1);
    for (int v = 0; v < 3; ++v) db->wave_occ[v] = wave_occupancy(kWaveRows[v], alphabet_size + 1);
    CU(cudaDeviceGetAttribute(&db->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (db->inter_occ[0] <= 0 || db->intra_occ <= 0)
        return fail(SW_ERR_CUDA, "kernels cannot be resident on device %d", dev);
    const char* forced = std::getenv("SWGB_VARIANT");
    if (forced) {
        const int v = std::atoi(forced);
        if (v >= 0 && v < inter_num_variants() && db->inter_occ[v] > 0) db->variant = v;
    }
    CU(cudaStreamCreateWithFlags(&db->stream, cudaStreamNonBlocking));
    CU(cudaStreamCreateWithFlags(&db->capture_stream, cudaStreamNonBlocking));
    for (auto& e : db->ev) CU(cudaEventCreate(&e));
    const Layout& L = db->layout;
    const size_t inter_bytes = static_cast<size_t>(std::max<int64_t>(L.inter_bytes, 16));
    if (db->placement == SW_PLACE_HOST) {
        // pinned host memory mapped into the device address space: kernels read it over the link
        CU(cudaHostAlloc(reinterpret_cast<void**>(&db->host_inter), inter_bytes, cudaHostAllocMapped));
        if (L.num_groups > 0) fill_inter(residues, offsets, alphabet_size, L, db->host_inter);
        void* dp = nullptr;
        CU(cudaHostGetDevicePointer(&dp, db->host_inter, 0));
        db->inter_ptr = static_cast<const uint8_t*>(dp);
    } else {
        std::vector<uint8_t> inter(inter_bytes);
        if (L.num_groups > 0) fill_inter(residues, offsets, alphabet_size, L, inter.data());
        CU(db->inter.ensure(inter.size()));
        CU(cudaMemcpy(db->inter.ptr, inter.data(), inter.size(), cudaMemcpyHostToDevice));
        db->inter_ptr = db->inter.ptr;
    }
    CU(db->group_off.ensure(L.group_off.size()));
    CU(db->group_len.ensure(L.group_len.size()));
    CU(db->group_cols.ensure(L.group_cols.size()));
    CU(db->perm.ensure(L.perm.size()));
    if (!L.group_off.empty()) {
        CU(cudaMemcpy(db->group_off.ptr, L.group_off.data(), sizeof(int64_t) * L.group_off.size(),
                      cudaMemcpyHostToDevice));
        CU(cudaMemcpy(db->group_len.ptr, L.group_len.data(), sizeof(int32_t) * L.group_len.size(),
                      cudaMemcpyHostToDevice));
        CU(cudaMemcpy(db->group_cols.ptr, L.group_cols.data(), sizeof(int32_t) * L.group_cols.size(),
                      cudaMemcpyHostToDevice));
        CU(cudaMemcpy(db->perm.ptr, L.perm.data(), sizeof(int32_t) * L.perm.size(),
                      cudaMemcpyHostToDevice));
    }
    if (db->placement == SW_PLACE_HOST) {
        CU(cudaHostAlloc(reinterpret_cast<void**>(&db->host_plain),
                         static_cast<size_t>(std::max<int64_t>(R, 16)), cudaHostAllocMapped));
        if (R > 0) std::memcpy(db->host_plain, residues, static_cast<size_t>(R));
        void* dp = nullptr;
        CU(cudaHostGetDevicePointer(&dp, db->host_plain, 0));
        db->plain_ptr = static_cast<const uint8_t*>(dp);
    } else {
        CU(db->plain.ensure(static_cast<size_t>(std::max<int64_t>(R, 16))));
        if (R > 0) CU(cudaMemcpy(db->plain.ptr, residues, static_cast<size_t>(R), cudaMemcpyHostToDevice));
        db->plain_ptr = db->plain.ptr;
    }
    CU(db->plain_off.ensure(static_cast<size_t>(num_seqs) + 1));
    CU(cudaMemcpy(db->plain_off.ptr, offsets, sizeof(int64_t) * (num_seqs + 1), cudaMemcpyHostToDevice));
    CU(db->long_ids.ensure(std::max<size_t>(L.long_ids.size(), 1)));
    if (!L.long_ids.empty())
        CU(cudaMemcpy(db->long_ids.ptr, L.long_ids.data(), sizeof(int32_t) * L.long_ids.size(),
                      cudaMemcpyHostToDevice));
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
        if (db->done_recorded) cudaEventSynchronize(db->ev[4]);
        destroy_plans(db);
        db->inter.release();
        db->plain.release();
        db->h_queries.release();
        db->group_off.release();
        db->group_len.release();
        db->group_cols.release();
        db->perm.release();
        db->plain_off.release();
        db->long_ids.release();
        db->ctrl.release();
        db->flags.release();
        db->bnd.release();
        db->spill.release();
        db->h_scores.release();
        for (auto& e : db->ev)
            if (e) cudaEventDestroy(e);
        if (db->stream) cudaStreamDestroy(db->stream);
        if (db->capture_stream) cudaStreamDestroy(db->capture_stream);
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

sw_status sw_search_async(const sw_db* db, const uint8_t* d_queries, const int64_t* query_offsets,
                          int32_t num_queries, const int8_t* matrix, int32_t gap_open,
                          int32_t gap_extend, int32_t* d_scores, void* stream) {
    return sw_search_batch_device(db, d_queries, query_offsets, num_queries, matrix, gap_open,
                                  gap_extend, d_scores, stream);
}

sw_status sw_search_batch(const sw_db* cdb, const uint8_t* const* queries,
                          const int32_t* query_lens, int32_t num_queries, const int8_t* matrix,
                          int32_t gap_open, int32_t gap_extend, int32_t* scores) {
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
    const size_t qbytes = static_cast<size_t>(std::max<int64_t>(qoff.back(), 1));
    if (db->done_recorded) CU(cudaEventSynchronize(db->ev[4]));   // staging buffers may move
    // the queries are concatenated into pinned host memory (an asynchronous copy; a pageable
    // source would be staged by the driver), checked, then copied to the device
    if (db->pinned_q_cap < qbytes) {
        if (db->pinned_q) cudaFreeHost(db->pinned_q);
        db->pinned_q = nullptr;
        db->pinned_q_cap = 0;
        CU(cudaHostAlloc(reinterpret_cast<void**>(&db->pinned_q), qbytes, cudaHostAllocDefault));
        db->pinned_q_cap = qbytes;
    }
    uint8_t* cat = db->pinned_q;
    for (int q = 0; q < num_queries; ++q)
        if (query_lens[q] > 0)
            std::memcpy(cat + qoff[static_cast<size_t>(q)], queries[q], static_cast<size_t>(query_lens[q]));
    for (int64_t i = 0; i < qoff.back(); ++i)
        if (cat[i] >= db->A)
            return fail(SW_ERR_CODE, "query residue %lld has code %d >= alphabet_size %d",
                        static_cast<long long>(i), cat[i], db->A);
    if (num_queries == 0 || N == 0) return SW_OK;
    CU(db->h_queries.ensure(qbytes));
    CU(db->h_scores.ensure(static_cast<size_t>(N * num_queries)));
    CU(cudaMemcpyAsync(db->h_queries.ptr, cat, qbytes, cudaMemcpyHostToDevice, db->stream));
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
