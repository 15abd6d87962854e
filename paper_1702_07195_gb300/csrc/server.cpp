// Continuous-batching search server (sw_server_*): admission by DP-state bytes, ticks that
// replay one captured CUDA graph over all in-flight requests, latency accounting.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/swgb.h"
#include "db_view.h"
#include "runtime_internal.h"
#include "swgb_device.cuh"

using namespace swgb;

namespace {

using Clock = std::chrono::steady_clock;

double now_s() {
    return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

struct Request {
    int64_t ticket = 0;
    std::vector<uint8_t> query;
    int32_t m = 0;
    int slot = -1;
    int32_t slices_left = 0;   // database slices still to scan (one per tick, cyclically)
    bool long_pending = false;
    int64_t state_bytes = 0;
    double t_submit = 0, t_done = 0;
    std::vector<int32_t> result;
    bool done = false;
};

}  // namespace

struct sw_server {
    sw_db* db = nullptr;
    int32_t A = 0;
    std::vector<int8_t> matrix;
    int32_t goe = 0, ge = 0, max_s = 0;
    sw_server_options opt{};
    int variant = 0, W = 4, T = 64;
    int64_t nchunks = 0;
    std::vector<int64_t> slice_chunk;   // slice k = chunks [slice_chunk[k], slice_chunk[k+1])
    int32_t cur_slice = 0;
    int inter_grid = 0, intra_grid = 0, mq_grid = 0;
    bool mq_ok = false;
    int64_t max_steps = 0, rows_pad = 0;
    int64_t N = 0, mpad_max = 0;
    // device
    DevBuf<uint8_t> q_buf;
    DevBuf<int16_t> qp_buf;
    DevBuf<int32_t> scores;
    DevBuf<QueryDesc> descs;
    DevBuf<int64_t> qoff;
    DevBuf<int64_t> qp_off;
    DevBuf<int32_t> mpad;
    DevBuf<int8_t> dmat;
    DevBuf<TickDesc> tick_d;
    DevBuf<int64_t> qstart;           // per slot: start of its query in q_buf
    DevBuf<int32_t> qlen;             // per slot: query length
    DevBuf<MqStep> steps_d;
    DevBuf<uint32_t> pp;
    MqStep* steps_h = nullptr;        // pinned
    DevBuf<Control> ctrl;
    DevBuf<FlagEntry> flags;
    DevBuf<uint4> bnd;
    DevBuf<int2> spill;
    TickDesc* tick_h = nullptr;       // pinned
    cudaStream_t st = nullptr, cap = nullptr;
    cudaGraphExec_t graph = nullptr;      // one request in flight: two subjects per register
    cudaGraphExec_t graph_mq = nullptr;   // two or more: two queries per register
    cudaEvent_t ev = nullptr;
    // host state
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> pending;
    std::vector<Request*> active;     // per slot, nullptr = free
    std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
    int64_t next_ticket = 1;
    int64_t state_used = 0;
    bool stop = false;
    std::thread worker;
    sw_status worker_status = SW_OK;
    // stats
    std::vector<double> latencies;
    int64_t submitted = 0, completed = 0, rejected = 0, ticks = 0, joined = 0, cells = 0;
    int64_t mq_ticks = 0;
    int32_t max_in_flight = 0;
    double t_first = 0, t_last = 0;
    // running mean of the gap between submissions (seconds), for the whole-database tick
    double last_submit = 0, mean_gap = 1.0;
};

namespace {

sw_status cerr(cudaError_t e, const char* what) {
    char msg[256];
    snprintf(msg, sizeof(msg), "%s: %s", what, cudaGetErrorString(e));
    return set_last_error(e == cudaErrorMemoryAllocation ? SW_ERR_OOM : SW_ERR_CUDA, msg);
}

#define SCU(call)                                          \
    do {                                                   \
        const cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cerr(e_, #call);     \
    } while (0)

int in_flight(const sw_server* s) {
    int n = 0;
    for (auto* r : s->active) n += r != nullptr;
    return n;
}

// Uploads an admitted request's query and builds its profile in its slot (server stream).
sw_status start_request(sw_server* s, Request* r) {
    const int slot = r->slot;
    const int64_t mp = (std::max<int64_t>(r->m, 1) + kQpRows - 1) / kQpRows * kQpRows;
    uint8_t* dq = s->q_buf.ptr + static_cast<int64_t>(slot) * s->opt.max_query_len;
    SCU(cudaMemcpyAsync(dq, r->query.data(), static_cast<size_t>(r->m), cudaMemcpyHostToDevice, s->st));
    const QueryDesc d{s->qp_buf.ptr + static_cast<int64_t>(slot) * (s->A + 1) * s->mpad_max,
                      s->scores.ptr + static_cast<int64_t>(slot) * s->N, r->m, static_cast<int32_t>(mp)};
    const int64_t qo[2] = {0, r->m};
    const int32_t mpv = static_cast<int32_t>(mp);
    SCU(cudaMemcpyAsync(s->descs.ptr + slot, &d, sizeof(d), cudaMemcpyHostToDevice, s->st));
    SCU(cudaMemcpyAsync(s->qoff.ptr + 2 * slot, qo, sizeof(qo), cudaMemcpyHostToDevice, s->st));
    SCU(cudaMemcpyAsync(s->mpad.ptr + slot, &mpv, sizeof(mpv), cudaMemcpyHostToDevice, s->st));
    const int32_t len = r->m;
    SCU(cudaMemcpyAsync(s->qlen.ptr + slot, &len, sizeof(len), cudaMemcpyHostToDevice, s->st));
    SCU(launch_build_qp(dq, s->qoff.ptr + 2 * slot, 1, s->dmat.ptr, s->A, s->goe, s->qp_off.ptr,
                        s->mpad.ptr + slot, const_cast<int16_t*>(d.qp), mp, s->ctrl.ptr, s->st));
    add_launches(1);
    // the copies read host memory owned by `r` and the stack: wait for them before returning
    SCU(cudaStreamSynchronize(s->st));
    return SW_OK;
}

sw_status capture_tick_graphs(sw_server* s, const DbView& v) {
    const Gaps gaps{s->goe, s->ge, std::min(s->goe, s->ge)};
    const int64_t bnd_stride = std::max<int64_t>(1, v.max_group_len / 2 * kWarp);
    InterParams ip{};
    ip.inter = v.inter;
    ip.group_off = v.group_off;
    ip.group_len = v.group_len;
    ip.group_cols = v.group_cols;
    ip.perm = v.perm;
    ip.queries = s->descs.ptr;
    ip.items = nullptr;
    ip.num_items = 0;
    ip.alphabet1 = s->A + 1;
    ip.ctrl = s->ctrl.ptr;
    ip.flags = s->flags.ptr;
    ip.flag_cap = static_cast<uint32_t>(s->flags.cap);
    ip.thresh = 32767 - std::max(0, s->max_s);
    ip.bnd = s->bnd.ptr;
    ip.bnd_stride = bnd_stride;
    ip.gaps = gaps;
    ip.tick = s->tick_d.ptr;
    ip.num_groups = static_cast<int32_t>(v.num_groups);
    InterMqParams mp{};
    mp.inter = v.inter;
    mp.group_off = v.group_off;
    mp.group_len = v.group_len;
    mp.group_cols = v.group_cols;
    mp.perm = v.perm;
    mp.queries = s->descs.ptr;
    mp.pp = s->pp.ptr;
    mp.rows_pad = s->rows_pad;
    mp.steps = s->steps_d.ptr;
    mp.num_steps = 0;
    mp.num_half_groups = 0;
    mp.alphabet1 = s->A + 1;
    mp.ctrl = s->ctrl.ptr;
    mp.flags = s->flags.ptr;
    mp.flag_cap = static_cast<uint32_t>(s->flags.cap);
    mp.thresh = ip.thresh;
    mp.bnd = s->bnd.ptr;
    mp.bnd_stride = bnd_stride;
    mp.gaps = gaps;
    mp.tick = s->tick_d.ptr;
    IntraParams jp{};
    jp.plain = v.plain;
    jp.plain_off = v.plain_off;
    jp.queries = s->descs.ptr;
    jp.num_queries = s->opt.max_inflight;
    jp.long_ids = v.long_ids;
    jp.num_long = v.num_long;
    jp.query_order = nullptr;
    jp.num_seqs = v.num_seqs;
    jp.flags = s->flags.ptr;
    jp.flag_cap = static_cast<uint32_t>(s->flags.cap);
    jp.alphabet1 = s->A + 1;
    jp.ctrl = s->ctrl.ptr;
    jp.spill = s->spill.ptr;
    jp.spill_stride = std::max<int64_t>(1, (v.max_len + 31) / 32 * 32 + 64);
    jp.gaps = gaps;
    jp.qp_add = 0;
    jp.tick = s->tick_d.ptr;
    for (int mode = 0; mode < (s->mq_ok ? 2 : 1); ++mode) {
        cudaGraph_t g = nullptr;
        SCU(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaMemcpyAsync(s->tick_d.ptr, s->tick_h, sizeof(TickDesc),
                                        cudaMemcpyHostToDevice, s->cap);
        if (e == cudaSuccess) e = cudaMemsetAsync(s->ctrl.ptr, 0, sizeof(Control), s->cap);
        if (mode == 1) {
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(s->steps_d.ptr, s->steps_h, sizeof(MqStep) * s->max_steps,
                                    cudaMemcpyHostToDevice, s->cap);
            if (e == cudaSuccess)
                e = launch_build_pp(s->q_buf.ptr, s->qstart.ptr, s->qlen.ptr, s->steps_d.ptr, 0,
                                    s->tick_d.ptr, s->T, s->dmat.ptr, s->A, s->goe, s->pp.ptr,
                                    s->rows_pad, s->ctrl.ptr, s->cap);
            if (e == cudaSuccess && v.num_groups > 0) e = launch_inter_mq(mp, s->variant, s->mq_grid, s->cap);
        } else if (e == cudaSuccess && v.num_groups > 0) {
            e = launch_inter(ip, s->variant, s->inter_grid, s->cap);
        }
        if (e == cudaSuccess && v.num_long > 0) {
            jp.mode = kIntraTickLong;
            e = launch_intra(jp, s->intra_grid, intra_block_threads(), s->cap);
        }
        if (e == cudaSuccess && v.num_groups > 0) {
            jp.mode = kIntraRescore;
            e = launch_intra(jp, s->intra_grid, intra_block_threads(), s->cap);
        }
        const cudaError_t e2 = cudaStreamEndCapture(s->cap, &g);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cerr(e, "tick capture");
        }
        if (e2 != cudaSuccess) return cerr(e2, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(mode == 1 ? &s->graph_mq : &s->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cerr(e, "cudaGraphInstantiate");
    }
    return SW_OK;
}

int64_t state_bytes(const sw_server* s, int32_t m) {
    const int64_t mp = (std::max<int64_t>(m, 1) + kQpRows - 1) / kQpRows * kQpRows;
    return (s->A + 1) * mp * 2 + s->N * 4;
}

void finish(sw_server* s, Request* r) {
    r->done = true;
    r->t_done = now_s();
    s->latencies.push_back(r->t_done - r->t_submit);
    s->t_last = r->t_done;
    s->cells += static_cast<int64_t>(r->m) * s->db->num_residues;
    ++s->completed;
}

// Fills the host tick descriptor (and, with two or more requests, the two query streams)
// for database slice `c`.  Returns true for a multi-query tick.
bool build_tick(sw_server* s, int32_t c, const std::vector<Request*>& act) {
    TickDesc& t = *s->tick_h;
    t.n = 0;
    t.n_long = 0;
    t.prefix[0] = 0;
    for (Request* r : act)
        if (r->long_pending) t.long_slot[t.n_long++] = r->slot;
    const int64_t c0 = s->slice_chunk[static_cast<size_t>(c)], c1 = s->slice_chunk[static_cast<size_t>(c) + 1];
    const bool mq = s->mq_ok && act.size() >= 2;
    if (!mq) {
        for (Request* r : act) {   // one request: its chunks of the slice, longest first
            t.slot[t.n] = r->slot;
            t.chunk_end[t.n] = static_cast<int32_t>(c1);
            t.prefix[t.n + 1] = t.prefix[t.n] + static_cast<int32_t>(c1 - c0);
            ++t.n;
        }
        t.mq_steps = 0;
        return false;
    }
    // Independent batches, each with two streams of T-row strips balanced by strip count,
    // longest query first.  As few batches as give ~12 waves of work items (larger batches
    // balance their two streams better), and at least four requests per batch.
    std::vector<Request*> order(act.begin(), act.end());
    std::stable_sort(order.begin(), order.end(), [](Request* a, Request* b) { return a->m > b->m; });
    const int64_t g0s = c0 * s->W, g1s = std::min<int64_t>(c1 * s->W, s->db->layout.num_groups);
    const int64_t n_hb = std::max<int64_t>(1, (2 * (g1s - g0s) + s->W - 1) / s->W);
    const int64_t want = (12 * static_cast<int64_t>(s->mq_grid) + n_hb - 1) / n_hb;
    const int nb = static_cast<int>(std::max<int64_t>(
        1, std::min<int64_t>(want, static_cast<int64_t>(order.size()) / 4)));
    std::vector<std::vector<Request*>> batch(static_cast<size_t>(nb));
    std::vector<int64_t> bload(static_cast<size_t>(nb), 0);
    for (Request* r : order) {
        const size_t b = static_cast<size_t>(std::min_element(bload.begin(), bload.end()) - bload.begin());
        batch[b].push_back(r);
        bload[b] += (r->m + s->T - 1) / s->T;
    }
    int64_t off = 0;
    t.n_batches = nb;
    for (int b = 0; b < nb; ++b) {
        t.batch_step_off[b] = static_cast<int32_t>(off);
        std::vector<Request*> stream[2];
        int64_t len[2] = {0, 0};
        for (Request* r : batch[static_cast<size_t>(b)]) {
            const int x = len[0] <= len[1] ? 0 : 1;
            stream[x].push_back(r);
            len[x] += (r->m + s->T - 1) / s->T;
        }
        const int64_t n = std::max(len[0], len[1]);
        for (int64_t k = 0; k < n; ++k) s->steps_h[off + k] = MqStep{-1, -1, 0, 0, kMqFirstA | kMqFirstB, 0};
        for (int x = 0; x < 2; ++x) {
            int64_t k = off;
            for (Request* r : stream[x]) {
                const int32_t S = (r->m + s->T - 1) / s->T;
                for (int32_t si = 0; si < S; ++si, ++k) {
                    MqStep& st = s->steps_h[k];
                    uint32_t fl = st.flags & (x == 0 ? (kMqFirstB | kMqLastB) : (kMqFirstA | kMqLastA));
                    if (si == 0) fl |= (x == 0 ? kMqFirstA : kMqFirstB);
                    if (si == S - 1) fl |= (x == 0 ? kMqLastA : kMqLastB);
                    st.flags = fl;
                    if (x == 0) {
                        st.qa = r->slot;
                        st.sa = si;
                    } else {
                        st.qb = r->slot;
                        st.sb = si;
                    }
                }
            }
        }
        off += n;
    }
    t.batch_step_off[nb] = static_cast<int32_t>(off);
    const int64_t n = off;
    const int64_t g0 = c0 * s->W, g1 = std::min<int64_t>(c1 * s->W, s->db->layout.num_groups);
    t.mq_steps = static_cast<int32_t>(n);
    t.hg_begin = static_cast<int32_t>(2 * g0);
    t.hg_end = static_cast<int32_t>(2 * g1);
    return true;
}

// Cell rate assumed for a lone request's whole-database tick (the single-query kernel).
constexpr double kWholeTickCellsPerS = 5.0e12;

void worker_loop(sw_server* s) {
    cudaSetDevice(s->db->device);
    DbView v;
    db_view(s->db, &v);
    const int64_t num_long = v.num_long;
    const int32_t K = static_cast<int32_t>(s->slice_chunk.size()) - 1;
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        // Admission: free slot and DP-state budget.
        std::vector<Request*> admitted;
        while (!s->pending.empty()) {
            Request* r = s->pending.front();
            if (s->state_used + r->state_bytes > s->opt.state_budget_bytes && in_flight(s) > 0) break;
            int slot = -1;
            for (int i = 0; i < s->opt.max_inflight; ++i)
                if (!s->active[i]) {
                    slot = i;
                    break;
                }
            if (slot < 0) break;
            s->pending.pop_front();
            if (in_flight(s) > 0) ++s->joined;
            r->slot = slot;
            r->slices_left = K;
            r->long_pending = num_long > 0;
            s->active[slot] = r;
            s->state_used += r->state_bytes;
            admitted.push_back(r);
        }
        std::vector<Request*> act;
        for (Request* r : s->active)
            if (r) act.push_back(r);
        s->max_in_flight = std::max<int32_t>(s->max_in_flight, static_cast<int32_t>(act.size()));
        if (act.empty()) {
            s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
            continue;
        }
        for (Request* r : admitted) {
            const sw_status st = start_request(s, r);
            if (st != SW_OK) {
                s->worker_status = st;
                s->stop = true;
                break;
            }
        }
        if (s->stop) break;
        // Tick: every in-flight request scans the current database slice.  A lone request just
        // admitted, with nothing pending, scans the whole database in this one tick instead when
        // that tick is unlikely to hold up an arrival (its estimated time below 30 % of the
        // running mean gap between submissions): slices only serve to let arrivals join a
        // running scan, and alone the request would pay K launches and K tails (p50 at 5 % of
        // capacity: 28 ms in 3 ticks, 20 ms in one).
        const int32_t c = s->cur_slice;
        bool mq = false;
        bool whole = false;
        const double whole_s = static_cast<double>(act[0]->m) * static_cast<double>(v.short_residues) /
                               kWholeTickCellsPerS;
        if (K > 1 && act.size() == 1 && s->pending.empty() && act[0]->slices_left == K &&
            whole_s < 0.3 * s->mean_gap) {
            whole = true;
            TickDesc& t = *s->tick_h;
            t.n = 1;
            t.n_long = act[0]->long_pending ? 1 : 0;
            t.long_slot[0] = act[0]->slot;
            t.slot[0] = act[0]->slot;
            t.chunk_end[0] = static_cast<int32_t>(s->nchunks);
            t.prefix[0] = 0;
            t.prefix[1] = static_cast<int32_t>(s->nchunks);
            t.mq_steps = 0;
            act[0]->slices_left = 1;
        } else if (K > 0) {
            mq = build_tick(s, c, act);
        } else {   // no interleaved groups: only long subjects
            TickDesc& t = *s->tick_h;
            t.n = 0;
            t.n_long = 0;
            t.prefix[0] = 0;
            t.mq_steps = 0;
            for (Request* r : act)
                if (r->long_pending) t.long_slot[t.n_long++] = r->slot;
        }
        lk.unlock();
        cudaError_t e = cudaSuccess;
        if (K > 0 || num_long > 0) {
            e = cudaGraphLaunch(mq ? s->graph_mq : s->graph, s->st);
            if (e == cudaSuccess) e = cudaEventRecord(s->ev, s->st);
            if (e == cudaSuccess) e = cudaEventSynchronize(s->ev);
            add_launches(mq ? 5 : 3);
        }
        lk.lock();
        if (e != cudaSuccess) {
            s->worker_status = cerr(e, "tick");
            s->stop = true;
            break;
        }
        ++s->ticks;
        s->mq_ticks += mq ? 1 : 0;
        if (K > 0 && !whole) s->cur_slice = (c + 1) % K;
        for (Request* r : act) {
            r->slices_left -= 1;
            r->long_pending = false;
            if (r->slices_left <= 0) {
                r->result.resize(static_cast<size_t>(s->N));
                e = cudaMemcpy(r->result.data(), s->scores.ptr + static_cast<int64_t>(r->slot) * s->N,
                               sizeof(int32_t) * s->N, cudaMemcpyDeviceToHost);
                if (e != cudaSuccess) {
                    s->worker_status = cerr(e, "score copy");
                    s->stop = true;
                }
                s->active[r->slot] = nullptr;
                s->state_used -= r->state_bytes;
                finish(s, r);
            }
        }
        s->cv_done.notify_all();
    }
    s->cv_done.notify_all();
}

double percentile(std::vector<double> v, double p) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double idx = p * static_cast<double>(v.size() - 1);
    const size_t lo = static_cast<size_t>(idx);
    const size_t hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (v[hi] - v[lo]) * (idx - static_cast<double>(lo));
}

}  // namespace

extern "C" {

sw_status sw_server_create(sw_db* db, const int8_t* matrix, int32_t gap_open, int32_t gap_extend,
                           const sw_server_options* opts, sw_server** out) {
    if (!db || !matrix || !out) return set_last_error(SW_ERR_ARG, "null pointer");
    *out = nullptr;
    if (gap_open < 0 || gap_extend < 0 || gap_open > 16383 || gap_extend > 16383)
        return set_last_error(SW_ERR_ARG, "server gap costs must be in [0, 16383]");
    DbView v;
    db_view(db, &v);
    auto s = std::make_unique<sw_server>();
    s->db = db;
    s->A = v.alphabet;
    s->matrix.assign(matrix, matrix + v.alphabet * v.alphabet);
    s->goe = gap_open;
    s->ge = gap_extend;
    for (int8_t x : s->matrix) s->max_s = std::max<int32_t>(s->max_s, x);
    s->opt.max_inflight = 32;
    s->opt.max_query_len = 8192;
    s->opt.state_budget_bytes = int64_t{1} << 30;
    s->opt.slices = 0;
    s->opt.max_pending = 4096;
    if (opts) {
        if (opts->max_inflight > 0) s->opt.max_inflight = opts->max_inflight;
        if (opts->max_query_len > 0) s->opt.max_query_len = opts->max_query_len;
        if (opts->state_budget_bytes > 0) s->opt.state_budget_bytes = opts->state_budget_bytes;
        if (opts->slices > 0) s->opt.slices = opts->slices;
        if (opts->max_pending > 0) s->opt.max_pending = opts->max_pending;
    }
    if (s->opt.max_inflight > kTickMax) return set_last_error(SW_ERR_ARG, "max_inflight > 128");
    if (static_cast<double>(std::min<int64_t>(s->opt.max_query_len, v.max_len)) * s->max_s > 2147483647.0)
        return set_last_error(SW_ERR_ARG, "scores could exceed the int32 range");
    DeviceGuard guard(v.device);
    s->N = v.num_seqs;
    s->variant = db->variant;
    s->W = inter_variant_warps(s->variant);
    s->T = inter_mq_variant_rows(s->variant);
    s->nchunks = (v.num_groups + s->W - 1) / s->W;
    // Slices of about equal residue work, whole chunks of W groups each.  Default: as many as
    // keep eight waves of multi-query work items per tick.
    {
        const int64_t warps = static_cast<int64_t>(v.sms) * std::max(1, db->inter_mq_occ[s->variant]) * s->W;
        const int64_t auto_k = std::max<int64_t>(1, std::min<int64_t>(16, 2 * v.num_groups / std::max<int64_t>(1, 8 * warps)));
        const int64_t want = s->opt.slices > 0 ? s->opt.slices : auto_k;
        s->opt.slices = static_cast<int32_t>(want);
        const int64_t K = std::max<int64_t>(1, std::min<int64_t>(want, s->nchunks));
        std::vector<int64_t> cres(static_cast<size_t>(s->nchunks) + 1, 0);
        for (int64_t c = 0; c < s->nchunks; ++c) {
            int64_t r = 0;
            for (int64_t g = c * s->W; g < std::min<int64_t>((c + 1) * s->W, v.num_groups); ++g)
                r += db->layout.group_res[static_cast<size_t>(g)];
            cres[static_cast<size_t>(c) + 1] = cres[static_cast<size_t>(c)] + r;
        }
        s->slice_chunk.assign(1, 0);
        for (int64_t k = 1; k < K; ++k) {
            const int64_t target = cres.back() * k / K;
            int64_t c = s->slice_chunk.back() + 1;
            while (c < s->nchunks && cres[static_cast<size_t>(c)] < target) ++c;
            if (c < s->nchunks) s->slice_chunk.push_back(c);
        }
        if (s->nchunks > 0) s->slice_chunk.push_back(s->nchunks);
    }
    s->inter_grid = v.sms * std::max(1, db->inter_occ[s->variant]);
    s->mq_grid = v.sms * std::max(1, db->inter_mq_occ[s->variant]);
    s->mq_ok = db->inter_mq_occ[s->variant] > 0 && v.num_groups > 0;
    s->intra_grid = v.sms * std::max(1, v.intra_occ);
    s->mpad_max = (s->opt.max_query_len + kQpRows - 1) / kQpRows * kQpRows;
    s->max_steps = std::max<int64_t>(1, static_cast<int64_t>(s->opt.max_inflight) *
                                            ((s->opt.max_query_len + s->T - 1) / s->T));
    // a batch may start at any step and its staging window reads kQpRows rows from there
    s->rows_pad = (s->max_steps * s->T + 2 * kQpRows - 1) / kQpRows * kQpRows;
    const int S = s->opt.max_inflight;
    SCU(s->q_buf.ensure(static_cast<size_t>(S) * s->opt.max_query_len));
    SCU(s->qp_buf.ensure(static_cast<size_t>(S) * (s->A + 1) * s->mpad_max));
    SCU(s->scores.ensure(static_cast<size_t>(S) * std::max<int64_t>(s->N, 1)));
    SCU(s->descs.ensure(static_cast<size_t>(S)));
    {   // every slot points at its own buffers from the start (an idle slot has m = 0)
        std::vector<QueryDesc> d0(static_cast<size_t>(S));
        for (int i = 0; i < S; ++i)
            d0[static_cast<size_t>(i)] = QueryDesc{s->qp_buf.ptr + static_cast<int64_t>(i) * (s->A + 1) * s->mpad_max,
                                                   s->scores.ptr + static_cast<int64_t>(i) * s->N, 0,
                                                   static_cast<int32_t>(kQpRows)};
        SCU(cudaMemcpy(s->descs.ptr, d0.data(), sizeof(QueryDesc) * S, cudaMemcpyHostToDevice));
    }
    SCU(s->qoff.ensure(static_cast<size_t>(2 * S)));
    SCU(s->qp_off.ensure(1));
    SCU(cudaMemset(s->qp_off.ptr, 0, sizeof(int64_t)));
    SCU(s->mpad.ensure(static_cast<size_t>(S)));
    SCU(s->dmat.ensure(s->matrix.size()));
    SCU(cudaMemcpy(s->dmat.ptr, s->matrix.data(), s->matrix.size(), cudaMemcpyHostToDevice));
    SCU(s->tick_d.ensure(1));
    SCU(s->qstart.ensure(static_cast<size_t>(S)));
    SCU(s->qlen.ensure(static_cast<size_t>(S)));
    {
        std::vector<int64_t> st0(static_cast<size_t>(S));
        for (int i = 0; i < S; ++i) st0[static_cast<size_t>(i)] = static_cast<int64_t>(i) * s->opt.max_query_len;
        SCU(cudaMemcpy(s->qstart.ptr, st0.data(), sizeof(int64_t) * S, cudaMemcpyHostToDevice));
        SCU(cudaMemset(s->qlen.ptr, 0, sizeof(int32_t) * S));
    }
    if (s->mq_ok) {
        SCU(s->steps_d.ensure(static_cast<size_t>(s->max_steps)));
        SCU(s->pp.ensure(static_cast<size_t>((s->A + 1) * s->rows_pad)));
        SCU(cudaMallocHost(reinterpret_cast<void**>(&s->steps_h), sizeof(MqStep) * s->max_steps));
        std::memset(s->steps_h, 0, sizeof(MqStep) * s->max_steps);
    }
    SCU(s->ctrl.ensure(1));
    SCU(s->flags.ensure(static_cast<size_t>(std::min<int64_t>(std::max<int64_t>(s->N * S, 1), 1 << 20))));
    const int64_t bnd_stride = std::max<int64_t>(1, v.max_group_len / 2 * kWarp);
    const int64_t spill_stride = std::max<int64_t>(1, (v.max_len + 31) / 32 * 32 + 64);
    SCU(s->bnd.ensure(static_cast<size_t>(static_cast<int64_t>(std::max(s->inter_grid, s->mq_grid)) *
                                          s->W * bnd_stride)));
    SCU(s->spill.ensure(static_cast<size_t>(static_cast<int64_t>(s->intra_grid) *
                                            (intra_block_threads() / kWarp) * spill_stride)));
    SCU(cudaMallocHost(reinterpret_cast<void**>(&s->tick_h), sizeof(TickDesc)));
    std::memset(s->tick_h, 0, sizeof(TickDesc));
    SCU(cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking));
    SCU(cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking));
    SCU(cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming));
    sw_status st = capture_tick_graphs(s.get(), v);
    if (st != SW_OK) return st;
    s->active.assign(static_cast<size_t>(S), nullptr);
    sw_server* raw = s.get();
    raw->worker = std::thread(worker_loop, raw);
    *out = s.release();
    return SW_OK;
}

sw_status sw_server_submit(sw_server* s, const uint8_t* query, int32_t query_len, int64_t* ticket) {
    if (!s || !ticket) return set_last_error(SW_ERR_ARG, "null pointer");
    if (query_len < 0 || query_len > s->opt.max_query_len)
        return set_last_error(SW_ERR_ARG, "query_len outside [0, max_query_len]");
    if (query_len > 0 && !query) return set_last_error(SW_ERR_ARG, "query is null");
    for (int32_t i = 0; i < query_len; ++i)
        if (query[i] >= s->A) return set_last_error(SW_ERR_CODE, "query residue code >= alphabet_size");
    auto r = std::make_unique<Request>();
    r->query.assign(query, query + query_len);
    r->m = query_len;
    r->state_bytes = state_bytes(s, query_len);
    r->t_submit = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return set_last_error(SW_ERR_STATE, "server stopped");
    if (static_cast<int64_t>(s->pending.size()) >= s->opt.max_pending) {
        ++s->rejected;
        return set_last_error(SW_ERR_BUSY, "pending queue full");
    }
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    if (s->submitted == 0 || s->t_first == 0) s->t_first = r->t_submit;
    if (s->last_submit > 0) s->mean_gap = 0.9 * s->mean_gap + 0.1 * (r->t_submit - s->last_submit);
    s->last_submit = r->t_submit;
    ++s->submitted;
    Request* raw = r.get();
    s->reqs.emplace(raw->ticket, std::move(r));
    if (query_len == 0 || s->N == 0) {   // nothing to align: every score is 0
        raw->result.assign(static_cast<size_t>(s->N), 0);
        finish(s, raw);
        s->cv_done.notify_all();
        return SW_OK;
    }
    s->pending.push_back(raw);
    s->cv_work.notify_one();
    return SW_OK;
}

static sw_status take_result(sw_server* s, int64_t ticket, int32_t* scores, int32_t* done,
                             std::unique_lock<std::mutex>& lk, int32_t timeout_ms) {
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_last_error(SW_ERR_ARG, "unknown ticket");
    Request* r = it->second.get();
    if (timeout_ms > 0 && !r->done) {
        s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                            [&] { return r->done || s->stop; });
    }
    if (!r->done) {
        if (s->worker_status != SW_OK) return s->worker_status;
        if (done) *done = 0;
        return timeout_ms > 0 ? set_last_error(SW_ERR_TIMEOUT, "request not done within the timeout")
                              : SW_OK;
    }
    if (scores && s->N > 0) std::memcpy(scores, r->result.data(), sizeof(int32_t) * s->N);
    if (done) *done = 1;
    s->reqs.erase(it);
    return SW_OK;
}

sw_status sw_server_poll(sw_server* s, int64_t ticket, int32_t* scores, int32_t* done) {
    if (!s || !done) return set_last_error(SW_ERR_ARG, "null pointer");
    std::unique_lock<std::mutex> lk(s->mu);
    return take_result(s, ticket, scores, done, lk, 0);
}

sw_status sw_server_wait(sw_server* s, int64_t ticket, int32_t* scores, int32_t timeout_ms) {
    if (!s) return set_last_error(SW_ERR_ARG, "null pointer");
    if (timeout_ms <= 0) timeout_ms = 1;
    std::unique_lock<std::mutex> lk(s->mu);
    int32_t done = 0;
    return take_result(s, ticket, scores, &done, lk, timeout_ms);
}

sw_status sw_server_get_stats(sw_server* s, sw_server_stats* out, int32_t reset) {
    if (!s || !out) return set_last_error(SW_ERR_ARG, "null pointer");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->ticks = s->ticks;
    out->in_flight = in_flight(s);
    out->max_in_flight = s->max_in_flight;
    out->joined_while_running = s->joined;
    out->latency_p50_ms = 1e3 * percentile(s->latencies, 0.50);
    out->latency_p99_ms = 1e3 * percentile(s->latencies, 0.99);
    double sum = 0, mx = 0;
    for (double x : s->latencies) {
        sum += x;
        mx = std::max(mx, x);
    }
    out->latency_mean_ms = s->latencies.empty() ? 0.0 : 1e3 * sum / s->latencies.size();
    out->latency_max_ms = 1e3 * mx;
    out->cells = s->cells;
    const double span = s->t_last - s->t_first;
    out->gcups = span > 0 ? s->cells / span / 1e9 : 0.0;
    if (reset) {
        s->latencies.clear();
        s->submitted = s->completed = s->rejected = s->ticks = s->joined = s->cells = 0;
        s->max_in_flight = 0;
        s->t_first = s->t_last = 0;
    }
    return s->worker_status;
}

void sw_server_destroy(sw_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    {
        DeviceGuard guard(s->db->device);
        if (s->st) cudaStreamSynchronize(s->st);
        if (s->graph) cudaGraphExecDestroy(s->graph);
        if (s->graph_mq) cudaGraphExecDestroy(s->graph_mq);
        if (s->steps_h) cudaFreeHost(s->steps_h);
        if (s->ev) cudaEventDestroy(s->ev);
        if (s->st) cudaStreamDestroy(s->st);
        if (s->cap) cudaStreamDestroy(s->cap);
        if (s->tick_h) cudaFreeHost(s->tick_h);
        s->q_buf.release();
        s->qp_buf.release();
        s->scores.release();
        s->descs.release();
        s->qoff.release();
        s->qp_off.release();
        s->mpad.release();
        s->dmat.release();
        s->tick_d.release();
        s->qstart.release();
        s->qlen.release();
        s->steps_d.release();
        s->pp.release();
        s->ctrl.release();
        s->flags.release();
        s->bnd.release();
        s->spill.release();
    }
    delete s;
}

}  // extern "C"
