// Internal state of a loaded database (sw_db) and of a cached launch plan.  Shared by the
// runtime's translation units; not part of the C ABI.
#pragma once

#include <algorithm>
#include <cstdint>
#include <memory>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/swgb.h"
#include "layout.h"
#include "swgb_device.cuh"

namespace swgb {

constexpr int kMaxVariants = 8;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
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
    ~DevBuf() { release(); }
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
};

// Everything one search shape needs besides the shared scratch: its own profile buffer and
// tables, the kernel parameters, and the instantiated CUDA graph of its launch sequence.
struct Plan {
    std::vector<int64_t> key;
    int nq = 0;
    std::vector<int32_t> m;
    int32_t* d_scores = nullptr;
    bool int16_ok = true;
    int32_t qp_bias = 0;
    int variant = 0;
    int64_t max_mpad = 0;
    int64_t num_items = 0;
    int inter_grid = 0, intra_grid = 0, intra_block_grid = 0;
    int intra_rows_per_lane = 16;
    int intra_block_warps = 4;
    uint32_t flag_cap = 0;
    int64_t cells = 0, inter_cells = 0, launches = 0;
    DevBuf<int16_t> qp;
    DevBuf<QueryDesc> descs;
    DevBuf<InterItem> items;
    DevBuf<int64_t> qp_off;
    DevBuf<int32_t> mpad;
    DevBuf<int64_t> qoff;
    DevBuf<int32_t> order;
    DevBuf<int8_t> matrix;
    InterParams inter{};
    IntraParams intra{};
    int64_t g_split = 0;      // groups [g_split, G) run on the int32 kernel (critical path)
    // multi-query kernel (two queries per register against one subject)
    bool mq = false;
    bool sp = false;              // score-profile single-query kernel
    DevBuf<int16_t> mt;           // its transposed biased matrix
    int32_t num_steps = 0;
    int64_t rows_pad = 0;
    DevBuf<MqStep> steps;
    DevBuf<uint32_t> pp;
    InterMqParams inter_mq{};
    // packed int16x2 wavefront kernel for the long subjects (two queries per register)
    bool wave = false;
    int wave_rows = 16;           // query rows per lane
    int wave_grid = 0;
    int32_t num_wpasses = 0;
    int64_t wrows_pad = 0;
    DevBuf<WavePass> wpasses;
    DevBuf<uint32_t> wpp;
    WaveParams wave_p{};
    // packed int16x2 wavefront kernel for routed groups of a one-query search (two subjects
    // per register); groups [g_split, g_pair_end) run there, [g_pair_end, G) on int32
    bool pair = false;
    int pair_rows = 5;            // rows per lane of the 32-lane wavefronts
    bool pair_half = false;       // bulk: two 16-lane wavefronts per warp for the shorter pairs
    int64_t pair_half_from = 0;   // ... from this pair index on (0 = the longest)
    int pair_grid = 0;
    int64_t g_pair_end = 0;
    int64_t pair_long_pairs = 0;  // longest slot pairs, run first with one warp per sub-partition
    int pair_long_blocks = 0;
    WaveParams pair_p{};
    cudaGraphExec_t exec = nullptr;
};

}  // namespace swgb

struct sw_db {
    int device = 0;
    int sms = 0;
    int32_t A = 0;
    int32_t long_cutoff = 0;
    int32_t flag_cap = 1 << 20;
    swgb::Layout layout;
    int64_t num_residues = 0;
    // device database
    swgb::DevBuf<uint8_t> inter;
    swgb::DevBuf<int64_t> group_off;
    swgb::DevBuf<int32_t> group_len;
    swgb::DevBuf<int32_t> group_cols;
    swgb::DevBuf<int32_t> perm;
    swgb::DevBuf<uint8_t> plain;
    swgb::DevBuf<int64_t> plain_off;
    swgb::DevBuf<int32_t> long_ids;
    int32_t placement = 0;
    uint8_t* host_inter = nullptr;   // SW_PLACE_HOST: pinned, mapped database copies
    uint8_t* host_plain = nullptr;
    const uint8_t* inter_ptr = nullptr;   // device view of the interleaved groups
    const uint8_t* plain_ptr = nullptr;   // device view of the plain copy
    // scratch shared by all searches on this database (ordered on the device by ev[4])
    swgb::DevBuf<swgb::Control> ctrl;
    swgb::DevBuf<swgb::FlagEntry> flags;
    swgb::DevBuf<uint4> bnd;
    swgb::DevBuf<int2> spill;
    // host-buffer API staging
    swgb::DevBuf<uint8_t> h_queries;
    swgb::DevBuf<int32_t> h_scores;
    uint8_t* pinned_q = nullptr;     // pinned host staging of the queries (grown on demand)
    size_t pinned_q_cap = 0;
    cudaStream_t stream = nullptr;           // stream of the host-buffer API
    cudaStream_t capture_stream = nullptr;   // graphs are captured here, launched on the caller's
    cudaEvent_t ev[5] = {};                  // per-kernel timing; ev[4] = end of the last search
    bool done_recorded = false;
    std::vector<std::unique_ptr<swgb::Plan>> plans;   // most recent last, at most 32
    // kernel choice
    int variant = 0;
    bool no_route = false;    // set by the autotuner: every group stays on the inter-task kernel
    int inter_occ[swgb::kMaxVariants] = {};
    int inter_mq_occ[swgb::kMaxVariants] = {};
    int intra_occ = 0;
    int intra_block_occ[3] = {0, 0, 0};   // 5, 8 and 16 query rows per lane
    int inter_sp_occ = 0;                 // score-profile inter-task kernel
    int wave_occ[3] = {0, 0, 0};          // packed wavefront kernel, 8, 12 and 16 rows per lane
    int max_smem = 0;                     // opt-in shared memory per block (bytes)
    // last search
    sw_stats stats{};
    bool stats_pending = false;
    bool stats_inter = false;    // the last search recorded the inter-task stage events
    bool stats_pair_only = false;  // ... and ran the two-subject kernel with a dependent rescore
    std::mutex mu;
    ~sw_db() {
        if (host_inter) cudaFreeHost(host_inter);
        if (host_plain) cudaFreeHost(host_plain);
        if (pinned_q) cudaFreeHost(pinned_q);
    }
};
