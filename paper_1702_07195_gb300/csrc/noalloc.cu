// sw_search_noalloc: the one-query search with no device allocation at all.
//
// Who needs it.  The regular entry points keep a per-database workspace that grows with
// cudaMalloc the first time a bigger search arrives.  Some callers cannot accept that:
//  * a service that overlaps many streams: cudaMalloc and cudaFree may synchronise the
//    whole device, stalling every other stream at an unpredictable moment;
//  * a process whose device memory is already handed out by another allocator (a deep
//    learning framework's caching allocator, a pool sized at start-up, a container with a
//    hard memory limit): a library-private cudaMalloc at search time can fail there;
//  * code that must not allocate after initialisation (latency-critical or certified
//    pipelines).
// This entry point keeps every piece of working memory -- the query profile, the work list,
// the counters, the list of saturated lanes and the strip and pass boundary buffers -- in
// one fixed array, `g_scratch` below, that is part of the library's device image.  The
// caller still passes the query and the output on the device.
//
// Cost of the fixed array: kScratchBytes (about 85 MiB) on every device where this entry
// point runs, held until the process exits.  (With CUDA's default lazy module loading the
// array is reserved when the first call on a device resolves its address.)  Because the
// boundary buffers are bounded, the inter-task kernel runs on as many blocks as fit in them
// (a warp's buffer takes 16 bytes per column pair and thread: 512 KB for a longest group of
// 2,000 columns, 2 MB for a 4-warp block, so about 32 blocks fit in kBndBytes), so this path
// is slower than sw_search_batch_device on large databases.
//
// The same kernels as the regular search run here (query profile, int16x2 inter-task
// kernel, int32 intra-task kernel for long subjects and for saturated lanes); only the
// scratch pointers differ.  The paper has no counterpart to this entry point.
#include <algorithm>
#include <cstdio>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/swgb.h"
#include "db_view.h"
#include "swgb_device.cuh"

namespace swgb {

namespace {

constexpr int64_t kAlign = 256;
constexpr int64_t align_up(int64_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

constexpr int64_t kMaxQuery = SW_NOALLOC_MAX_QUERY;
constexpr int64_t kMaxItems = 1 << 18;      // block work items: up to 2^20 groups (67M sequences)
constexpr int64_t kMaxFlags = 1 << 16;      // saturated lanes listed; beyond, the rescore sweeps
constexpr int64_t kBndBytes = int64_t{64} << 20;
constexpr int64_t kSpillBytes = int64_t{16} << 20;

// Byte offsets of each region inside the array (all 256-byte aligned).
constexpr int64_t kOffCtrl = 0;
constexpr int64_t kOffDesc = align_up(kOffCtrl + static_cast<int64_t>(sizeof(Control)));
constexpr int64_t kOffQpOff = align_up(kOffDesc + static_cast<int64_t>(sizeof(QueryDesc)));
constexpr int64_t kOffMpad = align_up(kOffQpOff + 8);
constexpr int64_t kOffQoff = align_up(kOffMpad + 4);
constexpr int64_t kOffOrder = align_up(kOffQoff + 16);
constexpr int64_t kOffMatrix = align_up(kOffOrder + 4);
constexpr int64_t kOffItems = align_up(kOffMatrix + kMaxAlphabet * kMaxAlphabet);
constexpr int64_t kOffFlags = align_up(kOffItems + kMaxItems * static_cast<int64_t>(sizeof(InterItem)));
constexpr int64_t kOffQp = align_up(kOffFlags + kMaxFlags * static_cast<int64_t>(sizeof(FlagEntry)));
constexpr int64_t kOffBnd = align_up(kOffQp + (kMaxAlphabet + 1) * kMaxQuery * 2);
constexpr int64_t kOffSpill = align_up(kOffBnd + kBndBytes);
constexpr int64_t kScratchBytes = align_up(kOffSpill + kSpillBytes);

static_assert(SW_NOALLOC_SCRATCH_BYTES == kScratchBytes, "header states the array size");
static_assert(kMaxQuery % kQpRows == 0, "profile rows are padded to kQpRows");

// The scratch array.  Host code must not use this name as a pointer: on the host it is a
// stand-in symbol, not a device address.  Its device address comes from
// cudaGetSymbolAddress, once per device (scratch_base below).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char* g_base[kMaxDevices] = {};

// Device address of g_scratch on the current device `dev`, resolved on the first call there.
sw_status scratch_base(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (dev < 0 || dev >= kMaxDevices) return set_last_error(SW_ERR_ARG, "device ordinal out of range");
    if (!g_base[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) {
            char msg[256];
            snprintf(msg, sizeof(msg), "cudaGetSymbolAddress(g_scratch): %s", cudaGetErrorString(e));
            return set_last_error(SW_ERR_CUDA, msg);
        }
        g_base[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_base[dev];
    return SW_OK;
}

// Per-call tables, passed by value as kernel parameters (about 1.1 KB) and written into the
// array by k_noalloc_setup: no host staging buffer and no host-to-device copy.
struct NoallocSetup {
    QueryDesc desc;
    int64_t query_len;
    int32_t m_pad;
    int32_t matrix_bytes;
    int8_t matrix[kMaxAlphabet * kMaxAlphabet];
};

// Writes the one-query tables (descriptor, profile offset and padded length, query offsets,
// query order, matrix) and zeroes the control block: the array keeps the previous call's
// contents, and the counters must start at zero.
__global__ void k_noalloc_setup(const NoallocSetup s, Control* ctrl, QueryDesc* desc,
                                int64_t* qp_off, int32_t* mpad, int64_t* qoff, int32_t* order,
                                int8_t* dmat) {
    for (int i = threadIdx.x; i < s.matrix_bytes; i += blockDim.x) dmat[i] = s.matrix[i];
    if (threadIdx.x == 0) {
        *ctrl = Control{};
        *desc = s.desc;
        *qp_off = 0;
        *mpad = s.m_pad;
        qoff[0] = 0;
        qoff[1] = s.query_len;
        *order = 0;
    }
}

// Work list for one query: chunks of `w` groups, longest groups first.
__global__ void k_noalloc_items(InterItem* items, int64_t num_groups, int w, int64_t nchunks) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < nchunks;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t g0 = (nchunks - 1 - i) * w;
        const int64_t ng = num_groups - g0 < w ? num_groups - g0 : w;
        items[i] = InterItem{0, static_cast<int32_t>(g0), static_cast<int32_t>(ng), 0};
    }
}

sw_status arg_error(const char* msg) { return set_last_error(SW_ERR_ARG, msg); }

sw_status cuda_error(cudaError_t e, const char* what) {
    char msg[256];
    snprintf(msg, sizeof(msg), "%s: %s", what, cudaGetErrorString(e));
    return set_last_error(SW_ERR_CUDA, msg);
}

#define NA_CU(call)                                          \
    do {                                                     \
        const cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_error(e_, #call); \
    } while (0)

struct CurrentDevice {
    int prev = -1;
    explicit CurrentDevice(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~CurrentDevice() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

}  // namespace swgb

using namespace swgb;

extern "C" sw_status sw_search_noalloc(const sw_db* db, const uint8_t* d_query, int32_t query_len,
                                       const int8_t* matrix, int32_t gap_open,
                                       int32_t gap_extend, int32_t* d_scores, void* stream) {
    DbView v;
    if (!db_view(db, &v)) return arg_error("db is null");
    if (!matrix) return arg_error("matrix is null");
    if (query_len < 0) return arg_error("query_len < 0");
    if (query_len > kMaxQuery) return arg_error("query_len exceeds SW_NOALLOC_MAX_QUERY (8192)");
    if (query_len > 0 && !d_query) return arg_error("d_query is null");
    if (gap_open < 0 || gap_extend < 0 || gap_open > 1000000 || gap_extend > 1000000)
        return arg_error("gap costs must be in [0, 1000000]");
    const int64_t N = v.num_seqs;
    if (N > 0 && !d_scores) return arg_error("d_scores is null");
    const int32_t A = v.alphabet;
    int max_s = 0;
    for (int i = 0; i < A * A; ++i) max_s = std::max<int>(max_s, matrix[i]);
    if (static_cast<double>(std::min<int64_t>(query_len, v.max_len)) * max_s > 2147483647.0)
        return arg_error("scores could exceed the int32 range");

    const int W = inter_variant_warps(0);
    const int IW = intra_block_threads() / kWarp;
    const int64_t nchunks = (v.num_groups + W - 1) / W;
    if (nchunks > kMaxItems) return arg_error("database has more groups than the fixed work list holds");
    const int64_t bnd_stride = std::max<int64_t>(1, v.max_group_len / 2 * kWarp);
    const int64_t inter_blocks =
        std::min<int64_t>(static_cast<int64_t>(v.sms) * std::max(1, v.inter_occ),
                          kBndBytes / (bnd_stride * static_cast<int64_t>(sizeof(uint4)) * W));
    if (v.num_groups > 0 && inter_blocks < 1)
        return arg_error("database groups are too long for the fixed boundary buffers");
    const int64_t spill_stride = std::max<int64_t>(1, (v.max_len + 31) / 32 * 32 + 64);
    const int64_t intra_blocks =
        std::min<int64_t>(static_cast<int64_t>(v.sms) * std::max(1, v.intra_occ),
                          kSpillBytes / (spill_stride * static_cast<int64_t>(sizeof(int2)) * IW));
    if (intra_blocks < 1) return arg_error("database sequences are too long for the fixed pass buffers");
    if (N == 0) return SW_OK;

    CurrentDevice guard(v.device);
    unsigned char* base = nullptr;
    const sw_status st0 = scratch_base(v.device, &base);
    if (st0 != SW_OK) return st0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (query_len == 0) {
        NA_CU(cudaMemsetAsync(d_scores, 0, sizeof(int32_t) * N, st));
        return SW_OK;
    }

    Control* ctrl = reinterpret_cast<Control*>(base + kOffCtrl);
    QueryDesc* desc = reinterpret_cast<QueryDesc*>(base + kOffDesc);
    int64_t* qp_off = reinterpret_cast<int64_t*>(base + kOffQpOff);
    int32_t* mpad = reinterpret_cast<int32_t*>(base + kOffMpad);
    int64_t* qoff = reinterpret_cast<int64_t*>(base + kOffQoff);
    int32_t* order = reinterpret_cast<int32_t*>(base + kOffOrder);
    int8_t* dmat = reinterpret_cast<int8_t*>(base + kOffMatrix);
    InterItem* items = reinterpret_cast<InterItem*>(base + kOffItems);
    FlagEntry* flags = reinterpret_cast<FlagEntry*>(base + kOffFlags);
    int16_t* qp = reinterpret_cast<int16_t*>(base + kOffQp);
    uint4* bnd = reinterpret_cast<uint4*>(base + kOffBnd);
    int2* spill = reinterpret_cast<int2*>(base + kOffSpill);

    const int32_t goe = gap_open, ge = gap_extend, gep = std::min(goe, ge);
    const bool int16_ok = goe <= 16383 && ge <= 16383;
    const int32_t qp_bias = (goe + 128 <= 32767) ? goe : 0;
    const int32_t m_pad = static_cast<int32_t>((query_len + kQpRows - 1) / kQpRows * kQpRows);
    const uint32_t flag_cap = static_cast<uint32_t>(std::min<int64_t>(std::min<int64_t>(N, kMaxFlags), v.flag_cap));

    // Small per-call tables travel as kernel parameters (captured by value at launch).
    NoallocSetup setup{};
    setup.desc = QueryDesc{qp, d_scores, query_len, m_pad};
    setup.query_len = query_len;
    setup.m_pad = m_pad;
    setup.matrix_bytes = A * A;
    for (int i = 0; i < A * A; ++i) setup.matrix[i] = matrix[i];
    k_noalloc_setup<<<1, 256, 0, st>>>(setup, ctrl, desc, qp_off, mpad, qoff, order, dmat);
    NA_CU(cudaGetLastError());

    int64_t launches = 1;
    NA_CU(launch_build_qp(d_query, qoff, 1, dmat, A, qp_bias, qp_off, mpad, qp, m_pad, ctrl, st));
    ++launches;
    const Gaps gaps{goe, ge, gep};
    if (int16_ok && v.num_groups > 0) {
        const int64_t grid = std::min<int64_t>(std::max<int64_t>(1, (nchunks + 255) / 256), 1024);
        k_noalloc_items<<<static_cast<unsigned>(grid), 256, 0, st>>>(items, v.num_groups, W, nchunks);
        NA_CU(cudaGetLastError());
        ++launches;
        InterParams p{};
        p.inter = v.inter;
        p.group_off = v.group_off;
        p.group_len = v.group_len;
        p.group_cols = v.group_cols;
        p.perm = v.perm;
        p.queries = desc;
        p.items = items;
        p.num_items = static_cast<int32_t>(nchunks);
        p.alphabet1 = A + 1;
        p.ctrl = ctrl;
        p.flags = flags;
        p.flag_cap = flag_cap;
        p.thresh = 32767 - std::max(0, max_s);
        p.bnd = bnd;
        p.bnd_stride = bnd_stride;
        p.gaps = gaps;
        NA_CU(launch_inter(p, 0, static_cast<int>(inter_blocks), st));
        ++launches;
    }
    IntraParams ip{};
    ip.plain = v.plain;
    ip.plain_off = v.plain_off;
    ip.queries = desc;
    ip.num_queries = 1;
    ip.long_ids = v.long_ids;
    ip.num_long = v.num_long;
    ip.query_order = order;
    ip.num_seqs = N;
    ip.flags = flags;
    ip.flag_cap = flag_cap;
    ip.alphabet1 = A + 1;
    ip.ctrl = ctrl;
    ip.spill = spill;
    ip.spill_stride = spill_stride;
    ip.gaps = gaps;
    ip.qp_add = goe - qp_bias;
    const int iblocks = static_cast<int>(intra_blocks);
    if (!int16_ok) {
        ip.mode = kIntraAll;
        NA_CU(launch_intra(ip, iblocks, intra_block_threads(), st));
        ++launches;
    } else {
        if (v.num_long > 0) {
            ip.mode = kIntraLong;
            NA_CU(launch_intra(ip, iblocks, intra_block_threads(), st));
            ++launches;
        }
        if (v.num_groups > 0) {
            ip.mode = kIntraRescore;
            NA_CU(launch_intra(ip, iblocks, intra_block_threads(), st));
            ++launches;
        }
    }
    add_launches(launches);
    return SW_OK;
}
