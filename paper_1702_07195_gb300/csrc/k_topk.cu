// Sorting stage (paper Section 4, step 3: alignment scores sorted in descending order): the
// k best database sequences of every query, descending score, ties by ascending sequence
// index.  One block per query:
//   1. radix select, most significant 8-bit digit first, of the k-th largest score t;
//   2. collection of every score > t and of the first (k - #greater) scores == t in index
//      order (block-wide ordered scan, so the lowest indices win ties);
//   3. a bitonic sort of the k (score, index) pairs in shared memory.
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/swgb.h"
#include "db_view.h"

namespace swgb {

namespace {

constexpr int kTopkThreads = 1024;
constexpr int kTopkMax = SW_TOPK_MAX;

__device__ __forceinline__ unsigned long long pack_key(int score, int id) {
    // descending score, then ascending index, as one ascending 64-bit key
    return (static_cast<unsigned long long>(0x7fffffffu - static_cast<unsigned>(score)) << 32) |
           static_cast<unsigned>(id);
}

__global__ void __launch_bounds__(kTopkThreads) k_topk(const int32_t* __restrict__ scores,
                                                       int64_t n, int32_t k,
                                                       int32_t* __restrict__ top_scores,
                                                       int32_t* __restrict__ top_ids) {
    __shared__ unsigned hist[256];
    __shared__ unsigned long long keys[kTopkMax];
    __shared__ unsigned s_prefix, s_mask, s_need, s_count, s_eq_taken;
    __shared__ unsigned s_warp[kTopkThreads / 32];
    __shared__ int s_max;
    const int tid = threadIdx.x;
    const int32_t* row = scores + static_cast<int64_t>(blockIdx.x) * n;

    // 0. maximum score: the radix select starts at its highest non-zero byte
    int mx = 0;
    for (int64_t i = tid; i < n; i += kTopkThreads) mx = max(mx, row[i]);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (tid == 0) s_max = 0;
    __syncthreads();
    if ((tid & 31) == 0) atomicMax(&s_max, mx);
    if (tid == 0) {
        s_prefix = 0;
        s_mask = 0;
        s_need = static_cast<unsigned>(k);
    }
    __syncthreads();
    int top_byte = 0;
    for (int b = 3; b > 0; --b)
        if (static_cast<unsigned>(s_max) >> (8 * b)) {
            top_byte = b;
            break;
        }

    // 1. radix select of the k-th largest score
    for (int b = top_byte; b >= 0; --b) {
        const int shift = 8 * b;
        for (int i = tid; i < 256; i += kTopkThreads) hist[i] = 0;
        __syncthreads();
        const unsigned prefix = s_prefix, mask = s_mask;
        for (int64_t i = tid; i < n; i += kTopkThreads) {
            const unsigned v = static_cast<unsigned>(row[i]);
            if ((v & mask) == prefix) atomicAdd(&hist[(v >> shift) & 0xFFu], 1u);
        }
        __syncthreads();
        if (tid == 0) {
            unsigned need = s_need, digit = 0;
            for (int d = 255; d >= 0; --d) {
                if (hist[d] >= need) {
                    digit = static_cast<unsigned>(d);
                    break;
                }
                need -= hist[d];
            }
            s_need = need;   // how many scores equal to the final threshold are still needed
            s_prefix = prefix | (digit << shift);
            s_mask = mask | (0xFFu << shift);
        }
        __syncthreads();
    }
    // Bytes above top_byte are zero for every score, and the select fixed the rest.
    const unsigned t = s_prefix;
    const unsigned need_eq = s_need;

    // 2. collection
    if (tid == 0) {
        s_count = 0;
        s_eq_taken = 0;
    }
    __syncthreads();
    for (int64_t i = tid; i < n; i += kTopkThreads) {
        const int v = row[i];
        if (static_cast<unsigned>(v) > t) {
            const unsigned pos = atomicAdd(&s_count, 1u);
            keys[pos] = pack_key(v, static_cast<int>(i));
        }
    }
    __syncthreads();
    const unsigned greater = s_count;
    // scores equal to t in index order: tiles of kTopkThreads, block prefix counts
    for (int64_t base = 0; base < n && s_eq_taken < need_eq; base += kTopkThreads) {
        const int64_t i = base + tid;
        const bool eq = i < n && static_cast<unsigned>(row[i]) == t;
        const unsigned ballot = __ballot_sync(0xffffffffu, eq);
        const int lane = tid & 31, warp = tid >> 5;
        if (lane == 0) s_warp[warp] = __popc(ballot);
        __syncthreads();
        unsigned before = 0;
        for (int w = 0; w < warp; ++w) before += s_warp[w];
        before += __popc(ballot & ((1u << lane) - 1u));
        const unsigned taken = s_eq_taken;
        if (eq && taken + before < need_eq)
            keys[greater + taken + before] = pack_key(static_cast<int>(t), static_cast<int>(i));
        __syncthreads();
        if (tid == 0) {
            unsigned tot = 0;
            for (int w = 0; w < kTopkThreads / 32; ++w) tot += s_warp[w];
            s_eq_taken = min(need_eq, taken + tot);
        }
        __syncthreads();
    }

    // 3. bitonic sort of the k keys (padded to a power of two with the largest key)
    int size = 1;
    while (size < k) size <<= 1;
    for (int i = k + tid; i < size; i += kTopkThreads) keys[i] = ~0ull;
    __syncthreads();
    for (int len = 2; len <= size; len <<= 1) {
        for (int stride = len >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < size; i += kTopkThreads) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = (i & len) == 0;
                    const unsigned long long a = keys[i], c = keys[j];
                    if ((a > c) == up) {
                        keys[i] = c;
                        keys[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int r = tid; r < k; r += kTopkThreads) {
        const unsigned long long key = keys[r];
        top_scores[static_cast<int64_t>(blockIdx.x) * k + r] =
            static_cast<int32_t>(0x7fffffffu - static_cast<unsigned>(key >> 32));
        top_ids[static_cast<int64_t>(blockIdx.x) * k + r] = static_cast<int32_t>(key & 0xffffffffu);
    }
}

}  // namespace

}  // namespace swgb

extern "C" sw_status sw_topk(const int32_t* d_scores, int64_t num_seqs, int32_t num_queries,
                             int32_t k, int32_t* d_top_scores, int32_t* d_top_ids, void* stream) {
    if (num_queries < 0 || num_seqs < 0 || k < 0)
        return swgb::set_last_error(SW_ERR_ARG, "negative size");
    if (k > SW_TOPK_MAX) return swgb::set_last_error(SW_ERR_ARG, "k exceeds SW_TOPK_MAX (4096)");
    if (k > num_seqs) return swgb::set_last_error(SW_ERR_ARG, "k exceeds num_seqs");
    if (num_seqs > INT32_MAX) return swgb::set_last_error(SW_ERR_ARG, "num_seqs exceeds INT32_MAX");
    if (num_queries == 0 || k == 0) return SW_OK;
    if (!d_scores || !d_top_scores || !d_top_ids) return swgb::set_last_error(SW_ERR_ARG, "null pointer");
    swgb::k_topk<<<num_queries, swgb::kTopkThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        d_scores, num_seqs, k, d_top_scores, d_top_ids);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return swgb::set_last_error(SW_ERR_CUDA, cudaGetErrorString(e));
    swgb::add_launches(1);
    return SW_OK;
}
