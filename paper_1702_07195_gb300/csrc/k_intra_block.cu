// Intra-task Smith-Waterman/Gotoh kernel in int32, block-shared profile variant.
//
// Same wavefront as k_intra_i32 (one warp per (query, subject) pair; lane l owns a strip of
// query rows and updates column t - l at step t; rows pass between lanes by __shfl_up_sync;
// a per-warp global buffer carries the bottom row to the next pass) but for the work sources
// where neighbouring pairs share the query -- subjects above the inter-task cutoff and groups
// routed off the inter-task kernel -- the warps of a block (8 with 16 rows per lane, else 4)
// take the same query against as many neighbouring subjects (longest first), so one copy of
// the pass's profile slice serves the block.  The slice is stored as int32 (sign-extended and
// biased once per pass, not once per cell) and each lane owns 5, 8 or 16 rows.
// Eqs. sw2-sw4, Section 2; the intra-task scheme of Section 1.
//
// Shared-memory layout of the slice: the 32 lanes read the rows of 32 different residues in
// the same step, so with a plain row-major slice the bank a lane hits depends on its residue
// and the 16-byte loads of a quarter-warp collide at random.  Here the row stride of a residue
// is a multiple of 32 words (the residue no longer moves the bank) and lane l's chunk of
// kTB words sits at a lane-dependent offset chosen so that the 8 lanes of every quarter-warp
// start in 8 different 16-byte bank groups: each 16-byte profile load is one wavefront per
// quarter-warp whatever the residues are.  With an odd number of rows per lane the chunks are
// packed (lane l at word 5 l for 5 rows) and read with 4-byte loads: 5 l mod 32 is a
// permutation of the banks, so those loads are conflict-free as they are.
#include <type_traits>

#include "slice_layout.cuh"
#include "swgb_device.cuh"

namespace swgb {

namespace {

constexpr int kMaxBW = 8;                   // warps per block = subjects per block item

struct BlockItem {
    int q;
    int seq[kMaxBW];
};

// Decodes block item `it` (longest subjects first); seq = -1 for absent / filler slots.
template <int kBW>
__device__ bool decode_item(const IntraParams& p, unsigned long long it, BlockItem& out) {
    if (p.mode == kIntraLong) {
        const int64_t per_q = (p.num_long + kBW - 1) / kBW;
        const unsigned long long total =
            static_cast<unsigned long long>(per_q) * static_cast<unsigned long long>(p.num_queries);
        if (it >= total) return false;
        const int64_t c = static_cast<int64_t>(it / static_cast<unsigned long long>(p.num_queries));
        const int qi = static_cast<int>(static_cast<int64_t>(it) - c * p.num_queries);
        out.q = p.query_order[qi];
        for (int w = 0; w < kBW; ++w) {
            const int64_t li = c * kBW + w;
            out.seq[w] = li < p.num_long ? p.long_ids[li] : -1;
        }
        return true;
    }
    // kIntraGroups: slots [slot_begin, slot_end), from the end (longest groups first)
    const int64_t nslots = p.slot_end - p.slot_begin;
    const int64_t per_q = (nslots + kBW - 1) / kBW;
    const unsigned long long total =
        static_cast<unsigned long long>(per_q) * static_cast<unsigned long long>(p.num_queries);
    if (it >= total) return false;
    const int64_t c = static_cast<int64_t>(it / static_cast<unsigned long long>(p.num_queries));
    const int qi = static_cast<int>(static_cast<int64_t>(it) - c * p.num_queries);
    out.q = p.query_order[qi];
    for (int w = 0; w < kBW; ++w) {
        const int64_t si = c * kBW + w;
        out.seq[w] = si < nslots ? p.perm[p.slot_end - 1 - si] : -1;
    }
    return true;
}

// One query row of the column step: the cell update of Eqs. sw2-sw4 on (H - Goe) state.
__device__ __forceinline__ int cell_i32(int& d, int& hm, int& e, int& f, int sc, int goe, int ge,
                                        int gep) {
    const int x = __viaddmax_s32_relu(d, sc, e);
    const int xm = x - goe;
    d = hm;
    hm = __viaddmax_s32(f, -goe, xm);
    e = __viaddmax_s32(e, -ge, hm);
    f = __viaddmax_s32(f, -gep, xm);
    return x;
}

// kTB query rows per lane: passes of 32 * kTB rows (160, 256 or 512); kBW warps per block.
template <int kTB, int kBW>
__global__ void __launch_bounds__(kBW * kWarp) k_intra_block_i32(const IntraParams p) {
    constexpr int kBBlock = kBW * kWarp;
    constexpr int kRowsB = kTB * kWarp;
    constexpr int kPStride = slice_stride<kTB>();   // int32 per shared-memory profile row
    extern __shared__ __align__(16) int32_t s_prof[];     // (A+1) x kPStride
    __shared__ BlockItem s_item;
    __shared__ int s_done;
    __shared__ int s_passes;
    const int lane = threadIdx.x & (kWarp - 1);
    const int warp = threadIdx.x >> 5;
    const int my_chunk = chunk_offset<kTB>(lane);
    int2* spill = p.spill + (static_cast<int64_t>(blockIdx.x) * kBW + warp) * p.spill_stride;
    const int goe = p.gaps.goe, ge = p.gaps.ge, gep = p.gaps.gep;
    unsigned long long* counter =
        p.mode == kIntraGroups ? &p.ctrl->next_groups : &p.ctrl->next_intra;

    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned long long it = atomicAdd(counter, 1ull);
            s_done = decode_item<kBW>(p, it, s_item) ? 0 : 1;
            if (!s_done) s_passes = (p.queries[s_item.q].m + kRowsB - 1) / kRowsB;
        }
        __syncthreads();
        if (s_done) break;
        const int q = s_item.q;
        const QueryDesc qd = p.queries[q];
        const int seq = s_item.seq[warp];
        const int passes = s_passes;
        int n = 0;
        const uint8_t* subj = nullptr;
        if (seq >= 0) {
            const int64_t off = p.plain_off[seq];
            n = static_cast<int>(p.plain_off[seq + 1] - off);
            subj = p.plain + off;
        }
        int best = 0;
        for (int pass = 0; pass < passes; ++pass) {
            const bool first = pass == 0, last = pass == passes - 1;
            __syncthreads();   // everyone is done with the previous slice
            for (int v = threadIdx.x; v < p.alphabet1 * kRowsB; v += kBBlock) {
                const int d = v / kRowsB;
                const int r = v - d * kRowsB;
                const int64_t row = static_cast<int64_t>(pass) * kRowsB + r;
                // rows past the profile score 0: S' = 0 + Goe, like the profile's own padding
                s_prof[d * kPStride + chunk_offset<kTB>(r / kTB) + r % kTB] =
                    row < qd.m_pad ? qd.qp[static_cast<int64_t>(d) * qd.m_pad + row] + p.qp_add : goe;
            }
            __syncthreads();
            if (n == 0 || qd.m == 0) continue;
            int Hm[kTB], E[kTB];
#pragma unroll
            for (int r = 0; r < kTB; ++r) {
                Hm[r] = -goe;
                E[r] = -gep;
            }
            int hm_prev = -goe;
            int out_hm = -goe, out_f = -gep;
            int2 sp_cur = make_int2(-goe, -gep), sp_next = make_int2(-goe, -gep);
            if (!first) {
                if (lane < n) sp_cur = spill[lane];
                if (32 + lane < n) sp_next = spill[32 + lane];
            }
            const int steps = n + kWarp - 1;
            // Step t: lane l updates column t - l.  `checked` steps skip lanes whose column is
            // outside [0, n); blocks of 32 steps in which every lane's column is inside skip the
            // test.  Lane 0 takes the previous pass's row of column t from lane (t mod 32) of
            // sp_cur, which holds columns [32 k, 32 k + 32) during steps [32 k, 32 k + 32); in the
            // first pass that row is the zero boundary, a constant (`on_first`: no shuffle).
            auto step = [&](const int t, const int src, auto checked, auto on_first) {
                const int up_hm = __shfl_up_sync(0xffffffffu, out_hm, 1);
                const int up_f = __shfl_up_sync(0xffffffffu, out_f, 1);
                int l0_hm = -goe, l0_f = -gep;
                if constexpr (!decltype(on_first)::value) {
                    l0_hm = __shfl_sync(0xffffffffu, sp_cur.x, src);
                    l0_f = __shfl_sync(0xffffffffu, sp_cur.y, src);
                }
                const int j = t - lane;
                if (decltype(checked)::value && !(j >= 0 && j < n)) return;
                int F = lane == 0 ? l0_f : up_f;                 // F(r0, j)
                int d = hm_prev;                                 // (H - Goe)(r0 - 1, j - 1)
                hm_prev = lane == 0 ? l0_hm : up_hm;             // (H - Goe)(r0 - 1, j)
                const int32_t* prow1 = s_prof + subj[j] * kPStride + my_chunk;
                if constexpr (kTB % 2 == 1) {
#pragma unroll
                    for (int r = 0; r + 1 < kTB; r += 2) {
                        const int x0 = cell_i32(d, Hm[r], E[r], F, prow1[r], goe, ge, gep);
                        const int x1 = cell_i32(d, Hm[r + 1], E[r + 1], F, prow1[r + 1], goe, ge, gep);
                        best = __vimax3_s32(best, x0, x1);
                    }
                    best = max(best, cell_i32(d, Hm[kTB - 1], E[kTB - 1], F, prow1[kTB - 1], goe, ge, gep));
                } else {
                    const int4* prow = reinterpret_cast<const int4*>(prow1);
#pragma unroll
                    for (int r4 = 0; r4 < kTB; r4 += 4) {
                        const int4 sv = prow[r4 >> 2];
                        const int x0 = cell_i32(d, Hm[r4], E[r4], F, sv.x, goe, ge, gep);
                        const int x1 = cell_i32(d, Hm[r4 + 1], E[r4 + 1], F, sv.y, goe, ge, gep);
                        best = __vimax3_s32(best, x0, x1);
                        const int x2 = cell_i32(d, Hm[r4 + 2], E[r4 + 2], F, sv.z, goe, ge, gep);
                        const int x3 = cell_i32(d, Hm[r4 + 3], E[r4 + 3], F, sv.w, goe, ge, gep);
                        best = __vimax3_s32(best, x2, x3);
                    }
                }
                out_hm = Hm[kTB - 1];
                out_f = F;
                if (lane == kWarp - 1 && !last) spill[j] = make_int2(out_hm, out_f);
            };
            auto run = [&](auto on_first) {
                for (int tb = 0; tb < steps; tb += kWarp) {
                    if constexpr (!decltype(on_first)::value) {
                        if (tb > 0) {
                            sp_cur = sp_next;
                            if (tb + 32 + lane < n) sp_next = spill[tb + 32 + lane];
                        }
                    }
                    if (tb >= kWarp && tb + kWarp <= n) {
                        // 5 or 8 rows per lane: four steps per loop iteration (plain config
                        // 0.283 -> 0.24-0.26 ms); 16 rows: one (two measured 1.5 % slower)
                        if constexpr (kTB < 16) {
#pragma unroll 4
                            for (int u = 0; u < kWarp; ++u) step(tb + u, u, std::false_type{}, on_first);
                        } else {
#pragma unroll 1
                            for (int u = 0; u < kWarp; ++u) step(tb + u, u, std::false_type{}, on_first);
                        }
                    } else {
                        const int ue = min(kWarp, steps - tb);
#pragma unroll 1
                        for (int u = 0; u < ue; ++u) step(tb + u, u, std::true_type{}, on_first);
                    }
                }
            };
            if (first)
                run(std::true_type{});
            else
                run(std::false_type{});
            __syncwarp();   // lane 31's spill writes are visible to the warp's next pass
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
        if (seq >= 0 && lane == 0) qd.scores[seq] = best;
    }
}

}  // namespace

// Warps per block: 8 with 16 rows per lane (three 54 KB blocks, 24 warps per SM; four 4-warp
// blocks gave 16 warps per SM and 5 % less throughput on long subjects), else 4.
int intra_block_warps(int rows_per_lane) { return rows_per_lane == 16 ? 8 : 4; }

namespace {

const void* block_fn(int rows_per_lane) {
    switch (rows_per_lane) {
        case 5: return reinterpret_cast<const void*>(&k_intra_block_i32<5, 4>);
        case 8: return reinterpret_cast<const void*>(&k_intra_block_i32<8, 4>);
        default: return reinterpret_cast<const void*>(&k_intra_block_i32<16, 8>);
    }
}

}  // namespace

size_t intra_block_smem_bytes(int rows_per_lane, int alphabet1) {
    const int stride = rows_per_lane == 5   ? slice_stride<5>()
                       : rows_per_lane == 8 ? slice_stride<8>()
                                            : slice_stride<16>();
    return static_cast<size_t>(alphabet1) * stride * sizeof(int32_t);
}

int intra_block_occupancy(int rows_per_lane, int alphabet1) {
    int n = 0;
    const size_t smem = intra_block_smem_bytes(rows_per_lane, alphabet1);
    const void* fn = block_fn(rows_per_lane);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, intra_block_warps(rows_per_lane) * kWarp,
                                                      smem) != cudaSuccess)
        return 0;
    return n;
}

// Runs the long-subject (kIntraLong) and routed-group (kIntraGroups) work sources with 5, 8 or
// 16 query rows per lane.
cudaError_t launch_intra_block(const IntraParams& p, int rows_per_lane, int grid, cudaStream_t st) {
    const size_t smem = intra_block_smem_bytes(rows_per_lane, p.alphabet1);
    const void* fn = block_fn(rows_per_lane);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    if (rows_per_lane == 5)
        k_intra_block_i32<5, 4><<<grid, 4 * kWarp, smem, st>>>(p);
    else if (rows_per_lane == 8)
        k_intra_block_i32<8, 4><<<grid, 4 * kWarp, smem, st>>>(p);
    else
        k_intra_block_i32<16, 8><<<grid, 8 * kWarp, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace swgb
