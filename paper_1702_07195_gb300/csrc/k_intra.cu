// Intra-task Smith-Waterman/Gotoh kernel in int32: one warp per (query, subject) pair.
//
// The paper names the intra-task scheme (parallelism inside one alignment matrix, Section 1)
// as the option for very long sequences.  Here it serves three work sources:
//   * kIntraLong    -- subjects longer than the inter-task cutoff, against every query;
//   * kIntraRescore -- (query, subject) pairs whose int16 lane reached the saturation
//                      threshold in the inter-task kernel: the exact recomputation at the
//                      next wider integer range of Section 4.2;
//   * kIntraAll     -- every pair, when the gap costs do not fit the int16 path.
//
// Layout of one pass: lane l owns query rows [p*256 + 8l, p*256 + 8l + 8) in registers.  At
// step t lane l updates column j = t - l (an anti-diagonal wavefront across the warp); the
// bottom row of lane l (H - Goe and F) reaches lane l + 1 through __shfl_up_sync one step
// later.  Lane 0 reads the previous pass's bottom row from a per-warp global buffer (one
// coalesced 32-column block at a time, distributed by shuffles) and lane 31 writes the
// pass's bottom row back in place.  The 256 rows of the query profile that a pass needs are
// staged in the warp's own slice of shared memory.  Same cell update as the inter-task
// kernel (Eqs. sw2-sw4 with the profile biased by Goe), on int32 DPX operations.
#include "swgb_device.cuh"

namespace swgb {

namespace {

constexpr int kTI = 8;                       // query rows per lane
constexpr int kRowsPerPass = kTI * kWarp;    // 256 == kQpRows
constexpr int kIW = 4;                       // warps per block
constexpr int kIBlock = kIW * kWarp;

static_assert(kRowsPerPass == kQpRows, "intra pass must match the profile padding");

struct Pair {
    int q;
    int seq;
};

// Claims the next (query, subject) pair of the long or all-pairs work sources.
__device__ __forceinline__ bool next_enumerated(const IntraParams& p, int lane, Pair& out) {
    if (p.mode == kIntraGroups) {   // layout slots, longest groups first, fillers skipped
        const int64_t nslots = p.slot_end - p.slot_begin;
        const unsigned long long total =
            static_cast<unsigned long long>(nslots) * static_cast<unsigned long long>(p.num_queries);
        for (;;) {
            unsigned long long k = 0;
            if (lane == 0) k = atomicAdd(&p.ctrl->next_groups, 1ull);
            k = __shfl_sync(0xffffffffu, k, 0);
            if (k >= total) return false;
            const int64_t si = static_cast<int64_t>(k / static_cast<unsigned long long>(p.num_queries));
            const int qi = static_cast<int>(static_cast<int64_t>(k) - si * p.num_queries);
            const int id = p.perm[p.slot_end - 1 - si];
            if (id < 0) continue;
            out.q = p.query_order[qi];
            out.seq = id;
            return true;
        }
    }
    const bool tick = p.mode == kIntraTickLong;
    const int64_t nsub = (p.mode == kIntraLong || tick) ? p.num_long : p.num_seqs;
    const int64_t nq = tick ? p.tick->n_long : p.num_queries;
    const unsigned long long total =
        static_cast<unsigned long long>(nsub) * static_cast<unsigned long long>(nq);
    unsigned long long k = 0;
    if (lane == 0) k = atomicAdd(&p.ctrl->next_intra, 1ull);
    k = __shfl_sync(0xffffffffu, k, 0);
    if (k >= total) return false;
    const int64_t si = static_cast<int64_t>(k / static_cast<unsigned long long>(nq));
    const int qi = static_cast<int>(static_cast<int64_t>(k) - si * nq);
    out.q = tick ? p.tick->long_slot[qi] : p.query_order[qi];
    out.seq = (p.mode == kIntraLong || tick) ? p.long_ids[si] : static_cast<int>(si);
    return true;
}

__device__ __forceinline__ void load_profile(const QueryDesc& qd, int pass, int alphabet1,
                                             int16_t* s_qp, int lane) {
    constexpr int kVecPerRow = kRowsPerPass / 8;
    const int stride = kRowsPerPass + kQpPad;
    for (int v = lane; v < alphabet1 * kVecPerRow; v += kWarp) {
        const int d = v / kVecPerRow;
        const int o = (v - d * kVecPerRow) * 8;
        *reinterpret_cast<uint4*>(s_qp + d * stride + o) = *reinterpret_cast<const uint4*>(
            qd.qp + static_cast<int64_t>(d) * qd.m_pad + pass * kRowsPerPass + o);
    }
}

template <bool kAdd>
__device__ int align_pair_t(const IntraParams& p, const Pair& pr, int16_t* s_qp, int2* spill,
                            int lane) {
    const QueryDesc qd = p.queries[pr.q];
    const int m = qd.m;
    const int64_t off = p.plain_off[pr.seq];
    const int n = static_cast<int>(p.plain_off[pr.seq + 1] - off);
    if (m == 0 || n == 0) return 0;
    const uint8_t* subj = p.plain + off;
    const int goe = p.gaps.goe, ge = p.gaps.ge, gep = p.gaps.gep;
    const int stride = kRowsPerPass + kQpPad;
    const int passes = (m + kRowsPerPass - 1) / kRowsPerPass;
    int best = 0;
    for (int pass = 0; pass < passes; ++pass) {
        const bool first = pass == 0, last = pass == passes - 1;
        __syncwarp();
        load_profile(qd, pass, p.alphabet1, s_qp, lane);
        __syncwarp();
        int Hm[kTI], E[kTI];
#pragma unroll
        for (int r = 0; r < kTI; ++r) {
            Hm[r] = -goe;
            E[r] = -gep;
        }
        int hm_prev = -goe;        // (H - Goe)(r0 - 1, j - 1) for this lane's first row
        int out_hm = -goe, out_f = -gep;
        // lane 0's upstream values for columns [blk, blk + 32), one per lane
        int2 sp_cur = make_int2(-goe, -gep), sp_next = make_int2(-goe, -gep);
        if (!first) {
            if (lane < n) sp_cur = spill[lane];
            if (32 + lane < n) sp_next = spill[32 + lane];
        }
        const int steps = n + kWarp - 1;
        for (int t = 0; t < steps; ++t) {
            if ((t & 31) == 0 && t > 0) {
                sp_cur = sp_next;
                if (!first && t + 32 + lane < n) sp_next = spill[t + 32 + lane];
            }
            const int up_hm = __shfl_up_sync(0xffffffffu, out_hm, 1);
            const int up_f = __shfl_up_sync(0xffffffffu, out_f, 1);
            const int src = t & 31;
            const int l0_hm = __shfl_sync(0xffffffffu, sp_cur.x, src);
            const int l0_f = __shfl_sync(0xffffffffu, sp_cur.y, src);
            const int j = t - lane;
            if (j >= 0 && j < n) {
                const int in_hm = lane == 0 ? l0_hm : up_hm;   // (H - Goe)(r0 - 1, j)
                int F = lane == 0 ? l0_f : up_f;               // F(r0, j)
                int d = hm_prev;
                hm_prev = in_hm;
                const int16_t* prow = s_qp + subj[j] * stride + lane * kTI;
                const uint4 sv = *reinterpret_cast<const uint4*>(prow);
                const unsigned w[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int r = 2 * h;
                    int s0 = static_cast<int>(static_cast<short>(w[h] & 0xFFFFu));
                    int s1 = static_cast<int>(w[h]) >> 16;
                    if (kAdd) {
                        s0 += p.qp_add;
                        s1 += p.qp_add;
                    }
                    const int x0 = __viaddmax_s32_relu(d, s0, E[r]);
                    const int xm0 = x0 - goe;
                    d = Hm[r];
                    Hm[r] = __viaddmax_s32(F, -goe, xm0);
                    E[r] = __viaddmax_s32(E[r], -ge, Hm[r]);
                    F = __viaddmax_s32(F, -gep, xm0);
                    const int x1 = __viaddmax_s32_relu(d, s1, E[r + 1]);
                    const int xm1 = x1 - goe;
                    d = Hm[r + 1];
                    Hm[r + 1] = __viaddmax_s32(F, -goe, xm1);
                    E[r + 1] = __viaddmax_s32(E[r + 1], -ge, Hm[r + 1]);
                    F = __viaddmax_s32(F, -gep, xm1);
                    best = __vimax3_s32(best, x0, x1);
                }
                out_hm = Hm[kTI - 1];
                out_f = F;
                if (lane == kWarp - 1 && !last) spill[j] = make_int2(out_hm, out_f);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    return best;
}

__device__ __forceinline__ int align_pair(const IntraParams& p, const Pair& pr, int16_t* s_qp,
                                          int2* spill, int lane) {
    return p.qp_add == 0 ? align_pair_t<false>(p, pr, s_qp, spill, lane)
                         : align_pair_t<true>(p, pr, s_qp, spill, lane);
}

__global__ void __launch_bounds__(kIBlock) k_intra_i32(const IntraParams p) {
    extern __shared__ __align__(16) int16_t s_all[];
    const int lane = threadIdx.x & (kWarp - 1);
    const int warp = threadIdx.x >> 5;
    int16_t* s_qp = s_all + static_cast<size_t>(warp) * p.alphabet1 * (kRowsPerPass + kQpPad);
    int2* spill = p.spill + (static_cast<int64_t>(blockIdx.x) * kIW + warp) * p.spill_stride;
    Pair pr;
    if (p.mode != kIntraRescore) {
        while (next_enumerated(p, lane, pr)) {
            const int v = align_pair(p, pr, s_qp, spill, lane);
            if (lane == 0) p.queries[pr.q].scores[pr.seq] = v;
            __syncwarp();
        }
        return;
    }
    // Launched as a programmatic dependent, the kernel may start while the kernel before it
    // still runs: wait here for its completion and memory (no effect after an ordinary launch).
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // Saturated lanes: the list first.  (Usually empty: then no warp touches the work counter,
    // whose atomics from every warp of the grid would otherwise serialise for microseconds.)
    const unsigned count = *reinterpret_cast<volatile unsigned*>(&p.ctrl->flag_count);
    const unsigned listed = count < p.flag_cap ? count : p.flag_cap;
    for (; listed > 0;) {
        unsigned k = 0;
        if (lane == 0) k = atomicAdd(&p.ctrl->next_rescore, 1u);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= listed) break;
        pr.q = p.flags[k].query;
        pr.seq = p.flags[k].seq;
        const int v = align_pair(p, pr, s_qp, spill, lane);
        if (lane == 0) p.queries[pr.q].scores[pr.seq] = v;
        __syncwarp();
    }
    if (count <= p.flag_cap) return;
    // The list overflowed: sweep every output row for the -1 marker the inter-task kernel
    // leaves on saturated lanes.  A pair seen by both phases is computed twice with the same
    // result.
    const int64_t per_q = (p.num_seqs + kWarp - 1) / kWarp;
    const unsigned long long blocks =
        static_cast<unsigned long long>(per_q) * static_cast<unsigned long long>(p.num_queries);
    for (;;) {
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(&p.ctrl->sweep_next, 1ull);
        b = __shfl_sync(0xffffffffu, b, 0);
        if (b >= blocks) break;
        const int qs = static_cast<int>(b / static_cast<unsigned long long>(per_q));
        const int64_t s0 = (static_cast<int64_t>(b) - static_cast<int64_t>(qs) * per_q) * kWarp;
        int32_t* row = p.queries[qs].scores;
        const bool marked = s0 + lane < p.num_seqs && row[s0 + lane] == -1;
        unsigned mask = __ballot_sync(0xffffffffu, marked);
        while (mask) {
            const int first = __ffs(mask) - 1;
            mask &= mask - 1;
            pr.q = qs;
            pr.seq = static_cast<int>(s0 + first);
            const int v = align_pair(p, pr, s_qp, spill, lane);
            if (lane == 0) row[pr.seq] = v;
            __syncwarp();
        }
    }
}

}  // namespace

int intra_block_threads() { return kIBlock; }
int intra_rows_per_pass() { return kRowsPerPass; }

size_t intra_smem_bytes(int alphabet1) {
    return static_cast<size_t>(kIW) * alphabet1 * (kRowsPerPass + kQpPad) * sizeof(int16_t);
}

int intra_occupancy(int alphabet1) {
    int n = 0;
    const size_t smem = intra_smem_bytes(alphabet1);
    cudaFuncSetAttribute(k_intra_i32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_intra_i32, kIBlock, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_intra(const IntraParams& p, int grid, int block, cudaStream_t st) {
    const size_t smem = intra_smem_bytes(p.alphabet1);
    cudaError_t e = cudaFuncSetAttribute(k_intra_i32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    k_intra_i32<<<grid, block, smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_intra_dependent(const IntraParams& p, int grid, int block, cudaStream_t st) {
    const size_t smem = intra_smem_bytes(p.alphabet1);
    cudaError_t e = cudaFuncSetAttribute(k_intra_i32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(grid));
    cfg.blockDim = dim3(static_cast<unsigned>(block));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_intra_i32, p);
}

}  // namespace swgb
