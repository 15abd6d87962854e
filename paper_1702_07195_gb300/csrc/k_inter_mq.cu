// Multi-query inter-task kernel: the two int16 lanes of a register are two queries against
// the same database sequence.
//
// Same recurrence and saturation rule as k_inter_i16x2 (Eqs. sw2-sw4; Section 4.2), same
// strips ("vertical blocks", Section 4.1) and the same interleaved database layout, but the
// lanes are laid out differently: a thread aligns ONE subject, and lane a / lane b run two
// streams of query strips (every query of the batch sits, strip by strip, in one of the two
// streams).  Both lanes then look up the same subject residue, so one 16-byte shared-memory load
// of the paired profile (pp[d][row] = (S'_a, S'_b)) yields four packed score pairs ready for
// the DPX update: the byte permute of the two-subject kernel disappears (5.5 instead of 6.5 ALU
// operations per cell pair).  A warp item is one slot parity of one 64-sequence group (32
// subjects) against every query; at a query boundary a lane restarts from the zero boundary
// (Section 2) and emits its score.
#include "swgb_device.cuh"

namespace swgb {

namespace {

struct PackedMq {
    unsigned ngoe, nge, ngep, floor;
};

__device__ __forceinline__ unsigned pack2mq(int v) {
    return (static_cast<unsigned>(v) & 0xFFFFu) * 0x00010001u;
}

// One column of one strip for both lanes (S' pairs read straight from the paired profile).
// Rows go in sub-blocks of four: first X (and X - Goe) of the four rows from the previous
// column's state -- row r's diagonal is row r - 1's H - Goe of the previous column, still in
// Hm[r - 1] (for the first row of a sub-block it was saved in d before the previous sub-block
// overwrote it) -- then the F chain down the sub-block, which overwrites Hm and E in place: the
// operations of a row-by-row update of Eqs. sw2-sw4, with the four X independent of F.
template <int kT>
__device__ __forceinline__ void column_mq(unsigned (&Hm)[kT], unsigned (&E)[kT], unsigned& f,
                                          unsigned d, const uint32_t* prow, const PackedMq& k,
                                          unsigned& best) {
    const uint4* p4 = reinterpret_cast<const uint4*>(prow);
    unsigned F = f;
#pragma unroll
    for (int r4 = 0; r4 < kT; r4 += 4) {
        const uint4 sv = p4[r4 >> 2];
        const unsigned x0 = __viaddmax_s16x2_relu(d, sv.x, E[r4]);
        const unsigned x1 = __viaddmax_s16x2_relu(Hm[r4], sv.y, E[r4 + 1]);
        const unsigned x2 = __viaddmax_s16x2_relu(Hm[r4 + 1], sv.z, E[r4 + 2]);
        const unsigned x3 = __viaddmax_s16x2_relu(Hm[r4 + 2], sv.w, E[r4 + 3]);
        const unsigned xm[4] = {__viaddmax_s16x2(x0, k.ngoe, k.floor), __viaddmax_s16x2(x1, k.ngoe, k.floor),
                                __viaddmax_s16x2(x2, k.ngoe, k.floor), __viaddmax_s16x2(x3, k.ngoe, k.floor)};
        best = __vimax3_s16x2(best, x0, x1);
        best = __vimax3_s16x2(best, x2, x3);
        d = Hm[r4 + 3];   // old H - Goe of the sub-block's last row: the next sub-block's diagonal
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            Hm[r4 + i] = __viaddmax_s16x2(F, k.ngoe, xm[i]);
            E[r4 + i] = __viaddmax_s16x2(E[r4 + i], k.nge, Hm[r4 + i]);
            F = __viaddmax_s16x2(F, k.ngep, xm[i]);
        }
    }
    f = F;
}

// One strip pair over all L columns of the thread's subject (slot parity `h` of the group).
// `keep` masks the boundary halves to read (0 for a lane that starts a query here).
template <int kT>
__device__ __forceinline__ void strip_mq(const uint4* __restrict__ res, int L, int h, uint4* bnd,
                                         const uint32_t* pp_strip, int pstride, unsigned keep,
                                         bool read, bool write, const PackedMq& k,
                                         unsigned& best, int lane) {
    unsigned Hm[kT], E[kT];
#pragma unroll
    for (int r = 0; r < kT; ++r) {
        Hm[r] = k.ngoe;
        E[r] = k.ngep;
    }
    const unsigned init_f = k.ngep, init_hm = k.ngoe;
    const uint4 init = make_uint4(init_hm, init_f, init_hm, init_f);
    unsigned hm_prev = k.ngoe;
    uint4 w_next = res[lane];
    // boundary records alternate between two registers sets (no copy per record)
    uint4 b_a = read ? bnd[lane] : init, b_b = init;
    // Columns j, j + 1: residues are bytes h and 2 + h of word wq; b holds the previous strip's
    // record of these columns, b_pref receives the next record.
    auto two_columns = [&](const unsigned wq, uint4 b, uint4& b_pref, const int j) {
        if (read && j + 2 < L) b_pref = bnd[((j >> 1) + 1) * kWarp + lane];
        if (keep != 0xFFFFFFFFu) {
            b.x = (b.x & keep) | (init.x & ~keep);
            b.y = (b.y & keep) | (init.y & ~keep);
            b.z = (b.z & keep) | (init.z & ~keep);
            b.w = (b.w & keep) | (init.w & ~keep);
        }
        const unsigned c0 = __byte_perm(wq, 0u, 0x4440u + h);
        const unsigned c1 = __byte_perm(wq, 0u, 0x4442u + h);
        unsigned f0 = b.y;
        column_mq<kT>(Hm, E, f0, hm_prev, pp_strip + c0 * pstride, k, best);
        const unsigned out_hm0 = Hm[kT - 1];
        unsigned f1 = b.w;
        column_mq<kT>(Hm, E, f1, b.x, pp_strip + c1 * pstride, k, best);
        hm_prev = b.z;
        if (write) bnd[(j >> 1) * kWarp + lane] = make_uint4(out_hm0, f0, Hm[kT - 1], f1);
    };
    // L (even) columns: whole 8-column chunks, then 1-3 column pairs of the last chunk (the
    // storage is padded to 8 columns; the sweep stops at the longest member)
    for (int jc = 0; jc < L; jc += 8) {
        const uint4 w = w_next;
        if (jc + 8 < L) w_next = res[((jc >> 3) + 1) * kWarp + lane];
        if (jc + 8 <= L) {
#pragma unroll 1
            for (int q2 = 0; q2 < 2; ++q2) {
                two_columns(q2 ? w.z : w.x, b_a, b_b, jc + 4 * q2);
                two_columns(q2 ? w.w : w.y, b_b, b_a, jc + 4 * q2 + 2);
            }
        } else {
            const int np = (L - jc) >> 1;
            two_columns(w.x, b_a, b_b, jc);
            if (np > 1) two_columns(w.y, b_b, b_a, jc + 2);
            if (np > 2) two_columns(w.z, b_a, b_b, jc + 4);
        }
    }
}

__device__ __forceinline__ void emit_mq(const InterMqParams& p, int q, int id, int v) {
    if (id < 0 || q < 0) return;
    int32_t* scores = p.queries[q].scores;
    if (v >= p.thresh) {
        scores[id] = -1;
        const unsigned slot = atomicAdd(&p.ctrl->flag_count, 1u);
        if (slot < p.flag_cap) p.flags[slot] = FlagEntry{q, id};
    } else {
        scores[id] = v;
    }
}

template <int kT, int kW, int kMinBlocks>
__global__ void __launch_bounds__(kW * kWarp, kMinBlocks) k_inter_mq_i16x2(const InterMqParams p) {
    constexpr int kBlock = kW * kWarp;
    constexpr int kChunk = kQpRows;            // profile rows staged per chunk
    constexpr int kStepsPerChunk = kChunk / kT;
    extern __shared__ __align__(16) uint32_t s_pp[];
    __shared__ int s_item;
    const int lane = threadIdx.x & (kWarp - 1);
    const int warp = threadIdx.x >> 5;
    const int pstride = kChunk + 4;            // uint32 per shared-memory profile row
    uint4* bnd = p.bnd + (static_cast<int64_t>(blockIdx.x) * kW + warp) * p.bnd_stride;
    PackedMq k;
    k.ngoe = pack2mq(-p.gaps.goe);
    k.nge = pack2mq(-p.gaps.ge);
    k.ngep = pack2mq(-p.gaps.gep);
    k.floor = 0x80008000u;
    const int num_steps = p.tick ? p.tick->mq_steps : p.num_steps;
    const int hg_begin = p.tick ? p.tick->hg_begin : 0;
    const int hg_end = p.tick ? p.tick->hg_end : p.num_half_groups;
    const int nb = p.tick ? p.tick->n_batches : 1;
    const int n_hb = (hg_end - hg_begin + kW - 1) / kW;   // blocks of kW half-groups
    const int num_items = n_hb * nb;

    for (;;) {
        if (threadIdx.x == 0) s_item = static_cast<int>(atomicAdd(&p.ctrl->next_inter, 1u));
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= num_items) break;
        // longest groups first (half-groups are in ascending length order), batches interleaved
        const int b = it % nb;
        const int hg = hg_begin + (n_hb - 1 - it / nb) * kW + warp;
        const bool active = hg < hg_end;
        const int s_begin = p.tick ? p.tick->batch_step_off[b] : 0;
        const int s_end = p.tick ? p.tick->batch_step_off[b + 1] : num_steps;
        const int g = hg >> 1, h = hg & 1;
        const int L = active ? p.group_cols[g] : 0;
        const uint4* res =
            active ? reinterpret_cast<const uint4*>(p.inter + p.group_off[g]) : nullptr;
        const int id = active ? p.perm[g * kGroupSeqs + 2 * lane + h] : -1;
        unsigned best = 0;
        for (int k0 = s_begin; k0 < s_end; k0 += kStepsPerChunk) {
            __syncthreads();
            constexpr int kVecPerRow = kChunk / 4;
            const int64_t row0 = static_cast<int64_t>(k0) * kT;
            for (int v = threadIdx.x; v < p.alphabet1 * kVecPerRow; v += kBlock) {
                const int d = v / kVecPerRow;
                const int o = (v - d * kVecPerRow) * 4;
                *reinterpret_cast<uint4*>(s_pp + d * pstride + o) =
                    *reinterpret_cast<const uint4*>(p.pp + static_cast<int64_t>(d) * p.rows_pad + row0 + o);
            }
            __syncthreads();
            if (!active || L == 0) continue;
            const int k_end = min(s_end, k0 + kStepsPerChunk);
            for (int ks = k0; ks < k_end; ++ks) {
                const MqStep st = p.steps[ks];
                const bool fa = st.flags & kMqFirstA, fb = st.flags & kMqFirstB;
                const unsigned keep = (fa ? 0u : 0x0000FFFFu) | (fb ? 0u : 0xFFFF0000u);
                strip_mq<kT>(res, L, h, bnd, s_pp + (ks - k0) * kT, pstride, keep,
                             keep != 0u, ks + 1 < s_end, k, best, lane);
                if (st.flags & kMqLastA) {
                    emit_mq(p, st.qa, id, static_cast<int>(static_cast<short>(best & 0xFFFFu)));
                    best &= 0xFFFF0000u;
                }
                if (st.flags & kMqLastB) {
                    emit_mq(p, st.qb, id, static_cast<int>(static_cast<short>(best >> 16)));
                    best &= 0x0000FFFFu;
                }
            }
        }
    }
}

struct MqVariant {
    int T, W;
    const void* fn;
};

const MqVariant kMqVariants[] = {
    {32, 4, reinterpret_cast<const void*>(&k_inter_mq_i16x2<32, 4, 3>)},
    {64, 4, reinterpret_cast<const void*>(&k_inter_mq_i16x2<64, 4, 2>)},
    {32, 8, reinterpret_cast<const void*>(&k_inter_mq_i16x2<32, 8, 2>)},
    {64, 8, reinterpret_cast<const void*>(&k_inter_mq_i16x2<64, 8, 1>)},
};
constexpr int kNumMq = sizeof(kMqVariants) / sizeof(kMqVariants[0]);

// Paired profile: pp[d * rows_pad + k*T + r] = (S'(qa, sa*T + r, d), S'(qb, sb*T + r, d)) with
// S' = SM + bias, and 0 + bias for the dummy code, rows past a query's end and absent lanes.
__global__ void k_build_pp(const uint8_t* __restrict__ queries, const int64_t* __restrict__ qoff,
                           const int32_t* __restrict__ qlen, const MqStep* __restrict__ steps,
                           int32_t num_steps_arg, const TickDesc* __restrict__ tick, int32_t T,
                           const int8_t* __restrict__ matrix, int32_t A, int32_t bias,
                           uint32_t* __restrict__ pp, int64_t rows_pad, Control* ctrl) {
    const int d = blockIdx.y;
    const int64_t row = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (row >= rows_pad) return;
    const int32_t num_steps = tick ? tick->mq_steps : num_steps_arg;
    const int64_t ks = row / T;
    const int r = static_cast<int>(row - ks * T);
    int sa = 0, sb = 0;
    if (ks < num_steps) {
        const MqStep st = steps[ks];
        const int qs[2] = {st.qa, st.qb};
        const int strips[2] = {st.sa, st.sb};
        int out[2] = {0, 0};
        for (int l = 0; l < 2; ++l) {
            const int q = qs[l];
            if (q < 0 || d >= A) continue;
            const int64_t q0 = qoff[q];
            const int64_t m = qlen ? qlen[q] : qoff[q + 1] - q0;
            const int64_t i = static_cast<int64_t>(strips[l]) * T + r;
            if (i >= m) continue;
            const int code = queries[q0 + i];
            if (code < A)
                out[l] = matrix[code * A + d];
            else
                atomicOr(&ctrl->status, 1u);
        }
        sa = out[0];
        sb = out[1];
    }
    pp[static_cast<int64_t>(d) * rows_pad + row] =
        (static_cast<unsigned>(sa + bias) & 0xFFFFu) | (static_cast<unsigned>(sb + bias) << 16);
}

template <int T, int W, int MB>
void launch_mq_variant(const InterMqParams& p, int grid, size_t smem, cudaStream_t st) {
    k_inter_mq_i16x2<T, W, MB><<<grid, W * kWarp, smem, st>>>(p);
}

}  // namespace

int inter_mq_num_variants() { return kNumMq; }
int inter_mq_variant_rows(int v) { return kMqVariants[v].T; }
int inter_mq_variant_warps(int v) { return kMqVariants[v].W; }

size_t inter_mq_smem_bytes(int alphabet1) {
    return static_cast<size_t>(alphabet1) * (kQpRows + 4) * sizeof(uint32_t);
}

int inter_mq_occupancy(int variant, int alphabet1) {
    if (variant < 0 || variant >= kNumMq) return 0;
    int n = 0;
    const size_t smem = inter_mq_smem_bytes(alphabet1);
    const void* fn = kMqVariants[variant].fn;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kMqVariants[variant].W * kWarp,
                                                      smem) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_inter_mq(const InterMqParams& p, int variant, int grid, cudaStream_t st) {
    if (variant < 0 || variant >= kNumMq) return cudaErrorInvalidValue;
    const size_t smem = inter_mq_smem_bytes(p.alphabet1);
    cudaError_t e = cudaFuncSetAttribute(kMqVariants[variant].fn,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    switch (variant) {
        case 0: launch_mq_variant<32, 4, 3>(p, grid, smem, st); break;
        case 1: launch_mq_variant<64, 4, 2>(p, grid, smem, st); break;
        case 2: launch_mq_variant<32, 8, 2>(p, grid, smem, st); break;
        default: launch_mq_variant<64, 8, 1>(p, grid, smem, st); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_build_pp(const uint8_t* d_queries, const int64_t* d_qoff, const int32_t* d_qlen,
                            const MqStep* d_steps, int32_t num_steps, const TickDesc* tick,
                            int32_t rows_per_strip, const int8_t* d_matrix, int32_t A,
                            int32_t bias, uint32_t* d_pp, int64_t rows_pad, Control* ctrl,
                            cudaStream_t st) {
    const int threads = 256;
    dim3 grid(static_cast<unsigned>((rows_pad + threads - 1) / threads), static_cast<unsigned>(A + 1));
    k_build_pp<<<grid, threads, 0, st>>>(d_queries, d_qoff, d_qlen, d_steps, num_steps, tick,
                                         rows_per_strip, d_matrix, A, bias, d_pp, rows_pad, ctrl);
    return cudaGetLastError();
}

}  // namespace swgb
