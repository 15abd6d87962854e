// Intra-task Smith-Waterman/Gotoh wavefront on packed int16x2 lanes.
//
// The int32 intra-task kernels (k_intra_i32, k_intra_block_i32) give one warp one (query,
// subject) pair: lane l owns kTB query rows of a pass and updates column t - l at step t, the
// bottom row of each lane reaching the next lane by __shfl_up_sync (the intra-task scheme of
// Section 1, on Eqs. sw2-sw4 of Section 2).  This kernel runs the same wavefront with the
// DPX int16x2 operations of the inter-task kernels, two alignments per register, and therefore
// two cells per lane-operation:
//
//  two-query mode (k_wave_mq_i16x2): a warp aligns ONE subject against two streams of query
//  passes, pass k of stream a in the low halves and pass k of stream b in the high halves of
//  its registers.  A stream chains its queries at lane granularity (a query of m rows takes
//  ceil(m / kTB) lanes, WavePass), so a pass wastes rows only at the end of each query's last
//  lane.  Both halves read the same subject residue, so one 16-byte load of the paired profile
//  pp[d][row] = (S'_a, S'_b) gives four packed score pairs: 5.5 DPX operations per cell pair,
//  the inter-task kernels' minimum.  A lane that holds row 0 of a query takes the zero
//  boundary as its row above (instead of the lane above, or the previous pass); after each
//  pass the lanes' bests are reduced per query and merged with the query's earlier passes,
//  and a query's score is emitted after the pass of its last row.
//
//  two-subject mode (k_wave_ss_i16x2): a search with one query; a warp aligns the query
//  against the two subjects in slots 2t and 2t + 1 of an interleaved 64-sequence group, one in
//  each half.  The group layout puts the two subjects' residues of a column in adjacent bytes
//  (one 16-bit load per step), and the two score rows come from the query profile: the slice
//  of a pass holds, per residue and lane, the lane's rows as int16 pairs (rows 2w, 2w + 1 in
//  word w), and a byte permute of the two residues' words gives each row's packed pair
//  (6.5 operations per cell pair instead of 5.5).  Beyond a subject's end its half reads the
//  dummy code, whose score 0 leaves its best unchanged.  This mode serves the groups that a
//  small database routes off the inter-task kernel (one warp per 64 subjects cannot fill the
//  GPU there).
//
// Saturation (Section 4.2): every intermediate lies in [-2 Goe - Ge, best + max SM] until the
// running best of a half reaches 32767 - max SM, so an alignment whose best stays below that
// threshold is exact; one that reaches it is written as -1 and listed for the int32 rescore,
// like the inter-task kernels' lanes.  The pass-boundary row (H - Goe, F) of each column goes
// through a per-warp global buffer as one int2 of packed pairs, written by lane 31 and read by
// lane 0 of the next pass, 32 columns at a time.
#include <algorithm>
#include <type_traits>

#include "slice_layout.cuh"
#include "swgb_device.cuh"

namespace swgb {

namespace {

constexpr int kWaveBW = 8;   // warps per block: the subjects that share one profile slice

struct PackedGaps {
    unsigned ngoe, nge, ngep, floor;
};

__device__ __forceinline__ unsigned pack2(int v) {
    return (static_cast<unsigned>(v) & 0xFFFFu) * 0x00010001u;
}

// One column step of a lane's kTB rows on both halves.  Rows go in sub-blocks of up to four:
// first X (and X - Goe) of the sub-block's rows from the previous column's state -- row r's
// diagonal is row r - 1's H - Goe of the previous column, still in Hm[r - 1] (for the first row
// of a sub-block it was saved before the previous sub-block overwrote it) -- then the F chain
// down the sub-block, which overwrites Hm and E in place.  The same operations as a row-by-row
// update of Eqs. sw2-sw4, without a register rotation per row.
// `score(rb, sc)` fills sc[0..3] with the packed scores S' of rows rb..rb+3.
template <int kTB, class ScoreFn>
__device__ __forceinline__ void column2(unsigned (&Hm)[kTB], unsigned (&E)[kTB], unsigned& F,
                                        const unsigned d, ScoreFn score, const PackedGaps& k,
                                        unsigned& best) {
    unsigned diag = d;
#pragma unroll
    for (int rb = 0; rb < kTB; rb += 4) {
        constexpr int kSub = 4;
        unsigned xm[kSub], sc[kSub];
        score(rb, sc);
#pragma unroll
        for (int i = 0; i < kSub; i += 2) {
            const int r = rb + i;
            if (r >= kTB) break;
            const unsigned xa = __viaddmax_s16x2_relu(i == 0 ? diag : Hm[r - 1], sc[i], E[r]);
            xm[i] = __viaddmax_s16x2(xa, k.ngoe, k.floor);
            if (r + 1 < kTB) {
                const unsigned xb = __viaddmax_s16x2_relu(Hm[r], sc[i + 1], E[r + 1]);
                xm[i + 1] = __viaddmax_s16x2(xb, k.ngoe, k.floor);
                best = __vimax3_s16x2(best, xa, xb);
            } else {
                best = __vmaxs2(best, xa);
            }
        }
        if (rb + kSub < kTB) diag = Hm[rb + kSub - 1];   // old H - Goe: diagonal of the next row
#pragma unroll
        for (int i = 0; i < kSub; ++i) {
            const int r = rb + i;
            if (r >= kTB) break;
            Hm[r] = __viaddmax_s16x2(F, k.ngoe, xm[i]);   // H - Goe = max(F, X) - Goe
            E[r] = __viaddmax_s16x2(E[r], k.nge, Hm[r]);  // E of the next column
            F = __viaddmax_s16x2(F, k.ngep, xm[i]);       // F of the next row
        }
    }
}

// The same column step with the F recurrence of Eq. sw4 unrolled down the lane's rows:
// F_r = max(F_in - r Ge', Y_r), Y_r = max over i < r of (X_i - Goe - (r - 1 - i) Ge'), Ge' =
// min(Ge, Goe).  Every F_r is then one operation from the F that arrives from the lane above
// (instead of r), which shortens the step's dependency chain -- what bounds a wavefront running
// alone on its SM sub-partition -- at the cost of kTB - 1 more operations per step (the Y
// chain).  ngep_r[i] holds -(i + 1) Ge' in both halves; the caller checks that
// Goe + kTB Ge' stays inside the int16 range, so no intermediate wraps.
template <int kTB, class ScoreFn>
__device__ __forceinline__ void column2_prefix(unsigned (&Hm)[kTB], unsigned (&E)[kTB], unsigned& F,
                                               const unsigned d, ScoreFn score,
                                               const PackedGaps& k, const unsigned (&ngep_r)[kTB],
                                               unsigned& best) {
    unsigned xm[kTB];
#pragma unroll
    for (int rb = 0; rb < kTB; rb += 4) {
        unsigned sc[4];
        score(rb, sc);
#pragma unroll
        for (int i = 0; i < 4; i += 2) {
            const int r = rb + i;
            if (r >= kTB) break;
            const unsigned xa = __viaddmax_s16x2_relu(r == 0 ? d : Hm[r - 1], sc[i], E[r]);
            xm[r] = __viaddmax_s16x2(xa, k.ngoe, k.floor);
            if (r + 1 < kTB) {
                const unsigned xb = __viaddmax_s16x2_relu(Hm[r], sc[i + 1], E[r + 1]);
                xm[r + 1] = __viaddmax_s16x2(xb, k.ngoe, k.floor);
                best = __vimax3_s16x2(best, xa, xb);
            } else {
                best = __vmaxs2(best, xa);
            }
        }
    }
    const unsigned f_in = F;
    unsigned y = xm[0];                                   // Y_1
    Hm[0] = __viaddmax_s16x2(f_in, k.ngoe, xm[0]);
    E[0] = __viaddmax_s16x2(E[0], k.nge, Hm[0]);
#pragma unroll
    for (int r = 1; r < kTB; ++r) {
        const unsigned fr = __viaddmax_s16x2(f_in, ngep_r[r - 1], y);   // F_r
        Hm[r] = __viaddmax_s16x2(fr, k.ngoe, xm[r]);
        E[r] = __viaddmax_s16x2(E[r], k.nge, Hm[r]);
        y = __viaddmax_s16x2(y, k.ngep, xm[r]);                          // Y_{r+1}
    }
    F = __viaddmax_s16x2(f_in, ngep_r[kTB - 1], y);                     // F of the row below
}

__device__ __forceinline__ void emit_score(const WaveParams& p, int q, int id, int v) {
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

__device__ __forceinline__ uint2 mask_boundary(uint2 v, unsigned keep, unsigned init_hm,
                                               unsigned init_f) {
    v.x = (v.x & keep) | (init_hm & ~keep);
    v.y = (v.y & keep) | (init_f & ~keep);
    return v;
}

// kTB query rows per lane (passes of 32 * kTB rows), kWaveBW warps per block: block item i
// takes subjects [i * kWaveBW, (i + 1) * kWaveBW) of the list (longest first), one per warp,
// and runs every pass of the two-stream pass list over them.
template <int kTB>
__global__ void __launch_bounds__(kWaveBW * kWarp, (kTB >= 12 ? 2 : 3)) k_wave_mq_i16x2(const WaveParams p) {
    constexpr int kBlock = kWaveBW * kWarp;
    constexpr int kRowsB = kTB * kWarp;
    constexpr int kPStride = slice_stride<kTB>();   // words per residue row of the slice
    static_assert(kTB % 4 == 0, "rows per lane: whole 16-byte profile loads");
    extern __shared__ __align__(16) uint32_t s_pp[];   // (A + 1) x kPStride
    __shared__ int s_item;
    __shared__ uint8_t s_ring[kWaveBW][256];           // per-warp residue rings
    __shared__ unsigned s_best[kWaveBW][kWarp];        // per-lane bests of a pass
    __shared__ int s_carry[kWaveBW][2];                // best so far of the query continuing
                                                       // into the next pass, per half
    const int lane = threadIdx.x & (kWarp - 1);
    const int warp = threadIdx.x >> 5;
    const int my_chunk = chunk_offset<kTB>(lane);
    int2* spill = p.spill + (static_cast<int64_t>(blockIdx.x) * kWaveBW + warp) * p.spill_stride;
    uint8_t* ring = s_ring[warp];
    PackedGaps k;
    k.ngoe = pack2(-p.gaps.goe);
    k.nge = pack2(-p.gaps.ge);
    k.ngep = pack2(-p.gaps.gep);
    k.floor = 0x80008000u;
    const unsigned init_hm = k.ngoe, init_f = k.ngep;   // (H - Goe, F) of the zero boundary

    for (;;) {
        __syncthreads();   // s_item of the previous item has been read by every warp
        if (threadIdx.x == 0) s_item = static_cast<int>(atomicAdd(&p.ctrl->next_wave, 1u));
        __syncthreads();
        const int64_t first_subject = static_cast<int64_t>(s_item) * kWaveBW;
        if (first_subject >= p.num_subjects) break;
        const int64_t si = first_subject + warp;
        const int seq = si < p.num_subjects ? p.subjects[si] : -1;
        int n = 0;
        const uint8_t* subj = nullptr;
        if (seq >= 0) {
            const int64_t off = p.plain_off[seq];
            n = static_cast<int>(p.plain_off[seq + 1] - off);
            subj = p.plain + off;
        }
        for (int ks = 0; ks < p.num_passes; ++ks) {
            __syncthreads();   // everyone is done with the previous slice
            const int64_t row0 = static_cast<int64_t>(ks) * kRowsB;
            for (int v = threadIdx.x; v < p.alphabet1 * kRowsB; v += kBlock) {
                const int d = v / kRowsB;
                const int r = v - d * kRowsB;
                s_pp[d * kPStride + chunk_offset<kTB>(r / kTB) + r % kTB] =
                    p.pp[static_cast<int64_t>(d) * p.rows_pad + row0 + r];
            }
            __syncthreads();
            const WavePass& wpass = p.passes[ks];
            const uint32_t first_a = wpass.first[0], first_b = wpass.first[1];
            // a half whose lane 0 starts a query takes the zero boundary instead of the previous
            // pass's row; lanes past 0 that start a query (`inner`) mask the lane above's row
            const unsigned keep = ((first_a & 1u) ? 0u : 0x0000FFFFu) | ((first_b & 1u) ? 0u : 0xFFFF0000u);
            const unsigned my_keep = (((first_a >> lane) & 1u) ? 0u : 0x0000FFFFu) |
                                     (((first_b >> lane) & 1u) ? 0u : 0xFFFF0000u);
            const bool inner_starts = ((first_a | first_b) & ~1u) != 0u;
            const bool write = ks + 1 < p.num_passes;
            unsigned best = 0;
            if (n > 0) {
                unsigned Hm[kTB], E[kTB];
#pragma unroll
                for (int r = 0; r < kTB; ++r) {
                    Hm[r] = init_hm;
                    E[r] = init_f;
                }
                unsigned hm_prev = init_hm;
                unsigned out_hm = init_hm, out_f = init_f;
                uint2 sp_cur = make_uint2(init_hm, init_f), sp_next = sp_cur;
                if (keep != 0u) {
                    if (lane < n)
                        sp_cur = mask_boundary(reinterpret_cast<const uint2*>(spill)[lane], keep,
                                               init_hm, init_f);
                    if (32 + lane < n)
                        sp_next = mask_boundary(reinterpret_cast<const uint2*>(spill)[32 + lane],
                                                keep, init_hm, init_f);
                }
                // Residue ring of this warp: column c at ring[c & 127] and ring[(c & 127) + 128]
                // (a mirror, so that a block of 32 steps reads without wrapping); columns
                // outside [0, n) hold the dummy code.  During the 32-step block starting at tb it
                // holds [tb - 31, tb + 33); at the block's start the lanes write the columns the
                // next block adds, loaded from global memory one block ahead.
                const unsigned dummy = static_cast<unsigned>(p.alphabet1 - 1);
                auto res_at = [&](const int c) -> unsigned {
                    return (c >= 0 && c < n) ? static_cast<unsigned>(subj[c]) : dummy;
                };
                auto ring_put = [&](const int c, const unsigned v) {
                    ring[c & 127] = static_cast<uint8_t>(v);
                    ring[(c & 127) + 128] = static_cast<uint8_t>(v);
                };
                ring_put(lane - 32, dummy);
                ring_put(lane, res_at(lane));
                if (lane == 0) ring_put(32, res_at(32));
                unsigned res_ahead = res_at(33 + lane);   // the next block's columns
                __syncwarp();
                unsigned res_next = ring[(-lane) & 127];   // column -lane: step 0
                const int steps = n + kWarp - 1;
                // Step t: lane l updates column j = t - l (every lane, every step: a column outside
                // the subject is a dummy column, exact as for the two-subject mode).  Lane 0 takes
                // the previous pass's row of column t from lane (t mod 32) of sp_cur (columns
                // [32 k, 32 k + 32) during steps [32 k, 32 k + 32)); when both halves start a
                // query (`on_first`) that row is the zero boundary, a constant.
                // store: 0 = no pass-boundary row (last step), 1 = lane 31 writes (its column is
                // inside the subject for the whole block), 2 = lane 31 writes if inside
                auto step = [&](const int t, const int src, const uint8_t* rnext, auto on_first,
                                auto inner, auto store) {
                    const unsigned up_hm = __shfl_up_sync(0xffffffffu, out_hm, 1);
                    const unsigned up_f = __shfl_up_sync(0xffffffffu, out_f, 1);
                    unsigned l0_hm = init_hm, l0_f = init_f;
                    if constexpr (!decltype(on_first)::value) {
                        l0_hm = __shfl_sync(0xffffffffu, sp_cur.x, src);
                        l0_f = __shfl_sync(0xffffffffu, sp_cur.y, src);
                    }
                    const unsigned res = res_next;
                    res_next = *rnext;                         // column j + 1
                    unsigned F = lane == 0 ? l0_f : up_f;     // F(r0, j)
                    const unsigned d = hm_prev;                // (H - Goe)(r0 - 1, j - 1)
                    hm_prev = lane == 0 ? l0_hm : up_hm;       // (H - Goe)(r0 - 1, j)
                    if constexpr (decltype(inner)::value) {   // row 0 of a query: zero boundary
                        F = (F & my_keep) | (init_f & ~my_keep);
                        hm_prev = (hm_prev & my_keep) | (init_hm & ~my_keep);
                    }
                    const uint4* prow = reinterpret_cast<const uint4*>(s_pp + res * kPStride + my_chunk);
                    column2<kTB>(Hm, E, F, d, [&](const int rb, unsigned (&sc)[4]) {
                        const uint4 sv = prow[rb >> 2];
                        sc[0] = sv.x;
                        sc[1] = sv.y;
                        sc[2] = sv.z;
                        sc[3] = sv.w;
                    }, k, best);
                    out_hm = Hm[kTB - 1];
                    out_f = F;
                    if constexpr (decltype(store)::value == 1) {
                        if (lane == kWarp - 1)
                            spill[t - lane] = make_int2(static_cast<int>(out_hm), static_cast<int>(out_f));
                    } else if constexpr (decltype(store)::value == 2) {
                        const int j = t - lane;
                        if (lane == kWarp - 1 && static_cast<unsigned>(j) < static_cast<unsigned>(n))
                            spill[j] = make_int2(static_cast<int>(out_hm), static_cast<int>(out_f));
                    }
                };
                auto run = [&](auto on_first, auto inner) {
                    for (int tb = 0; tb < steps; tb += kWarp) {
                        if constexpr (!decltype(on_first)::value) {
                            if (tb > 0) {
                                sp_cur = sp_next;
                                if (tb + 32 + lane < n)
                                    sp_next = mask_boundary(
                                        reinterpret_cast<const uint2*>(spill)[tb + 32 + lane],
                                        keep, init_hm, init_f);
                            }
                        }
                        ring_put(tb + 33 + lane, res_ahead);
                        res_ahead = res_at(tb + 65 + lane);
                        __syncwarp();
                        const uint8_t* rbase = ring + ((tb - lane) & 127) + 1;   // column j + 1 at u
                        using NoStore = std::integral_constant<int, 0>;
                        using Store = std::integral_constant<int, 1>;
                        using CheckedStore = std::integral_constant<int, 2>;
                        if (tb + kWarp <= steps) {
                            if (!write) {
#pragma unroll 4
                                for (int u = 0; u < kWarp; ++u) step(tb + u, u, rbase + u, on_first, inner, NoStore{});
                            } else if (tb >= kWarp && tb < n) {
#pragma unroll 4
                                for (int u = 0; u < kWarp; ++u) step(tb + u, u, rbase + u, on_first, inner, Store{});
                            } else {
#pragma unroll 4
                                for (int u = 0; u < kWarp; ++u) step(tb + u, u, rbase + u, on_first, inner, CheckedStore{});
                            }
                        } else {
                            const int ue = steps - tb;
#pragma unroll 1
                            for (int u = 0; u < ue; ++u) step(tb + u, u, rbase + u, on_first, inner, CheckedStore{});
                        }
                    }
                };
                if (keep == 0u) {
                    if (inner_starts)
                        run(std::true_type{}, std::true_type{});
                    else
                        run(std::true_type{}, std::false_type{});
                } else {
                    if (inner_starts)
                        run(std::false_type{}, std::true_type{});
                    else
                        run(std::false_type{}, std::false_type{});
                }
                __syncwarp();   // lane 31's spill writes are visible to the next pass
            }
            // Per half, the lanes of one query are contiguous: the first of them reduces their
            // bests (and, for a query that began in an earlier pass, the carried best) and
            // emits the score if the query ends in this pass, else carries it to the next.
            s_best[warp][lane] = best;
            __syncwarp();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int q = wpass.q[h][lane];
                const bool head = q >= 0 && (lane == 0 || wpass.q[h][lane - 1] != q);
                if (head) {
                    const uint32_t fbits = h == 0 ? first_a : first_b;
                    int v = (lane == 0 && !(fbits & 1u)) ? s_carry[warp][h] : 0;
                    int l2 = lane;
                    for (; l2 < kWarp && wpass.q[h][l2] == q; ++l2) {
                        const unsigned w = s_best[warp][l2];
                        v = max(v, static_cast<int>(static_cast<short>(h == 0 ? (w & 0xFFFFu) : (w >> 16))));
                    }
                    if ((wpass.last[h] >> (l2 - 1)) & 1u) {
                        if (seq >= 0) emit_score(p, q, seq, v);
                    } else {
                        s_carry[warp][h] = v;
                    }
                }
            }
            __syncwarp();
        }
    }
}

// Two-subject mode.  kTB query rows per lane (passes of 32 * kTB rows), kW = ceil(kTB / 2)
// words of int16 row pairs per lane and residue.  The whole query profile (every pass) sits in
// shared memory, staged once per block, and each warp copies the residue pairs of its current
// slot pair into its own shared-memory buffer, so the warps of a block are independent: each
// takes one slot pair at a time from a work counter, with no block-wide synchronisation, and a
// step reads only shared memory (the residues of the next column, then their profile words).
//
// Every step of the wavefront runs on all 32 lanes.  A lane whose column lies before the
// subject (j < 0) or past its end (j >= n) computes a column of the dummy code (score 0) from
// the boundary values: before column 0 that leaves H at 0 and only lowers E and F, which stay
// at or below 0 and reach H only through max(0, ...) (and never below -Goe - Ge); past the end
// every H is bounded by a real cell.  So the scores are exact and no lane branches.
//
// Work: the 32 slot pairs of every group in [group_begin, group_end), numbered longest first.
// The first `long_pairs` of them form a separate queue served in a first phase by the first
// kSsLongWarps warps of blocks [0, long_blocks) while the block's other warps wait at a
// barrier: the wavefronts of the longest subjects set the length of a search on a small
// database, and alone on an SM sub-partition their steps run at the latency of the step's
// dependency chain rather than sharing the sub-partition's issue with other warps.  Then every
// warp serves the remaining pairs, longest first.
constexpr int kSsBW = 16;         // warps per block (one block per SM)
constexpr int kSsBlocksPerSM = 1;
constexpr int kSsLongWarps = 4;   // warps of a long block that run the first phase
constexpr int kResPad = 32;       // dummy columns kept before column 0 in a residue buffer
constexpr int kSsBulkRows = 9;    // rows per lane of the 16-lane bulk wavefronts (144-row passes)
constexpr int kSsBulkLanes = 16;

// kTBL query rows per lane of the 32-lane wavefronts (first phase and the longer bulk pairs);
// kHalf: the bulk's shorter pairs run two 16-lane wavefronts per warp (two slot pairs,
// kSsBulkRows rows per lane).  With 16 lanes a slot pair fills and drains its wavefront in 15
// steps instead of 31, and a 144-row query fits one pass exactly, but a warp's item (two pairs,
// 9 rows per lane and step) lasts longer than a 32-lane one.
template <int kTBL, bool kHalf>
__global__ void __launch_bounds__(kSsBW * kWarp, kSsBlocksPerSM) k_wave_ss_i16x2(const WaveParams p) {
    constexpr int kWL = (kTBL + 1) / 2;
    constexpr int kWB = (kSsBulkRows + 1) / 2;
    extern __shared__ __align__(16) uint32_t s_sl[];   // profiles, then residue buffers
    const int lane = threadIdx.x & (kWarp - 1);
    const int warp = threadIdx.x >> 5;
    const int64_t gwarp = static_cast<int64_t>(blockIdx.x) * kSsBW + warp;
    PackedGaps k;
    k.ngoe = pack2(-p.gaps.goe);
    k.nge = pack2(-p.gaps.ge);
    k.ngep = pack2(-p.gaps.gep);
    k.floor = 0x80008000u;
    const unsigned init_hm = k.ngoe, init_f = k.ngep;
    // a rescore launched as a programmatic dependent may be scheduled now; it waits for this
    // kernel's completion before it reads anything
    asm volatile("griddepcontrol.launch_dependents;");
    const QueryDesc qd = p.queries[p.query];
    const int passes_l = max(1, (qd.m + kWarp * kTBL - 1) / (kWarp * kTBL));
    const int passes_b = kHalf ? max(1, (qd.m + kSsBulkLanes * kSsBulkRows - 1) / (kSsBulkLanes * kSsBulkRows)) : 0;
    const int words_l = p.alphabet1 * slice_stride<kWL>();
    const int words_b = p.alphabet1 * slice_stride<kWB>();
    uint32_t* prof_l = s_sl;
    uint32_t* prof_b = s_sl + passes_l * words_l;
    const int64_t total_pairs = (p.group_end - p.group_begin) * (kGroupSeqs / 2);
    const int64_t long_pairs = min(p.long_pairs, total_pairs);
    const bool long_block = static_cast<int>(blockIdx.x) < p.long_blocks;
    const int bias = p.gaps.goe;   // score 0 of rows past the profile: S' = 0 + Goe
    const uint16_t dummy2 = static_cast<uint16_t>((p.alphabet1 - 1) * 0x0101);
    // residue buffers of this warp (one per wavefront): column c of a pair at index c + kResPad
    const int res_stride = wave_ss_res_stride(p.max_group_len);
    uint16_t* rbuf = reinterpret_cast<uint16_t*>(prof_b + passes_b * words_b) + warp * (kHalf ? 2 : 1) * res_stride;

    // The query profile (Section 4.3), built here from the query and the matrix, for each
    // wavefront shape in use: pass, residue d, lane chunk, word w = rows (2w, 2w + 1) of the
    // lane, each S'(q_i, d) = SM(q_i, d) + Goe; the dummy code and rows past the query score 0
    // (S' = Goe).  A 16-lane profile stores every lane's chunk twice (chunks l and l + 16), so
    // the two wavefronts of a warp read it with the 32-lane bank pattern.  A query residue
    // outside the alphabet sets status bit 0 (reported by the host after the search) and
    // scores 0 here.  The matrix goes to shared memory first, so that building a word costs
    // shared-memory reads only.
    const int A = p.alphabet1 - 1;
    __shared__ int8_t s_mat[kMaxAlphabet * kMaxAlphabet];
    for (int i = threadIdx.x; i < A * A; i += blockDim.x) s_mat[i] = p.matrix[i];
    __syncthreads();
    const uint8_t* qres = p.qres + p.qres_off[p.query];
    auto build = [&](auto tb_c, auto lanes_c, uint32_t* base, const int passes) {
        constexpr int kTB = decltype(tb_c)::value, kL = decltype(lanes_c)::value;
        constexpr int kW = (kTB + 1) / 2;
        constexpr int kStride = slice_stride<kW>();
        const int words = p.alphabet1 * kStride;
        for (int v = threadIdx.x; v < passes * kW * kWarp; v += blockDim.x) {
            const int ps = v / (kW * kWarp);                 // pass, chunk, word of the lane's rows
            const int rem = v - ps * (kW * kWarp);
            const int ln = rem / kW, wi = rem - ln * kW;
            const int r0 = ps * (kL * kTB) + (ln % kL) * kTB + 2 * wi;
            const bool has1 = 2 * wi + 1 < kTB;
            int c0 = r0 < qd.m ? qres[r0] : -1;              // -1: a row past the query
            int c1 = has1 && r0 + 1 < qd.m ? qres[r0 + 1] : -1;
            if (c0 >= A || c1 >= A) {
                atomicOr(&p.ctrl->status, 1u);
                c0 = c0 >= A ? -1 : c0;
                c1 = c1 >= A ? -1 : c1;
            }
            uint32_t* dst = base + ps * words + chunk_offset<kW>(ln) + wi;
            for (int d = 0; d < p.alphabet1; ++d) {
                const int s0 = (c0 >= 0 && d < A) ? s_mat[c0 * A + d] + bias : bias;
                const int s1 = (c1 >= 0 && d < A) ? s_mat[c1 * A + d] + bias : bias;
                dst[d * kStride] = (static_cast<unsigned>(s0) & 0xFFFFu) | (static_cast<unsigned>(s1) << 16);
            }
        }
    };
    build(std::integral_constant<int, kTBL>{}, std::integral_constant<int, kWarp>{}, prof_l, passes_l);
    if constexpr (kHalf)
        build(std::integral_constant<int, kSsBulkRows>{}, std::integral_constant<int, kSsBulkLanes>{},
              prof_b, passes_b);
    // The int16 profile of the int32 rescore (query-major: qp_out[d * qp_mpad + i]), spread
    // over the grid, when no separate kernel builds it.
    if (p.qp_out) {
        const int total = p.alphabet1 * p.qp_mpad;
        for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < total; v += gridDim.x * blockDim.x) {
            const int d = v / p.qp_mpad, i = v - d * p.qp_mpad;
            const int c = (d < A && i < qd.m) ? qres[i] : -1;
            p.qp_out[v] = static_cast<int16_t>((c >= 0 && c < A ? s_mat[c * A + d] : 0) + p.qp_bias);
        }
    }
    __syncthreads();

    // Slot pair pi (0 = the longest): its group, pair index t, subject ids and lengths; an
    // index outside [0, total_pairs) is an empty pair.
    struct PairRef {
        int64_t g;
        int t, id[2], n[2];
    };
    auto pair_ref = [&](const int64_t pi) {
        PairRef r;
        r.g = -1;
        r.t = 0;
        r.id[0] = r.id[1] = -1;
        r.n[0] = r.n[1] = 0;
        if (pi >= 0 && pi < total_pairs) {
            r.g = p.group_end - 1 - pi / (kGroupSeqs / 2);
            r.t = kGroupSeqs / 2 - 1 - static_cast<int>(pi % (kGroupSeqs / 2));
            for (int h = 0; h < 2; ++h) {
                r.id[h] = p.perm[r.g * kGroupSeqs + 2 * r.t + h];
                r.n[h] = r.id[h] >= 0 ? static_cast<int>(p.plain_off[r.id[h] + 1] - p.plain_off[r.id[h]]) : 0;
            }
        }
        return r;
    };
    // Residue pairs of columns [0, n rounded up to 8) from the interleaved group (16 bytes = 8
    // columns per load; past each subject's end the layout holds the dummy code), the dummy pair
    // elsewhere in [-kResPad, n_fill + kWarp + 1).  Uniform trip counts (predicated bodies): the
    // warp stays converged.
    auto stage_residues = [&](const PairRef& r, const int n, const int n_fill, uint16_t* buf) {
        const int chunks = (n + 7) >> 3;
        if (r.g >= 0) {
            const uint4* src = reinterpret_cast<const uint4*>(p.inter + p.group_off[r.g] + r.t * 16);
            for (int c0 = 0; c0 < chunks; c0 += kWarp) {
                const int c = c0 + lane;
                if (c < chunks)
                    *reinterpret_cast<uint4*>(buf + kResPad + 8 * c) = src[static_cast<int64_t>(c) * (kGroupChunk / 16)];
            }
        }
        buf[lane] = dummy2;                                   // columns [-kResPad, 0)
        for (int c0 = kResPad + 8 * chunks; c0 < kResPad + n_fill + kWarp + 2; c0 += kWarp)
            if (c0 + lane < kResPad + n_fill + kWarp + 2) buf[c0 + lane] = dummy2;
    };

    // Slot pairs pi0 (and pi1: the second 16-lane wavefront) over every pass, both subjects of a
    // pair packed in the halves of the registers.  kL lanes per wavefront; `prefix`: the F
    // recurrence unrolled down the lane's rows (a shorter dependency chain).
    auto align = [&](auto tb_c, auto lanes_c, auto prefix, const int64_t pi0, const int64_t pi1) {
        constexpr int kTB = decltype(tb_c)::value, kL = decltype(lanes_c)::value;
        constexpr int kW = (kTB + 1) / 2;
        constexpr int kPStride = slice_stride<kW>();
        const uint32_t* prof = kL == kWarp ? prof_l : prof_b;
        const int passes = kL == kWarp ? passes_l : passes_b;
        const int words = p.alphabet1 * kPStride;
        const int seg = lane / kL, sl = lane % kL;
        const PairRef r0 = pair_ref(pi0);
        const PairRef r1 = pair_ref(kL < kWarp ? pi1 : -1);
        const int n0 = max(r0.n[0], r0.n[1]), n1 = max(r1.n[0], r1.n[1]);
        const int N = max(n0, n1);
        __syncwarp();   // the previous item's steps have read the buffers
        stage_residues(r0, n0, N, rbuf);
        if constexpr (kL < kWarp) stage_residues(r1, n1, N, rbuf + res_stride);
        __syncwarp();
        const int n_me = seg == 0 ? n0 : n1;
        const uint16_t* rcol = rbuf + seg * res_stride + kResPad - sl;   // rcol[t]: column t - sl
        int2* spill = p.spill + (gwarp * 2 + seg) * p.spill_stride;
        unsigned ngep_r[kTB];
        if constexpr (decltype(prefix)::value) {
#pragma unroll
            for (int r = 0; r < kTB; ++r) ngep_r[r] = pack2(-(r + 1) * p.gaps.gep);
        }
        unsigned best = 0;
        for (int pass = 0; N > 0 && pass < passes; ++pass) {
            const uint32_t* slp = prof + pass * words + chunk_offset<kW>(lane);
            unsigned Hm[kTB], E[kTB];
#pragma unroll
            for (int r = 0; r < kTB; ++r) {
                Hm[r] = init_hm;
                E[r] = init_f;
            }
            unsigned hm_prev = init_hm;
            unsigned out_hm = init_hm, out_f = init_f;
            uint2 sp_cur = make_uint2(init_hm, init_f), sp_next = sp_cur;
            if (pass > 0) {
                if (sl < n_me) sp_cur = reinterpret_cast<const uint2*>(spill)[sl];
                if (kL + sl < n_me) sp_next = reinterpret_cast<const uint2*>(spill)[kL + sl];
            }
            // Pipeline: at step t a lane holds the profile words of its column (loaded during
            // step t - 1) and loads its next column's residues, then their words.
            unsigned wa[kW], wb[kW];
            {
                const unsigned rr = rcol[0];
#pragma unroll
                for (int wi = 0; wi < kW; ++wi) {
                    wa[wi] = slp[(rr & 0xFFu) * kPStride + wi];
                    wb[wi] = slp[(rr >> 8) * kPStride + wi];
                }
            }
            const int steps = N + kL - 1;
            auto step = [&](const int t, const int src_lane, auto on_first, auto write) {
                const unsigned up_hm = __shfl_up_sync(0xffffffffu, out_hm, 1, kL);
                const unsigned up_f = __shfl_up_sync(0xffffffffu, out_f, 1, kL);
                unsigned l0_hm = init_hm, l0_f = init_f;
                if constexpr (!decltype(on_first)::value) {
                    l0_hm = __shfl_sync(0xffffffffu, sp_cur.x, src_lane, kL);
                    l0_f = __shfl_sync(0xffffffffu, sp_cur.y, src_lane, kL);
                }
                unsigned ca[kW], cb[kW];
                const unsigned rn = rcol[t + 1];
#pragma unroll
                for (int wi = 0; wi < kW; ++wi) {
                    ca[wi] = wa[wi];
                    cb[wi] = wb[wi];
                    wa[wi] = slp[(rn & 0xFFu) * kPStride + wi];   // step t + 1
                    wb[wi] = slp[(rn >> 8) * kPStride + wi];
                }
                unsigned F = sl == 0 ? l0_f : up_f;
                const unsigned d = hm_prev;
                hm_prev = sl == 0 ? l0_hm : up_hm;
                auto score = [&](const int rb, unsigned (&sc)[4]) {
#pragma unroll
                    for (int i = 0; i < 4; i += 2) {
                        const int wi = (rb + i) >> 1;
                        if (wi < kW) {
                            sc[i] = __byte_perm(ca[wi], cb[wi], 0x5410);
                            sc[i + 1] = __byte_perm(ca[wi], cb[wi], 0x7632);
                        }
                    }
                };
                if constexpr (decltype(prefix)::value)
                    column2_prefix<kTB>(Hm, E, F, d, score, k, ngep_r, best);
                else
                    column2<kTB>(Hm, E, F, d, score, k, best);
                out_hm = Hm[kTB - 1];
                out_f = F;
                if constexpr (decltype(write)::value) {
                    const int j = t - sl;
                    if (sl == kL - 1 && static_cast<unsigned>(j) < static_cast<unsigned>(n_me))
                        spill[j] = make_int2(static_cast<int>(out_hm), static_cast<int>(out_f));
                }
            };
            auto run = [&](auto on_first, auto write) {
                if constexpr (decltype(on_first)::value) {
                    // constant lane-0 boundary: no kL-step blocks; an extra step past the end
                    // (every lane on a dummy column) is harmless
#pragma unroll 1
                    for (int t = 0; t < steps; t += 2) {
                        step(t, 0, on_first, write);
                        step(t + 1, 0, on_first, write);
                    }
                } else {
                    for (int tb = 0; tb < steps; tb += kL) {
                        if (tb > 0) {
                            sp_cur = sp_next;
                            if (tb + kL + sl < n_me)
                                sp_next = reinterpret_cast<const uint2*>(spill)[tb + kL + sl];
                        }
                        const int ue = min(kL, steps - tb);
                        if (ue == kL) {
#pragma unroll 2
                            for (int u = 0; u < kL; ++u) step(tb + u, u, on_first, write);
                        } else {
#pragma unroll 1
                            for (int u = 0; u < ue; ++u) step(tb + u, u, on_first, write);
                        }
                    }
                }
            };
            const bool last = pass == passes - 1;
            if (pass == 0) {
                if (last)
                    run(std::true_type{}, std::false_type{});
                else
                    run(std::true_type{}, std::true_type{});
            } else {
                if (last)
                    run(std::false_type{}, std::false_type{});
                else
                    run(std::false_type{}, std::true_type{});
            }
            __syncwarp();
        }
        unsigned b = best;
#pragma unroll
        for (int o = kL / 2; o > 0; o >>= 1) b = __vmaxs2(b, __shfl_xor_sync(0xffffffffu, b, o));
        if (sl == 0) {
            const PairRef& r = seg == 0 ? r0 : r1;
            emit_score(p, p.query, r.id[0], static_cast<int>(static_cast<short>(b & 0xFFFFu)));
            emit_score(p, p.query, r.id[1], static_cast<int>(static_cast<short>(b >> 16)));
        }
        __syncwarp();
    };

    // First phase: the longest slot pairs, alone on their SM sub-partitions.
    using TBL = std::integral_constant<int, kTBL>;
    using Full = std::integral_constant<int, kWarp>;
    if (long_block) {
        // Warps w, w + 4, w + 8, w + 12 share a sub-partition (warp w of the block on
        // sub-partition w mod 4); each group waits at its own named barrier (ids 1-4, 128
        // threads) until its first-phase warp has drained the queue, so a sub-partition returns
        // to the bulk as soon as its own first-phase warp is done.
        static_assert(kSsLongWarps == 4 && kSsBW % kSsLongWarps == 0, "one first-phase warp per sub-partition");
        const int sub = warp % kSsLongWarps;
        constexpr int kGroupThreads = kSsBW / kSsLongWarps * kWarp;
        if (warp < kSsLongWarps) {
            for (;;) {
                unsigned it = 0;
                if (lane == 0) it = atomicAdd(&p.ctrl->next_wave_long, 1u);
                it = __shfl_sync(0xffffffffu, it, 0);
                if (it >= long_pairs) break;
                if (p.prefix_f)
                    align(TBL{}, Full{}, std::true_type{}, static_cast<int64_t>(it), int64_t{-1});
                else
                    align(TBL{}, Full{}, std::false_type{}, static_cast<int64_t>(it), int64_t{-1});
            }
            __syncwarp();
            asm volatile("bar.arrive %0, %1;" ::"r"(1 + sub), "r"(kGroupThreads) : "memory");
        } else {
            asm volatile("bar.sync %0, %1;" ::"r"(1 + sub), "r"(kGroupThreads) : "memory");
        }
    }
    // Bulk: the remaining pairs, longest first: one per item on the 32-lane wavefront up to
    // pair half_from, then (kHalf) two per item on 16-lane wavefronts.  A 16-lane item takes
    // longer than a 32-lane one, so only the short pairs, whose items end well before the
    // search does, run that way.
    const int64_t half_from = kHalf ? max(long_pairs, min(p.half_from, total_pairs)) : total_pairs;
    const int64_t full_items = half_from - long_pairs;
    for (;;) {
        unsigned it = 0;
        if (lane == 0) it = atomicAdd(&p.ctrl->next_wave, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (static_cast<int64_t>(it) < full_items) {
            align(TBL{}, Full{}, std::false_type{}, long_pairs + static_cast<int64_t>(it), int64_t{-1});
            continue;
        }
        const int64_t pi = half_from + 2 * (static_cast<int64_t>(it) - full_items);
        if (pi >= total_pairs) break;
        if constexpr (kHalf)
            align(std::integral_constant<int, kSsBulkRows>{}, std::integral_constant<int, kSsBulkLanes>{},
                  std::false_type{}, pi, pi + 1);
    }
}

const void* wave_ss_fn(int rows_per_lane, bool half) {
    if (half)
        return rows_per_lane == 5 ? reinterpret_cast<const void*>(&k_wave_ss_i16x2<5, true>)
                                  : reinterpret_cast<const void*>(&k_wave_ss_i16x2<8, true>);
    return rows_per_lane == 5 ? reinterpret_cast<const void*>(&k_wave_ss_i16x2<5, false>)
                              : reinterpret_cast<const void*>(&k_wave_ss_i16x2<8, false>);
}

// Paired profile of the two-query wavefront: for lane l of pass k,
// pp[d * rows_pad + k * 32 kTB + l * kTB + r] = (S'(q_a, row0_a + r, d), S'(q_b, row0_b + r, d))
// with S' = SM + bias, and 0 + bias for the dummy code, rows past a query's end and lanes
// without a query.
__global__ void k_build_pp_wave(const uint8_t* __restrict__ queries, const int64_t* __restrict__ qoff,
                                const WavePass* __restrict__ passes, int32_t num_passes, int32_t kTB,
                                const int8_t* __restrict__ matrix, int32_t A, int32_t bias,
                                uint32_t* __restrict__ pp, int64_t rows_pad, Control* ctrl) {
    const int d = blockIdx.y;
    const int64_t row = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (row >= rows_pad) return;
    const int T = kWarp * kTB;
    const int64_t k = row / T;
    const int within = static_cast<int>(row - k * T);
    const int l = within / kTB;
    const int r = within - l * kTB;
    int out[2] = {0, 0};
    if (k < num_passes && d < A) {
        for (int h = 0; h < 2; ++h) {
            const int q = passes[k].q[h][l];
            if (q < 0) continue;
            const int64_t q0 = qoff[q];
            const int64_t i = static_cast<int64_t>(passes[k].row0[h][l]) + r;
            if (i >= qoff[q + 1] - q0) continue;
            const int code = queries[q0 + i];
            if (code < A)
                out[h] = matrix[code * A + d];
            else
                atomicOr(&ctrl->status, 1u);
        }
    }
    pp[static_cast<int64_t>(d) * rows_pad + row] =
        (static_cast<unsigned>(out[0] + bias) & 0xFFFFu) | (static_cast<unsigned>(out[1] + bias) << 16);
}

const void* wave_mq_fn(int rows_per_lane) {
    return rows_per_lane == 8    ? reinterpret_cast<const void*>(&k_wave_mq_i16x2<8>)
           : rows_per_lane == 12 ? reinterpret_cast<const void*>(&k_wave_mq_i16x2<12>)
                                 : reinterpret_cast<const void*>(&k_wave_mq_i16x2<16>);
}

}  // namespace

int wave_warps() { return kWaveBW; }

size_t wave_smem_bytes(int rows_per_lane, int alphabet1) {
    const int stride = rows_per_lane == 8    ? slice_stride<8>()
                       : rows_per_lane == 12 ? slice_stride<12>()
                                             : slice_stride<16>();
    return static_cast<size_t>(alphabet1) * stride * sizeof(uint32_t);
}

int wave_occupancy(int rows_per_lane, int alphabet1) {
    int n = 0;
    const size_t smem = wave_smem_bytes(rows_per_lane, alphabet1);
    const void* fn = wave_mq_fn(rows_per_lane);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kWaveBW * kWarp, smem) != cudaSuccess)
        return 0;
    return n;
}

size_t wave_ss_smem_bytes(int rows_per_lane, int alphabet1, int m, int max_group_len, bool half) {
    const int stride_l = rows_per_lane == 5 ? slice_stride<3>() : slice_stride<4>();
    const int passes_l = std::max(1, (m + kWarp * rows_per_lane - 1) / (kWarp * rows_per_lane));
    constexpr int kRowsB = kSsBulkLanes * kSsBulkRows;
    const int passes_b = half ? std::max(1, (m + kRowsB - 1) / kRowsB) : 0;
    return (static_cast<size_t>(passes_l) * stride_l +
            static_cast<size_t>(passes_b) * slice_stride<(kSsBulkRows + 1) / 2>()) *
               alphabet1 * sizeof(uint32_t) +
           static_cast<size_t>(kSsBW) * (half ? 2 : 1) * wave_ss_res_stride(max_group_len) * sizeof(uint16_t);
}

int wave_ss_warps() { return kSsBW; }
int wave_ss_blocks_per_sm() { return kSsBlocksPerSM; }
int wave_ss_long_warps() { return kSsLongWarps; }
int wave_ss_bulk_rows() { return kSsBulkRows; }
int wave_ss_bulk_lanes() { return kSsBulkLanes; }

bool wave_ss_fits(int rows_per_lane, int alphabet1, int m, int max_group_len, int max_smem, bool half) {
    if (m <= 0) return false;
    const size_t smem = wave_ss_smem_bytes(rows_per_lane, alphabet1, m, max_group_len, half);
    if (smem * kSsBlocksPerSM > static_cast<size_t>(max_smem)) return false;
    const void* fn = wave_ss_fn(rows_per_lane, half);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) !=
        cudaSuccess)
        return false;
    int n = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kSsBW * kWarp, smem) == cudaSuccess &&
           n >= kSsBlocksPerSM;
}

cudaError_t launch_wave_ss(const WaveParams& p, int rows_per_lane, bool half, int m, int grid,
                           cudaStream_t st) {
    const size_t smem = wave_ss_smem_bytes(rows_per_lane, p.alphabet1, m, p.max_group_len, half);
    const void* fn = wave_ss_fn(rows_per_lane, half);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    if (half) {
        if (rows_per_lane == 5)
            k_wave_ss_i16x2<5, true><<<grid, kSsBW * kWarp, smem, st>>>(p);
        else
            k_wave_ss_i16x2<8, true><<<grid, kSsBW * kWarp, smem, st>>>(p);
    } else {
        if (rows_per_lane == 5)
            k_wave_ss_i16x2<5, false><<<grid, kSsBW * kWarp, smem, st>>>(p);
        else
            k_wave_ss_i16x2<8, false><<<grid, kSsBW * kWarp, smem, st>>>(p);
    }
    return cudaGetLastError();
}

cudaError_t launch_build_pp_wave(const uint8_t* d_queries, const int64_t* d_qoff,
                                 const WavePass* d_passes, int32_t num_passes, int32_t rows_per_lane,
                                 const int8_t* d_matrix, int32_t A, int32_t bias, uint32_t* d_pp,
                                 int64_t rows_pad, Control* ctrl, cudaStream_t st) {
    const int threads = 256;
    dim3 grid(static_cast<unsigned>((rows_pad + threads - 1) / threads), static_cast<unsigned>(A + 1));
    k_build_pp_wave<<<grid, threads, 0, st>>>(d_queries, d_qoff, d_passes, num_passes, rows_per_lane,
                                              d_matrix, A, bias, d_pp, rows_pad, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_wave_mq(const WaveParams& p, int rows_per_lane, int grid, cudaStream_t st) {
    const size_t smem = wave_smem_bytes(rows_per_lane, p.alphabet1);
    const void* fn = wave_mq_fn(rows_per_lane);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    if (rows_per_lane == 8)
        k_wave_mq_i16x2<8><<<grid, kWaveBW * kWarp, smem, st>>>(p);
    else if (rows_per_lane == 12)
        k_wave_mq_i16x2<12><<<grid, kWaveBW * kWarp, smem, st>>>(p);
    else
        k_wave_mq_i16x2<16><<<grid, kWaveBW * kWarp, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace swgb
