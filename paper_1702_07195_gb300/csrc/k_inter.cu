// Inter-task Smith-Waterman/Gotoh kernel: packed int16x2 lanes, Blackwell DPX max-plus ops.
//
// Paper Section 4 (inter-task scheme, Section 4.1 vertical blocking, Section 4.2 narrow
// integer ranges with recomputation, Section 4.3 query profile), redesigned for sm_103a:
//  * one warp aligns one query against a group of 64 database sequences: 32 threads, each
//    holding two sequences in the two 16-bit halves of every register (int16x2 lanes);
//  * the query is cut into strips of T rows ("vertical blocks"); a thread keeps the strip's
//    H - Goe and E columns in registers and sweeps the whole subject, one column at a time;
//    the strip's bottom row (H - Goe, F) goes to a per-warp global buffer that the next
//    strip reads (coalesced 16-byte accesses, L2 resident for typical lengths);
//  * the query profile for 256 rows at a time sits in shared memory; one 16-byte load
//    serves 8 rows of one lane, and a byte permute packs the two lanes' scores;
//  * the cell update is five DPX operations per cell pair plus half a three-way max for the
//    running best (Eqs. sw2-sw4, rearranged as shown in `cell` below);
//  * blocks are persistent and take (query, 4 groups) items from an atomic queue, longest
//    items first (the paper's dynamic distribution to idle threads, Section 4.1);
//  * a lane whose best score reaches 32767 - max(SM) may have wrapped and is flagged; its
//    exact score comes from the int32 rescore kernel (Section 4.2's recomputation at the
//    next wider range).  Below that threshold no intermediate can leave the int16 range.
#include "swgb_device.cuh"

namespace swgb {

namespace {


struct Packed {
    unsigned ngoe;   // (-Goe, -Goe)
    unsigned nge;    // (-Ge, -Ge)
    unsigned ngep;   // (-min(Ge, Goe), ...)
    unsigned e0;     // E(i, 1) = -min(Ge, Goe): Eq. sw3 with the zero boundary
    unsigned floor;  // (-32768, -32768)
};

__device__ __forceinline__ unsigned pack2(int v) {
    return (static_cast<unsigned>(v) & 0xFFFFu) * 0x00010001u;
}

// One column of one strip for both lanes (kT query rows per strip).
//   diag : (H - Goe)(r0 - 1, j - 1)       f : F(r0, j)
// returns, through hm_out / f, (H - Goe)(r_last, j) and F(r_last + 1, j).
// Per row r with S' = SM + Goe from the profile:
//   X      = max(Hm(r-1, j-1) + S', E(r, j), 0)        = max(0, H_diag + SM, E)    Eq. sw2 part
//   H      = max(X, F(r, j))                            Eq. sw2
//   Hm     = H - Goe = max(F - Goe, X - Goe)
//   E(r, j+1) = max(E(r, j) - Ge, Hm)                   Eq. sw3
//   F(r+1, j) = max(F - Ge, H - Goe) = max(F - min(Ge, Goe), X - Goe)   Eq. sw4
//   best   = max(best, X)     (max H = max X: every F is bounded by an earlier X or by 0)
template <int kT>
__device__ __forceinline__ void column(unsigned (&Hm)[kT], unsigned (&E)[kT], unsigned& f,
                                       unsigned& diag, const int16_t* qa, const int16_t* qb,
                                       const Packed& k, unsigned& best) {
    const uint4* pa = reinterpret_cast<const uint4*>(qa);
    const uint4* pb = reinterpret_cast<const uint4*>(qb);
    unsigned F = f;
    unsigned d = diag;
#pragma unroll
    for (int r8 = 0; r8 < kT; r8 += 8) {
        const uint4 a = pa[r8 >> 3];
        const uint4 b = pb[r8 >> 3];
        const unsigned wa[4] = {a.x, a.y, a.z, a.w};
        const unsigned wb[4] = {b.x, b.y, b.z, b.w};
        // rows in sub-blocks of four: the four X (diagonals from the previous column's Hm,
        // the first saved in d) before the F chain, which then overwrites Hm and E in place
#pragma unroll
        for (int h4 = 0; h4 < 4; h4 += 2) {
            const int r = r8 + 2 * h4;
            unsigned sc[4];
            sc[0] = __byte_perm(wa[h4], wb[h4], 0x5410);           // row r:   (lane a, lane b)
            sc[1] = __byte_perm(wa[h4], wb[h4], 0x7632);           // row r + 1
            sc[2] = __byte_perm(wa[h4 + 1], wb[h4 + 1], 0x5410);
            sc[3] = __byte_perm(wa[h4 + 1], wb[h4 + 1], 0x7632);
            const unsigned x0 = __viaddmax_s16x2_relu(d, sc[0], E[r]);
            const unsigned x1 = __viaddmax_s16x2_relu(Hm[r], sc[1], E[r + 1]);
            const unsigned x2 = __viaddmax_s16x2_relu(Hm[r + 1], sc[2], E[r + 2]);
            const unsigned x3 = __viaddmax_s16x2_relu(Hm[r + 2], sc[3], E[r + 3]);
            const unsigned xm[4] = {__viaddmax_s16x2(x0, k.ngoe, k.floor), __viaddmax_s16x2(x1, k.ngoe, k.floor),
                                    __viaddmax_s16x2(x2, k.ngoe, k.floor), __viaddmax_s16x2(x3, k.ngoe, k.floor)};
            best = __vimax3_s16x2(best, x0, x1);
            best = __vimax3_s16x2(best, x2, x3);
            d = Hm[r + 3];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                Hm[r + i] = __viaddmax_s16x2(F, k.ngoe, xm[i]);
                E[r + i] = __viaddmax_s16x2(E[r + i], k.nge, Hm[r + i]);
                F = __viaddmax_s16x2(F, k.ngep, xm[i]);
            }
        }
    }
    f = F;
}

// One strip (query rows [s*kT, s*kT + kT)) of one group: sweeps all L columns.
template <int kT>
__device__ __forceinline__ void strip(const uint4* __restrict__ res, int L, uint4* bnd,
                                      const int16_t* qp_strip, int qstride, bool first,
                                      bool last, const Packed& k, unsigned& best, int lane) {
    unsigned Hm[kT], E[kT];
#pragma unroll
    for (int r = 0; r < kT; ++r) {
        Hm[r] = k.ngoe;   // H(r, 0) - Goe
        E[r] = k.e0;      // E(r, 1)
    }
    const unsigned f_top = k.ngep;   // F(1, j) = max(0 - Goe, 0 - Ge) on the first strip
    unsigned hm_prev = k.ngoe;       // (H - Goe)(r0 - 1, j - 1), column 0
    uint4 w_next = res[lane];
    // boundary records alternate between two register sets (no copy per record)
    uint4 b_a = first ? make_uint4(k.ngoe, f_top, k.ngoe, f_top) : bnd[lane];
    uint4 b_b = b_a;
    // Columns j and j + 1: residue bytes of word wq (lane a, lane b per column); b holds the
    // previous strip's record of these columns, b_pref receives the next record.
    auto two_columns = [&](const unsigned wq, const uint4 b, uint4& b_pref, const int j) {
        if (!first && j + 2 < L) b_pref = bnd[((j >> 1) + 1) * kWarp + lane];
        unsigned f0 = b.y;
        unsigned d0 = hm_prev;
        column(Hm, E, f0, d0, qp_strip + __byte_perm(wq, 0u, 0x4440u) * qstride,
               qp_strip + __byte_perm(wq, 0u, 0x4441u) * qstride, k, best);
        const unsigned out_hm0 = Hm[kT - 1];
        unsigned f1 = b.w;
        unsigned d1 = b.x;
        column(Hm, E, f1, d1, qp_strip + __byte_perm(wq, 0u, 0x4442u) * qstride,
               qp_strip + __byte_perm(wq, 0u, 0x4443u) * qstride, k, best);
        hm_prev = b.z;
        if (!last) bnd[(j >> 1) * kWarp + lane] = make_uint4(out_hm0, f0, Hm[kT - 1], f1);
    };
    // L (even) columns: whole 8-column chunks, then 1-3 column pairs of the last chunk
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

__device__ __forceinline__ void emit(const InterParams& p, int q, int32_t* scores, int id, int v) {
    if (id < 0) return;
    if (v >= p.thresh) {
        scores[id] = -1;
        const unsigned slot = atomicAdd(&p.ctrl->flag_count, 1u);
        if (slot < p.flag_cap) p.flags[slot] = FlagEntry{q, id};
    } else {
        scores[id] = v;
    }
}

template <int kT, int kW, int kMinBlocks>
__global__ void __launch_bounds__(kW * kWarp, kMinBlocks) k_inter_i16x2(const InterParams p) {
    constexpr int kBlock = kW * kWarp;
    extern __shared__ __align__(16) int16_t s_qp[];
    const int lane = threadIdx.x & (kWarp - 1);
    const int warp = threadIdx.x >> 5;
    const int qstride = kQpRows + kQpPad;
    uint4* bnd = p.bnd + (static_cast<int64_t>(blockIdx.x) * kW + warp) * p.bnd_stride;
    Packed k;
    k.ngoe = pack2(-p.gaps.goe);
    k.nge = pack2(-p.gaps.ge);
    k.ngep = pack2(-p.gaps.gep);
    k.e0 = pack2(-p.gaps.gep);
    k.floor = 0x80008000u;

    __shared__ InterItem s_it;
    for (;;) {
        if (threadIdx.x == 0) {
            const int it = static_cast<int>(atomicAdd(&p.ctrl->next_inter, 1u));
            InterItem next{-1, 0, 0, 0};   // query -1: no work left
            if (p.tick) {   // serving tick: decode (request, chunk) from the descriptor
                const TickDesc* t = p.tick;
                if (it < t->prefix[t->n]) {
                    int s = 0;
                    while (t->prefix[s + 1] <= it) ++s;
                    const int g0 = (t->chunk_end[s] - 1 - (it - t->prefix[s])) * kW;
                    next = InterItem{t->slot[s], g0, min(kW, p.num_groups - g0), 0};
                }
            } else if (it < p.num_items) {
                next = p.items[it];
            }
            s_it = next;
        }
        __syncthreads();
        const InterItem item = s_it;
        __syncthreads();
        if (item.query < 0) break;
        const QueryDesc qd = p.queries[item.query];
        const bool active = warp < item.ngroups;
        const int g = item.group + warp;
        const int L = active ? p.group_cols[g] : 0;
        const uint4* res =
            active ? reinterpret_cast<const uint4*>(p.inter + p.group_off[g]) : nullptr;
        const int S = (qd.m + kT - 1) / kT;
        unsigned best = 0;
        for (int c0 = 0; c0 < S * kT; c0 += kQpRows) {
            __syncthreads();
            constexpr int kVecPerRow = kQpRows / 8;
            for (int v = threadIdx.x; v < p.alphabet1 * kVecPerRow; v += kBlock) {
                const int d = v / kVecPerRow;
                const int o = (v - d * kVecPerRow) * 8;
                const uint4 x = *reinterpret_cast<const uint4*>(
                    qd.qp + static_cast<int64_t>(d) * qd.m_pad + c0 + o);
                *reinterpret_cast<uint4*>(s_qp + d * qstride + o) = x;
            }
            __syncthreads();
            if (active && L > 0) {
                const int s_end = min(S, (c0 + kQpRows) / kT);
                for (int s = c0 / kT; s < s_end; ++s)
                    strip<kT>(res, L, bnd, s_qp + (s * kT - c0), qstride, s == 0, s == S - 1,
                              k, best, lane);
            }
        }
        if (active) {
            const int base = g * kGroupSeqs + 2 * lane;
            const int b0 = static_cast<int>(static_cast<short>(best & 0xFFFFu));
            const int b1 = static_cast<int>(static_cast<short>(best >> 16));
            emit(p, item.query, qd.scores, p.perm[base], b0);
            emit(p, item.query, qd.scores, p.perm[base + 1], b1);
        }
    }
}

// Variants: (rows per strip, warps per block).  Register budgets: 32 rows -> 128 registers
// (4 blocks of 4 warps per SM); 64 rows -> <= 255 registers (2 blocks of 4 warps, or 1 of 8).
struct InterVariant {
    int T, W;
    const void* fn;
};

template <int T, int W, int MB>
void launch_variant(const InterParams& p, int grid, size_t smem, cudaStream_t st) {
    k_inter_i16x2<T, W, MB><<<grid, W * kWarp, smem, st>>>(p);
}

const InterVariant kVariants[] = {
    {32, 4, reinterpret_cast<const void*>(&k_inter_i16x2<32, 4, 4>)},
    {64, 4, reinterpret_cast<const void*>(&k_inter_i16x2<64, 4, 2>)},
    {32, 8, reinterpret_cast<const void*>(&k_inter_i16x2<32, 8, 2>)},
    {64, 8, reinterpret_cast<const void*>(&k_inter_i16x2<64, 8, 1>)},
};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

}  // namespace

int inter_num_variants() { return kNumVariants; }
int inter_variant_rows(int v) { return kVariants[v].T; }
int inter_variant_warps(int v) { return kVariants[v].W; }

size_t inter_smem_bytes(int alphabet1) {
    return static_cast<size_t>(alphabet1) * (kQpRows + kQpPad) * sizeof(int16_t);
}

int inter_occupancy(int variant, int alphabet1) {
    if (variant < 0 || variant >= kNumVariants) return 0;
    int n = 0;
    const size_t smem = inter_smem_bytes(alphabet1);
    const void* fn = kVariants[variant].fn;
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kVariants[variant].W * kWarp, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_inter(const InterParams& p, int variant, int grid, cudaStream_t st) {
    if (variant < 0 || variant >= kNumVariants) return cudaErrorInvalidValue;
    const size_t smem = inter_smem_bytes(p.alphabet1);
    cudaError_t e = cudaFuncSetAttribute(kVariants[variant].fn,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    switch (variant) {
        case 0: launch_variant<32, 4, 4>(p, grid, smem, st); break;
        case 1: launch_variant<64, 4, 2>(p, grid, smem, st); break;
        case 2: launch_variant<32, 8, 2>(p, grid, smem, st); break;
        default: launch_variant<64, 8, 1>(p, grid, smem, st); break;
    }
    return cudaGetLastError();
}

}  // namespace swgb
