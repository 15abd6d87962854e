// Inter-task kernel with a score profile instead of a query profile (Section 4.3).
//
// The paper offers two ways to fetch substitution scores in the inter-task loop: a query
// profile (scores indexed by query position, one table per query) and a score profile (for a
// group of database sequences and each alphabet letter a, the vector of scores of a against the
// group's residues at column j, rebuilt for every group; one vector load per cell).  This kernel
// is the score-profile form of k_inter_i16x2 (same strips, interleaved database, int16x2 DPX
// update, saturation flag and boundary buffers):
//  * every 4 columns a thread builds, in its own slice of shared memory, sp[a][c] = (S'(a, s_a),
//    S'(a, s_b)) for every letter a and its two subjects' residues s_a, s_b at the 4 columns,
//    from the transposed biased matrix (S' = SM + Goe, one 16-byte load serves 8 letters and a
//    byte permute per letter packs the two lanes);
//  * the cell update of row r reads sp[q_r][c] with one 4-byte load: no permute per cell pair
//    (5.5 ALU operations per cell pair instead of 6.5), but 32 permutes and 32 stores per column
//    to build the profile, amortised over the 32 rows of a strip rather than over the whole
//    query as on the CPU, where the profile of a group is built once for all query rows.
// Selected for single-query launches by SWGB_SCORE_PROFILE=1; the query profile remains the
// default (measured comparison in the design notes).
#include "swgb_device.cuh"

namespace swgb {

namespace {

constexpr int kT = 32;             // rows per strip
constexpr int kW = 4;              // warps per block
constexpr int kSpCols = 4;         // columns per profile build
constexpr int kMtStride = 40;      // int16 per transposed-matrix row (80 B: spreads the banks)

struct PackedSp {
    unsigned ngoe, nge, ngep, e0, floor;
};

__device__ __forceinline__ unsigned pack2_sp(int v) {
    return (static_cast<unsigned>(v) & 0xFFFFu) * 0x00010001u;
}

// Score-profile build for 4 columns: `words` holds the residue bytes of columns c = 0..3
// (byte 2c: lane a, byte 2c + 1: lane b); sp points at this thread's word of letter 0, column 0.
__device__ __forceinline__ void build_sp(unsigned word_lo, unsigned word_hi, const int16_t* s_mt,
                                         uint32_t* sp, int nvec) {
#pragma unroll
    for (int c = 0; c < kSpCols; ++c) {
        const unsigned w = c < 2 ? word_lo : word_hi;
        const int sh = 16 * (c & 1);
        const unsigned ra = (w >> sh) & 0xFFu, rb = (w >> (sh + 8)) & 0xFFu;
        const uint4* ma = reinterpret_cast<const uint4*>(s_mt + ra * kMtStride);
        const uint4* mb = reinterpret_cast<const uint4*>(s_mt + rb * kMtStride);
        for (int v = 0; v < nvec; ++v) {
            const uint4 x = ma[v], y = mb[v];
            const unsigned xa[4] = {x.x, x.y, x.z, x.w}, ya[4] = {y.x, y.y, y.z, y.w};
            uint32_t* o = sp + (8 * v) * (kSpCols * kWarp) + c * kWarp;
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                o[(2 * h) * (kSpCols * kWarp)] = __byte_perm(xa[h], ya[h], 0x5410);
                o[(2 * h + 1) * (kSpCols * kWarp)] = __byte_perm(xa[h], ya[h], 0x7632);
            }
        }
    }
}

// One column of one strip: the update of k_inter_i16x2 with the score pair of row r read from
// the score profile at qo[r] (letter q_r's word for this column).
__device__ __forceinline__ void column_sp(unsigned (&Hm)[kT], unsigned (&E)[kT], unsigned& f,
                                          unsigned& diag, const uint32_t* spc, const int (&qo)[kT],
                                          const PackedSp& k, unsigned& best) {
    unsigned F = f;
    unsigned d = diag;
#pragma unroll
    for (int r = 0; r < kT; r += 2) {
        const unsigned s0 = spc[qo[r]];
        const unsigned s1 = spc[qo[r + 1]];
        const unsigned x0 = __viaddmax_s16x2_relu(d, s0, E[r]);
        const unsigned xm0 = __viaddmax_s16x2(x0, k.ngoe, k.floor);
        d = Hm[r];
        Hm[r] = __viaddmax_s16x2(F, k.ngoe, xm0);
        E[r] = __viaddmax_s16x2(E[r], k.nge, Hm[r]);
        F = __viaddmax_s16x2(F, k.ngep, xm0);
        const unsigned x1 = __viaddmax_s16x2_relu(d, s1, E[r + 1]);
        const unsigned xm1 = __viaddmax_s16x2(x1, k.ngoe, k.floor);
        d = Hm[r + 1];
        Hm[r + 1] = __viaddmax_s16x2(F, k.ngoe, xm1);
        E[r + 1] = __viaddmax_s16x2(E[r + 1], k.nge, Hm[r + 1]);
        F = __viaddmax_s16x2(F, k.ngep, xm1);
        best = __vimax3_s16x2(best, x0, x1);
    }
    f = F;
}

// One strip of one group over all L columns (L is a multiple of 8).
__device__ __forceinline__ void strip_sp(const uint4* __restrict__ res, int L, uint4* bnd,
                                         uint32_t* sp, const int (&qo)[kT], const int16_t* s_mt,
                                         int nvec, bool first, bool last, const PackedSp& k,
                                         unsigned& best, int lane) {
    unsigned Hm[kT], E[kT];
#pragma unroll
    for (int r = 0; r < kT; ++r) {
        Hm[r] = k.ngoe;
        E[r] = k.e0;
    }
    const unsigned f_top = k.ngep;
    unsigned hm_prev = k.ngoe;
    uint4 w_next = res[lane];
    uint4 b_next = first ? make_uint4(k.ngoe, f_top, k.ngoe, f_top) : bnd[lane];
    for (int jc = 0; jc < L; jc += 8) {
        const uint4 w = w_next;
        if (jc + 8 < L) w_next = res[((jc >> 3) + 1) * kWarp + lane];
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            build_sp(half ? w.z : w.x, half ? w.w : w.y, s_mt, sp, nvec);
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {
                const int j = jc + 4 * half + 2 * h2;   // columns j and j + 1
                const uint4 b = b_next;
                if (!first && j + 2 < L) b_next = bnd[((j >> 1) + 1) * kWarp + lane];
                unsigned f0 = b.y;
                unsigned d0 = hm_prev;
                column_sp(Hm, E, f0, d0, sp + (2 * h2) * kWarp, qo, k, best);
                const unsigned out_hm0 = Hm[kT - 1];
                unsigned f1 = b.w;
                unsigned d1 = b.x;
                column_sp(Hm, E, f1, d1, sp + (2 * h2 + 1) * kWarp, qo, k, best);
                hm_prev = b.z;
                if (!last) bnd[(j >> 1) * kWarp + lane] = make_uint4(out_hm0, f0, Hm[kT - 1], f1);
            }
        }
    }
}

__device__ __forceinline__ void emit_sp(const InterParams& p, int q, int32_t* scores, int id, int v) {
    if (id < 0) return;
    if (v >= p.thresh) {
        scores[id] = -1;
        const unsigned slot = atomicAdd(&p.ctrl->flag_count, 1u);
        if (slot < p.flag_cap) p.flags[slot] = FlagEntry{q, id};
    } else {
        scores[id] = v;
    }
}

__global__ void __launch_bounds__(kW * kWarp, 3) k_inter_sp_i16x2(const InterParams p) {
    constexpr int kBlock = kW * kWarp;
    extern __shared__ __align__(16) uint32_t s_dyn[];
    const int lane = threadIdx.x & (kWarp - 1);
    const int warp = threadIdx.x >> 5;
    const int A1 = p.alphabet1;
    const int nvec = (A1 + 7) / 8;                       // 8 letters per 16-byte matrix load
    const int mt_words = (A1 * kMtStride * 2 + 15) / 16 * 4;
    int16_t* s_mt = reinterpret_cast<int16_t*>(s_dyn);
    // this thread's profile words: [letter][column][lane], letters padded to 8
    uint32_t* sp = s_dyn + mt_words + warp * (nvec * 8 * kSpCols * kWarp) + lane;
    uint4* bnd = p.bnd + (static_cast<int64_t>(blockIdx.x) * kW + warp) * p.bnd_stride;
    PackedSp k;
    k.ngoe = pack2_sp(-p.gaps.goe);
    k.nge = pack2_sp(-p.gaps.ge);
    k.ngep = pack2_sp(-p.gaps.gep);
    k.e0 = pack2_sp(-p.gaps.gep);
    k.floor = 0x80008000u;
    for (int v = threadIdx.x; v < A1 * kMtStride; v += kBlock) s_mt[v] = p.mt[v];

    __shared__ InterItem s_it;
    for (;;) {
        __syncthreads();   // also orders the matrix staging before the first use
        if (threadIdx.x == 0) {
            const int it = static_cast<int>(atomicAdd(&p.ctrl->next_inter, 1u));
            s_it = it < p.num_items ? p.items[it] : InterItem{-1, 0, 0, 0};
        }
        __syncthreads();
        const InterItem item = s_it;
        if (item.query < 0) break;
        const QueryDesc qd = p.queries[item.query];
        const bool active = warp < item.ngroups;
        if (!active) continue;
        const int g = item.group + warp;
        const int L = p.group_len[g];
        const uint4* res = reinterpret_cast<const uint4*>(p.inter + p.group_off[g]);
        const uint8_t* qres = p.qres + p.qres_off[item.query];
        const int S = (qd.m + kT - 1) / kT;
        unsigned best = 0;
        if (L > 0) {
            for (int s = 0; s < S; ++s) {
                int qo[kT];   // word offset of row r's letter in this thread's profile slice
#pragma unroll
                for (int r = 0; r < kT; ++r) {
                    const int row = s * kT + r;
                    // rows past the query take the dummy letter (score 0); codes are checked
                    // by the profile build, the clamp only keeps the read inside the slice
                    const int a = row < qd.m ? min(static_cast<int>(qres[row]), A1 - 1) : A1 - 1;
                    qo[r] = a * (kSpCols * kWarp);
                }
                strip_sp(res, L, bnd, sp, qo, s_mt, nvec, s == 0, s == S - 1, k, best, lane);
            }
        }
        const int base = g * kGroupSeqs + 2 * lane;
        emit_sp(p, item.query, qd.scores, p.perm[base],
                static_cast<int>(static_cast<short>(best & 0xFFFFu)));
        emit_sp(p, item.query, qd.scores, p.perm[base + 1],
                static_cast<int>(static_cast<short>(best >> 16)));
    }
}

}  // namespace

int inter_sp_mt_stride() { return kMtStride; }
int inter_sp_warps() { return kW; }

size_t inter_sp_smem_bytes(int alphabet1) {
    const int nvec = (alphabet1 + 7) / 8;
    const size_t mt = static_cast<size_t>((alphabet1 * kMtStride * 2 + 15) / 16 * 16);
    return mt + static_cast<size_t>(kW) * nvec * 8 * kSpCols * kWarp * sizeof(uint32_t);
}

int inter_sp_occupancy(int alphabet1) {
    int n = 0;
    const size_t smem = inter_sp_smem_bytes(alphabet1);
    const void* fn = reinterpret_cast<const void*>(&k_inter_sp_i16x2);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kW * kWarp, smem) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_inter_sp(const InterParams& p, int grid, cudaStream_t st) {
    const size_t smem = inter_sp_smem_bytes(p.alphabet1);
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_inter_sp_i16x2),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    k_inter_sp_i16x2<<<grid, kW * kWarp, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace swgb
