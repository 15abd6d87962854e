// Device-side data structures and launch entry points shared by the kernels and the host
// runtime of libswgb.  Not part of the public C ABI (include/swgb.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace swgb {

constexpr int kWarp = 32;
constexpr int kGroupSeqs = 64;     // sequences per interleaved group: 32 threads x 2 int16 lanes
constexpr int kGroupChunk = 512;   // bytes per 8 columns of a group (32 threads x 16 B)
constexpr int kQpRows = 256;       // query rows staged in shared memory per chunk; profiles are
                                   // padded to a multiple of this
constexpr int kQpPad = 8;          // int16 padding per shared-memory profile row (16 B)
constexpr int kMaxAlphabet = 32;

// One query of a search.  The profile is biased by the gap-open cost so that the int16x2
// update can keep H - Goe instead of H (one DPX operation less per cell pair):
//   qp[d * m_pad + i] = SM(q_i, d) + bias   for d < A, i < m
//   qp[d * m_pad + i] = 0 + bias            for the dummy code d = A, or i >= m
// with bias = Goe whenever Goe + 127 fits int16 (always on the int16x2 path); otherwise
// bias = 0 and the int32 kernel adds Goe itself.
// A score of 0 for the dummy code and the padded rows leaves every score unchanged (cells
// there are bounded by cells of the real matrix).
struct QueryDesc {
    const int16_t* qp;
    int32_t* scores;     // output row, indexed by original database sequence id
    int32_t m;
    int32_t m_pad;
};

// Block-level work item of the inter-task kernel: `ngroups` (<= warps per block) consecutive
// groups starting at `group`, all against query slot `query`.
struct InterItem {
    int32_t query;
    int32_t group;
    int32_t ngroups;
    int32_t cost;        // unused on the device; the host sorts by it
};

// One tick of the serving loop (continuous batching): every in-flight request contributes a
// range of its database chunks (W groups each); requests admitted this tick also get their
// long subjects.  Uploaded to the device before each replay of the tick graph.
constexpr int kTickMax = 128;
struct TickDesc {
    int32_t n;                        // requests in this tick
    int32_t n_long;                   // requests whose long subjects run in this tick
    int32_t mq_steps;                 // multi-query ticks: strip pairs of all batches
    int32_t hg_begin, hg_end;         // multi-query ticks: half-groups of the database slice
    int32_t n_batches;                // multi-query ticks: independent two-stream batches
    int32_t batch_step_off[kTickMax + 1];   // batch b owns steps [off[b], off[b+1])
    int32_t slot[kTickMax];           // query slot of request s
    int32_t chunk_end[kTickMax];      // its chunks [chunk_end - count, chunk_end), longest first
    int32_t prefix[kTickMax + 1];     // item offsets: request s owns items [prefix[s], prefix[s+1])
    int32_t long_slot[kTickMax];
};

struct FlagEntry {
    int32_t query;
    int32_t seq;
};

// Zeroed before every launch sequence.
struct Control {
    unsigned long long next_intra;   // intra-task pair counter (long subjects, all pairs)
    unsigned long long next_groups;  // intra-task pair counter (routed groups)
    unsigned long long sweep_next;   // rescore sweep block counter
    unsigned int next_inter;         // inter-task item counter
    unsigned int next_rescore;       // saturation-list counter
    unsigned int flag_count;         // saturated lanes seen by the int16x2 kernels
    unsigned int status;             // bit 0: a query residue code was out of range
    unsigned int next_wave;          // packed wavefront kernel's item counter
    unsigned int next_wave_long;     // its queue of the longest slot pairs (two-subject mode)
};

struct Gaps {
    int32_t goe;         // Goe
    int32_t ge;          // Ge
    int32_t gep;         // min(Ge, Goe): the cost a continuing F position pays in Eq. sw4
};

struct InterParams {
    const uint8_t* inter;
    const int64_t* group_off;
    const int32_t* group_len;
    const int32_t* group_cols;  // columns to sweep per group (longest member, rounded to 2)
    const int32_t* perm;
    const QueryDesc* queries;
    const InterItem* items;
    int32_t num_items;
    int32_t alphabet1;   // A + 1 profile rows (the last is the dummy code)
    Control* ctrl;
    FlagEntry* flags;
    uint32_t flag_cap;
    int32_t thresh;      // int16 saturation threshold: 32767 - max(0, max SM)
    uint4* bnd;          // strip-boundary buffers, one per resident warp
    int64_t bnd_stride;  // uint4 per warp slot
    Gaps gaps;
    const TickDesc* tick;   // non-null: items come from this tick descriptor, not `items`
    int32_t num_groups;     // groups in the database (tick mode)
    // score-profile kernel only: query residues, their offsets, the biased transposed matrix
    const uint8_t* qres;
    const int64_t* qres_off;
    const int16_t* mt;      // mt[s * inter_sp_mt_stride() + a] = SM(a, s) + bias
};

// Multi-query inter-task kernel: the two int16 lanes of a register hold two different queries
// against the same subject.  The queries are laid out in two "streams" of T-row strips; step k
// pairs strip k of stream a (lane a) with strip k of stream b (lane b).
struct MqStep {
    int32_t qa, qb;      // query slots (-1: the lane has no query at this step)
    int32_t sa, sb;      // strip index within that query
    uint32_t flags;      // kMqFirstA | kMqLastA | kMqFirstB | kMqLastB
    int32_t pad;
};
constexpr uint32_t kMqFirstA = 1u, kMqLastA = 2u, kMqFirstB = 4u, kMqLastB = 8u;

struct InterMqParams {
    const uint8_t* inter;
    const int64_t* group_off;
    const int32_t* group_len;
    const int32_t* group_cols;  // columns to sweep per group (longest member, rounded to 2)
    const int32_t* perm;
    const QueryDesc* queries;   // output rows (qp unused)
    const uint32_t* pp;         // paired profile: pp[d * rows_pad + k * T + r] = (S'_a, S'_b)
    int64_t rows_pad;           // multiple of kQpRows
    const MqStep* steps;
    int32_t num_steps;
    int32_t num_half_groups;    // 2 x groups: each warp item is one slot parity of one group
    int32_t alphabet1;
    Control* ctrl;
    FlagEntry* flags;
    uint32_t flag_cap;
    int32_t thresh;
    uint4* bnd;
    int64_t bnd_stride;
    Gaps gaps;
    const TickDesc* tick;       // non-null: num_steps and the half-group range come from here
};

// Work source of the int32 intra-task kernel.
enum IntraMode : int32_t {
    kIntraLong = 0,      // (query, long subject) pairs: num_queries x num_long
    kIntraRescore = 1,   // entries of the saturation list, then a sweep if it overflowed
    kIntraAll = 2,       // every (query, sequence) pair (int16 path not applicable)
    kIntraTickLong = 3,  // serving: long subjects of the requests admitted in this tick
    kIntraGroups = 4     // group slots [slot_begin, slot_end) of the layout, every query
};

struct IntraParams {
    const uint8_t* plain;       // all sequences, original order
    const int64_t* plain_off;
    const QueryDesc* queries;
    int32_t num_queries;
    int32_t mode;
    const int32_t* long_ids;    // kIntraLong: subject ids, longest first
    int64_t num_long;
    const int32_t* query_order; // query slots, longest first
    int64_t num_seqs;
    const FlagEntry* flags;
    uint32_t flag_cap;
    int32_t alphabet1;
    Control* ctrl;
    int2* spill;                // per resident warp: (H - Goe, F) of the pass boundary row
    int64_t spill_stride;       // int2 per warp slot
    Gaps gaps;
    int32_t qp_add;             // Goe minus the profile's bias (0 unless Goe is too large)
    const TickDesc* tick;       // kIntraTickLong
    const int32_t* perm;        // kIntraGroups: group slot -> sequence id (-1 filler)
    int64_t slot_begin, slot_end;
};

// Packed int16x2 intra-task wavefront kernel (k_wave.cu).  Two int16 lanes per register:
//  * two-query mode (queries != two-subject): one subject per warp against two streams of
//    query passes (pass k of stream a in the low lanes, of stream b in the high lanes; the
//    pass structure is a WavePass list, 32 x rows per lane rows per pass), scores from the
//    paired profile pp;
//  * two-subject mode: one query, the subjects in slots 2t and 2t + 1 of an interleaved group
//    per warp, scores from the query profile qp (two lookups packed by a byte permute).
// One pass of the two-query wavefront.  Each of the two streams (a: low int16 halves, b: high)
// is a chain of queries packed at lane granularity -- a query of m rows takes ceil(m / kTB)
// consecutive lanes -- cut into passes of 32 lanes, so one pass can hold the end of a query,
// whole short queries and the start of the next.
struct WavePass {
    uint32_t first[2];     // bit l: lane l holds row 0 of its query, or no query (zero boundary above)
    uint32_t last[2];      // bit l: lane l holds the last row of its query
    int32_t q[2][32];      // query slot of lane l, -1: none
    int32_t row0[2][32];   // query row of lane l's first row
};

struct WaveParams {
    const uint8_t* plain;       // two-query mode: subjects in original order
    const int64_t* plain_off;
    const int32_t* subjects;    // two-query mode: subject ids, longest first
    int64_t num_subjects;
    const QueryDesc* queries;   // score rows (and the profile in two-subject mode)
    const uint32_t* pp;         // two-query mode: pp[d * rows_pad + k * 32 kTB + l * kTB + r]
    int64_t rows_pad;
    const WavePass* passes;     // two-query mode: the passes of the two streams
    int32_t num_passes;
    int32_t query;              // two-subject mode: the query slot
    const uint8_t* inter;       // two-subject mode: interleaved groups [group_begin, group_end)
    const int64_t* group_off;
    const int32_t* group_len;
    const int32_t* perm;
    int64_t group_begin, group_end;
    int32_t max_group_len;      // two-subject mode: sizes the residue buffers
    const uint8_t* qres;        // two-subject mode: query residues (query q at qres_off[q]),
    const int64_t* qres_off;    //   from which the kernel builds its own profile, with
    const int8_t* matrix;       //   the A x A matrix (device)
    int64_t long_pairs;         // two-subject mode: the longest slot pairs, served first ...
    int32_t long_blocks;        // ... by a few warps of blocks [0, long_blocks)
    int32_t prefix_f;           // first phase: F recurrence unrolled (Goe + rows x Ge' < 2^15)
    int32_t alphabet1;
    Control* ctrl;
    FlagEntry* flags;
    uint32_t flag_cap;
    int32_t thresh;             // int16 saturation threshold: 32767 - max(0, max SM)
    int2* spill;                // per resident warp: pass-boundary row, one int2 per column
    int64_t spill_stride;
    Gaps gaps;
    // (the two-subject fields below come last: placed before alphabet1, which shifts the
    // fields the two-query kernel reads, they cost that kernel 1.6 % on the long-subject mix)
    int64_t half_from;          // two-subject mode: pairs from here on run two per warp item
                                //   on 16-lane wavefronts (kernels built for it)
    int16_t* qp_out;            // two-subject mode, non-null: also write the query's int16
    int32_t qp_mpad;            //   profile (qp_out[d * qp_mpad + i] = SM + qp_bias) for the
    int32_t qp_bias;            //   int32 rescore that follows as a dependent launch
};
constexpr int kWaveRows[3] = {8, 12, 16};   // query rows per lane of the two-query variants
int wave_warps();
size_t wave_smem_bytes(int rows_per_lane, int alphabet1);
int wave_occupancy(int rows_per_lane, int alphabet1);
cudaError_t launch_wave_mq(const WaveParams& p, int rows_per_lane, int grid, cudaStream_t st);
// Paired profile of the two-query wavefront from its pass list (pp of WaveParams).
cudaError_t launch_build_pp_wave(const uint8_t* d_queries, const int64_t* d_qoff,
                                 const WavePass* d_passes, int32_t num_passes, int32_t rows_per_lane,
                                 const int8_t* d_matrix, int32_t A, int32_t bias, uint32_t* d_pp,
                                 int64_t rows_pad, Control* ctrl, cudaStream_t st);
constexpr int kWaveSsRows[2] = {5, 8};  // query rows per lane of the two-subject variants
// Two-subject mode holds the whole query profile in shared memory (one block of
// wave_ss_warps() warps per SM): wave_ss_fits says whether a query of m rows fits.  rows_per_lane
// is the 32-lane wavefronts'; `half`: the bulk's shorter pairs run two 16-lane wavefronts of
// wave_ss_bulk_rows() rows per lane in each warp.
size_t wave_ss_smem_bytes(int rows_per_lane, int alphabet1, int m, int max_group_len, bool half);
int wave_ss_warps();
int wave_ss_blocks_per_sm();
int wave_ss_long_warps();
int wave_ss_bulk_rows();
int wave_ss_bulk_lanes();
bool wave_ss_fits(int rows_per_lane, int alphabet1, int m, int max_group_len, int max_smem, bool half);
// uint16 entries of a warp's residue buffer: dummy columns, the longest group, and the
// columns the wavefront's last lanes read past the end, rounded to 16 bytes
__host__ __device__ constexpr int wave_ss_res_stride(int max_group_len) {
    return (32 + max_group_len + 64 + 7) / 8 * 8;
}
// (spill: two regions per resident warp, one per 16-lane wavefront)
cudaError_t launch_wave_ss(const WaveParams& p, int rows_per_lane, bool half, int m, int grid,
                           cudaStream_t st);

// Launchers (return the CUDA error of the launch).
cudaError_t launch_build_qp(const uint8_t* d_queries, const int64_t* d_qoff, int32_t nq,
                            const int8_t* d_matrix, int32_t A, int32_t bias,
                            const int64_t* d_qp_off, const int32_t* d_mpad, int16_t* d_qp,
                            int64_t max_mpad, Control* ctrl, cudaStream_t st);
// Inter-task kernel variants (rows per strip x warps per block), chosen by the autotuner.
int inter_num_variants();
int inter_variant_rows(int variant);
int inter_variant_warps(int variant);
size_t inter_smem_bytes(int alphabet1);
int inter_occupancy(int variant, int alphabet1);
cudaError_t launch_inter(const InterParams& p, int variant, int grid, cudaStream_t st);
// Score-profile form of the single-query inter-task kernel (32 rows per strip, 4 warps).
int inter_sp_mt_stride();
int inter_sp_warps();
size_t inter_sp_smem_bytes(int alphabet1);
int inter_sp_occupancy(int alphabet1);
cudaError_t launch_inter_sp(const InterParams& p, int grid, cudaStream_t st);
int inter_mq_num_variants();
int inter_mq_variant_rows(int variant);
int inter_mq_variant_warps(int variant);
size_t inter_mq_smem_bytes(int alphabet1);
int inter_mq_occupancy(int variant, int alphabet1);
cudaError_t launch_inter_mq(const InterMqParams& p, int variant, int grid, cudaStream_t st);
// Query q's residues start at d_queries[d_qoff[q]]; its length is d_qlen[q] when d_qlen is
// given, else d_qoff[q + 1] - d_qoff[q].  With `tick`, the step count comes from the device.
cudaError_t launch_build_pp(const uint8_t* d_queries, const int64_t* d_qoff, const int32_t* d_qlen,
                            const MqStep* d_steps, int32_t num_steps, const TickDesc* tick,
                            int32_t rows_per_strip, const int8_t* d_matrix, int32_t A,
                            int32_t bias, uint32_t* d_pp, int64_t rows_pad, Control* ctrl,
                            cudaStream_t st);
cudaError_t launch_intra(const IntraParams& p, int grid, int block, cudaStream_t st);
// The same launch as a programmatic dependent of the kernel launched just before it on `st`: its
// blocks may become resident while that kernel runs and wait (griddepcontrol.wait) for its
// completion and memory before reading anything it wrote.
cudaError_t launch_intra_dependent(const IntraParams& p, int grid, int block, cudaStream_t st);
// Block-shared-profile variant for the kIntraLong and kIntraGroups work sources (4 warps,
// 8 or 16 query rows per lane).
// Query rows per lane of the block int32 kernel's variants (passes of 160, 256 and 512 rows).
constexpr int kIntraBlockRows[3] = {5, 8, 16};
size_t intra_block_smem_bytes(int rows_per_lane, int alphabet1);
int intra_block_warps(int rows_per_lane);
int intra_block_occupancy(int rows_per_lane, int alphabet1);
cudaError_t launch_intra_block(const IntraParams& p, int rows_per_lane, int grid, cudaStream_t st);
int intra_block_threads();
int intra_rows_per_pass();
size_t intra_smem_bytes(int alphabet1);
int intra_occupancy(int alphabet1);

}  // namespace swgb
