// Shared-memory layout of a wavefront kernel's profile slice (the rows of one pass, 32 lanes
// x kTB rows per lane, one 32-bit word per row and residue code), used by the int32 block
// kernel and the packed int16x2 wavefront kernel.
//
// In one step the 32 lanes read the rows of 32 different residues, so with a plain row-major
// slice the bank a lane hits depends on its residue and the 16-byte loads of a quarter-warp
// collide at random.  Here the row stride of a residue is a multiple of 32 words (the residue
// no longer moves the bank) and lane l's chunk of kTB words sits at a lane-dependent offset
// chosen so that the 8 lanes of every quarter-warp start in 8 different 16-byte bank groups.
// With an odd number of rows per lane the chunks are packed (lane l at word kTB * l) and read
// with 4-byte loads: kTB * l mod 32 is then a permutation of the banks.  Two-word chunks (also
// read with 4-byte loads) put lanes 16..31 one word further, on the odd banks.
#pragma once

#include "swgb_device.cuh"

namespace swgb {

// Word offset of lane `lane`'s chunk of kTB rows inside one residue's slice row.  Chunks are
// w = kTB / 4 bank groups (16 bytes each) wide and packed in w segments of 32 / w chunks, each
// segment one group further along than a packed layout would put it; the lane -> (segment,
// chunk) map gives the 8 lanes of a quarter-warp 8 distinct starting groups modulo 8.
// kTB: an odd count (4-byte loads), a multiple of 4 with an odd number of 16-byte groups
// (12: lane l at group 3 l, and 3 l mod 8 is a permutation of a quarter-warp's groups), or 8 or
// 16 (the segment layout below).
template <int kTB>
__host__ __device__ constexpr int chunk_offset(int lane) {
    if constexpr (kTB == 2) {   // 4-byte loads: lanes 16..31 one word further, onto the odd banks
        return 2 * lane + (lane >> 4);
    } else if constexpr (kTB % 2 == 1 || (kTB % 4 == 0 && (kTB / 4) % 2 == 1)) {
        return kTB * lane;
    } else {
        constexpr int w = kTB / 4;
        constexpr int per_q = 8 / w;               // lanes of a quarter-warp per segment
        const int q = lane >> 3, i = lane & 7;
        const int seg = i / per_q, c = q * per_q + i % per_q;
        return 4 * (33 * seg + w * c);
    }
}

// Words per residue row of the slice: the span of the chunks rounded up to 32 words.
template <int kTB>
__host__ __device__ constexpr int slice_stride() {
    if constexpr (kTB == 2)
        return (2 * kWarp + 1 + 31) / 32 * 32;
    else if constexpr (kTB % 2 == 1 || (kTB % 4 == 0 && (kTB / 4) % 2 == 1))
        return (kTB * kWarp + 31) / 32 * 32;
    else
        return (4 * (33 * (kTB / 4) - 1) + 31) / 32 * 32;
}

template <int kTB>
constexpr bool chunks_conflict_free() {
    bool ok = slice_stride<kTB>() % 32 == 0;   // the residue does not move the bank
    if (kTB % 2 == 1 || kTB == 2) {
        for (int k = 0; k < kTB; ++k) {        // 4-byte loads: one bank per lane
            unsigned long long seen = 0;
            for (int l = 0; l < kWarp; ++l) seen |= 1ull << ((chunk_offset<kTB>(l) + k) % 32);
            ok = ok && seen == 0xFFFFFFFFull;
        }
    } else {
        for (int q = 0; q < 4; ++q) {          // 16-byte loads: 8 groups per quarter-warp
            unsigned seen = 0;
            for (int i = 0; i < 8; ++i) {
                const int off = chunk_offset<kTB>(8 * q + i);
                ok = ok && off % 4 == 0;
                seen |= 1u << ((off / 4) % 8);
            }
            ok = ok && seen == 0xFFu;
        }
    }
    for (int l = 0; l < kWarp; ++l)            // chunks lie inside the row, disjoint
        for (int m = 0; m < kWarp; ++m) {
            const int a = chunk_offset<kTB>(l), b = chunk_offset<kTB>(m);
            ok = ok && a + kTB <= slice_stride<kTB>();
            ok = ok && (l == m || a >= b + kTB || b >= a + kTB);
        }
    return ok;
}
static_assert(chunks_conflict_free<1>() && chunks_conflict_free<2>() && chunks_conflict_free<3>() &&
                  chunks_conflict_free<4>() && chunks_conflict_free<5>() &&
                  chunks_conflict_free<8>() && chunks_conflict_free<12>() && chunks_conflict_free<16>(),
              "profile slice layout");

}  // namespace swgb
