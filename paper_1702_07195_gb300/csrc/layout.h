// Host-side preprocessing stage (paper Section 4): database sequences are sorted by length
// in ascending order, cut into groups of 64 (one warp's lanes) and interleaved so that a
// thread's two sequences advance together, 16 bytes per 8 columns; the tail of each shorter
// sequence is padded with a dummy code.  Sequences longer than a cutoff are listed apart for
// the intra-task kernel.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace swgb {

struct Layout {
    int64_t num_seqs = 0;
    int64_t num_groups = 0;
    int64_t inter_bytes = 0;
    int32_t max_group_len = 0;   // padded columns of the longest group
    int32_t max_len = 0;         // longest sequence overall
    int64_t short_residues = 0;  // residues covered by the interleaved groups
    std::vector<int64_t> group_off;
    std::vector<int32_t> group_len;   // columns of the group's storage (multiple of 8)
    std::vector<int32_t> group_cols;  // columns the kernels sweep: longest member, rounded to 2
    std::vector<int64_t> group_res;   // real residues per group
    std::vector<int32_t> perm;      // num_groups * 64, -1 for fillers
    std::vector<int32_t> long_ids;  // longest first
};

// Validates `offsets` and computes the grouping.  Returns an empty string or an error.
std::string plan_layout(const int64_t* offsets, int64_t num_seqs, int32_t long_cutoff,
                        Layout& out);

// Checks every residue code against the alphabet (parallel).  Returns the index of the first
// bad residue or -1.
int64_t find_bad_code(const uint8_t* residues, int64_t count, int32_t alphabet_size);

// Writes the interleaved residues of all groups into `inter` (layout.inter_bytes bytes).
void fill_inter(const uint8_t* residues, const int64_t* offsets, int32_t alphabet_size,
                const Layout& layout, uint8_t* inter);

}  // namespace swgb
