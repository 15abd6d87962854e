// Internal read-only view of a loaded database (for translation units other than the
// runtime that owns sw_db).
#pragma once

#include <cstdint>

#include "../../include/swgb.h"

namespace swgb {

struct DbView {
    int device;
    int sms;
    int32_t alphabet;
    int64_t num_seqs;
    int64_t num_residues;
    int64_t short_residues;
    int64_t num_groups;
    int32_t max_group_len;
    int32_t max_len;
    int64_t num_long;
    int32_t flag_cap;
    int inter_occ;
    int intra_occ;
    const uint8_t* inter;
    const int64_t* group_off;
    const int32_t* group_len;
    const int32_t* group_cols;
    const int32_t* perm;
    const uint8_t* plain;
    const int64_t* plain_off;
    const int32_t* long_ids;
};

bool db_view(const sw_db* db, DbView* v);
sw_status set_last_error(sw_status st, const char* msg);
void add_launches(int64_t n);

}  // namespace swgb
