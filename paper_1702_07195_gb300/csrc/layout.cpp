#include "layout.h"

#include <algorithm>
#include <atomic>
#include <cstring>
#include <thread>

namespace swgb {

namespace {

constexpr int kGroup = 64;
constexpr int kChunkBytes = 512;   // 8 columns x 32 threads x 2 lanes

int worker_count(int64_t work) {
    unsigned hw = std::thread::hardware_concurrency();
    if (hw == 0) hw = 4;
    int64_t n = std::min<int64_t>(hw, 32);
    n = std::min<int64_t>(n, std::max<int64_t>(1, work / (1 << 16)));
    return static_cast<int>(std::max<int64_t>(1, n));
}

template <class F>
void parallel_for(int64_t n, F&& fn) {
    const int w = worker_count(n);
    if (w <= 1) {
        fn(0, n);
        return;
    }
    std::vector<std::thread> th;
    const int64_t step = (n + w - 1) / w;
    for (int t = 0; t < w; ++t) {
        const int64_t lo = t * step, hi = std::min(n, lo + step);
        if (lo >= hi) break;
        th.emplace_back([&fn, lo, hi] { fn(lo, hi); });
    }
    for (auto& x : th) x.join();
}

}  // namespace

std::string plan_layout(const int64_t* offsets, int64_t num_seqs, int32_t long_cutoff,
                        Layout& out) {
    if (num_seqs < 0) return "num_seqs < 0";
    if (num_seqs > (int64_t{1} << 31) - kGroup) return "num_seqs too large (max 2^31 - 64)";
    if (!offsets) return "offsets is null";
    if (offsets[0] != 0) return "offsets[0] must be 0";
    if (long_cutoff <= 0 || long_cutoff % 8 != 0) return "long_cutoff must be a positive multiple of 8";
    out = Layout();
    out.num_seqs = num_seqs;
    int32_t max_len = 0;
    for (int64_t k = 0; k < num_seqs; ++k) {
        const int64_t len = offsets[k + 1] - offsets[k];
        if (len < 0) return "offsets must be non-decreasing";
        if (len > (int64_t{1} << 30)) return "sequence longer than 2^30 residues";
        max_len = std::max<int32_t>(max_len, static_cast<int32_t>(len));
    }
    out.max_len = max_len;
    // Stable counting sort of the short sequences by length (ascending).
    std::vector<int64_t> count(static_cast<size_t>(long_cutoff) + 2, 0);
    int64_t n_short = 0;
    for (int64_t k = 0; k < num_seqs; ++k) {
        const int64_t len = offsets[k + 1] - offsets[k];
        if (len <= long_cutoff) {
            ++count[static_cast<size_t>(len) + 1];
            ++n_short;
        } else {
            out.long_ids.push_back(static_cast<int32_t>(k));
        }
    }
    for (size_t i = 1; i < count.size(); ++i) count[i] += count[i - 1];
    std::vector<int32_t> order(static_cast<size_t>(n_short));
    for (int64_t k = 0; k < num_seqs; ++k) {
        const int64_t len = offsets[k + 1] - offsets[k];
        if (len <= long_cutoff) order[static_cast<size_t>(count[static_cast<size_t>(len)]++)] =
            static_cast<int32_t>(k);
    }
    std::stable_sort(out.long_ids.begin(), out.long_ids.end(), [offsets](int32_t a, int32_t b) {
        return offsets[a + 1] - offsets[a] > offsets[b + 1] - offsets[b];
    });
    out.num_groups = (n_short + kGroup - 1) / kGroup;
    out.group_off.resize(static_cast<size_t>(out.num_groups));
    out.group_len.resize(static_cast<size_t>(out.num_groups));
    out.group_cols.resize(static_cast<size_t>(out.num_groups));
    out.group_res.assign(static_cast<size_t>(out.num_groups), 0);
    out.perm.assign(static_cast<size_t>(out.num_groups * kGroup), -1);
    int64_t off = 0;
    for (int64_t g = 0; g < out.num_groups; ++g) {
        const int64_t lo = g * kGroup, hi = std::min(n_short, lo + kGroup);
        int64_t glen = 0;
        for (int64_t s = lo; s < hi; ++s) {
            const int32_t id = order[static_cast<size_t>(s)];
            out.perm[static_cast<size_t>(s)] = id;
            glen = std::max(glen, offsets[id + 1] - offsets[id]);
            out.short_residues += offsets[id + 1] - offsets[id];
            out.group_res[static_cast<size_t>(g)] += offsets[id + 1] - offsets[id];
        }
        out.group_cols[static_cast<size_t>(g)] = static_cast<int32_t>((glen + 1) / 2 * 2);
        glen = (glen + 7) / 8 * 8;
        out.group_len[static_cast<size_t>(g)] = static_cast<int32_t>(glen);
        out.group_off[static_cast<size_t>(g)] = off;
        off += glen * kGroup;   // 64 bytes per column
        out.max_group_len = std::max<int32_t>(out.max_group_len, static_cast<int32_t>(glen));
    }
    out.inter_bytes = off;
    return std::string();
}

int64_t find_bad_code(const uint8_t* residues, int64_t count, int32_t alphabet_size) {
    std::atomic<int64_t> first{-1};
    parallel_for(count, [&](int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i) {
            if (residues[i] >= alphabet_size) {
                int64_t cur = first.load();
                while ((cur < 0 || i < cur) && !first.compare_exchange_weak(cur, i)) {
                }
                return;
            }
        }
    });
    return first.load();
}

void fill_inter(const uint8_t* residues, const int64_t* offsets, int32_t alphabet_size,
                const Layout& L, uint8_t* inter) {
    const uint8_t dummy = static_cast<uint8_t>(alphabet_size);
    parallel_for(L.num_groups * 64, [&](int64_t lo, int64_t hi) {
        // work unit: one group (units are groups * 64 so the split has enough granularity)
        for (int64_t g = lo / 64; g < (hi + 63) / 64 && g < L.num_groups; ++g) {
            if (g * 64 < lo) continue;   // the group belongs to the previous range
            const int64_t glen = L.group_len[static_cast<size_t>(g)];
            uint8_t* base = inter + L.group_off[static_cast<size_t>(g)];
            for (int s = 0; s < kGroup; ++s) {
                const int32_t id = L.perm[static_cast<size_t>(g * kGroup + s)];
                const uint8_t* src = id >= 0 ? residues + offsets[id] : nullptr;
                const int64_t len = id >= 0 ? offsets[id + 1] - offsets[id] : 0;
                const int t = s >> 1, lane = s & 1;
                for (int64_t j = 0; j < glen; ++j) {
                    base[(j >> 3) * kChunkBytes + t * 16 + (j & 7) * 2 + lane] =
                        j < len ? src[j] : dummy;
                }
            }
        }
    });
}

}  // namespace swgb
