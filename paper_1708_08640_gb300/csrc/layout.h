// Host-side layout build of the S3CMTF path: the items (tensor entries and coupled-matrix
// entries) are visited in a given order and cut into groups (minibatches, HOGWILD tiles or
// gradient chunks).  Inside each group, the occurrences of every factor row are sorted by
// row into segments, so that the device can sum a row's gradients in a fixed order
// (minibatch, gradient) or combine them in shared memory before one atomic (HOGWILD).
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

namespace s3 {

struct HostInput {
    int N = 0, M = 0;
    int64_t I[4] = {};
    int cmode[8] = {};
    int64_t K[8] = {};
    int64_t nnz = 0;
    const int32_t* idx[4] = {};
    const float* val = nullptr;
    int64_t ynnz[8] = {};
    const int32_t* yr[8] = {};
    const int32_t* yc[8] = {};
    const float* yv[8] = {};   // nullptr: all ones
};

enum GroupRule {
    RULE_UNION = 0,    // consecutive runs of `size` items of the order (minibatches, chunks)
    RULE_TENSOR = 1    // runs holding `size` tensor entries each (HOGWILD tiles)
};
enum PosKind {
    POS_SLOT = 0,      // an event's position is its slot (sorted position) in the group
    POS_SEG = 1        // an event's position is its segment (row) index in the group
};

struct HostGrouping {
    int pos_kind = POS_SLOT;
    int long_thr = 0;          // > 0 (POS_SLOT only): each group lists its segments of more than
    int huge_thr = 0;          // huge_thr events first, then those of more than long_thr, then
                               // the others, each class in row order (huge_thr 0: no huge class)
    int64_t ngroups = 0;
    int nF = 0;
    std::vector<int64_t> t_off;
    std::vector<int32_t> tidx[4];
    std::vector<float> tval;
    std::vector<int32_t> tpos[4];
    std::vector<int64_t> t_src;
    std::vector<int64_t> c_off[8];
    std::vector<int32_t> cr[8], cc[8];
    std::vector<float> cval[8];
    std::vector<int32_t> cpos_u[8], cpos_v[8];
    std::vector<int64_t> c_src[8];
    std::vector<int64_t> seg_off[12], slot_off[12];
    std::vector<int32_t> seg_row[12], seg_start[12], seg_cnt[12];
    std::vector<int32_t> seg_nlong[12];   // [groups] segments of more than long_thr events
    std::vector<int32_t> seg_nhuge[12];   // [groups] segments of more than huge_thr events
    int64_t max_t = 0;
    int64_t max_c[8] = {};
    int64_t max_seg[12] = {};
    int64_t max_ev[12] = {};
};

// order: n_union items (nullptr = identity order).  Items k < nnz are tensor entries,
// then the entries of coupled matrix 0, 1, ...  Returns an empty string on success.
// long_thr, huge_thr: see HostGrouping.
std::string build_grouping(const HostInput& in, const int64_t* order, int64_t n_union, int rule,
                           int64_t size, int pos_kind, HostGrouping& out, int long_thr = 0,
                           int huge_thr = 0);

// The visiting order derived from a seed: items sorted by a counter-based 64-bit key
// (splitmix64 of seed and item, stream 63), ties by item.
void seeded_order(uint64_t seed, int64_t n, std::vector<int64_t>& order);

}  // namespace s3
