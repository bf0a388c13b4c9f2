// Host interface of the grouped multi-pair cell-grouped pose path (rs_group.cu).
#pragma once

#include <vector>

#include "rs_common.cuh"

namespace rs {

// One pair's consecutive poses inside a chunk.
struct GroupSeg {
    int pair;            // index into the pair-descriptor array
    int pc;              // poses
    long long p0;        // first pose (index within the pair)
    int pose_off;        // first chunk pose
    int cell_base;       // first record key of this segment's cells
    long long atom_off;  // first chunk pose-atom
};

struct GroupChunk {
    int seg_begin, seg_end;  // segments [seg_begin, seg_end) of the plan
    int npose;
    long long natom;
    int nkey;                // cells (sum over segments of n - 1)
    int ksub;                // sort sub-buckets per cell (a power of two <= 32)
};

// Chunks and segments of the pairs `members` (all Tucker-reduced, one padded rank).
struct GroupPlan {
    int RP = 0;
    std::vector<GroupSeg> segs;
    std::vector<GroupChunk> chunks;
    size_t scratch = 0;      // device bytes one chunk needs
};

rs_status group_plan(const std::vector<PairDesc>& pairs, const std::vector<int>& members, long long max_atoms,
                     GroupPlan* out);
// Enqueues every chunk of the plan on `st`.  d_pairs and d_segs are device copies of
// the pair descriptors and of plan.segs; ws holds at least plan.scratch bytes; wpb is
// the warps per CTA of the W-form kernel (4 or 8).
rs_status group_launch(const GroupPlan& plan, const PairDesc* d_pairs, const GroupSeg* d_segs, void* ws,
                       size_t ws_bytes, int wpb, cudaStream_t st, bool events);

}  // namespace rs
