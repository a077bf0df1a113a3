// xr_batch_plan.h -- host plans of batched requests (shared by the batch API
// and the server): the request table, the (generator, dtype) groups, the warp
// tasks and the segment-start level lists, and their device copies.
#pragma once

#include <vector>

#include "xr_internal.h"

namespace xr {

typedef unsigned long long u64_t;

struct BReq {
    u64_t n, out_offset, slot, seg_base;
    int variant, dtype;
};

struct BGroup {
    int variant, dtype;
    unsigned int nreq, req_first;
    u64_t nseg, prefix_first;
};

struct BLevelItem {
    u64_t parent, limit;  // parent segment index (absolute) and end of its request's segments
};

// Items of one launch are sorted by the segments they span, longest first;
// maxj is the largest power-set index any of them uses.
struct LevelLaunch {
    int engine, level;
    size_t first, count;
    unsigned int maxj;
};

// Segment starts of the engines without power sets (xoshiro512,
// xoroshiro1024) by a doubling tree over every such request at once: at
// level L, segment 2^L + i of a request is T^(2^(10 + L)) applied to segment
// i, for i < min(2^L, P - 2^L).  An item is one request's work at a level;
// `prefix` numbers the work of the launch's items consecutively.
struct BTreeItem {
    u64_t seg_base, prefix;
};
struct TreeLaunch {
    int engine, level;
    size_t first, count;  // items
    u64_t work;           // products in the launch
};

struct HostPlan {
    std::vector<BReq> reqs;
    std::vector<BGroup> groups;
    std::vector<unsigned int> group_reqs;
    std::vector<u64_t> prefix;
    std::vector<u64_t> tasks;
    std::vector<BLevelItem> items;
    std::vector<LevelLaunch> levels;
    std::vector<BTreeItem> titems;
    std::vector<TreeLaunch> trees;
    u64_t nseg = 0, arena_bytes = 0, max_slot = 0;
    // Tasks [0, ntasks_small) are of the generators with states up to 32
    // bytes, the rest of xoshiro512 / xoroshiro1024 (a kernel of their own).
    u64_t ntasks_small = 0;
    // 32-bit words per state slot and per segment state: 8 (states up to 32
    // bytes), 16 (xoshiro512) or 32 (xoroshiro1024), by the largest state in
    // the plan.
    unsigned int slot_words = 8;
};

// Device copy of a plan: one blob (arrays at 256-byte aligned offsets), the
// segment-state scratch and the task counter; a pinned host blob of the same
// layout feeds one asynchronous copy per upload.
struct DevPlan {
    unsigned char *blob = nullptr, *pinned = nullptr;
    size_t blob_cap = 0;
    unsigned int *segstates = nullptr;
    size_t seg_cap = 0;
    unsigned long long *counter = nullptr;
    size_t off_reqs = 0, off_groups = 0, off_group_reqs = 0, off_prefix = 0, off_tasks = 0, off_items = 0;
    size_t off_titems = 0;
    size_t off_extra = 0, off_counter = 0;  // caller's records; two task counters uploaded as zero
    // launch facts reused while the output allocation and the configuration
    // stay the same (a server runs every round on one arena)
    CUtensorMap maps[2];
    const void *maps_out = nullptr;
    u64_t maps_rows_bytes = 0;
    int maps_ok = 0;
    int occ_opt = 0, occ_block = 0, occ_per_sm = 0, occ_sms = 0;
    int occ_large_opt = 0, occ_large_block = 0, occ_large_per_sm = 0;
};

int check_requests(const xr_request *h, size_t nreq);
// Slot words (8, 16 or 32) of a generator's state, and of a set of requests.
unsigned int slot_words_of(int variant);
void build_plan(const xr_request *in, size_t nreq, HostPlan &p);
// `extra` (extra_bytes, may be empty) is copied into the blob at d.off_extra
// with the plan, and a zeroed task counter at d.off_counter.
cudaError_t upload_plan(const HostPlan &p, DevPlan &d, cudaStream_t st, const void *extra = nullptr,
                        size_t extra_bytes = 0);
void free_devplan(DevPlan &d);
size_t batch_smem_bytes(int opt, int block);
// round_ready: the plan was just uploaded (its counter is zero) and segment 0
// of every request already holds the request's start state, so neither the
// counter reset nor the seed step is enqueued.
cudaError_t enqueue_plan(xr_ctx *ctx, const HostPlan &p, DevPlan &dp, const uint64_t *d_seeds, void *d_slots,
                         void *d_out, u64_t rows_bytes, int opt, int block, cudaStream_t st,
                         bool round_ready = false);

}  // namespace xr
