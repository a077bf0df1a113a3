// xr_batch.cu -- many uneven generation requests in one persistent launch.
//
// A request is "the first n outputs of the sequence in state slot s" (the
// semantics of xr_fill_seq).  The host plan cuts every request into segments
// of 2^10 outputs.  Segment q of a request starts at T^(q 2^10) s, computed by
// the three-level power-set scheme (xr_jump.cu), batched over requests.
// Requests with the same (generator, dtype) form a group whose segments are
// numbered consecutively; a warp task is 32 consecutive segments of a group,
// so small requests share warps without divergent code paths.  One persistent
// kernel pulls tasks from a device counter.  The generators with 64- and
// 128-byte states (xoshiro512, xoroshiro1024) have no power sets: their
// segment starts come from a doubling tree batched over their requests, and
// their tasks run in a second instance of the persistent kernel, so the
// kernel of the other generators keeps its registers.  Each lane stages its rows in its
// own shared-memory buffers and writes them with its own bulk copies
// (cp.async.bulk), so lanes of different requests never wait for each other.
#include <algorithm>
#include <stdlib.h>
#include <string.h>
#include <vector>

#include "xr_device.cuh"
#include "xr_f2.cuh"
#include "xr_fill_impl.cuh"
#include "xr_internal.h"
#include "xr_batch_plan.h"

namespace xr {

constexpr int BSEG_LOG2 = 10;            // outputs per segment = 1024
constexpr u64 BSEG = 1ull << BSEG_LOG2;
constexpr int BATCH_NBUF = 2;            // staged rows per lane
constexpr int TILE_BYTES_B = 32 * 128;   // one 32-row x 128-byte tile

struct BatchDev {
    const BReq *reqs;
    const BGroup *groups;
    const u32 *group_reqs;
    const u64 *prefix;
    const u64 *tasks;
    u64 ntasks;
    unsigned long long *counter;
    u32 *segstates;
    unsigned char *slots;
    u32 sw;             // 32-bit words per state slot and per segment state (8, 16 or 32)
    unsigned char *out;
    const u64 *seeds;
    int *status;
    int opt;            // outputs per staged row (per-lane path)
    u32 bufstride;      // bytes between consecutive lanes' buffers
    u32 warpbytes;      // shared memory per warp (1024-byte multiple)
    int rows_ok;        // tensor maps over 1024-element rows are valid
};

constexpr u64 TASK_FULL = 1ull << 63;  // 32 full segments of one row-aligned request

// ---------------------------------------------------------------- seeding / copy-in

// State bytes of a generator (the order of enum xr_variant).
__device__ __forceinline__ int batch_state_bytes(int v)
{
    return v <= 2 ? 32 : v <= 9 ? 16 : v <= 11 ? 8 : v <= 14 ? 64 : 128;
}

// Slot state (or SplitMix64 of the request's seed, also written to the slot)
// becomes segment 0 of the request.  Slots and segment states are d.sw words;
// the words past the state are written as zero.
__global__ void k_batch_seed(BatchDev d, size_t nreq)
{
    const size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nreq) return;
    const BReq q = d.reqs[r];
    uint4 *slot = reinterpret_cast<uint4 *>(d.slots + q.slot * (u64)d.sw * 4u);
    uint4 *dst = q.n > 0 ? reinterpret_cast<uint4 *>(d.segstates + q.seg_base * (u64)d.sw) : nullptr;
    // 64-bit SplitMix64 outputs per state: one per 8 state bytes (32-bit words
    // take each output's low half first, so the u32 words come out in the same
    // order either way)
    const int sb = batch_state_bytes(q.variant), outs = (sb + 7) / 8;
    u64 x = d.seeds ? d.seeds[r] : 0ull;
    u32 any = 0;
    for (u32 k = 0; k < d.sw / 4; ++k) {  // 16 bytes = two SplitMix64 outputs at a time
        u32 w[4];
        if (d.seeds) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const bool used = (int)(2 * k + h) < outs;
                const u64 z = used ? splitmix64_next(x) : 0ull;
                w[2 * h] = (u32)z;
                w[2 * h + 1] = (u32)(z >> 32);
            }
            slot[k] = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
            const uint4 a = (int)(16 * k) < sb ? slot[k] : make_uint4(0u, 0u, 0u, 0u);
            w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
            if ((int)(16 * k + 8) >= sb) w[2] = w[3] = 0u;  // an 8-byte state in a 16-byte piece
        }
        any |= w[0] | w[1] | w[2] | w[3];
        if (dst) dst[k] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    if (!any) atomicCAS(d.status, 0, XR_EZERO_STATE);
}

// ---------------------------------------------------------------- segment starts

// One level of the power-set scheme over many requests:
// segstates[parent + j * stride] = P[j] segstates[parent] when inside the
// request (below `limit`).  One launch serves every engine of the level: the
// x-range of each engine's CTAs is a field of LevelArgs.  A CTA shares j,
// builds the Four-Russians tables of P[j] in shared memory and handles two
// items per thread.  Items come longest first, so a CTA whose first item has
// no child j has nothing to do and leaves before building its tables.
constexpr int BLEVEL_ITEMS_PER_THREAD = 2;
constexpr int BLEVEL_THREADS = 256;

struct LevelEngine {
    const u32 *P;             // the level's power set of this engine's distance
    const BLevelItem *items;  // this engine's items, longest first
    u64 nitems;
    unsigned cta_first;       // first blockIdx.x of this engine
    unsigned maxj;            // largest power-set index in use
    int nw;                   // state words
};
struct LevelArgs {
    LevelEngine e[NUM_PSET_ENGINES];
    int n;
    u32 sw;  // words per segment state
    u64 stride;
};

template <int NW>
__device__ __forceinline__ void batch_level_cta(const LevelEngine &E, unsigned x, int j, u64 stride, u32 sw,
                                                u32 *segstates, u32 *T)
{
    typedef Russians<NW> RT;
    {
        const BLevelItem lead = E.items[(size_t)x * BLEVEL_ITEMS_PER_THREAD * BLEVEL_THREADS];
        if (lead.parent + (u64)j * stride >= lead.limit) return;
    }
    russians_build<NW>(E.P + (size_t)j * RT::n * NW, T);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BLEVEL_ITEMS_PER_THREAD; ++k) {
        const size_t idx = ((size_t)x * BLEVEL_ITEMS_PER_THREAD + k) * BLEVEL_THREADS + threadIdx.x;
        if (idx >= E.nitems) return;
        const BLevelItem it = E.items[idx];
        const u64 child = it.parent + (u64)j * stride;
        if (child >= it.limit) continue;
        // whole 16-byte loads and stores of the first 32 bytes of a segment
        // state (the unused words among them are written as zero)
        u32 v[NW], r[NW];
        const uint4 *ps = reinterpret_cast<const uint4 *>(segstates + it.parent * sw);
        const uint4 a = ps[0];
        v[0] = a.x; v[1] = a.y;
        if constexpr (NW >= 4) { v[2] = a.z; v[3] = a.w; }
        if constexpr (NW == 8) {
            const uint4 b = ps[1];
            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        }
        russians_matvec<NW>(T, v, r);
        uint4 *cs = reinterpret_cast<uint4 *>(segstates + child * sw);
        if constexpr (NW == 8) {
            cs[0] = make_uint4(r[0], r[1], r[2], r[3]);
            cs[1] = make_uint4(r[4], r[5], r[6], r[7]);
        } else if constexpr (NW == 4) {
            cs[0] = make_uint4(r[0], r[1], r[2], r[3]);
            cs[1] = make_uint4(0u, 0u, 0u, 0u);
        } else {
            cs[0] = make_uint4(r[0], r[1], 0u, 0u);
            cs[1] = make_uint4(0u, 0u, 0u, 0u);
        }
    }
}

__global__ void __launch_bounds__(BLEVEL_THREADS) k_batch_level(const LevelArgs a, u32 *segstates)
{
    __shared__ __align__(16) u32 T[Russians<8>::WORDS];
    int k = 0;
    while (k + 1 < a.n && blockIdx.x >= a.e[k + 1].cta_first) ++k;
    const LevelEngine &E = a.e[k];
    const int j = blockIdx.y + 1;
    if ((unsigned)j > E.maxj) return;
    const unsigned x = blockIdx.x - E.cta_first;
    if (E.nw == 8) batch_level_cta<8>(E, x, j, a.stride, a.sw, segstates, T);
    else if (E.nw == 4) batch_level_cta<4>(E, x, j, a.stride, a.sw, segstates, T);
    else batch_level_cta<2>(E, x, j, a.stride, a.sw, segstates, T);
}

// One level of the doubling tree of the engines without power sets: product
// t of the launch belongs to the item k with prefix[k] <= t < prefix[k + 1];
// segment seg_base + half + i = M (segment seg_base + i), i = t - prefix[k].
// M = T^(2^(10 + L)) is read through the read-only cache by every thread in
// the same order (warp-uniform loads).
template <int NW>
__global__ void __launch_bounds__(128)
    k_batch_tree(const u32 *__restrict__ M, const BTreeItem *items, u32 nitems, u64 work, u64 half, u32 sw,
                 u32 *segstates)
{
    const u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= work) return;
    u32 lo = 0, hi = nitems;  // prefix[lo] <= t < prefix[hi] (prefix[nitems] = work)
    while (hi - lo > 1) {
        const u32 mid = (lo + hi) >> 1;
        if (items[mid].prefix <= t) lo = mid;
        else hi = mid;
    }
    const u64 parent = items[lo].seg_base + (t - items[lo].prefix);
    u32 v[NW], r[NW];
    load_vec<NW>(v, segstates + parent * sw);
    f2_matvec<NW, false>(M, v, r);
    store_vec<NW>(r, segstates + (parent + half) * sw);
}

// ---------------------------------------------------------------- persistent fill

__device__ __forceinline__ void bulk_store_s2g(void *gdst, u32 ssrc, u32 bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(ssrc),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ u64 lds_u64(u32 a)
{
    u64 v;
    asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ u32 lds_u32(u32 a)
{
    u32 v;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}

// One lane, one segment: `count` outputs from the state at `st`, written at
// `out`; rows of opt outputs are staged in two shared buffers and written by
// bulk copies (a trailing piece under 16 bytes by plain stores).  With
// `slot` non-null the final state is stored there.
template <int V, int DT>
__device__ __forceinline__ void batch_lane(const u32 *st, unsigned char *slot, unsigned char *out,
                                           u64 count, u32 buf0, u32 bufnext, int opt)
{
    typedef Gen<V> G;
    typedef typename G::E E;
    typedef typename OutElem<DT>::type OT;
    constexpr int ES = (int)sizeof(OT), PER = 16 / ES;
    E e;
    load_state(e, st);
    const int chunks = opt * ES / 16;
    int it = 0;
    for (u64 j0 = 0; j0 < count; j0 += (u64)opt, ++it) {
        const u32 buf = buf0 + (u32)(it & 1) * bufnext;
        if (it >= BATCH_NBUF) bulk_wait_read<BATCH_NBUF - 1>();
        const u64 left = count - j0;
        const int cnt = left < (u64)opt ? (int)left : opt;
        if (cnt == opt) {
            for (int c = 0; c < chunks; ++c) {
                u32 w[4];
                gen16<G, DT>(e, w);
                st_shared_v4(buf + (u32)c * 16u, w[0], w[1], w[2], w[3]);
            }
        } else {
            for (int c = 0; c * PER < cnt; ++c) {
                u32 w[4];
                gen16_partial<G, DT>(e, w, cnt - c * PER);
                st_shared_v4(buf + (u32)c * 16u, w[0], w[1], w[2], w[3]);
            }
        }
        fence_proxy_async_shared();
        const u32 bytes = (u32)cnt * ES, full = bytes & ~15u;
        unsigned char *dst = out + j0 * ES;
        if (full) {
            bulk_store_s2g(dst, buf, full);
            bulk_commit();
        }
        for (u32 b = full; b < bytes; b += ES) {
            if (ES == 8) *reinterpret_cast<u64 *>(dst + b) = lds_u64(buf + b);
            else *reinterpret_cast<u32 *>(dst + b) = lds_u32(buf + b);
        }
    }
    bulk_wait_read<0>();
    if (slot) store_state(e, slot);
}

// Wait until at most n (1..7) committed bulk groups still read shared memory;
// the count must be an immediate, so each depth has its own instruction.
__device__ __forceinline__ void bulk_wait_read_n(int n)
{
    switch (n) {
    case 1: bulk_wait_read<1>(); break;
    case 2: bulk_wait_read<2>(); break;
    case 3: bulk_wait_read<3>(); break;
    case 4: bulk_wait_read<4>(); break;
    case 5: bulk_wait_read<5>(); break;
    case 6: bulk_wait_read<6>(); break;
    default: bulk_wait_read<7>(); break;
    }
}

// A warp whose 32 lanes hold 32 consecutive full segments of one request:
// the segments are 32 consecutive 1024-element rows of the arena, written as
// 32-row x 128-byte tiles by 2D TMA stores, exactly like the bulk fill.
// `ntiles` (2..8) tiles rotate, so up to ntiles stores are in flight.
template <int V, int DT>
__device__ __forceinline__ void batch_warp_rows(const u32 *st, unsigned char *slot, const CUtensorMap *map,
                                                int row0, u32 tiles, int ntiles, int lane)
{
    typedef Gen<V> G;
    typedef typename G::E E;
    constexpr int COLS = 128 / (int)sizeof(typename OutElem<DT>::type);
    E e;
    load_state(e, st);
    int it = 0, k = 0;
    for (int j0 = 0; j0 < (int)BSEG; j0 += COLS, ++it) {
        const u32 tile = tiles + (u32)(k * TILE_BYTES_B);
        k = k + 1 == ntiles ? 0 : k + 1;
        if (it >= ntiles) {
            if (lane == 0) bulk_wait_read_n(ntiles - 1);
            __syncwarp();
        }
        fill_tile_row<G, DT>(e, tile, lane, (size_t)COLS, true, st, (size_t)j0);  // st is read only here
        fence_proxy_async_shared();
        __syncwarp();
        if (lane == 0) {
            tma_store_2d(map, tile, j0, row0);
            bulk_commit();
        }
    }
    if (lane == 0) bulk_wait_read<0>();
    __syncwarp();
    if (slot) store_state(e, slot);
}

#define XR_BATCH_CASE(V, DT)                                                              \
    case (V) * 4 + (DT):                                                                  \
        if (full) batch_warp_rows<V, DT>(st, slot, (DT == DT_U32 || DT == DT_F32) ? &map32 : &map64, row0, tiles, ntiles, lane); \
        else batch_lane<V, DT>(st, slot, out, count, buf0, bufnext, d.opt);               \
        break;

// LARGE = false: the generators with states of up to 32 bytes (0 .. 11);
// LARGE = true: xoshiro512 and xoroshiro1024 (12 .. 17).
template <bool LARGE>
__global__ void __launch_bounds__(512)
    k_batch_fill(BatchDev d, const __grid_constant__ CUtensorMap map64, const __grid_constant__ CUtensorMap map32)
{
    extern __shared__ unsigned char bsmem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const u32 wbase = ((smem_addr(bsmem) + 1023u) & ~1023u) + (u32)warp * d.warpbytes;
    const u32 tiles = wbase;                       // 4 KiB tiles (full tasks)
    // full tasks rotate as many tiles as the warp's share holds (at most 8)
    const int ntiles = (int)min(8u, d.warpbytes / (u32)TILE_BYTES_B);
    const u32 buf0 = wbase + (u32)lane * d.bufstride;  // per-lane rows (other tasks)
    const u32 bufnext = 32u * d.bufstride;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(d.counter, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= d.ntasks) break;
        const u64 code = d.tasks[t];
        const bool full = (code & TASK_FULL) && d.rows_ok;
        const BGroup g = d.groups[(code & ~TASK_FULL) >> 40];
        const u64 s = (code & ((1ull << 40) - 1)) * 32 + (u64)lane;
        if (s >= g.nseg) continue;  // never taken by full tasks
        const u64 *pre = d.prefix + g.prefix_first;
        u32 lo = 0, hi = g.nreq;  // pre[lo] <= s < pre[hi]
        while (hi - lo > 1) {
            const u32 mid = (lo + hi) >> 1;
            if (pre[mid] <= s) lo = mid;
            else hi = mid;
        }
        const BReq q = d.reqs[d.group_reqs[g.req_first + lo]];
        const u64 seg = s - pre[lo];
        const u64 start = seg << BSEG_LOG2;
        const u64 count = (q.n - start) < BSEG ? (q.n - start) : BSEG;
        const u32 *st = d.segstates + (q.seg_base + seg) * (u64)d.sw;
        unsigned char *slot = (start + count == q.n) ? d.slots + q.slot * (u64)d.sw * 4u : nullptr;
        const int es = (g.dtype == DT_U64 || g.dtype == DT_F64) ? 8 : 4;
        unsigned char *out = d.out + q.out_offset + start * (u64)es;
        const int row0 = (int)(q.out_offset / (BSEG * (u64)es) + seg - (u64)lane);
        if constexpr (LARGE) {
            switch (g.variant * 4 + g.dtype) {
                XR_BATCH_CASE(12, DT_U64) XR_BATCH_CASE(12, DT_F64) XR_BATCH_CASE(12, DT_F32)
                XR_BATCH_CASE(13, DT_U64) XR_BATCH_CASE(13, DT_F64) XR_BATCH_CASE(13, DT_F32)
                XR_BATCH_CASE(14, DT_U64) XR_BATCH_CASE(14, DT_F64) XR_BATCH_CASE(14, DT_F32)
                XR_BATCH_CASE(15, DT_U64) XR_BATCH_CASE(15, DT_F64) XR_BATCH_CASE(15, DT_F32)
                XR_BATCH_CASE(16, DT_U64) XR_BATCH_CASE(16, DT_F64) XR_BATCH_CASE(16, DT_F32)
                XR_BATCH_CASE(17, DT_U64) XR_BATCH_CASE(17, DT_F64) XR_BATCH_CASE(17, DT_F32)
            default:
                break;
            }
            continue;
        }
        switch (g.variant * 4 + g.dtype) {
            XR_BATCH_CASE(0, DT_U64) XR_BATCH_CASE(0, DT_F64) XR_BATCH_CASE(0, DT_F32)
            XR_BATCH_CASE(1, DT_U64) XR_BATCH_CASE(1, DT_F64) XR_BATCH_CASE(1, DT_F32)
            XR_BATCH_CASE(2, DT_U64) XR_BATCH_CASE(2, DT_F64) XR_BATCH_CASE(2, DT_F32)
            XR_BATCH_CASE(3, DT_U64) XR_BATCH_CASE(3, DT_F64) XR_BATCH_CASE(3, DT_F32)
            XR_BATCH_CASE(4, DT_U64) XR_BATCH_CASE(4, DT_F64) XR_BATCH_CASE(4, DT_F32)
            XR_BATCH_CASE(5, DT_U64) XR_BATCH_CASE(5, DT_F64) XR_BATCH_CASE(5, DT_F32)
            XR_BATCH_CASE(6, DT_U32) XR_BATCH_CASE(6, DT_F64) XR_BATCH_CASE(6, DT_F32)
            XR_BATCH_CASE(7, DT_U32) XR_BATCH_CASE(7, DT_F64) XR_BATCH_CASE(7, DT_F32)
            XR_BATCH_CASE(8, DT_U32) XR_BATCH_CASE(8, DT_F64) XR_BATCH_CASE(8, DT_F32)
            XR_BATCH_CASE(9, DT_U64) XR_BATCH_CASE(9, DT_F64) XR_BATCH_CASE(9, DT_F32)
            XR_BATCH_CASE(10, DT_U32) XR_BATCH_CASE(10, DT_F64) XR_BATCH_CASE(10, DT_F32)
            XR_BATCH_CASE(11, DT_U32) XR_BATCH_CASE(11, DT_F64) XR_BATCH_CASE(11, DT_F32)
        default:
            break;
        }
    }
    bulk_wait_all<0>();
}
#undef XR_BATCH_CASE

}  // namespace xr

using namespace xr;

// ---------------------------------------------------------------- host side: plans

namespace xr {

static int es_of(int dtype) { return (dtype == XR_U64 || dtype == XR_F64) ? 8 : 4; }
static bool word32(int v) { return (v >= 6 && v <= 8) || v == 10 || v == 11; }
static bool dtype_ok_b(int v, int dt)
{
    if (dt == XR_F64 || dt == XR_F32) return true;
    if (dt == XR_U64) return !word32(v);
    if (dt == XR_U32) return word32(v);
    return false;
}

unsigned int slot_words_of(int variant)
{
    const int b = xr_state_bytes(variant);
    return b <= 32 ? 8u : (unsigned)b / 4u;
}

int check_requests(const xr_request *h, size_t nreq)
{
    std::vector<u64> slots;
    slots.reserve(nreq);
    for (size_t r = 0; r < nreq; ++r) {
        const xr_request &q = h[r];
        if (q.variant < 0 || q.variant >= XR_NUM_VARIANTS || !dtype_ok_b(q.variant, q.dtype)) return XR_EINVAL;
        if (q.out_offset % 16) return XR_EINVAL;
        if (q.n > (1ull << 50)) return XR_EINVAL;
        slots.push_back(q.slot);
    }
    std::sort(slots.begin(), slots.end());
    for (size_t i = 1; i < slots.size(); ++i)
        if (slots[i] == slots[i - 1]) return XR_EINVAL;
    return XR_OK;
}

// O(requests + tasks): tasks are 32-segment windows of each group; a window
// lying inside the full segments of one row-aligned request is a full task.
// Full tasks go first; the others follow by their longest lane, longest first.
void build_plan(const xr_request *in, size_t nreq, HostPlan &p)
{
    p.reqs.resize(nreq);
    p.groups.clear();
    p.group_reqs.clear();
    p.prefix.clear();
    p.tasks.clear();
    p.items.clear();
    p.levels.clear();
    p.titems.clear();
    p.trees.clear();
    p.slot_words = 8;
    u64 segs = 0, arena = 0, maxslot = 0;
    for (size_t r = 0; r < nreq; ++r) {
        BReq &q = p.reqs[r];
        q.n = in[r].n;
        q.out_offset = in[r].out_offset;
        q.slot = in[r].slot;
        q.seg_base = segs;
        q.variant = in[r].variant;
        q.dtype = in[r].dtype;
        segs += (q.n + BSEG - 1) / BSEG;
        arena = std::max<u64>(arena, q.out_offset + q.n * (u64)es_of(q.dtype));
        maxslot = std::max<u64>(maxslot, q.slot);
        p.slot_words = std::max(p.slot_words, slot_words_of(q.variant));
    }
    p.nseg = segs;
    p.arena_bytes = arena;
    p.max_slot = maxslot;

    std::vector<u32> bucket[XR_NUM_VARIANTS * 4];
    for (size_t r = 0; r < nreq; ++r)
        if (p.reqs[r].n) bucket[p.reqs[r].variant * 4 + p.reqs[r].dtype].push_back((u32)r);
    // partial tasks by longest lane; [1] for the large generators
    std::vector<u64> partial[2][BSEG + 1];
    std::vector<u64> full_tasks[2];
    for (int bi = 0; bi < XR_NUM_VARIANTS * 4; ++bi) {
        if (bucket[bi].empty()) continue;
        const int big = engine_of(bi / 4) >= NUM_PSET_ENGINES ? 1 : 0;
        BGroup g;
        g.variant = bi / 4;
        g.dtype = bi % 4;
        g.nreq = (u32)bucket[bi].size();
        g.req_first = (u32)p.group_reqs.size();
        g.prefix_first = p.prefix.size();
        u64 acc = 0;
        for (u32 r : bucket[bi]) {
            p.group_reqs.push_back(r);
            p.prefix.push_back(acc);
            acc += (p.reqs[r].n + BSEG - 1) / BSEG;
        }
        p.prefix.push_back(acc);
        g.nseg = acc;
        const u64 gi = p.groups.size();
        p.groups.push_back(g);
        const u64 T = (acc + 31) / 32, rowbytes = BSEG * (u64)es_of(g.dtype);
        std::vector<unsigned short> len(T, 0);
        std::vector<char> full(T, 0);
        u64 pre = 0;
        for (u32 r : bucket[bi]) {
            const BReq &q = p.reqs[r];
            const u64 P = (q.n + BSEG - 1) / BSEG, fullseg = q.n / BSEG, last = q.n - (P - 1) * BSEG;
            if (q.out_offset % rowbytes == 0) {
                const u64 t0 = (pre + 31) / 32, t1 = (pre + fullseg) / 32;
                for (u64 t = t0; t < t1; ++t) full[t] = 1;
            }
            for (u64 t = pre / 32; t <= (pre + P - 1) / 32; ++t) {
                const u64 lo = std::max<u64>(pre, t * 32);
                const u64 l = lo < pre + fullseg ? BSEG : last;
                if (l > len[t]) len[t] = (unsigned short)l;
            }
            pre += P;
        }
        for (u64 t = 0; t < T; ++t) {
            if (full[t]) full_tasks[big].push_back((gi << 40) | t | TASK_FULL);
            else partial[big][len[t]].push_back((gi << 40) | t);
        }
    }
    for (int big = 0; big < 2; ++big) {
        p.tasks.insert(p.tasks.end(), full_tasks[big].begin(), full_tasks[big].end());
        for (int l = (int)BSEG; l >= 0; --l)
            p.tasks.insert(p.tasks.end(), partial[big][l].begin(), partial[big][l].end());
        if (big == 0) p.ntasks_small = p.tasks.size();
    }

    // levels of the segment-start scheme, per (level, engine)
    for (int l = PSET_LEVELS - 1; l >= 0; --l) {
        const u64 stride = 1ull << (PSET_BITS * l), span = stride << PSET_BITS;
        for (int e = 0; e < NUM_PSET_ENGINES; ++e) {
            LevelLaunch L;
            L.engine = e;
            L.level = l;
            L.first = p.items.size();
            for (size_t r = 0; r < nreq; ++r) {
                if (engine_of(p.reqs[r].variant) != e) continue;
                const u64 P = (p.reqs[r].n + BSEG - 1) / BSEG;
                if (P <= stride) continue;
                for (u64 k = 0; k * span < P; ++k)
                    p.items.push_back({p.reqs[r].seg_base + k * span, p.reqs[r].seg_base + P});
            }
            L.count = p.items.size() - L.first;
            if (!L.count) continue;
            std::sort(p.items.begin() + L.first, p.items.end(), [](const BLevelItem &a, const BLevelItem &b) {
                return a.limit - a.parent > b.limit - b.parent;
            });
            const u64 kids = (p.items[L.first].limit - p.items[L.first].parent + stride - 1) / stride;
            L.maxj = (unsigned)std::min<u64>(kids - 1, PSET_SIZE - 1);
            p.levels.push_back(L);
        }
    }
    // doubling-tree levels of the engines without power sets
    for (int e = NUM_PSET_ENGINES; e < NUM_ENGINES_H; ++e) {
        for (int L = 0; L < 64; ++L) {
            const u64 half = 1ull << L;
            TreeLaunch t;
            t.engine = e;
            t.level = L;
            t.first = p.titems.size();
            u64 work = 0;
            for (size_t r = 0; r < nreq; ++r) {
                if (engine_of(p.reqs[r].variant) != e) continue;
                const u64 P = (p.reqs[r].n + BSEG - 1) / BSEG;
                if (P <= half) continue;
                p.titems.push_back({p.reqs[r].seg_base, work});
                work += std::min<u64>(half, P - half);
            }
            t.count = p.titems.size() - t.first;
            t.work = work;
            if (!t.count) break;
            p.trees.push_back(t);
        }
    }
}

void free_devplan(DevPlan &d)
{
    cudaFree(d.blob);
    cudaFreeHost(d.pinned);
    cudaFree(d.segstates);
    cudaFree(d.counter);
    d = DevPlan();
}

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Copy the plan to the device: all arrays in one blob, one asynchronous copy
// from pinned memory.  Buffers grow (after waiting for `st`) only when a plan
// is larger than any before; the pinned blob is reused, so the caller must
// not upload again before this copy has completed.
cudaError_t upload_plan(const HostPlan &p, DevPlan &d, cudaStream_t st, const void *extra, size_t extra_bytes)
{
    d.off_reqs = 0;
    d.off_groups = up256(d.off_reqs + p.reqs.size() * sizeof(BReq));
    d.off_group_reqs = up256(d.off_groups + p.groups.size() * sizeof(BGroup));
    d.off_prefix = up256(d.off_group_reqs + p.group_reqs.size() * sizeof(u32));
    d.off_tasks = up256(d.off_prefix + p.prefix.size() * sizeof(u64));
    d.off_items = up256(d.off_tasks + p.tasks.size() * sizeof(u64));
    d.off_titems = up256(d.off_items + p.items.size() * sizeof(BLevelItem));
    d.off_extra = up256(d.off_titems + p.titems.size() * sizeof(BTreeItem));
    d.off_counter = up256(d.off_extra + extra_bytes);
    const size_t total = d.off_counter + 256;
    cudaError_t err = cudaSuccess;
    if (total > d.blob_cap) {
        err = cudaStreamSynchronize(st);
        cudaFree(d.blob);
        cudaFreeHost(d.pinned);
        d.blob = d.pinned = nullptr;
        d.blob_cap = 0;
        const size_t cap = total + total / 2;
        if (err == cudaSuccess) err = cudaMalloc((void **)&d.blob, cap);
        if (err == cudaSuccess) err = cudaMallocHost((void **)&d.pinned, cap);
        if (err != cudaSuccess) return err;
        d.blob_cap = cap;
    }
    const size_t segbytes = (size_t)p.nseg * p.slot_words * 4;
    if (segbytes > d.seg_cap) {
        err = cudaStreamSynchronize(st);
        cudaFree(d.segstates);
        d.segstates = nullptr;
        d.seg_cap = 0;
        if (err == cudaSuccess) err = cudaMalloc((void **)&d.segstates, segbytes);
        if (err != cudaSuccess) return err;
        d.seg_cap = segbytes;
    }
    if (!d.counter) {  // two task counters: the small and the large generators
        err = cudaMalloc((void **)&d.counter, 2 * sizeof(unsigned long long));
        if (err != cudaSuccess) return err;
    }
    auto put = [&](size_t off, const void *src, size_t bytes) {
        if (bytes) memcpy(d.pinned + off, src, bytes);
    };
    put(d.off_reqs, p.reqs.data(), p.reqs.size() * sizeof(BReq));
    put(d.off_groups, p.groups.data(), p.groups.size() * sizeof(BGroup));
    put(d.off_group_reqs, p.group_reqs.data(), p.group_reqs.size() * sizeof(u32));
    put(d.off_prefix, p.prefix.data(), p.prefix.size() * sizeof(u64));
    put(d.off_tasks, p.tasks.data(), p.tasks.size() * sizeof(u64));
    put(d.off_items, p.items.data(), p.items.size() * sizeof(BLevelItem));
    put(d.off_titems, p.titems.data(), p.titems.size() * sizeof(BTreeItem));
    put(d.off_extra, extra, extra_bytes);
    memset(d.pinned + d.off_counter, 0, 2 * sizeof(unsigned long long));
    return cudaMemcpyAsync(d.blob, d.pinned, total, cudaMemcpyHostToDevice, st);
}

static u32 bufstride_for(int opt) { return (u32)(opt * 8 + 16); }
// Per warp: two 32 x 128-byte tiles (full tasks) or 32 lanes x two staged
// rows (other tasks), whichever is larger, in 1024-byte units.  Full tasks
// then rotate as many tiles as that share holds.
static u32 warpbytes_for(int opt)
{
    const u32 rows = (u32)BATCH_NBUF * 32u * bufstride_for(opt);
    const u32 w = rows > 2u * TILE_BYTES_B ? rows : 2u * TILE_BYTES_B;
    return (w + 1023u) & ~1023u;
}
size_t batch_smem_bytes(int opt, int block) { return (size_t)(block / 32) * warpbytes_for(opt) + 1024; }

// Enqueue one run of an uploaded plan on `st` (also under stream capture):
// reset the task counter, seed or copy in segment 0 of every request, the
// segment-start levels, then the persistent fill.  `rows_bytes` is the size
// of the output allocation the row tensor maps may cover.
cudaError_t enqueue_plan(xr_ctx *ctx, const HostPlan &p, DevPlan &dp, const uint64_t *d_seeds, void *d_slots,
                         void *d_out, u64 rows_bytes, int opt, int block, cudaStream_t st, bool round_ready)
{
    BatchDev d;
    d.reqs = (const BReq *)(dp.blob + dp.off_reqs);
    d.groups = (const BGroup *)(dp.blob + dp.off_groups);
    d.group_reqs = (const u32 *)(dp.blob + dp.off_group_reqs);
    d.prefix = (const u64 *)(dp.blob + dp.off_prefix);
    d.tasks = (const u64 *)(dp.blob + dp.off_tasks);
    const BLevelItem *items = (const BLevelItem *)(dp.blob + dp.off_items);
    const BTreeItem *titems = (const BTreeItem *)(dp.blob + dp.off_titems);
    d.ntasks = p.ntasks_small;
    d.counter = round_ready ? reinterpret_cast<unsigned long long *>(dp.blob + dp.off_counter) : dp.counter;
    d.segstates = dp.segstates;
    d.sw = p.slot_words;
    d.slots = (unsigned char *)d_slots;
    d.out = (unsigned char *)d_out;
    d.seeds = reinterpret_cast<const u64 *>(d_seeds);
    d.status = ctx->d_status;
    d.opt = opt;
    d.bufstride = bufstride_for(opt);
    d.warpbytes = warpbytes_for(opt);
    // tensor maps over the output as 1024-element rows: encoded again only
    // when the output allocation changes
    if (dp.maps_out != d_out || dp.maps_rows_bytes != rows_bytes) {
        memset(dp.maps, 0, sizeof(dp.maps));
        dp.maps_ok = 0;
        if (ctx->encode && d_out && ((uintptr_t)d_out % 16) == 0) {
            dp.maps_ok = 1;
            for (int k = 0; k < 2; ++k) {
                const u64 es = k == 0 ? 8 : 4, rows = rows_bytes / (BSEG * es);
                if (rows == 0) continue;
                if (rows >= (1ull << 31)) {
                    dp.maps_ok = 0;
                    continue;
                }
                const cuuint64_t dims[2] = {(cuuint64_t)BSEG, (cuuint64_t)rows};
                const cuuint64_t strides[1] = {(cuuint64_t)(BSEG * es)};
                const cuuint32_t box[2] = {(cuuint32_t)(128 / es), 32u};
                const cuuint32_t estr[2] = {1u, 1u};
                if (ctx->encode(&dp.maps[k], k == 0 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32,
                                2, d_out, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                    dp.maps_ok = 0;
            }
        }
        dp.maps_out = d_out;
        dp.maps_rows_bytes = rows_bytes;
    }
    d.rows_ok = dp.maps_ok;
    const size_t nreq = p.reqs.size();
    if (nreq == 0) return cudaSuccess;
    cudaError_t err = cudaSuccess;
    if (!round_ready) {
        err = cudaMemsetAsync(dp.counter, 0, 2 * sizeof(unsigned long long), st);
        if (err != cudaSuccess) return err;
        k_batch_seed<<<(unsigned)((nreq + 127) / 128), 128, 0, st>>>(d, nreq);
        count_launch();
        err = cudaGetLastError();
    }
    // one launch per level, every engine of the level in it (p.levels is
    // ordered by level, highest first)
    for (size_t i = 0; i < p.levels.size() && err == cudaSuccess;) {
        LevelArgs a;
        a.n = 0;
        a.sw = p.slot_words;
        a.stride = 1ull << (PSET_BITS * p.levels[i].level);
        unsigned ctas = 0, maxj = 0;
        const size_t per_cta = (size_t)BLEVEL_THREADS * BLEVEL_ITEMS_PER_THREAD;
        const int level = p.levels[i].level;
        for (; i < p.levels.size() && p.levels[i].level == level; ++i) {
            const LevelLaunch &L = p.levels[i];
            const int n = engine_bits(L.engine);
            const size_t set_words = (size_t)PSET_SIZE * n * (n / 32);
            LevelEngine &E = a.e[a.n++];
            E.P = pset_sets(ctx, L.engine, pset_index(L.engine, BSEG_LOG2)) + (size_t)L.level * set_words;
            E.items = items + L.first;
            E.nitems = L.count;
            E.cta_first = ctas;
            E.maxj = L.maxj;
            E.nw = n / 32;
            ctas += (unsigned)((L.count + per_cta - 1) / per_cta);
            maxj = std::max(maxj, L.maxj);
        }
        k_batch_level<<<dim3(ctas, maxj), BLEVEL_THREADS, 0, st>>>(a, dp.segstates);
        count_launch();
        err = cudaGetLastError();
    }
    // doubling-tree levels of xoshiro512 / xoroshiro1024 (in level order)
    for (size_t i = 0; i < p.trees.size() && err == cudaSuccess; ++i) {
        const TreeLaunch &L = p.trees[i];
        const int n = engine_bits(L.engine);
        const u32 *M = ctx->tables[L.engine] + (size_t)((BSEG_LOG2 + L.level) % n) * n * (n / 32);
        const unsigned grid = (unsigned)((L.work + 127) / 128);
        if (n == 512)
            k_batch_tree<16><<<grid, 128, 0, st>>>(M, titems + L.first, (u32)L.count, L.work, 1ull << L.level,
                                                   p.slot_words, dp.segstates);
        else
            k_batch_tree<32><<<grid, 128, 0, st>>>(M, titems + L.first, (u32)L.count, L.work, 1ull << L.level,
                                                   p.slot_words, dp.segstates);
        count_launch();
        err = cudaGetLastError();
    }
    if (err != cudaSuccess || p.tasks.empty()) return err;
    const size_t smem = batch_smem_bytes(opt, block);
    const u64 warps_per_block = (u64)block / 32;
    // the persistent fill of the small generators, then of the large ones
    for (int big = 0; big < 2 && err == cudaSuccess; ++big) {
        const u64 first = big ? p.ntasks_small : 0, ntasks = big ? p.tasks.size() - p.ntasks_small : p.ntasks_small;
        if (!ntasks) continue;
        BatchDev db = d;
        db.tasks = d.tasks + first;
        db.ntasks = ntasks;
        db.counter = d.counter + big;
        auto kern = big ? k_batch_fill<true> : k_batch_fill<false>;
        static std::atomic<uint64_t> attr[2];
        err = set_smem_once(attr[big], kern, 227 * 1024);
        if (err != cudaSuccess) return err;
        int &occ_opt = big ? dp.occ_large_opt : dp.occ_opt, &occ_block = big ? dp.occ_large_block : dp.occ_block;
        int &occ_per_sm = big ? dp.occ_large_per_sm : dp.occ_per_sm;
        if (occ_opt != opt || occ_block != block) {  // occupancy per configuration, once
            int per_sm = 0, sms = 0;
            err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem);
            if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
            if (err != cudaSuccess) return err;
            if (per_sm < 1) return cudaErrorInvalidConfiguration;
            occ_opt = opt;
            occ_block = block;
            occ_per_sm = per_sm;
            dp.occ_sms = sms;
        }
        const u64 grid = std::min<u64>((u64)occ_per_sm * dp.occ_sms, (ntasks + warps_per_block - 1) / warps_per_block);
        kern<<<(unsigned)grid, block, smem, st>>>(db, dp.maps[0], dp.maps[1]);
        count_launch();
        err = cudaGetLastError();
    }
    return err;
}

}  // namespace xr

using namespace xr;

// ---------------------------------------------------------------- the public batch

struct xr_batch {
    xr_ctx *ctx = nullptr;
    HostPlan plan;
    DevPlan dev;
    int opt = 16, block = 128;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void *g_seeds = nullptr, *g_slots = nullptr, *g_out = nullptr;
    int g_opt = 0, g_block = 0;
    cudaStream_t cap = nullptr;
    void *d_slot_backup = nullptr;
    size_t slot_backup_bytes = 0;
};

static int st_of(cudaError_t e)
{
    if (e == cudaSuccess) return XR_OK;
    if (e == cudaErrorMemoryAllocation) return XR_ENOMEM;
    return XR_ECUDA;
}

extern "C" int xr_batch_destroy(xr_batch *b)
{
    if (!b) return XR_OK;
    DeviceScope dscope(b->ctx->device);
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    free_devplan(b->dev);
    cudaFree(b->d_slot_backup);
    delete b;
    return XR_OK;
}

extern "C" int xr_batch_create(xr_ctx *ctx, const xr_request *h_reqs, size_t nreq, xr_batch **out)
{
    if (!ctx || !out || (nreq && !h_reqs)) return XR_EINVAL;
    *out = nullptr;
    const int rc = check_requests(h_reqs, nreq);
    if (rc != XR_OK) return rc;
    DeviceScope dscope(ctx->device);
    for (size_t r = 0; r < nreq; ++r) {  // the large engines' tables are built on first use
        const int erc = ensure_engine(ctx, engine_of(h_reqs[r].variant));
        if (erc != XR_OK) return erc;
    }
    xr_batch *b = new xr_batch();
    b->ctx = ctx;
    build_plan(h_reqs, nreq, b->plan);
    cudaError_t err = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = upload_plan(b->plan, b->dev, b->cap);
    if (err == cudaSuccess) err = cudaStreamSynchronize(b->cap);
    if (err != cudaSuccess) {
        xr_batch_destroy(b);
        return st_of(err);
    }
    *out = b;
    return XR_OK;
}

extern "C" uint64_t xr_batch_arena_bytes(const xr_batch *b) { return b ? b->plan.arena_bytes : 0; }
extern "C" uint64_t xr_batch_tasks(const xr_batch *b) { return b ? (uint64_t)b->plan.tasks.size() : 0; }
extern "C" uint64_t xr_batch_slot_bytes(const xr_batch *b) { return b ? (uint64_t)b->plan.slot_words * 4u : 0; }

extern "C" int xr_batch_set_config(xr_batch *b, int opt, int block)
{
    if (!b) return XR_EINVAL;
    if (opt != 4 && opt != 8 && opt != 16 && opt != 32 && opt != 64) return XR_EINVAL;
    if (block != 128 && block != 256 && block != 512) return XR_EINVAL;
    if (batch_smem_bytes(opt, block) > 227 * 1024) return XR_EINVAL;
    b->opt = opt;
    b->block = block;
    return XR_OK;
}

extern "C" int xr_batch_get_config(const xr_batch *b, int *opt, int *block)
{
    if (!b || !opt || !block) return XR_EINVAL;
    *opt = b->opt;
    *block = b->block;
    return XR_OK;
}

static cudaError_t batch_enqueue(xr_batch *b, const uint64_t *d_seeds, void *d_slots, void *d_out, cudaStream_t st)
{
    return enqueue_plan(b->ctx, b->plan, b->dev, d_seeds, d_slots, d_out, b->plan.arena_bytes, b->opt, b->block, st);
}

extern "C" int xr_batch_run(xr_batch *b, const uint64_t *d_seeds, void *d_slots, void *d_out, int use_graph,
                            void *stream)
{
    if (!b) return XR_EINVAL;
    if (b->plan.reqs.empty()) return XR_OK;
    DeviceScope dscope(b->ctx->device);
    NvtxRange nvtx("xr_batch_run");
    if (!d_slots || ((uintptr_t)d_slots % 16)) return XR_EINVAL;
    if (b->plan.arena_bytes && (!d_out || ((uintptr_t)d_out % 16))) return XR_EINVAL;
    const cudaStream_t st = (cudaStream_t)stream;
    if (!use_graph) return st_of(batch_enqueue(b, d_seeds, d_slots, d_out, st));
    if (!b->exec || b->g_seeds != d_seeds || b->g_slots != d_slots || b->g_out != d_out || b->g_opt != b->opt ||
        b->g_block != b->block) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        cudaError_t err = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (err != cudaSuccess) return st_of(err);
        cudaError_t e1 = batch_enqueue(b, d_seeds, d_slots, d_out, b->cap);
        err = cudaStreamEndCapture(b->cap, &b->graph);
        if (e1 != cudaSuccess) return st_of(e1);
        if (err != cudaSuccess) return st_of(err);
        err = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (err != cudaSuccess) return st_of(err);
        b->g_seeds = d_seeds;
        b->g_slots = d_slots;
        b->g_out = d_out;
        b->g_opt = b->opt;
        b->g_block = b->block;
    }
    return st_of(cudaGraphLaunch(b->exec, st));
}

extern "C" int xr_batch_tune(xr_batch *b, const uint64_t *d_seeds, void *d_slots, void *d_out, void *stream,
                             float *best_ms)
{
    if (!b || !d_slots) return XR_EINVAL;
    DeviceScope dscope(b->ctx->device);
    NvtxRange nvtx("xr_batch_tune");
    const cudaStream_t st = (cudaStream_t)stream;
    const size_t nbytes = (size_t)(b->plan.max_slot + 1) * b->plan.slot_words * 4;
    cudaError_t err = cudaSuccess;
    if (b->slot_backup_bytes < nbytes) {
        cudaFree(b->d_slot_backup);
        b->d_slot_backup = nullptr;
        err = cudaMalloc(&b->d_slot_backup, nbytes);
        if (err != cudaSuccess) return st_of(err);
        b->slot_backup_bytes = nbytes;
    }
    err = cudaMemcpyAsync(b->d_slot_backup, d_slots, nbytes, cudaMemcpyDeviceToDevice, st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int opts[5] = {4, 8, 16, 32, 64}, blocks[3] = {128, 256, 512};
    float best = 1e30f;
    int bo = b->opt, bb = b->block;
    for (int oi = 0; oi < 5 && err == cudaSuccess; ++oi)
        for (int bi = 0; bi < 3 && err == cudaSuccess; ++bi) {
            if (batch_smem_bytes(opts[oi], blocks[bi]) > 227 * 1024) continue;
            b->opt = opts[oi];
            b->block = blocks[bi];
            float ms = 1e30f;
            for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {
                err = cudaMemcpyAsync(d_slots, b->d_slot_backup, nbytes, cudaMemcpyDeviceToDevice, st);
                if (err == cudaSuccess) err = cudaEventRecord(e0, st);
                if (err == cudaSuccess) err = batch_enqueue(b, d_seeds, d_slots, d_out, st);
                if (err == cudaSuccess) err = cudaEventRecord(e1, st);
                if (err == cudaSuccess) err = cudaEventSynchronize(e1);
                float t = 0;
                if (err == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0) ms = std::min(ms, t);  // the first repetition warms up
            }
            if (err == cudaSuccess && ms < best) {
                best = ms;
                bo = opts[oi];
                bb = blocks[bi];
            }
        }
    b->opt = bo;
    b->block = bb;
    if (err == cudaSuccess) err = cudaMemcpyAsync(d_slots, b->d_slot_backup, nbytes, cudaMemcpyDeviceToDevice, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms) *best_ms = best;
    return st_of(err);
}
