// xr_internal.h -- host-side declarations shared by the libxr translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <atomic>

#include <nvtx3/nvToolsExt.h>

#include "xr.h"

namespace xr {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Count one kernel launch (host-side, process-wide).
void count_launch();

// Number of engines (xoshiro256, xoroshiro128, xoroshiro128 for ++, xoshiro128,
// xoroshiro64, xoshiro512, xoroshiro1024) and how many of them (the first
// ones, states of 256 bits or less) have power sets and serve batches.
constexpr int NUM_ENGINES_H = 7;
constexpr int NUM_PSET_ENGINES = 5;

// Largest state of any generator (xoroshiro1024: 16 x 64 bits).
constexpr int XR_MAX_STATE_BYTES = 128;

// Engine of each variant and its state size in bits.
int engine_of(int variant);
int engine_bits(int engine);

// Fill S streams x m outputs, row pitch ld elements (stream-major) or S
// (interleaved).  `encode` may be NULL (plain-store path only).
cudaError_t launch_fill(int variant, int dtype, int layout, void *states, size_t S, size_t m,
                        size_t ld, void *out, int write_back, int *status, cudaStream_t stream,
                        EncodeTiledFn encode);

// Jump tables: tables holds n matrices T^(2^k), k = 0..n-1, each n columns of
// n/32 words.  Built on `stream`.
cudaError_t launch_build_tables(int engine, uint32_t *tables, cudaStream_t stream);

// states[i] <- (prod over t of T^(2^ks[t])) states[i], i < count.
struct KList {
    int n;
    int k[64];
};
cudaError_t launch_apply_pow(int engine, const uint32_t *tables, const KList &ks, void *states,
                             size_t count, cudaStream_t stream);

// Doubling tree: given states[0], fill states[1 .. S-1] with
// states[i] = (T^(2^kbase))^i states[0] using T^(2^(kbase + L)) at level L.
cudaError_t launch_tree(int engine, const uint32_t *tables, int kbase, void *states, size_t S,
                        cudaStream_t stream);

// Power sets for three-level stream starts: per engine, for each jump distance
// 2^d in `dists` and level l < PSET_LEVELS, PSET_SIZE matrices P_l[j] =
// (T^(2^(d + PSET_BITS l)))^j, stored set after set (distance-major).
constexpr int PSET_BITS = 9;
constexpr int PSET_SIZE = 1 << PSET_BITS;
constexpr int PSET_LEVELS = 3;
cudaError_t launch_build_power_sets(int engine, const uint32_t *tables, const int *dists, int ndist,
                                    uint32_t *sets, cudaStream_t stream);
// Given states[0], fill states[1 .. S-1] (S <= 2^(PSET_BITS * PSET_LEVELS))
// with states[i] = (T^(2^d))^i states[0], sets3 = the three sets of distance d.
cudaError_t launch_streams_psets(int engine, const uint32_t *sets3, void *states, size_t S,
                                 cudaStream_t stream);
// Given states[0 .. P-1], fill states[P .. 512 P - 1] with
// states[p + P j] = Q_j states[p], Q = the level-0 power set of distance 2^d P.
cudaError_t launch_streams_jmajor(int engine, const uint32_t *Q, void *states, size_t P, cudaStream_t stream);
// out = (T^(2^d))^e base by one warp through the three power sets of distance
// 2^d (engines with power sets only: 256, 128 or 64 state bits).
cudaError_t launch_warp_jump(int engine, const uint32_t *psets_d, const uint32_t *tables, int d, const void *base,
                             void *out, uint64_t e, cudaStream_t stream);

// SplitMix64 seeding: count states from d_seeds (or from `seed` when d_seeds
// is NULL and count == 1).
cudaError_t launch_seed(int variant, const uint64_t *d_seeds, uint64_t seed, size_t count,
                        void *states, int *status, cudaStream_t stream);

}  // namespace xr

// Jump distances with power sets, per engine: jump, long jump, xr_fill_seq
// segment (2^10), and single steps (2^0, used to advance by any n).
static const int NUM_PSET_DISTS = 4;

// The context (opaque in include/xr.h).
struct xr_ctx {
    int device;
    uint32_t *tables[xr::NUM_ENGINES_H];
    uint32_t *psets[xr::NUM_ENGINES_H];  // NUM_PSET_DISTS x PSET_LEVELS power sets
    int *d_status;
    void *scratch;            // segment start states of xr_fill_seq
    size_t scratch_bytes;
    void *staging[2];         // output staging of xr_fill_host
    void *chunk_states[2];    // stream start states of xr_fill_host
    void *base_state;         // one state (xr_fill_host)
    size_t staging_bytes, chunk_states_bytes;
    cudaStream_t side;        // copy stream of xr_fill_host
    cudaEvent_t ev_gen[2], ev_copy[2];
    xr::EncodeTiledFn encode;
    void *lazy_mutex;         // guards the lazy build of the large engines' tables
    // power sets of further distances 2^d (index d < 256), built on first use
    // by xr_fill_streams: the PSET_LEVELS level sets of that distance
    uint32_t *dist_sets[xr::NUM_ENGINES_H][256];
};

namespace xr {
// Build the jump tables of an engine if it has none yet (large engines are
// built on first use); XR_OK or an error status.
int ensure_engine(xr_ctx *ctx, int engine);
// Index of the power sets of distance log2 d for an engine (-1 if none).
int pset_index(int engine, int d);
// The three level sets of distance index di of an engine.
const uint32_t *pset_sets(const xr_ctx *ctx, int engine, int di);
// The level-0 power set P_0[j] = T^(2^d j), j < 512, of any distance 2^d
// (d < engine bits) of an engine with power sets, built and cached on first
// use (the first use waits for the device); NULL on failure.
const uint32_t *dist_sets(xr_ctx *ctx, int engine, int d);
// The same when already built; otherwise built now unless `st` is capturing
// (NULL then, and nothing is built).
const uint32_t *dist_sets_outside_capture(xr_ctx *ctx, int engine, int d, cudaStream_t st);
// An NVTX range named after the entry point for its duration, so a timeline
// (Nsight Systems, or ncu's NVTX filters) groups each call's launches.  Costs
// a branch when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Makes the context's device current for the duration of an entry point and
// restores the caller's device afterwards (nothing to do when they agree), so
// calls on contexts of different devices need no cudaSetDevice from the caller.
struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int device)
    {
        int cur = -1;
        if (cudaGetDevice(&cur) == cudaSuccess && cur != device && cudaSetDevice(device) == cudaSuccess)
            prev = cur;
    }
    ~DeviceScope()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DeviceScope(const DeviceScope &) = delete;
    DeviceScope &operator=(const DeviceScope &) = delete;
};

// Raises a kernel's dynamic shared-memory limit on the current device once.
// The attribute belongs to the kernel in each device's context, so `done`
// keeps one bit per device; concurrent first calls both set it, harmlessly.
template <typename Kernel>
cudaError_t set_smem_once(std::atomic<uint64_t> &done, Kernel kernel, int bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

}  // namespace xr
