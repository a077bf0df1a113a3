// xr_fill_impl.cuh -- bulk generation kernels (engine step + scrambler +
// conversion + store), instantiated per generator by xr_fill_*.cu.
//
// One thread owns one stream: its state stays in registers for the whole call
// and it emits the stream's outputs in order (next() = scramble the current
// state, then step; Sec. 2).  Stream-major output (out[i * ld + j]) makes each
// thread write its own row, so rows are staged per warp in shared memory as a
// 32-row x 128-byte tile in the 128-byte swizzled layout and written by one
// TMA tile store (cp.async.bulk.tensor.2d) per tile; two tiles per warp let
// the warp generate the next tile while the previous one drains.  Rows and
// columns past the tensor's extent are clipped by the TMA unit, so ragged S
// and m need no extra code.  Output shapes TMA cannot describe take the
// plain-store path (same staging, then warp-wide stores); the interleaved
// layout (out[j * S + i]) is already coalesced and stores directly.
#pragma once

#include "xr_device.cuh"
#include "xr_internal.h"

namespace xr {

constexpr int FILL_WARPS = 4;          // warps per CTA (plain-store path)
constexpr int FILL_NBUF = 2;           // shared-memory tiles per warp (plain-store path)
constexpr int TILE_BYTES = 32 * 128;   // 32 rows x 128 bytes
constexpr int FILL_SMEM = FILL_WARPS * FILL_NBUF * TILE_BYTES + 1024;  // + alignment slack

// Tile-store path: warps per CTA and tiles in flight per warp, by how much
// integer work a byte costs.  The store pattern alone (nothing generated)
// reaches 7.49 TB/s with 1 warp x 8 tiles, 7.35 with 2 x 6 and 7.02 with 1 x
// 3; with the generation included, measured on GB300 per output class:
//   - native words without a multiplying scrambler, and every output of the
//     32-bit generators, leave the ALU and FMA pipes idle enough for the
//     deepest queue: 8 tiles x 1 warp;
//   - native words of the 64-bit * and ** generators need the warps: 6 tiles
//     x 2 warps (1 x 8 measured 3 % slower for xoshiro256**);
//   - the exact doubles of the 64-bit + generators: 6 tiles x 1 warp (2-3 %
//     faster than the classes below, which were 3-11 % slower with it for
//     ++ and **);
//   - the other exact doubles of 128-bit states: 4 tiles x 2 warps; of
//     256-bit states, and every output of xoshiro512 (whose 8-word step is the
//     costliest; the 16-word xoroshiro1024 step touches only 3 words): 3 tiles
//     x 1 warp, the most CTAs per SM.
// Short rows (at most FILL_SHORT_TILES tiles, so a warp lives only a few
// tiles) take 4 warps x 2 tiles instead: there the warps per SM count, not the
// depth of the store queue.
constexpr int FILL_SHORT_TILES = 4;

// Generators whose scrambler multiplies (* and **), and whose scrambler is +.
constexpr bool fill_mul_scrambler(int v)
{
    return v == 2 || v == 5 || v == 7 || v == 9 || v == 10 || v == 11 || v == 14 || v == 15 || v == 17;
}
constexpr bool fill_plus_scrambler(int v) { return v == 0 || v == 3 || v == 8 || v == 12; }

template <int V, int DT, bool SHORT>
struct FillCfg {
    static constexpr bool word64 = sizeof(typename Gen<V>::word) == 8;
    static constexpr bool f64w = DT == DT_F64 && word64;
    static constexpr bool e512 = Gen<V>::E::NBITS == 512;
    static constexpr bool heavy = (f64w && Gen<V>::E::NBITS >= 256) || e512;
    static constexpr bool deep = !e512 && !f64w && !(word64 && fill_mul_scrambler(V));
    static constexpr bool plus_f64 = !e512 && f64w && fill_plus_scrambler(V);
    static constexpr int WARPS = SHORT ? 4 : (deep || plus_f64 || heavy) ? 1 : 2;
    static constexpr int NBUF = SHORT ? 2 : deep ? 8 : plus_f64 ? 6 : heavy ? 3 : (f64w ? 4 : 6);
    static constexpr int SMEM = WARPS * NBUF * TILE_BYTES + 1024;
};

// The double (x >> 11) * 2^-53 of a 64-bit output whose high word is nonzero,
// with no branch: unit_f64_bits without its rare case.  `hmin` collects the
// high words; a row whose smallest high word is zero (x < 2^32, probability
// 2^-32 per value) is regenerated with the exact conversion (redo_row_f64).
__device__ __forceinline__ u64 unit_f64_bits_hi(u64 x, u32 &hmin)
{
    u32 lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(x));
    hmin = min(hmin, hi);
    const u32 vl = __funnelshift_r(lo, hi, 11);
    const u32 vh = hi >> 11;
    const u32 lz = (u32)__clz(hi);  // 32 when hi == 0; that row is replaced
    const u32 mh = __funnelshift_l(vl, vh, lz) + ((1021u - lz) << 20);
    u32 ml;
    asm("shl.b32 %0, %1, %2;" : "=r"(ml) : "r"(vl), "r"(lz));  // 0 for a shift of 32
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(ml), "r"(mh));
    return r;
}

// Regenerate this lane's f64 row at column j0 with the exact conversion: the
// stream's start state (still in global memory until write-back) stepped j0
// times.  Taken about once per 2^32 values.
template <typename G>
static __device__ __noinline__ void redo_row_f64(u32 row, u32 sw, const void *state0, size_t j0)
{
    typename G::E e;
    load_state(e, state0);
    for (size_t j = 0; j < j0; ++j) e.step();
#pragma unroll 1
    for (int c = 0; c < 8; ++c) {
        u32 w[4];
        gen16<G, DT_F64>(e, w);
        st_shared_v4(row + (((u32)c ^ sw) << 4), w[0], w[1], w[2], w[3]);
    }
}

// Generate one 32 x 128 B tile row for this lane into the swizzled tile:
// 16-byte chunk c of row r lives at r * 128 + ((c ^ (r & 7)) * 16), so the 8
// lanes of each quarter-warp hit 8 different bank groups.  Full f64 rows of
// 64-bit generators take the branch-free conversion and the row check above;
// `state0` and `j0` locate the row for the rare redo (live lanes only).
template <typename G, int DT>
__device__ __forceinline__ void fill_tile_row(typename G::E &e, u32 tile, int lane, size_t left, bool live,
                                              const void *state0, size_t j0)
{
    typedef typename OutElem<DT>::type OT;
    constexpr int COLS = 128 / (int)sizeof(OT);
    constexpr int PER = 16 / (int)sizeof(OT);
    const u32 row = tile + (u32)lane * 128u;
    const u32 sw = (u32)(lane & 7);
    if (left >= (size_t)COLS) {
        if constexpr (DT == DT_F64 && sizeof(typename G::word) == 8) {
            u32 hmin = 0xffffffffu;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                u32 w[4];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const u64 o = unit_f64_bits_hi((u64)G::out(e), hmin);
                    e.step();
                    w[2 * q] = (u32)o;
                    w[2 * q + 1] = (u32)(o >> 32);
                }
                st_shared_v4(row + (((u32)c ^ sw) << 4), w[0], w[1], w[2], w[3]);
            }
            if (__builtin_expect(hmin == 0u, 0) && live) redo_row_f64<G>(row, sw, state0, j0);
        } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                u32 w[4];
                gen16<G, DT>(e, w);
                st_shared_v4(row + (((u32)c ^ sw) << 4), w[0], w[1], w[2], w[3]);
            }
        }
    } else {
        const int cnt = (int)left;
        for (int c = 0; c < 8; ++c) {
            u32 w[4];
            gen16_partial<G, DT>(e, w, cnt - c * PER);
            st_shared_v4(row + (((u32)c ^ sw) << 4), w[0], w[1], w[2], w[3]);
        }
    }
}

template <int V, int DT, bool SHORT>
__global__ void __launch_bounds__(FillCfg<V, DT, SHORT>::WARPS * 32)
    k_fill_tma(const __grid_constant__ CUtensorMap map, void *states, size_t S, size_t m,
               int write_back, int *status)
{
    typedef Gen<V> G;
    typedef typename G::E E;
    typedef FillCfg<V, DT, SHORT> CF;
    constexpr int COLS = 128 / (int)sizeof(typename OutElem<DT>::type);
    extern __shared__ unsigned char dyn_smem[];
    const u32 base = (smem_addr(dyn_smem) + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t row0 = ((size_t)blockIdx.x * CF::WARPS + warp) * 32;
    if (row0 >= S) return;
    const size_t i = row0 + lane;
    const bool live = i < S;
    E e;
    if (live) {
        load_state(e, (const char *)states + i * sizeof(e.s));
        if (state_is_zero(e)) atomicCAS(status, 0, XR_EZERO_STATE);
    } else {
#pragma unroll
        for (int j = 0; j < E::K; ++j) e.s[j] = 0;
    }
    const u32 tiles = base + (u32)(warp * CF::NBUF * TILE_BYTES);
    int it = 0;
    for (size_t j0 = 0; j0 < m; j0 += COLS, ++it) {
        const u32 tile = tiles + (u32)((it % CF::NBUF) * TILE_BYTES);
        if (it >= CF::NBUF) {
            if (lane == 0) bulk_wait_read<CF::NBUF - 1>();
            __syncwarp();
        }
        fill_tile_row<G, DT>(e, tile, lane, m - j0, live, (const char *)states + i * sizeof(e.s), j0);
        fence_proxy_async_shared();
        __syncwarp();
        if (lane == 0) {
            tma_store_2d(&map, tile, (int)j0, (int)row0);
            bulk_commit();
        }
    }
    if (lane == 0) bulk_wait_read<0>();  // the tiles may be released; the writes land by the grid's end
    if (write_back && live) store_state(e, (char *)states + i * sizeof(e.s));
}

__device__ __forceinline__ u64 ld_shared_u64(u32 a)
{
    u64 v;
    asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ u32 ld_shared_u32(u32 a)
{
    u32 v;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}

// Same staging, then the warp writes its tile with element stores: any pitch,
// any element-aligned pointer.
template <int V, int DT>
__global__ void __launch_bounds__(FILL_WARPS * 32)
    k_fill_plain(void *states, size_t S, size_t m, size_t ld,
                 typename OutElem<DT>::type *__restrict__ out, int write_back, int *status)
{
    typedef Gen<V> G;
    typedef typename G::E E;
    typedef typename OutElem<DT>::type OT;
    constexpr int ES = (int)sizeof(OT);
    constexpr int COLS = 128 / ES;
    extern __shared__ unsigned char dyn_smem[];
    const u32 base = (smem_addr(dyn_smem) + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t row0 = ((size_t)blockIdx.x * FILL_WARPS + warp) * 32;
    if (row0 >= S) return;
    const size_t i = row0 + lane;
    const bool live = i < S;
    E e;
    if (live) {
        load_state(e, (const char *)states + i * sizeof(e.s));
        if (state_is_zero(e)) atomicCAS(status, 0, XR_EZERO_STATE);
    } else {
#pragma unroll
        for (int j = 0; j < E::K; ++j) e.s[j] = 0;
    }
    const u32 tile = base + (u32)(warp * FILL_NBUF * TILE_BYTES);
    for (size_t j0 = 0; j0 < m; j0 += COLS) {
        fill_tile_row<G, DT>(e, tile, lane, m - j0, live, (const char *)states + i * sizeof(e.s), j0);
        __syncwarp();
        const int cols = (int)((m - j0) < (size_t)COLS ? (m - j0) : (size_t)COLS);
        for (int f = lane; f < 32 * COLS; f += 32) {
            const int r = f / COLS, c = f % COLS;
            if (c >= cols || row0 + r >= S) continue;
            const u32 byte = (u32)(c * ES);
            const u32 a = tile + (u32)r * 128u + ((((byte >> 4) ^ (u32)(r & 7))) << 4) + (byte & 15u);
            OT v;
            if (ES == 8) v = (OT)ld_shared_u64(a);
            else v = (OT)ld_shared_u32(a);
            out[(row0 + r) * ld + j0 + c] = v;
        }
        __syncwarp();
    }
    if (write_back && live) store_state(e, (char *)states + i * sizeof(e.s));
}

// Interleaved layout: output j of all streams is contiguous, so the 32 lanes
// of a warp store 32 consecutive elements per output.
template <int V, int DT>
__global__ void __launch_bounds__(256)
    k_fill_interleaved(void *states, size_t S, size_t m,
                       typename OutElem<DT>::type *__restrict__ out, int write_back, int *status)
{
    typedef Gen<V> G;
    typedef typename G::E E;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S) return;
    E e;
    load_state(e, (const char *)states + i * sizeof(e.s));
    if (state_is_zero(e)) atomicCAS(status, 0, XR_EZERO_STATE);
    size_t j = 0;
    if constexpr (DT == DT_F64 && sizeof(typename G::word) == 8 && E::NBITS <= 512) {
        // doubles of 64-bit words in chunks of 16 with the branch-free
        // conversion; a chunk holding an output below 2^32 (probability 2^-28
        // per chunk) is written again exactly from its start state
        for (; j + 16 <= m; j += 16) {
            const E e0 = e;
            u32 hmin = 0xffffffffu;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                out[(j + q) * S + i] = unit_f64_bits_hi((u64)G::out(e), hmin);
                e.step();
            }
            if (__builtin_expect(hmin == 0u, 0)) {
                E r = e0;
#pragma unroll 1
                for (int q = 0; q < 16; ++q) {
                    out[(j + q) * S + i] = unit_f64_bits((u64)G::out(r));
                    r.step();
                }
            }
        }
    }
#pragma unroll 4
    for (; j < m; ++j) {
        out[j * S + i] = convert<DT>(G::out(e));
        e.step();
    }
    if (write_back) store_state(e, (char *)states + i * sizeof(e.s));
}

template <int V, int DT>
cudaError_t launch_fill_vd(int layout, void *states, size_t S, size_t m, size_t ld, void *out,
                           int write_back, int *status, cudaStream_t stream, EncodeTiledFn encode)
{
    typedef typename OutElem<DT>::type OT;
    constexpr int ES = (int)sizeof(OT);
    constexpr int COLS = 128 / ES;
    if (S == 0) return cudaSuccess;
    if (layout == XR_INTERLEAVED) {
        const size_t grid = (S + 255) / 256;
        k_fill_interleaved<V, DT><<<(unsigned)grid, 256, 0, stream>>>(states, S, m, (OT *)out,
                                                                     write_back, status);
        count_launch();
        return cudaGetLastError();
    }
    typedef FillCfg<V, DT, false> CL;
    typedef FillCfg<V, DT, true> CS;
    static std::atomic<uint64_t> attr_long{0}, attr_short{0}, attr_plain{0};
    cudaError_t ea = set_smem_once(attr_long, k_fill_tma<V, DT, false>, CL::SMEM);
    if (ea == cudaSuccess) ea = set_smem_once(attr_short, k_fill_tma<V, DT, true>, CS::SMEM);
    if (ea == cudaSuccess) ea = set_smem_once(attr_plain, k_fill_plain<V, DT>, FILL_SMEM);
    if (ea != cudaSuccess) return ea;
    const size_t rows_per_cta = (size_t)FILL_WARPS * 32;
    const size_t grid = (S + rows_per_cta - 1) / rows_per_cta;
    const bool short_rows = (m + COLS - 1) / COLS <= (size_t)FILL_SHORT_TILES;
    const size_t tma_rows = (size_t)(short_rows ? CS::WARPS : CL::WARPS) * 32;
    const size_t tma_grid = (S + tma_rows - 1) / tma_rows;
    // The tile store clips columns past the extent only to a 16-byte boundary
    // (seen on GB300: a 4-byte row received 16 bytes), so the row length must
    // be a multiple of 16 bytes as well as the pitch.
    const bool tma_ok = encode != nullptr && ((uintptr_t)out % 16) == 0 && ((ld * ES) % 16) == 0 &&
                        ((m * ES) % 16) == 0 && m < (1ull << 31) && S < (1ull << 31) &&
                        ld * ES < (1ull << 40) && m > 0;
    if (tma_ok) {
        CUtensorMap map;
        const cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)S};
        const cuuint64_t strides[1] = {(cuuint64_t)(ld * ES)};
        const cuuint32_t box[2] = {(cuuint32_t)COLS, 32u};
        const cuuint32_t estr[2] = {1u, 1u};
        const CUresult r = encode(&map, ES == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32,
                                  2, out, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r == CUDA_SUCCESS) {
            if (short_rows)
                k_fill_tma<V, DT, true><<<(unsigned)tma_grid, CS::WARPS * 32, CS::SMEM, stream>>>(
                    map, states, S, m, write_back, status);
            else
                k_fill_tma<V, DT, false><<<(unsigned)tma_grid, CL::WARPS * 32, CL::SMEM, stream>>>(
                    map, states, S, m, write_back, status);
            count_launch();
            return cudaGetLastError();
        }
    }
    k_fill_plain<V, DT><<<(unsigned)grid, FILL_WARPS * 32, FILL_SMEM, stream>>>(
        states, S, m, ld, (OT *)out, write_back, status);
    count_launch();
    return cudaGetLastError();
}

// Entry per generator: dtype dispatch over the element types it supports.
template <int V>
cudaError_t launch_fill_v(int dtype, int layout, void *states, size_t S, size_t m, size_t ld,
                          void *out, int write_back, int *status, cudaStream_t stream,
                          EncodeTiledFn encode)
{
    constexpr bool w64 = sizeof(typename Gen<V>::word) == 8;
    switch (dtype) {
    case DT_U64:
        if constexpr (w64)
            return launch_fill_vd<V, DT_U64>(layout, states, S, m, ld, out, write_back, status, stream, encode);
        return cudaErrorInvalidValue;
    case DT_U32:
        if constexpr (!w64)
            return launch_fill_vd<V, DT_U32>(layout, states, S, m, ld, out, write_back, status, stream, encode);
        return cudaErrorInvalidValue;
    case DT_F64:
        return launch_fill_vd<V, DT_F64>(layout, states, S, m, ld, out, write_back, status, stream, encode);
    case DT_F32:
        return launch_fill_vd<V, DT_F32>(layout, states, S, m, ld, out, write_back, status, stream, encode);
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace xr
