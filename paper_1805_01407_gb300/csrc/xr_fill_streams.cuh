// xr_fill_streams.cuh -- stream starts fused with the fill (xr_fill_streams):
// the fill kernels' tile staging (xr_fill_impl.cuh) fed by start states that
// each thread computes from the power sets (xr_f2.cuh).
#pragma once

#include "xr_f2.cuh"
#include "xr_fill_impl.cuh"

namespace xr {

// ---------------------------------------------------------------- stream starts fused with the fill
//
// A chunk of 512 P streams (P a power of two, at least 32) whose first P
// streams, the parents, are given: stream p + P j starts at P_0[j] parent_p,
// with P_0[j] = T^(2^d P j) the level-0 power set of the distance 2^d P
// (Sec. 5, 6).  A CTA takes one j: it builds the Four-Russians tables of
// P_0[j] once, and the lanes of each warp are 32 consecutive parents, hence
// 32 consecutive streams (rows p0 + P j ..), written by 2D tile stores like
// k_fill_tma.  The start states never reach global memory.  A warp takes
// `groups` groups of 32 parents in turn, so the tile stores of one group
// drain while the next group's products run; for doubles of 64-bit words a
// lane also keeps its start state in a shared-memory slot, for the rare exact
// redo of a row.  One tile per warp and 16 warps per CTA measured best (2^24
// x 64, 4 groups: u64 1.63 ms, f64 1.81 ms; 8 warps x 1 tile 1.64 / 1.88 ms;
// 8 warps x 2 tiles, u64 1.73 ms): shared memory, not the store queue, limits
// the warps per SM.  More groups per CTA spread each table build over more
// streams but leave fewer CTAs for the tail, so the count is a template
// argument: 8 from 2^15 parents (2^24 streams) on, else 4 (2^24 x 64 u64 with
// 2, 3, 4, 6, 8, 10, 12, 16 groups: 1.635, 1.617, 1.612, 1.577, 1.547, 1.561,
// 1.554, 1.588 ms; 2^21 x 64 u64 with 4 and 8 groups: 0.249 and 0.267 ms; a
// count passed at run time cost 2 % on the doubles).  Only rows
// of at most FILL_SHORT_TILES tiles come here: for longer rows the start
// states are a small part of the work, and a state table followed by the
// fill's own configuration (many small CTAs for the exact doubles, which a
// resident 32 KB table rules out) measured faster.
constexpr int FS_WARPS = 16;
constexpr int FS_NBUF = 1;
constexpr int FS_CHILDREN = PSET_SIZE;  // streams per parent (j < 512)

template <int V>
struct FuseCfg {
    typedef typename Gen<V>::E E;
    static constexpr int NW = (int)sizeof(E::s) / 4;
    static constexpr int TABLE_BYTES = Russians<NW>::WORDS * 4;
    static constexpr int SMEM = FS_WARPS * FS_NBUF * TILE_BYTES + TABLE_BYTES + FS_WARPS * 32 * 32 + 1024;
};

template <int V, int DT, int GROUPS>
__global__ void __launch_bounds__(FS_WARPS * 32)
    k_fill_streams(const __grid_constant__ CUtensorMap map, const u32 *__restrict__ P0, const u32 *parents,
                   size_t npar, size_t m, int *status)  // npar = P
{
    typedef Gen<V> G;
    typedef typename G::E E;
    constexpr int NW = FuseCfg<V>::NW;
    typedef Russians<NW> RT;
    constexpr int COLS = 128 / (int)sizeof(typename OutElem<DT>::type);
    extern __shared__ unsigned char dyn_smem[];
    const u32 pad = ((smem_addr(dyn_smem) + 1023u) & ~1023u) - smem_addr(dyn_smem);
    const u32 base = smem_addr(dyn_smem) + pad;                     // tiles, 1024-byte aligned
    u32 *T = reinterpret_cast<u32 *>(dyn_smem + pad + FS_WARPS * FS_NBUF * TILE_BYTES);
    unsigned char *slots = reinterpret_cast<unsigned char *>(T + RT::WORDS);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x;
    russians_build<NW>(P0 + (size_t)j * RT::n * NW, T);
    __syncthreads();
    const u32 tiles = base + (u32)(warp * FS_NBUF * TILE_BYTES);
    unsigned char *slot = slots + (warp * 32 + lane) * 32;
    int it = 0;
    for (int g = 0; g < GROUPS; ++g) {
        const size_t p0 = (((size_t)blockIdx.y * GROUPS + g) * FS_WARPS + warp) * 32;
        if (p0 >= npar) break;
        const bool live = p0 + lane < npar;
        u32 v[NW], r[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) v[w] = 0u;
        if (live) {
            const u32 *ps = parents + (p0 + lane) * NW;  // 16-byte loads (8-byte for 64-bit states)
            if constexpr (NW >= 4) {
#pragma unroll
                for (int q = 0; q < NW / 4; ++q) {
                    const uint4 a = reinterpret_cast<const uint4 *>(ps)[q];
                    v[4 * q] = a.x; v[4 * q + 1] = a.y; v[4 * q + 2] = a.z; v[4 * q + 3] = a.w;
                }
            } else {
                const uint2 a = reinterpret_cast<const uint2 *>(ps)[0];
                v[0] = a.x; v[1] = a.y;
            }
        }
        russians_matvec<NW>(T, v, r);
        // the start state goes to the lane's slot only where a row may need
        // its exact redo (doubles of 64-bit words); the engine takes it from
        // registers
        if constexpr (DT == DT_F64 && sizeof(typename G::word) == 8) {
#pragma unroll
            for (int q = 0; q < NW / 4; ++q)
                reinterpret_cast<uint4 *>(slot)[q] = make_uint4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
        }
        E e;
        if constexpr (sizeof(typename E::word) == 8) {
#pragma unroll
            for (int k = 0; k < E::K; ++k) e.s[k] = (u64)r[2 * k] | ((u64)r[2 * k + 1] << 32);
        } else {
#pragma unroll
            for (int k = 0; k < E::K; ++k) e.s[k] = r[k];
        }
        if (live && state_is_zero(e)) atomicCAS(status, 0, XR_EZERO_STATE);
        for (size_t j0 = 0; j0 < m; j0 += COLS, ++it) {
            const u32 tile = tiles + (u32)((it % FS_NBUF) * TILE_BYTES);
            if (it >= FS_NBUF) {
                if (lane == 0) bulk_wait_read<FS_NBUF - 1>();
                __syncwarp();
            }
            fill_tile_row<G, DT>(e, tile, lane, m - j0, live, slot, j0);
            fence_proxy_async_shared();
            __syncwarp();
            if (lane == 0) {
                tma_store_2d(&map, tile, (int)j0, (int)(p0 + npar * (size_t)j));
                bulk_commit();
            }
        }
    }
    if (lane == 0) bulk_wait_read<0>();
}

// P = npar parents (contiguous states, P a power of two, at least 32) ->
// 512 P streams x m outputs in d_out (stream-major), rows of at most
// FILL_SHORT_TILES tiles.  cudaErrorNotSupported for other shapes.
template <int V, int DT>
cudaError_t launch_fill_streams_vd(const u32 *P0, const void *parents, size_t npar, size_t m, void *out,
                                   int *status, cudaStream_t stream, EncodeTiledFn encode)
{
    constexpr int ES = (int)sizeof(typename OutElem<DT>::type);
    constexpr int COLS = 128 / ES;
    typedef FuseCfg<V> FC;
    const bool rows_ok = m > 0 && (m * ES) % 16 == 0 && (m + COLS - 1) / COLS <= (size_t)FILL_SHORT_TILES;
    const bool parents_ok = npar >= 32 && (npar & (npar - 1)) == 0 && (size_t)FS_CHILDREN * npar < (1ull << 31);
    if (!encode || ((uintptr_t)out % 16) || !rows_ok || !parents_ok) return cudaErrorNotSupported;
    // groups per CTA: 4, or 8 from 2^15 parents (2^24 streams) on
    const int groups = npar >= 32768 ? 8 : 4;
    const size_t gy = (npar + (size_t)groups * FS_WARPS * 32 - 1) / ((size_t)groups * FS_WARPS * 32);
    if (gy > 65535) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)(FS_CHILDREN * npar)};
    const cuuint64_t strides[1] = {(cuuint64_t)(m * ES)};
    const cuuint32_t box[2] = {(cuuint32_t)COLS, 32u};
    const cuuint32_t estr[2] = {1u, 1u};
    if (encode(&map, ES == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, out, dims,
               strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorNotSupported;
    static std::atomic<uint64_t> attr4{0}, attr8{0};
    cudaError_t ea = set_smem_once(attr4, k_fill_streams<V, DT, 4>, FC::SMEM);
    if (ea == cudaSuccess) ea = set_smem_once(attr8, k_fill_streams<V, DT, 8>, FC::SMEM);
    if (ea != cudaSuccess) return ea;
    const dim3 grid(FS_CHILDREN, (unsigned)gy);
    if (groups == 8)
        k_fill_streams<V, DT, 8><<<grid, FS_WARPS * 32, FC::SMEM, stream>>>(map, P0, (const u32 *)parents, npar, m, status);
    else
        k_fill_streams<V, DT, 4><<<grid, FS_WARPS * 32, FC::SMEM, stream>>>(map, P0, (const u32 *)parents, npar, m, status);
    count_launch();
    return cudaGetLastError();
}

template <int V>
cudaError_t launch_fill_streams_v(int dtype, const uint32_t *P0, const void *parents, size_t npar, size_t m,
                                  void *out, int *status, cudaStream_t stream, EncodeTiledFn encode)
{
    constexpr bool w64 = sizeof(typename Gen<V>::word) == 8;
    switch (dtype) {
    case DT_U64:
        if constexpr (w64) return launch_fill_streams_vd<V, DT_U64>(P0, parents, npar, m, out, status, stream, encode);
        return cudaErrorInvalidValue;
    case DT_U32:
        if constexpr (!w64) return launch_fill_streams_vd<V, DT_U32>(P0, parents, npar, m, out, status, stream, encode);
        return cudaErrorInvalidValue;
    case DT_F64:
        return launch_fill_streams_vd<V, DT_F64>(P0, parents, npar, m, out, status, stream, encode);
    case DT_F32:
        return launch_fill_streams_vd<V, DT_F32>(P0, parents, npar, m, out, status, stream, encode);
    default:
        return cudaErrorInvalidValue;
    }
}

}  // namespace xr
