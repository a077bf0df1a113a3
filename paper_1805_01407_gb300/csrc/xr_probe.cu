// xr_probe.cu -- measurement probes (include/xr_probe.h): the HBM write
// ceiling (a store-only kernel, cudaMemsetAsync) and the integer-ALU ceiling
// (independent lop3 chains) of the GPU the fill runs on.
#include <stdint.h>

#include "xr_device.cuh"
#include "xr_internal.h"
#include "xr_probe.h"

namespace {

using xr::u32;

// Thread t stores the 16-byte words t, t + G, t + 2G, ... (G = grid threads):
// each warp store covers 512 contiguous bytes.
__global__ void __launch_bounds__(512) k_probe_store(uint4 *p, size_t n16)
{
    const size_t G = (size_t)gridDim.x * blockDim.x;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint4 v = make_uint4((uint32_t)i, 0x5a5a5a5au, (uint32_t)(i >> 32), 0xa5a5a5a5u);
    for (; i + 3 * G < n16; i += 4 * G) {
        p[i] = v;
        p[i + G] = v;
        p[i + 2 * G] = v;
        p[i + 3 * G] = v;
    }
    for (; i < n16; i += G) p[i] = v;
}

// 8 chains of lop3 (xor of three words) per thread, two rounds of 8 per
// iteration, 8 iterations per loop trip: 128 lop3 per trip against about
// three loop instructions.
__global__ void __launch_bounds__(256) k_probe_alu(uint32_t *sink, int trips)
{
    uint32_t a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = threadIdx.x * (2u * j + 1u) + blockIdx.x * 0x9e3779b9u + j;
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int it = 0; it < 8 * 2; ++it) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[j]) : "r"(a[(j + 1) & 7]), "r"(a[(j + 3) & 7]));
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) x ^= a[j] * (2u * j + 1u);
    // a store that depends on every chain and practically never happens
    if (x == 0x2545f491u) *sink = x;
}

// The fill's tile-store pattern with nothing generated: each warp owns 32
// consecutive rows and writes them as 32-row x 128-byte swizzled tiles, column
// after column, staging each tile with st.shared first, NBUF tiles in flight
// per warp; one warp per 32 rows over the grid.  Coordinates stay inside the
// tensor: x below the row length in steps of 16 u64, row0 below `rows` (the
// grid is rows / (32 WARPS)).
template <int WARPS, int NBUF>
__global__ void __launch_bounds__(WARPS * 32) k_probe_tiles(const __grid_constant__ CUtensorMap map, int cols)
{
    extern __shared__ unsigned char probe_smem[];
    const u32 base = (xr::smem_addr(probe_smem) + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = (blockIdx.x * WARPS + warp) * 32;
    const u32 tiles = base + (u32)(warp * NBUF * 4096);
    int it = 0;
    for (int j0 = 0; j0 < cols; j0 += 16, ++it) {
        const u32 tile = tiles + (u32)((it % NBUF) * 4096);
        if (it >= NBUF) {
            if (lane == 0) xr::bulk_wait_read<NBUF - 1>();
            __syncwarp();
        }
        const u32 row = tile + (u32)lane * 128u, sw = (u32)(lane & 7);
#pragma unroll
        for (int c = 0; c < 8; ++c) xr::st_shared_v4(row + (((u32)c ^ sw) << 4), (u32)j0, (u32)c, (u32)lane, (u32)it);
        xr::fence_proxy_async_shared();
        __syncwarp();
        if (lane == 0) {
            xr::tma_store_2d(&map, tile, j0, row0);
            xr::bulk_commit();
        }
    }
    if (lane == 0) xr::bulk_wait_read<0>();
}

int status_of(cudaError_t e)
{
    if (e == cudaSuccess) return XR_OK;
    if (e == cudaErrorInvalidValue) return XR_EINVAL;
    return XR_ECUDA;
}

int sm_count(int *sms)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return XR_ECUDA;
    if (cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return XR_ECUDA;
    return XR_OK;
}

}  // namespace

extern "C" int xr_probe_store(void *d_buf, size_t bytes, int ctas_per_sm, void *stream)
{
    if (!d_buf || (bytes % 16) || ((uintptr_t)d_buf % 16) || ctas_per_sm < 0 || ctas_per_sm > 64) return XR_EINVAL;
    if (bytes == 0) return XR_OK;
    int sms = 0;
    const int rc = sm_count(&sms);
    if (rc != XR_OK) return rc;
    const int grid = sms * (ctas_per_sm ? ctas_per_sm : 4);
    k_probe_store<<<grid, 512, 0, (cudaStream_t)stream>>>((uint4 *)d_buf, bytes / 16);
    xr::count_launch();
    return status_of(cudaGetLastError());
}

extern "C" int xr_probe_memset(void *d_buf, size_t bytes, void *stream)
{
    if (!d_buf) return XR_EINVAL;
    return status_of(cudaMemsetAsync(d_buf, 0, bytes, (cudaStream_t)stream));
}

extern "C" int xr_probe_alu(uint32_t *d_sink, int blocks, int iters, void *stream)
{
    if (!d_sink || blocks < 1 || iters < 8 || (iters % 8)) return XR_EINVAL;
    // a loop trip is 8 iterations of 16 lop3
    k_probe_alu<<<blocks, 256, 0, (cudaStream_t)stream>>>(d_sink, iters / 8);
    xr::count_launch();
    return status_of(cudaGetLastError());
}

template <int WARPS, int NBUF>
static int probe_tiles(const CUtensorMap &map, size_t rows, int cols, cudaStream_t st)
{
    const int smem = WARPS * NBUF * 4096 + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_probe_tiles<WARPS, NBUF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return status_of(e);
    k_probe_tiles<WARPS, NBUF><<<(unsigned)(rows / (32 * WARPS)), WARPS * 32, smem, st>>>(map, cols);
    xr::count_launch();
    return status_of(cudaGetLastError());
}

extern "C" int xr_probe_tile_store(void *d_buf, size_t rows, size_t row_bytes, int config, void *stream)
{
    static const int warps_of[3] = {2, 1, 1};
    if (!d_buf || ((uintptr_t)d_buf % 128) || config < 0 || config > 2 || row_bytes == 0 || (row_bytes % 128) ||
        row_bytes > ((size_t)1 << 30) || rows == 0 || rows >= ((size_t)1 << 31) ||
        (rows % (32 * (size_t)warps_of[config])))
        return XR_EINVAL;
    // looked up once, thread-safely (a function-local static)
    static const xr::EncodeTiledFn encode = [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (xr::EncodeTiledFn) nullptr;
        return (xr::EncodeTiledFn)fn;
    }();
    if (!encode) return XR_ECUDA;
    CUtensorMap map;
    const cuuint64_t dims[2] = {(cuuint64_t)(row_bytes / 8), (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
    const cuuint32_t box[2] = {16u, 32u};
    const cuuint32_t estr[2] = {1u, 1u};
    if (encode(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, d_buf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
        return XR_EINVAL;
    const int cols = (int)(row_bytes / 8);
    const cudaStream_t st = (cudaStream_t)stream;
    switch (config) {
    case 0: return probe_tiles<2, 6>(map, rows, cols, st);
    case 1: return probe_tiles<1, 8>(map, rows, cols, st);
    default: return probe_tiles<1, 3>(map, rows, cols, st);
    }
}
