// xr_probe.cu -- measurement probes (include/xr_probe.h): the HBM write
// ceiling (a store-only kernel, cudaMemsetAsync) and the integer-ALU ceiling
// (independent lop3 chains) of the GPU the fill runs on.
#include <stdint.h>

#include "xr_internal.h"
#include "xr_probe.h"

namespace {

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
