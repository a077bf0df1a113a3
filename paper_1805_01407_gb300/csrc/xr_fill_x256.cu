// xr_fill_x256.cu -- fill kernels of generators 0, 1, 2 (see xr_fill_impl.cuh).
#include "xr_fill_streams.cuh"

namespace xr {
template cudaError_t launch_fill_v<0>(int, int, void *, size_t, size_t, size_t, void *, int, int *, cudaStream_t, EncodeTiledFn);
template cudaError_t launch_fill_v<1>(int, int, void *, size_t, size_t, size_t, void *, int, int *, cudaStream_t, EncodeTiledFn);
template cudaError_t launch_fill_v<2>(int, int, void *, size_t, size_t, size_t, void *, int, int *, cudaStream_t, EncodeTiledFn);
template cudaError_t launch_fill_streams_v<0>(int, const uint32_t *, const void *, size_t, size_t, void *, int *, cudaStream_t, EncodeTiledFn);
template cudaError_t launch_fill_streams_v<1>(int, const uint32_t *, const void *, size_t, size_t, void *, int *, cudaStream_t, EncodeTiledFn);
template cudaError_t launch_fill_streams_v<2>(int, const uint32_t *, const void *, size_t, size_t, void *, int *, cudaStream_t, EncodeTiledFn);
}  // namespace xr
