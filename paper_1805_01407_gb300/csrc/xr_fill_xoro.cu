// xr_fill_xoro.cu -- fill kernels of generators 3, 4, 5 (see xr_fill_impl.cuh).
#include "xr_fill_streams.cuh"

namespace xr {
template cudaError_t launch_fill_v<3>(int, int, void *, size_t, size_t, size_t, void *, int, int *, cudaStream_t, EncodeTiledFn);
template cudaError_t launch_fill_v<4>(int, int, void *, size_t, size_t, size_t, void *, int, int *, cudaStream_t, EncodeTiledFn);
template cudaError_t launch_fill_v<5>(int, int, void *, size_t, size_t, size_t, void *, int, int *, cudaStream_t, EncodeTiledFn);
template cudaError_t launch_fill_streams_v<3>(int, const uint32_t *, const void *, size_t, size_t, void *, int *, cudaStream_t, EncodeTiledFn);
template cudaError_t launch_fill_streams_v<4>(int, const uint32_t *, const void *, size_t, size_t, void *, int *, cudaStream_t, EncodeTiledFn);
template cudaError_t launch_fill_streams_v<5>(int, const uint32_t *, const void *, size_t, size_t, void *, int *, cudaStream_t, EncodeTiledFn);
}  // namespace xr
