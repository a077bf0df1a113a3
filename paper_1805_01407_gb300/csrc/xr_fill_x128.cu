// xr_fill_x128.cu -- fill kernels of generators 6, 7, 8 (see xr_fill_impl.cuh).
#include "xr_fill_streams.cuh"

namespace xr {
template cudaError_t launch_fill_v<6>(int, int, void *, size_t, size_t, size_t, void *, int, int *, cudaStream_t, EncodeTiledFn);
template cudaError_t launch_fill_v<7>(int, int, void *, size_t, size_t, size_t, void *, int, int *, cudaStream_t, EncodeTiledFn);
template cudaError_t launch_fill_v<8>(int, int, void *, size_t, size_t, size_t, void *, int, int *, cudaStream_t, EncodeTiledFn);
template cudaError_t launch_fill_streams_v<6>(int, const uint32_t *, const void *, size_t, size_t, void *, int *, cudaStream_t, EncodeTiledFn);
template cudaError_t launch_fill_streams_v<7>(int, const uint32_t *, const void *, size_t, size_t, void *, int *, cudaStream_t, EncodeTiledFn);
template cudaError_t launch_fill_streams_v<8>(int, const uint32_t *, const void *, size_t, size_t, void *, int *, cudaStream_t, EncodeTiledFn);
}  // namespace xr
