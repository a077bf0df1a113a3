// xr_fill_more.cu -- fill kernels of generators 9 .. 17 (xoroshiro128*, the
// 32-bit xoroshiro64 pair, xoshiro512 and xoroshiro1024; see xr_fill_impl.cuh).
#include "xr_fill_streams.cuh"

namespace xr {
#define XR_FILL_INST(V) \
    template cudaError_t launch_fill_v<V>(int, int, void *, size_t, size_t, size_t, void *, int, int *, cudaStream_t, EncodeTiledFn);
XR_FILL_INST(9) XR_FILL_INST(10) XR_FILL_INST(11) XR_FILL_INST(12) XR_FILL_INST(13)
XR_FILL_INST(14) XR_FILL_INST(15) XR_FILL_INST(16) XR_FILL_INST(17)
#undef XR_FILL_INST
template cudaError_t launch_fill_streams_v<9>(int, const uint32_t *, const void *, size_t, size_t, void *, int *, cudaStream_t, EncodeTiledFn);
template cudaError_t launch_fill_streams_v<10>(int, const uint32_t *, const void *, size_t, size_t, void *, int *, cudaStream_t, EncodeTiledFn);
template cudaError_t launch_fill_streams_v<11>(int, const uint32_t *, const void *, size_t, size_t, void *, int *, cudaStream_t, EncodeTiledFn);
}  // namespace xr
