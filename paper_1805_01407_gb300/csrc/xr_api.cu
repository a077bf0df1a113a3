// xr_api.cu -- the C ABI of libxr (declared in include/xr.h): argument checks,
// the context (jump tables, status word, scratch), and dispatch to kernels.
#include <stdlib.h>
#include <atomic>
#include <mutex>
#include <string.h>

#include "xr_device.cuh"
#include "xr_internal.h"

namespace xr {

template <int V>
cudaError_t launch_fill_v(int dtype, int layout, void *states, size_t S, size_t m, size_t ld,
                          void *out, int write_back, int *status, cudaStream_t stream,
                          EncodeTiledFn encode);
extern template cudaError_t launch_fill_v<0>(int, int, void *, size_t, size_t, size_t, void *, int, int *, cudaStream_t, EncodeTiledFn);
extern template cudaError_t launch_fill_v<1>(int, int, void *, size_t, size_t, size_t, void *, int, int *, cudaStream_t, EncodeTiledFn);
extern template cudaError_t launch_fill_v<2>(int, int, void *, size_t, size_t, size_t, void *, int, int *, cudaStream_t, EncodeTiledFn);
extern template cudaError_t launch_fill_v<3>(int, int, void *, size_t, size_t, size_t, void *, int, int *, cudaStream_t, EncodeTiledFn);
extern template cudaError_t launch_fill_v<4>(int, int, void *, size_t, size_t, size_t, void *, int, int *, cudaStream_t, EncodeTiledFn);
extern template cudaError_t launch_fill_v<5>(int, int, void *, size_t, size_t, size_t, void *, int, int *, cudaStream_t, EncodeTiledFn);
extern template cudaError_t launch_fill_v<6>(int, int, void *, size_t, size_t, size_t, void *, int, int *, cudaStream_t, EncodeTiledFn);
extern template cudaError_t launch_fill_v<7>(int, int, void *, size_t, size_t, size_t, void *, int, int *, cudaStream_t, EncodeTiledFn);
extern template cudaError_t launch_fill_v<8>(int, int, void *, size_t, size_t, size_t, void *, int, int *, cudaStream_t, EncodeTiledFn);
#define XR_EXTERN_FILL(V) \
    extern template cudaError_t launch_fill_v<V>(int, int, void *, size_t, size_t, size_t, void *, int, int *, cudaStream_t, EncodeTiledFn);
XR_EXTERN_FILL(9) XR_EXTERN_FILL(10) XR_EXTERN_FILL(11) XR_EXTERN_FILL(12) XR_EXTERN_FILL(13)
XR_EXTERN_FILL(14) XR_EXTERN_FILL(15) XR_EXTERN_FILL(16) XR_EXTERN_FILL(17)
#undef XR_EXTERN_FILL

static const int kEngineOf[XR_NUM_VARIANTS] = {
    ENG_XOSHIRO256, ENG_XOSHIRO256, ENG_XOSHIRO256, ENG_XOROSHIRO128, ENG_XOROSHIRO128PP, ENG_XOROSHIRO128,
    ENG_XOSHIRO128, ENG_XOSHIRO128, ENG_XOSHIRO128, ENG_XOROSHIRO128, ENG_XOROSHIRO64, ENG_XOROSHIRO64,
    ENG_XOSHIRO512, ENG_XOSHIRO512, ENG_XOSHIRO512, ENG_XOROSHIRO1024, ENG_XOROSHIRO1024, ENG_XOROSHIRO1024};
static const int kEngineBits[NUM_ENGINES] = {256, 128, 128, 128, 64, 512, 1024};
static const int kEngineWords[NUM_ENGINES] = {4, 2, 2, 4, 2, 8, 16};
static const int kEngineWordBits[NUM_ENGINES] = {64, 64, 64, 32, 32, 64, 64};
static_assert(NUM_ENGINES == NUM_ENGINES_H, "engine count");

static std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int engine_of(int variant) { return kEngineOf[variant]; }
int engine_bits(int engine) { return kEngineBits[engine]; }

cudaError_t launch_fill(int variant, int dtype, int layout, void *states, size_t S, size_t m,
                        size_t ld, void *out, int write_back, int *status, cudaStream_t stream,
                        EncodeTiledFn encode)
{
    switch (variant) {
    case 0: return launch_fill_v<0>(dtype, layout, states, S, m, ld, out, write_back, status, stream, encode);
    case 1: return launch_fill_v<1>(dtype, layout, states, S, m, ld, out, write_back, status, stream, encode);
    case 2: return launch_fill_v<2>(dtype, layout, states, S, m, ld, out, write_back, status, stream, encode);
    case 3: return launch_fill_v<3>(dtype, layout, states, S, m, ld, out, write_back, status, stream, encode);
    case 4: return launch_fill_v<4>(dtype, layout, states, S, m, ld, out, write_back, status, stream, encode);
    case 5: return launch_fill_v<5>(dtype, layout, states, S, m, ld, out, write_back, status, stream, encode);
    case 6: return launch_fill_v<6>(dtype, layout, states, S, m, ld, out, write_back, status, stream, encode);
    case 7: return launch_fill_v<7>(dtype, layout, states, S, m, ld, out, write_back, status, stream, encode);
    case 8: return launch_fill_v<8>(dtype, layout, states, S, m, ld, out, write_back, status, stream, encode);
    case 9: return launch_fill_v<9>(dtype, layout, states, S, m, ld, out, write_back, status, stream, encode);
    case 10: return launch_fill_v<10>(dtype, layout, states, S, m, ld, out, write_back, status, stream, encode);
    case 11: return launch_fill_v<11>(dtype, layout, states, S, m, ld, out, write_back, status, stream, encode);
    case 12: return launch_fill_v<12>(dtype, layout, states, S, m, ld, out, write_back, status, stream, encode);
    case 13: return launch_fill_v<13>(dtype, layout, states, S, m, ld, out, write_back, status, stream, encode);
    case 14: return launch_fill_v<14>(dtype, layout, states, S, m, ld, out, write_back, status, stream, encode);
    case 15: return launch_fill_v<15>(dtype, layout, states, S, m, ld, out, write_back, status, stream, encode);
    case 16: return launch_fill_v<16>(dtype, layout, states, S, m, ld, out, write_back, status, stream, encode);
    case 17: return launch_fill_v<17>(dtype, layout, states, S, m, ld, out, write_back, status, stream, encode);
    default: return cudaErrorInvalidValue;
    }
}

template <int V>
cudaError_t launch_fill_streams_v(int dtype, const uint32_t *P0, const void *parents, size_t npar, size_t m,
                                  void *out, int *status, cudaStream_t stream, EncodeTiledFn encode);
#define XR_FS_EXTERN(V)                                                                                         \
    extern template cudaError_t launch_fill_streams_v<V>(int, const uint32_t *, const void *, size_t, size_t, \
                                                         void *, int *, cudaStream_t, EncodeTiledFn);
XR_FS_EXTERN(0) XR_FS_EXTERN(1) XR_FS_EXTERN(2) XR_FS_EXTERN(3) XR_FS_EXTERN(4) XR_FS_EXTERN(5)
XR_FS_EXTERN(6) XR_FS_EXTERN(7) XR_FS_EXTERN(8) XR_FS_EXTERN(9) XR_FS_EXTERN(10) XR_FS_EXTERN(11)
#undef XR_FS_EXTERN

// Fused stream starts + fill for the generators with power sets (0 .. 11).
static cudaError_t launch_fill_streams(int variant, int dtype, const uint32_t *P0, const void *parents, size_t npar,
                                       size_t m, void *out, int *status, cudaStream_t st, EncodeTiledFn encode)
{
#define XR_FS_CASE(V) \
    case V: return launch_fill_streams_v<V>(dtype, P0, parents, npar, m, out, status, st, encode);
    switch (variant) {
        XR_FS_CASE(0) XR_FS_CASE(1) XR_FS_CASE(2) XR_FS_CASE(3) XR_FS_CASE(4) XR_FS_CASE(5)
        XR_FS_CASE(6) XR_FS_CASE(7) XR_FS_CASE(8) XR_FS_CASE(9) XR_FS_CASE(10) XR_FS_CASE(11)
    default: return cudaErrorNotSupported;
    }
#undef XR_FS_CASE
}

}  // namespace xr

using namespace xr;

// Segment length of xr_fill_seq: 2^SEQ_LOG2 outputs per segment.
static const int SEQ_LOG2 = 10;
// Segment length of xr_fill_seq_noalloc (same as xr_fill_seq).
#define SEQ_LOG2_NOALLOC 10
// Largest staging buffer of xr_fill_host (two of them).
static const size_t HOST_STAGING_BYTES = (size_t)256 << 20;

static const char *kNames[XR_NUM_VARIANTS] = {
    "xoshiro256+", "xoshiro256++", "xoshiro256**", "xoroshiro128+", "xoroshiro128++", "xoroshiro128**",
    "xoshiro128++", "xoshiro128**", "xoshiro128+", "xoroshiro128*", "xoroshiro64*", "xoroshiro64**",
    "xoshiro512+", "xoshiro512++", "xoshiro512**", "xoroshiro1024*", "xoroshiro1024++", "xoroshiro1024**"};

static bool variant_ok(int v) { return v >= 0 && v < XR_NUM_VARIANTS; }

static int status_of(cudaError_t e)
{
    if (e == cudaSuccess) return XR_OK;
    if (e == cudaErrorMemoryAllocation) return XR_ENOMEM;
    if (e == cudaErrorInvalidValue) return XR_EINVAL;
    return XR_ECUDA;
}

// ---------------------------------------------------------------- properties

extern "C" uint64_t xr_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" int xr_state_words(int variant)
{
    if (!variant_ok(variant)) return -1;
    return kEngineWords[engine_of(variant)];
}

extern "C" int xr_word_bits(int variant)
{
    if (!variant_ok(variant)) return -1;
    return kEngineWordBits[engine_of(variant)];
}

extern "C" int xr_state_bytes(int variant)
{
    if (!variant_ok(variant)) return -1;
    return xr_state_words(variant) * xr_word_bits(variant) / 8;
}

extern "C" int xr_state_bits(int variant)
{
    if (!variant_ok(variant)) return -1;
    return engine_bits(engine_of(variant));
}

extern "C" int xr_dtype_bytes(int dtype)
{
    switch (dtype) {
    case XR_U64: case XR_F64: return 8;
    case XR_U32: case XR_F32: return 4;
    default: return -1;
    }
}

extern "C" const char *xr_variant_name(int variant)
{
    return variant_ok(variant) ? kNames[variant] : NULL;
}

extern "C" const char *xr_error_string(int status)
{
    switch (status) {
    case XR_OK: return "ok";
    case XR_EINVAL: return "invalid argument";
    case XR_EZERO_STATE: return "all-zero generator state";
    case XR_ENOMEM: return "out of device memory";
    case XR_ECUDA: return "CUDA error";
    case XR_ETIMEOUT: return "device-side wait timed out";
    case XR_EUNSUPPORTED: return "not supported";
    default: return "unknown status";
    }
}

extern "C" int xr_jump_log2(int variant, int kind)
{
    if (!variant_ok(variant)) return -1;
    const int n = xr_state_bits(variant);
    if (kind == XR_JUMP) return n / 2;
    if (kind == XR_LONG_JUMP) return 3 * n / 4;
    return -1;
}

static bool dtype_ok(int variant, int dtype)
{
    if (dtype == XR_F64 || dtype == XR_F32) return true;
    if (dtype == XR_U64) return xr_word_bits(variant) == 64;
    if (dtype == XR_U32) return xr_word_bits(variant) == 32;
    return false;
}

// ---------------------------------------------------------------- context

// Jump distances (log2) that get power sets: jump, long jump, fill_seq segment.
static void pset_dists(int engine, int *d)
{
    const int n = engine_bits(engine);
    d[0] = n / 2;
    d[1] = 3 * n / 4;
    d[2] = 10;
    d[3] = 0;
}

namespace xr {
int ensure_engine(xr_ctx *ctx, int engine)
{
    if (ctx->tables[engine]) return XR_OK;
    std::lock_guard<std::mutex> lk(*(std::mutex *)ctx->lazy_mutex);
    if (ctx->tables[engine]) return XR_OK;
    const size_t n = (size_t)engine_bits(engine);
    uint32_t *t = nullptr;
    cudaError_t e = cudaMalloc((void **)&t, n * n * n / 8);
    if (e == cudaSuccess) e = launch_build_tables(engine, t, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(t);
        return status_of(e);
    }
    ctx->tables[engine] = t;
    return XR_OK;
}

int pset_index(int engine, int d)
{
    if (engine >= NUM_PSET_ENGINES) return -1;
    int dists[NUM_PSET_DISTS];
    pset_dists(engine, dists);
    for (int di = 0; di < NUM_PSET_DISTS; ++di)
        if (dists[di] == d) return di;
    return -1;
}

const uint32_t *pset_sets(const xr_ctx *ctx, int engine, int di)
{
    const size_t n = (size_t)engine_bits(engine);
    const size_t set_words = (size_t)PSET_SIZE * n * (n / 32);
    return ctx->psets[engine] + (size_t)di * PSET_LEVELS * set_words;
}

const uint32_t *dist_sets(xr_ctx *ctx, int engine, int d)
{
    if (engine >= NUM_PSET_ENGINES || d < 0 || d >= engine_bits(engine) || !ctx->tables[engine]) return nullptr;
    uint32_t *p = __atomic_load_n(&ctx->dist_sets[engine][d], __ATOMIC_ACQUIRE);
    if (p) return p;
    std::lock_guard<std::mutex> lk(*(std::mutex *)ctx->lazy_mutex);
    p = ctx->dist_sets[engine][d];
    if (p) return p;
    const size_t n = (size_t)engine_bits(engine);
    cudaError_t e = cudaMalloc((void **)&p, (size_t)PSET_LEVELS * PSET_SIZE * n * (n / 32) * 4);
    if (e == cudaSuccess) e = launch_build_power_sets(engine, ctx->tables[engine], &d, 1, p, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(p);
        return nullptr;
    }
    __atomic_store_n(&ctx->dist_sets[engine][d], p, __ATOMIC_RELEASE);
    return p;
}

const uint32_t *dist_sets_outside_capture(xr_ctx *ctx, int engine, int d, cudaStream_t st)
{
    if (engine >= NUM_PSET_ENGINES || d < 0 || d >= engine_bits(engine)) return nullptr;
    uint32_t *p = __atomic_load_n(&ctx->dist_sets[engine][d], __ATOMIC_ACQUIRE);
    if (p) return p;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
    return dist_sets(ctx, engine, d);
}
}  // namespace xr

extern "C" int xr_ctx_destroy(xr_ctx *ctx)
{
    if (!ctx) return XR_OK;
    DeviceScope dscope(ctx->device);
    cudaDeviceSynchronize();
    for (int e = 0; e < NUM_ENGINES; ++e) {
        cudaFree(ctx->tables[e]);
        cudaFree(ctx->psets[e]);
        for (int d = 0; d < 256; ++d) cudaFree(ctx->dist_sets[e][d]);
    }
    cudaFree(ctx->d_status);
    cudaFree(ctx->scratch);
    for (int b = 0; b < 2; ++b) {
        cudaFree(ctx->staging[b]);
        cudaFree(ctx->chunk_states[b]);
        if (ctx->ev_gen[b]) cudaEventDestroy(ctx->ev_gen[b]);
        if (ctx->ev_copy[b]) cudaEventDestroy(ctx->ev_copy[b]);
    }
    cudaFree(ctx->base_state);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    delete (std::mutex *)ctx->lazy_mutex;
    free(ctx);
    return XR_OK;
}

extern "C" int xr_ctx_create(int device, xr_ctx **out)
{
    if (!out) return XR_EINVAL;
    *out = NULL;
    if (cudaSetDevice(device) != cudaSuccess) return XR_ECUDA;
    xr_ctx *ctx = (xr_ctx *)calloc(1, sizeof(xr_ctx));
    if (!ctx) return XR_ENOMEM;
    ctx->device = device;
    ctx->lazy_mutex = new std::mutex();
    cudaDriverEntryPointQueryResult q;
    void *fn = NULL;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        ctx->encode = (EncodeTiledFn)fn;
    cudaGetLastError();
    int rc = XR_OK;
    for (int e = 0; e < NUM_PSET_ENGINES && rc == XR_OK; ++e) {
        const size_t n = (size_t)engine_bits(e);
        rc = status_of(cudaMalloc((void **)&ctx->tables[e], n * n * n / 8));
        if (rc == XR_OK) rc = status_of(launch_build_tables(e, ctx->tables[e], 0));
        const size_t pset_bytes = (size_t)NUM_PSET_DISTS * PSET_LEVELS * PSET_SIZE * n * n / 8;
        if (rc == XR_OK) rc = status_of(cudaMalloc((void **)&ctx->psets[e], pset_bytes));
        int dists[NUM_PSET_DISTS];
        pset_dists(e, dists);
        if (rc == XR_OK)
            rc = status_of(launch_build_power_sets(e, ctx->tables[e], dists, NUM_PSET_DISTS, ctx->psets[e], 0));
    }
    if (rc == XR_OK) rc = status_of(cudaMalloc((void **)&ctx->d_status, sizeof(int)));
    if (rc == XR_OK) rc = status_of(cudaMemset(ctx->d_status, 0, sizeof(int)));
    if (rc == XR_OK) rc = status_of(cudaMalloc(&ctx->base_state, XR_MAX_STATE_BYTES));
    if (rc == XR_OK) rc = status_of(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
    for (int b = 0; b < 2 && rc == XR_OK; ++b) {
        rc = status_of(cudaEventCreateWithFlags(&ctx->ev_gen[b], cudaEventDisableTiming));
        if (rc == XR_OK) rc = status_of(cudaEventCreateWithFlags(&ctx->ev_copy[b], cudaEventDisableTiming));
    }
    if (rc == XR_OK) rc = status_of(cudaDeviceSynchronize());
    if (rc != XR_OK) {
        xr_ctx_destroy(ctx);
        return rc == XR_EINVAL ? XR_ECUDA : rc;
    }
    *out = ctx;
    return XR_OK;
}

extern "C" int xr_status(xr_ctx *ctx, int reset)
{
    if (!ctx) return XR_EINVAL;
    DeviceScope dscope(ctx->device);
    int h = 0;
    if (cudaMemcpy(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return XR_ECUDA;
    if (reset && cudaMemset(ctx->d_status, 0, sizeof(int)) != cudaSuccess) return XR_ECUDA;
    return h;
}

extern "C" int xr_jump_table(xr_ctx *ctx, int variant, int k, void *h_out)
{
    if (!ctx || !variant_ok(variant) || !h_out) return XR_EINVAL;
    DeviceScope dscope(ctx->device);
    {
        const int erc = ensure_engine(ctx, engine_of(variant));
        if (erc != XR_OK) return erc;
    }
    const int e = engine_of(variant);
    const size_t n = (size_t)engine_bits(e);
    if (k < 0 || (size_t)k >= n) return XR_EINVAL;
    const size_t bytes = n * n / 8;
    return status_of(cudaMemcpy(h_out, (const char *)ctx->tables[e] + (size_t)k * bytes, bytes,
                                cudaMemcpyDeviceToHost));
}

// ---------------------------------------------------------------- seeding, states

extern "C" int xr_seed(xr_ctx *ctx, int variant, uint64_t seed, void *d_state, void *stream)
{
    if (!ctx || !variant_ok(variant) || !d_state || ((uintptr_t)d_state % 16)) return XR_EINVAL;
    DeviceScope dscope(ctx->device);
    NvtxRange nvtx("xr_seed");
    return status_of(launch_seed(variant, NULL, seed, 1, d_state, ctx->d_status, (cudaStream_t)stream));
}

extern "C" int xr_seed_many(xr_ctx *ctx, int variant, const uint64_t *d_seeds, size_t count,
                            void *d_states, void *stream)
{
    if (!ctx || !variant_ok(variant)) return XR_EINVAL;
    DeviceScope dscope(ctx->device);
    NvtxRange nvtx("xr_seed_many");
    if (count == 0) return XR_OK;
    if (!d_seeds || !d_states || ((uintptr_t)d_states % 16) || ((uintptr_t)d_seeds % 8))
        return XR_EINVAL;
    return status_of(launch_seed(variant, d_seeds, 0, count, d_states, ctx->d_status, (cudaStream_t)stream));
}

extern "C" int xr_set_state(xr_ctx *ctx, int variant, const void *h_words, void *d_state, void *stream)
{
    if (!ctx || !variant_ok(variant) || !h_words || !d_state) return XR_EINVAL;
    DeviceScope dscope(ctx->device);
    const int nb = xr_state_bytes(variant);
    unsigned char any = 0;
    for (int b = 0; b < nb; ++b) any |= ((const unsigned char *)h_words)[b];
    if (!any) return XR_EZERO_STATE;
    return status_of(cudaMemcpyAsync(d_state, h_words, (size_t)nb, cudaMemcpyHostToDevice,
                                     (cudaStream_t)stream));
}

extern "C" int xr_get_state(xr_ctx *ctx, int variant, const void *d_state, void *h_words, void *stream)
{
    if (!ctx || !variant_ok(variant) || !h_words || !d_state) return XR_EINVAL;
    DeviceScope dscope(ctx->device);
    cudaError_t e = cudaMemcpyAsync(h_words, d_state, (size_t)xr_state_bytes(variant),
                                    cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    return status_of(e);
}

// ---------------------------------------------------------------- jumps

// Matrix indices k = (d + b) mod n for the set bits b of e.
static KList klist(uint64_t e, int d, int n)
{
    KList ks;
    ks.n = 0;
    for (int b = 0; b < 64; ++b)
        if ((e >> b) & 1u) ks.k[ks.n++] = (d + b) % n;
    return ks;
}

static bool states_ok(const void *p) { return p && ((uintptr_t)p % 16) == 0; }

extern "C" int xr_jump(xr_ctx *ctx, int variant, int kind, void *d_states, size_t count,
                       uint64_t times, void *stream)
{
    if (!ctx || !variant_ok(variant) || (kind != XR_JUMP && kind != XR_LONG_JUMP)) return XR_EINVAL;
    DeviceScope dscope(ctx->device);
    NvtxRange nvtx("xr_jump");
    if (count == 0 || times == 0) return XR_OK;
    if (!states_ok(d_states)) return XR_EINVAL;
    {
        const int erc = ensure_engine(ctx, engine_of(variant));
        if (erc != XR_OK) return erc;
    }
    const int e = engine_of(variant);
    return status_of(launch_apply_pow(e, ctx->tables[e], klist(times, xr_jump_log2(variant, kind), engine_bits(e)),
                                      d_states, count, (cudaStream_t)stream));
}

extern "C" int xr_advance(xr_ctx *ctx, int variant, void *d_states, size_t count, uint64_t nsteps,
                          void *stream)
{
    if (!ctx || !variant_ok(variant)) return XR_EINVAL;
    DeviceScope dscope(ctx->device);
    NvtxRange nvtx("xr_advance");
    if (count == 0 || nsteps == 0) return XR_OK;
    if (!states_ok(d_states)) return XR_EINVAL;
    {
        const int erc = ensure_engine(ctx, engine_of(variant));
        if (erc != XR_OK) return erc;
    }
    const int e = engine_of(variant);
    return status_of(launch_apply_pow(e, ctx->tables[e], klist(nsteps, 0, engine_bits(e)), d_states,
                                      count, (cudaStream_t)stream));
}

// out[i] = (T^(2^d))^(first + i) base for i < S.  With `cached`, a chunk of
// 512 P streams (P the largest power of two, at least 32, that fits) takes
// its P parents from the path below and its other streams p + P j from one
// launch over the level-0 power set of the distance 2^d P (built once and
// kept in the context; not built under stream capture), whose warps load
// and store contiguous states; the rest of the range follows the same way.
// Callers that must not allocate pass cached = false.
static cudaError_t make_streams(xr_ctx *ctx, int variant, int d, const void *d_base, uint64_t first,
                                size_t S, void *out, cudaStream_t st, bool cached = true)
{
    if (S == 0) return cudaSuccess;
    const int e = engine_of(variant);
    const int di = pset_index(e, d);
    cudaError_t err;
    if (cached && e < NUM_PSET_ENGINES && S >= (size_t)PSET_SIZE * 32 && first <= UINT64_MAX - (S - 1)) {
        size_t P = 32;
        int k = 5;
        while (P * 2 * PSET_SIZE <= S) {
            P *= 2;
            ++k;
        }
        const uint32_t *Q = dist_sets_outside_capture(ctx, e, (d + k) % engine_bits(e), st);
        if (Q) {
            const size_t sb = (size_t)xr_state_bytes(variant), chunk = P * PSET_SIZE;
            err = make_streams(ctx, variant, d, d_base, first, P, out, st, false);
            if (err == cudaSuccess) err = launch_streams_jmajor(e, Q, out, P, st);
            if (err == cudaSuccess && S > chunk)
                err = make_streams(ctx, variant, d, d_base, first + chunk, S - chunk, (char *)out + chunk * sb, st,
                                   true);
            return err;
        }
    }
    if (first && di >= 0) {
        // J^first(base) by one warp from the power sets of this distance
        err = launch_warp_jump(e, pset_sets(ctx, e, di), ctx->tables[e], d, d_base, out, first, st);
    } else {
        err = cudaMemcpyAsync(out, d_base, (size_t)xr_state_bytes(variant), cudaMemcpyDeviceToDevice, st);
        if (err == cudaSuccess && first)
            err = launch_apply_pow(e, ctx->tables[e], klist(first, d, engine_bits(e)), out, 1, st);
    }
    if (err != cudaSuccess) return err;
    if (di >= 0 && S <= ((size_t)1 << (PSET_BITS * PSET_LEVELS)))
        return launch_streams_psets(e, pset_sets(ctx, e, di), out, S, st);
    return launch_tree(e, ctx->tables[e], d, out, S, st);
}

extern "C" int xr_make_streams(xr_ctx *ctx, int variant, int kind, const void *d_base, uint64_t first,
                               size_t S, void *d_states_out, void *stream)
{
    if (!ctx || !variant_ok(variant) || (kind != XR_JUMP && kind != XR_LONG_JUMP)) return XR_EINVAL;
    DeviceScope dscope(ctx->device);
    NvtxRange nvtx("xr_make_streams");
    if (S == 0) return XR_OK;
    if (!states_ok(d_base) || !states_ok(d_states_out)) return XR_EINVAL;
    const size_t sb = (size_t)xr_state_bytes(variant);
    const char *b = (const char *)d_base, *o = (const char *)d_states_out;
    if (b < o + S * sb && o < b + sb) return XR_EINVAL;  // overlap
    {
        const int erc = ensure_engine(ctx, engine_of(variant));
        if (erc != XR_OK) return erc;
    }
    return status_of(make_streams(ctx, variant, xr_jump_log2(variant, kind), d_base, first, S,
                                  d_states_out, (cudaStream_t)stream));
}

// Streams J^(first + i)(base), i < S, m outputs each, without a state table
// in global memory.  In chunks of 512 P streams, P the largest power of two
// (at least 32) that fits: the P parents are streams first + done + p
// (xr_make_streams over the scratch), and stream p + P j of the chunk starts
// at P_0[j] parent_p with P_0 the level-0 power set of the distance
// 2^(d + log2 P) (built once per distance and cached).  The lanes of a warp
// are then 32 consecutive streams sharing one matrix.  Rows over 512 bytes,
// fewer than 512 x 32 streams left, engines without power sets and shapes
// the tile store cannot describe go through a state table in the scratch.
static cudaError_t ensure(void **p, size_t *have, size_t want);

static cudaError_t fill_streams(xr_ctx *ctx, int variant, int d, const void *d_base, uint64_t first, size_t S,
                                size_t m, int dtype, void *out, cudaStream_t st)
{
    const int e = engine_of(variant);
    const int n = engine_bits(e);
    const size_t sb = (size_t)xr_state_bytes(variant), es = (size_t)xr_dtype_bytes(dtype);
    // short rows (at most 4 tiles of 128 bytes) that the tile store can take;
    // the launcher checks the same
    const bool tiles_ok = ctx->encode && ((uintptr_t)out % 16) == 0 && ((m * es) % 16) == 0 && m * es <= 512 &&
                          S < (1ull << 31);
    const size_t min_chunk = (size_t)PSET_SIZE * 32;
    cudaError_t err = cudaSuccess;
    size_t done = 0;  // streams written by the fused kernels
    if (e < NUM_PSET_ENGINES && tiles_ok) {
        while (S - done >= min_chunk) {
            size_t P = 32;
            int k = 5;
            while (P * 2 * PSET_SIZE <= S - done) {
                P *= 2;
                ++k;
            }
            // not built under stream capture (or if building fails): the rest
            // of the range then takes the state table
            const uint32_t *Q = dist_sets_outside_capture(ctx, e, (d + k) % n, st);
            if (!Q) break;
            size_t cap = ctx->scratch_bytes;
            err = ensure(&ctx->scratch, &cap, P * sb);
            ctx->scratch_bytes = cap;
            if (err == cudaSuccess) err = make_streams(ctx, variant, d, d_base, first + done, P, ctx->scratch, st);
            if (err == cudaSuccess)
                err = launch_fill_streams(variant, dtype, Q, ctx->scratch, P, m, (char *)out + done * m * es,
                                          ctx->d_status, st, ctx->encode);
            if (err != cudaSuccess) return err;
            done += P * PSET_SIZE;
        }
    }
    const size_t rest = S - done;
    if (rest == 0) return cudaSuccess;
    // the remaining streams through a state table
    size_t cap = ctx->scratch_bytes;
    err = ensure(&ctx->scratch, &cap, rest * sb);
    ctx->scratch_bytes = cap;
    if (err != cudaSuccess) return err;
    err = make_streams(ctx, variant, d, d_base, first + done, rest, ctx->scratch, st);
    if (err == cudaSuccess)
        err = launch_fill(variant, dtype, XR_STREAM_MAJOR, ctx->scratch, rest, m, m, (char *)out + done * m * es, 0,
                          ctx->d_status, st, ctx->encode);
    return err;
}

extern "C" int xr_fill_streams(xr_ctx *ctx, int variant, int kind, const void *d_base, uint64_t first, size_t S,
                               size_t m, int dtype, void *d_out, void *stream)
{
    if (!ctx || !variant_ok(variant) || !dtype_ok(variant, dtype)) return XR_EINVAL;
    if (kind != XR_JUMP && kind != XR_LONG_JUMP) return XR_EINVAL;
    DeviceScope dscope(ctx->device);
    NvtxRange nvtx("xr_fill_streams");
    if (S == 0 || m == 0) return XR_OK;
    const size_t es = (size_t)xr_dtype_bytes(dtype);
    if (!states_ok(d_base) || !d_out || ((uintptr_t)d_out % es) || m > (SIZE_MAX / es) / S) return XR_EINVAL;
    if (first > UINT64_MAX - (S - 1)) return XR_EINVAL;  // stream indices first .. first + S - 1 in 64 bits
    {
        const int erc = ensure_engine(ctx, engine_of(variant));
        if (erc != XR_OK) return erc;
    }
    return status_of(fill_streams(ctx, variant, xr_jump_log2(variant, kind), d_base, first, S, m, dtype, d_out,
                                  (cudaStream_t)stream));
}

// ---------------------------------------------------------------- generation

static int fill_args_ok(int variant, void *d_states, size_t S, size_t m, int dtype, int layout, void *d_out)
{
    if (!variant_ok(variant) || !dtype_ok(variant, dtype)) return 0;
    if (layout != XR_STREAM_MAJOR && layout != XR_INTERLEAVED) return 0;
    if (S == 0) return 1;
    if (!states_ok(d_states)) return 0;
    if (m == 0) return 1;
    const size_t es = (size_t)xr_dtype_bytes(dtype);
    if (!d_out || ((uintptr_t)d_out % es)) return 0;
    if (m > (SIZE_MAX / es) / S) return 0;
    return 1;
}

extern "C" int xr_fill(xr_ctx *ctx, int variant, void *d_states, size_t S, size_t m, int dtype,
                       int layout, void *d_out, int write_back, void *stream)
{
    if (!ctx || !fill_args_ok(variant, d_states, S, m, dtype, layout, d_out)) return XR_EINVAL;
    DeviceScope dscope(ctx->device);
    NvtxRange nvtx("xr_fill");
    if (S == 0 || m == 0) return XR_OK;
    return status_of(launch_fill(variant, dtype, layout, d_states, S, m, m, d_out, write_back,
                                 ctx->d_status, (cudaStream_t)stream, ctx->encode));
}

static cudaError_t ensure(void **p, size_t *have, size_t want)
{
    if (*have >= want && *p) return cudaSuccess;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    cudaFree(*p);
    *p = NULL;
    *have = 0;
    e = cudaMalloc(p, want);
    if (e == cudaSuccess) *have = want;
    return e;
}

extern "C" int xr_fill_seq(xr_ctx *ctx, int variant, void *d_state, size_t n, int dtype, void *d_out,
                           void *stream)
{
    if (!ctx || !variant_ok(variant) || !dtype_ok(variant, dtype)) return XR_EINVAL;
    DeviceScope dscope(ctx->device);
    NvtxRange nvtx("xr_fill_seq");
    if (n == 0) return XR_OK;
    const size_t es = (size_t)xr_dtype_bytes(dtype);
    if (!states_ok(d_state) || !d_out || ((uintptr_t)d_out % es)) return XR_EINVAL;
    {
        const int erc = ensure_engine(ctx, engine_of(variant));
        if (erc != XR_OK) return erc;
    }
    const cudaStream_t st = (cudaStream_t)stream;
    const size_t seg = (size_t)1 << SEQ_LOG2;
    const size_t full = n / seg, tail = n % seg, P = full + (tail ? 1 : 0);
    const size_t sb = (size_t)xr_state_bytes(variant);
    size_t cap = ctx->scratch_bytes;
    cudaError_t err = ensure(&ctx->scratch, &cap, P * sb);
    ctx->scratch_bytes = cap;
    if (err != cudaSuccess) return status_of(err);
    // segment p starts at T^(p * 2^SEQ_LOG2) s
    err = make_streams(ctx, variant, SEQ_LOG2, d_state, 0, P, ctx->scratch, st, false);
    if (err == cudaSuccess && full)
        err = launch_fill(variant, dtype, XR_STREAM_MAJOR, ctx->scratch, full, seg, seg, d_out, 1,
                          ctx->d_status, st, ctx->encode);
    if (err == cudaSuccess && tail)
        err = launch_fill(variant, dtype, XR_STREAM_MAJOR, (char *)ctx->scratch + full * sb, 1, tail,
                          seg, (char *)d_out + full * seg * es, 1, ctx->d_status, st, ctx->encode);
    // the last segment's written-back state is T^n s
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(d_state, (char *)ctx->scratch + (P - 1) * sb, sb,
                              cudaMemcpyDeviceToDevice, st);
    return status_of(err);
}

extern "C" int xr_fill_host(xr_ctx *ctx, int variant, int kind, const void *h_base, uint64_t first,
                            size_t S, size_t m, int dtype, void *h_out, void *stream)
{
    if (!ctx || !variant_ok(variant) || !dtype_ok(variant, dtype) || !h_base) return XR_EINVAL;
    DeviceScope dscope(ctx->device);
    NvtxRange nvtx("xr_fill_host");
    if (kind != XR_JUMP && kind != XR_LONG_JUMP) return XR_EINVAL;
    if (S == 0 || m == 0) return XR_OK;
    if (!h_out) return XR_EINVAL;
    const size_t es = (size_t)xr_dtype_bytes(dtype);
    if (m > (SIZE_MAX / es) / S) return XR_EINVAL;
    if (first > UINT64_MAX - (S - 1)) return XR_EINVAL;  // stream indices first .. first + S - 1 in 64 bits
    const size_t sb = (size_t)xr_state_bytes(variant);
    unsigned char any = 0;
    for (size_t b = 0; b < sb; ++b) any |= ((const unsigned char *)h_base)[b];
    if (!any) return XR_EZERO_STATE;
    {
        const int erc = ensure_engine(ctx, engine_of(variant));
        if (erc != XR_OK) return erc;
    }
    const cudaStream_t st = (cudaStream_t)stream;
    const size_t row = m * es;
    size_t ch = HOST_STAGING_BYTES / row;
    if (ch == 0) ch = 1;
    if (ch > S) ch = S;
    cudaError_t err = cudaSuccess;
    if (ctx->staging_bytes < ch * row || ctx->chunk_states_bytes < ch * sb) {
        err = cudaDeviceSynchronize();
        for (int b = 0; b < 2; ++b) {
            cudaFree(ctx->staging[b]);
            cudaFree(ctx->chunk_states[b]);
            ctx->staging[b] = ctx->chunk_states[b] = NULL;
        }
        ctx->staging_bytes = ctx->chunk_states_bytes = 0;
        for (int b = 0; b < 2 && err == cudaSuccess; ++b) {
            err = cudaMalloc(&ctx->staging[b], ch * row);
            if (err == cudaSuccess) err = cudaMalloc(&ctx->chunk_states[b], ch * sb);
        }
        if (err != cudaSuccess) return status_of(err);
        ctx->staging_bytes = ch * row;
        ctx->chunk_states_bytes = ch * sb;
    }
    const int d = xr_jump_log2(variant, kind);
    err = cudaMemcpyAsync(ctx->base_state, h_base, sb, cudaMemcpyHostToDevice, st);
    size_t c = 0;
    for (size_t s0 = 0; s0 < S && err == cudaSuccess; s0 += ch, ++c) {
        const int b = (int)(c & 1);
        const size_t cnt = (S - s0) < ch ? (S - s0) : ch;
        if (c >= 2) err = cudaStreamWaitEvent(st, ctx->ev_copy[b], 0);
        if (err == cudaSuccess)
            err = make_streams(ctx, variant, d, ctx->base_state, first + s0, cnt, ctx->chunk_states[b], st);
        if (err == cudaSuccess)
            err = launch_fill(variant, dtype, XR_STREAM_MAJOR, ctx->chunk_states[b], cnt, m, m,
                              ctx->staging[b], 0, ctx->d_status, st, ctx->encode);
        if (err == cudaSuccess) err = cudaEventRecord(ctx->ev_gen[b], st);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(ctx->side, ctx->ev_gen[b], 0);
        if (err == cudaSuccess)
            err = cudaMemcpyAsync((char *)h_out + s0 * row, ctx->staging[b], cnt * row,
                                  cudaMemcpyDeviceToHost, ctx->side);
        if (err == cudaSuccess) err = cudaEventRecord(ctx->ev_copy[b], ctx->side);
    }
    cudaError_t e2 = cudaStreamSynchronize(ctx->side);
    cudaError_t e3 = cudaStreamSynchronize(st);
    if (err == cudaSuccess) err = e2;
    if (err == cudaSuccess) err = e3;
    return status_of(err);
}

// ---------------------------------------------------------------- no-allocation variant
//
// xr_fill_seq_noalloc: the same computation as xr_fill_seq, for callers that
// must not allocate device memory while they run (see include/xr.h).  The
// segment start states live in the file-scope device array below instead of
// context scratch, so the call itself never calls cudaMalloc or cudaFree.

static __device__ __align__(256) unsigned char g_noalloc_segments[XR_NOALLOC_SCRATCH_BYTES];
static_assert(((XR_NOALLOC_MAX_OUTPUTS >> SEQ_LOG2_NOALLOC) * 32) == XR_NOALLOC_SCRATCH_BYTES,
              "the largest call of a 32-byte state fills the array exactly");

// Device address of g_noalloc_segments on each device, looked up once per
// device (with that device current) by the first call made on it.  In host
// code the array's name is only a host-side stand-in, never a device address.
static std::atomic<void *> g_noalloc_addr[64];

static int noalloc_scratch(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return XR_ECUDA;
    void *p = g_noalloc_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        if (cudaGetSymbolAddress(&p, g_noalloc_segments) != cudaSuccess || !p) return XR_ECUDA;
        g_noalloc_addr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return XR_OK;
}

extern "C" int xr_fill_seq_noalloc(xr_ctx *ctx, int variant, void *d_state, size_t n, int dtype,
                                   void *d_out, void *stream)
{
    if (!ctx || !variant_ok(variant) || !dtype_ok(variant, dtype)) return XR_EINVAL;
    DeviceScope dscope(ctx->device);
    NvtxRange nvtx("xr_fill_seq_noalloc");
    const size_t sb = (size_t)xr_state_bytes(variant);
    // P segment states of sb bytes must fit the array: n <= 2^26 for states of
    // up to 32 bytes, 2^25 for xoshiro512, 2^24 for xoroshiro1024
    if (n > XR_NOALLOC_MAX_OUTPUTS_FOR(sb)) return XR_EINVAL;
    if (n == 0) return XR_OK;
    const size_t es = (size_t)xr_dtype_bytes(dtype);
    if (!states_ok(d_state) || !d_out || ((uintptr_t)d_out % es)) return XR_EINVAL;
    // the jump tables must exist already: building them would allocate
    if (!ctx->tables[engine_of(variant)]) return XR_EUNSUPPORTED;
    void *scratch = NULL;
    const int rc = noalloc_scratch(&scratch);
    if (rc != XR_OK) return rc;
    const cudaStream_t st = (cudaStream_t)stream;
    const size_t seg = (size_t)1 << SEQ_LOG2_NOALLOC;
    const size_t full = n / seg, tail = n % seg, P = full + (tail ? 1 : 0);
    if (P * sb > sizeof(g_noalloc_segments)) return XR_EINVAL;
    // Every slot read below is written first in this call (make_streams fills
    // slots 0 .. P-1: the base copy, then the stream starts), so nothing has
    // to start at zero.
    cudaError_t err = make_streams(ctx, variant, SEQ_LOG2_NOALLOC, d_state, 0, P, scratch, st, false);
    if (err == cudaSuccess && full)
        err = launch_fill(variant, dtype, XR_STREAM_MAJOR, scratch, full, seg, seg, d_out, 1,
                          ctx->d_status, st, ctx->encode);
    if (err == cudaSuccess && tail)
        err = launch_fill(variant, dtype, XR_STREAM_MAJOR, (char *)scratch + full * sb, 1, tail, seg,
                          (char *)d_out + full * seg * es, 1, ctx->d_status, st, ctx->encode);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(d_state, (char *)scratch + (P - 1) * sb, sb, cudaMemcpyDeviceToDevice, st);
    return status_of(err);
}
