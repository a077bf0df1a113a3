// xr_analysis.cu -- the paper's analysis workloads on the device.
//
// Escaping zeroland (Sec. 8): starting from each of the n states with
// exactly one bit set, how fast do the outputs reach half ones?  One thread
// per one-bit state keeps a running count of one bits over a window of
// `window` consecutive outputs and adds it to counts[t] for every window start
// t; the curve in the paper is counts[t] / (n * window * w).
#include <algorithm>

#include "xr_device.cuh"
#include "xr_internal.h"

namespace xr {

template <int V>
__global__ void k_zeroland(size_t nout, int window, unsigned long long *counts)
{
    typedef Gen<V> G;
    typedef typename G::E E;
    typedef typename G::word W;
    constexpr int w = 8 * (int)sizeof(W);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= E::NBITS) return;
    E e;
#pragma unroll
    for (int k = 0; k < E::K; ++k) e.s[k] = (k == j / w) ? ((W)1 << (j % w)) : (W)0;
    u32 ring[64];  // popcounts of the last `window` outputs
    u32 sum = 0;
    for (size_t i = 0; i < nout; ++i) {
        const u32 c = (u32)__popcll((u64)G::out(e));
        e.step();
        if (i >= (size_t)window) sum -= ring[i % window];
        ring[i % window] = c;
        sum += c;
        if (i + 1 >= (size_t)window) atomicAdd(counts + (i + 1 - window), (unsigned long long)sum);
    }
}

template <int V>
static cudaError_t zeroland_v(size_t nout, int window, unsigned long long *counts, cudaStream_t st)
{
    constexpr int n = Gen<V>::E::NBITS;
    k_zeroland<V><<<(n + 127) / 128, 128, 0, st>>>(nout, window, counts);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_zeroland(int variant, size_t nout, int window, unsigned long long *counts, cudaStream_t st)
{
    switch (variant) {
    case 0: return zeroland_v<0>(nout, window, counts, st);
    case 1: return zeroland_v<1>(nout, window, counts, st);
    case 2: return zeroland_v<2>(nout, window, counts, st);
    case 3: return zeroland_v<3>(nout, window, counts, st);
    case 4: return zeroland_v<4>(nout, window, counts, st);
    case 5: return zeroland_v<5>(nout, window, counts, st);
    case 6: return zeroland_v<6>(nout, window, counts, st);
    case 7: return zeroland_v<7>(nout, window, counts, st);
    case 8: return zeroland_v<8>(nout, window, counts, st);
    case 9: return zeroland_v<9>(nout, window, counts, st);
    case 10: return zeroland_v<10>(nout, window, counts, st);
    case 11: return zeroland_v<11>(nout, window, counts, st);
    case 12: return zeroland_v<12>(nout, window, counts, st);
    case 13: return zeroland_v<13>(nout, window, counts, st);
    case 14: return zeroland_v<14>(nout, window, counts, st);
    case 15: return zeroland_v<15>(nout, window, counts, st);
    case 16: return zeroland_v<16>(nout, window, counts, st);
    case 17: return zeroland_v<17>(nout, window, counts, st);
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------- linear complexity

static constexpr size_t LC_SMEM_BYTES = 226 * 1024;
//
// Berlekamp-Massey over F2 (Sec. 9.3; the paper computes Table 13's lowest
// values this way) on bit `bit` of the first N outputs.  The bit sequence is
// stored reversed and packed (bit j of rev = s_{N-1-j}), so the window s_n,
// s_{n-1}, ..., s_{n-L} lines up with the connection polynomial's
// coefficients c_0 .. c_L starting at bit N-1-n.
//
// Thread p produces outputs p * chunk .. (p + 1) * chunk - 1: it jumps its
// copy of the state by T^(p * chunk) with the context's tables of T^(2^k)
// (one F2 matrix-vector product per set bit), then steps.  Words shared with
// the neighbouring chunks are merged with atomicOr into the zeroed array.
template <int V>
__global__ void __launch_bounds__(128)
    k_lc_bits(const u32 *__restrict__ tables, const void *state, int bit, size_t N, size_t chunk, u32 *rev)
{
    typedef Gen<V> G;
    typedef typename G::E E;
    constexpr int n = E::NBITS, NW = n / 32;
    const size_t t0 = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * chunk;
    if (t0 >= N) return;
    E e;
    load_state(e, state);
    u32 v[NW], r[NW];
    to_words(e, v);
    for (int k = 0; (t0 >> k) != 0; ++k) {
        if (!((t0 >> k) & 1)) continue;
        f2_matvec<NW, false>(tables + (size_t)k * n * NW, v, r);
#pragma unroll
        for (int j = 0; j < NW; ++j) v[j] = r[j];
    }
    from_words(e, v);
    const size_t t1 = t0 + chunk < N ? t0 + chunk : N;
    u32 acc = 0u;
    for (size_t t = t0; t < t1; ++t) {
        const size_t pos = N - 1 - t;
        acc |= (u32)((G::out(e) >> bit) & 1u) << (pos & 31);
        e.step();
        if ((pos & 31) == 0 || t + 1 == t1) {
            atomicOr(rev + (pos >> 5), acc);
            acc = 0u;
        }
    }
}

// One CTA.  C (the connection polynomial), B (C before the last length
// change) and a free buffer X live in shared memory, W words each; a length
// change writes C ^ x^m B into X and rotates the three roles instead of
// copying.  deg C <= L and deg B <= L_B always (so each buffer is zero above
// those words), and deg x^m B = m + L_B <= n + 1 - L at step n: every update
// stays within (max(L, n + 1 - L) >> 5) + 1 words.  A complexity that needs
// more than 32 W - 1 bits sets *overflow instead of a result.
//
// One pass and one barrier per sequence bit: step n applies its update
// (known from d_n) to the words a thread owns and, on the same words,
// accumulates the next discrepancy d_{n+1} = <C_{n+1}, s_{n+1} .. s_{n+1-L}>.
// Word w belongs to thread w mod blockDim.x in every role, so a thread only
// reads back C words it wrote itself; B and X are not written while read.
// Warp parities go to one byte per warp in slot (n + 1) % 2; a slot is
// rewritten two barriers after it was read.
//
// With SREV the packed sequence is staged in shared memory after the three
// polynomials; otherwise it is read through the read-only cache.
template <bool SREV>
__global__ void __launch_bounds__(1024) k_berlekamp_massey(const u32 *__restrict__ grev, size_t N, u32 W,
                                                          unsigned long long *out_L, int *overflow)
{
    extern __shared__ u32 bm[];
    __shared__ __align__(16) unsigned char wpar[2][32];
    const int tid = threadIdx.x, nth = blockDim.x, warp = tid >> 5;
    const size_t rev_words = (N + 31) / 32 + 2;
    for (u32 w = tid; w < 3 * W; w += nth) bm[w] = 0u;
    const u32 *rev = grev;
    if constexpr (SREV) {
        u32 *srev = bm + 3 * (size_t)W;
        for (size_t w = tid; w < rev_words; w += nth) srev[w] = grev[w];
        rev = srev;
    }
    for (int i = tid; i < 64; i += nth) (&wpar[0][0])[i] = 0;
    __syncthreads();
    if (tid == 0) bm[0] = 1u, bm[W] = 1u;
    // d_0 = s_0, bit N - 1 of the packed sequence
    int d = (int)((rev[(N - 1) >> 5] >> ((N - 1) & 31)) & 1u);
    __syncthreads();
    int ci = 0, bi = 1, xi = 2;
    size_t L = 0, LB = 0, m = 1;
    for (size_t n = 0; n < N; ++n) {
        // window of step n + 1: s_{n+1-i} is packed bit off + i
        const bool more = n + 1 < N;
        const size_t off = more ? N - 2 - n : 0;
        const size_t q0 = off >> 5;
        const int sh = (int)(off & 31);
        u32 acc = 0u;
        if (d) {
            const bool grow = 2 * L <= n;
            const size_t Lnew = grow ? n + 1 - L : L;
            if (Lnew >= (size_t)W * 32) {  // uniform
                if (tid == 0) *overflow = 1;
                return;
            }
            const u32 ws = (u32)(m >> 5), bs = (u32)(m & 31);
            const u32 lenB = (u32)(LB >> 5) + 1, lenC = (u32)(L >> 5) + 1;
            const u32 upto = (u32)(Lnew >> 5) + 1;
            const u32 *C = bm + ci * W;
            const u32 *B = bm + bi * W;
            u32 *X = bm + (grow ? xi : ci) * W;
            for (u32 w = tid; w < upto; w += nth) {
                u32 v = 0u;
                if (w >= ws && w - ws < lenB) v = B[w - ws] << bs;
                if (bs && w >= ws + 1 && w - ws - 1 < lenB) v |= B[w - ws - 1] >> (32 - bs);
                const u32 c = (w < lenC ? C[w] : 0u) ^ v;
                X[w] = c;
                if (more) {
                    u32 lo, hi;
                    if constexpr (SREV) {
                        lo = rev[q0 + w];
                        hi = rev[q0 + w + 1];
                    } else {
                        lo = __ldg(rev + q0 + w);
                        hi = __ldg(rev + q0 + w + 1);
                    }
                    acc ^= c & __funnelshift_r(lo, hi, sh);
                }
            }
            if (grow) {
                const int old_c = ci;
                ci = xi;
                xi = bi;
                bi = old_c;
                LB = L;
                L = Lnew;
                m = 1;
            } else {
                ++m;
            }
        } else {
            ++m;
            const u32 *C = bm + ci * W;
            const u32 nw = (u32)(L >> 5) + 1;
            if (more)
                for (u32 w = tid; w < nw; w += nth) {
                    u32 lo, hi;
                    if constexpr (SREV) {
                        lo = rev[q0 + w];
                        hi = rev[q0 + w + 1];
                    } else {
                        lo = __ldg(rev + q0 + w);
                        hi = __ldg(rev + q0 + w + 1);
                    }
                    acc ^= C[w] & __funnelshift_r(lo, hi, sh);
                }
        }
        const unsigned ball = __ballot_sync(0xffffffffu, __popc(acc) & 1);
        const int slot = (int)((n + 1) & 1);
        if ((tid & 31) == 0) wpar[slot][warp] = (unsigned char)(__popc(ball) & 1);
        __syncthreads();
        const uint4 p0 = *reinterpret_cast<const uint4 *>(&wpar[slot][0]);
        const uint4 p1 = *reinterpret_cast<const uint4 *>(&wpar[slot][16]);
        u32 x = p0.x ^ p0.y ^ p0.z ^ p0.w ^ p1.x ^ p1.y ^ p1.z ^ p1.w;
        d = __popc(x) & 1;
    }
    if (tid == 0) *out_L = (unsigned long long)L;
}

template <int V>
static int lc_bits_v(xr_ctx *ctx, const void *state, int bit, size_t N, u32 *rev, cudaStream_t st)
{
    constexpr int eng = Gen<V>::engine;
    const int rc = ensure_engine(ctx, eng);
    if (rc != XR_OK) return rc;
    // at least 256 outputs per thread, at most 2048 threads
    size_t chunk = (N + 2047) / 2048;
    chunk = chunk < 256 ? 256 : (chunk + 31) / 32 * 32;
    const size_t threads = (N + chunk - 1) / chunk;
    k_lc_bits<V><<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(ctx->tables[eng], state, bit, N, chunk, rev);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? XR_OK : XR_ECUDA;
}

static int launch_lc_bits(xr_ctx *ctx, int variant, const void *state, int bit, size_t N, u32 *rev,
                          cudaStream_t st)
{
    switch (variant) {
    case 0: return lc_bits_v<0>(ctx, state, bit, N, rev, st);
    case 1: return lc_bits_v<1>(ctx, state, bit, N, rev, st);
    case 2: return lc_bits_v<2>(ctx, state, bit, N, rev, st);
    case 3: return lc_bits_v<3>(ctx, state, bit, N, rev, st);
    case 4: return lc_bits_v<4>(ctx, state, bit, N, rev, st);
    case 5: return lc_bits_v<5>(ctx, state, bit, N, rev, st);
    case 6: return lc_bits_v<6>(ctx, state, bit, N, rev, st);
    case 7: return lc_bits_v<7>(ctx, state, bit, N, rev, st);
    case 8: return lc_bits_v<8>(ctx, state, bit, N, rev, st);
    case 9: return lc_bits_v<9>(ctx, state, bit, N, rev, st);
    case 10: return lc_bits_v<10>(ctx, state, bit, N, rev, st);
    case 11: return lc_bits_v<11>(ctx, state, bit, N, rev, st);
    case 12: return lc_bits_v<12>(ctx, state, bit, N, rev, st);
    case 13: return lc_bits_v<13>(ctx, state, bit, N, rev, st);
    case 14: return lc_bits_v<14>(ctx, state, bit, N, rev, st);
    case 15: return lc_bits_v<15>(ctx, state, bit, N, rev, st);
    case 16: return lc_bits_v<16>(ctx, state, bit, N, rev, st);
    case 17: return lc_bits_v<17>(ctx, state, bit, N, rev, st);
    default: return XR_EINVAL;
    }
}

}  // namespace xr

using namespace xr;

extern "C" int xr_linear_complexity(xr_ctx *ctx, int variant, int bit, size_t N, const void *d_state,
                                    void *d_scratch, size_t scratch_bytes, uint64_t *h_lc, void *stream)
{
    if (!ctx || variant < 0 || variant >= XR_NUM_VARIANTS || !d_state || !h_lc || !d_scratch) return XR_EINVAL;
    if (bit < 0 || bit >= xr_word_bits(variant) || N < 2 || N > XR_LC_MAX_BITS) return XR_EINVAL;
    if (((uintptr_t)d_state % 16) || ((uintptr_t)d_scratch % 16)) return XR_EINVAL;
    const size_t rev_words = (N + 31) / 32 + 2;
    const size_t l_off = (rev_words * 4 + 15) & ~(size_t)15;
    if (scratch_bytes < l_off + 16) return XR_EINVAL;
    // An N-bit prefix determines complexities up to N / 2: the polynomials get
    // N / 2 + 160 bits, and a larger complexity is reported, not computed.
    const u32 W = (u32)(N / 64 + 5);
    const size_t smem_poly = (size_t)3 * W * 4, smem_all = smem_poly + rev_words * 4;
    const bool srev = smem_all <= LC_SMEM_BYTES;
    const cudaStream_t st = (cudaStream_t)stream;
    u32 *rev = (u32 *)d_scratch;
    unsigned long long *dL = (unsigned long long *)((char *)d_scratch + l_off);
    int *dflag = (int *)(dL + 1);
    cudaError_t err = cudaMemsetAsync(d_scratch, 0, l_off + 16, st);
    if (err != cudaSuccess) return XR_ECUDA;
    const int rc = launch_lc_bits(ctx, variant, d_state, bit, N, rev, st);
    if (rc != XR_OK) return rc;
    err = cudaFuncSetAttribute(k_berlekamp_massey<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)LC_SMEM_BYTES);
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_berlekamp_massey<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)LC_SMEM_BYTES);
    if (err == cudaSuccess) {
        // about eight polynomial words per thread at the largest complexity
        unsigned threads = (unsigned)((W + 7) / 8 + 31) / 32 * 32;
        threads = threads < 32 ? 32 : threads > 1024 ? 1024 : threads;
        if (srev)
            k_berlekamp_massey<true><<<1, threads, smem_all, st>>>(rev, N, W, dL, dflag);
        else
            k_berlekamp_massey<false><<<1, threads, smem_poly, st>>>(rev, N, W, dL, dflag);
        count_launch();
        err = cudaGetLastError();
    }
    unsigned long long res[2] = {0, 0};
    if (err == cudaSuccess) err = cudaMemcpyAsync(res, dL, sizeof(res), cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return XR_ECUDA;
    if ((int)(res[1] & 0xffffffffu)) return XR_EUNSUPPORTED;
    *h_lc = res[0];
    return XR_OK;
}

extern "C" int xr_zeroland(xr_ctx *ctx, int variant, size_t nout, size_t window, uint64_t *d_counts, void *stream)
{
    if (!ctx || variant < 0 || variant >= XR_NUM_VARIANTS || !d_counts) return XR_EINVAL;
    if (window < 1 || window > 64 || nout < window || nout > ((size_t)1 << 32)) return XR_EINVAL;
    if ((uintptr_t)d_counts % 8) return XR_EINVAL;
    const cudaStream_t st = (cudaStream_t)stream;
    cudaError_t err = cudaMemsetAsync(d_counts, 0, (nout - window + 1) * sizeof(uint64_t), st);
    if (err == cudaSuccess)
        err = launch_zeroland(variant, nout, (int)window, reinterpret_cast<unsigned long long *>(d_counts), st);
    return err == cudaSuccess ? XR_OK : XR_ECUDA;
}
