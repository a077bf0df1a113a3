// xr_jump.cu -- jump tables, jump-ahead and seeding kernels of libxr.
//
// Every engine is F2-linear (Sec. 3): one step is s' = T s for an n x n matrix
// T over F2, so advancing e steps is T^e s.  The context keeps the powers
// T^(2^k), k = 0 .. n-1 (T^(2^n) = T because the characteristic polynomial
// is primitive, Sec. 6, so exponents wrap modulo n in k).  A jump by e * 2^d
// steps multiplies by T^(2^(d+b)) for each set bit b of e; start states of
// consecutive streams come from a doubling tree, one matrix-vector product per
// stream: x_{2^L + i} = T^(2^(d+L)) x_i.
#include <algorithm>

#include "xr_device.cuh"
#include "xr_f2.cuh"
#include "xr_internal.h"

namespace xr {

// ---------------------------------------------------------------- table build

// Column c of T is the step of the unit state e_c (bit c set).
template <int ENG>
__global__ void k_build_T(u32 *T)
{
    typedef typename EngineOf<ENG>::type E;
    constexpr int n = E::NBITS, NW = n / 32;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    u32 w[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) w[j] = (j == c / 32) ? (1u << (c % 32)) : 0u;
    E e;
    from_words(e, w);
    e.step();
    to_words(e, w);
#pragma unroll
    for (int j = 0; j < NW; ++j) T[(size_t)c * NW + j] = w[j];
}

// T^(2^(k+1)) = T^(2^k) T^(2^k): column c of the square is T^(2^k) applied to
// column c of T^(2^k).  One CTA of n threads walks k = 0 .. n-2, keeping the
// current matrix in shared memory (ping-pong) and writing every power out.
template <int NW>
__global__ void __launch_bounds__(NW * 32) k_square_chain(u32 *tables)
{
    constexpr int n = NW * 32;
    __shared__ __align__(16) u32 M[2][n * NW];
    const int c = threadIdx.x;
    for (int t = c; t < n * NW; t += n) M[0][t] = tables[t];
    __syncthreads();
    for (int k = 0; k + 1 < n; ++k) {
        const u32 *cur = M[k & 1];
        u32 v[NW], r[NW];
#pragma unroll
        for (int j = 0; j < NW; ++j) v[j] = cur[c * NW + j];
        f2_matvec<NW, true>(cur, v, r);
        u32 *dst = tables + (size_t)(k + 1) * n * NW + (size_t)c * NW;
#pragma unroll
        for (int j = 0; j < NW; ++j) {
            dst[j] = r[j];
            M[(k + 1) & 1][c * NW + j] = r[j];
        }
        __syncthreads();
    }
}

// For the large engines (512 and 1024 bits) one launch per power: column c
// of T^(2^(k+1)) = T^(2^k) (column c of T^(2^k)), the matrix read through
// the read-only cache with warp-uniform loads.
template <int NW>
__global__ void __launch_bounds__(128) k_square_step(const u32 *__restrict__ A, u32 *B)
{
    constexpr int n = NW * 32;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    u32 v[NW], r[NW];
    load_vec<NW>(v, A + (size_t)c * NW);
    f2_matvec<NW, false>(A, v, r);
    store_vec<NW>(r, B + (size_t)c * NW);
}

template <int ENG>
static cudaError_t build_tables_e(uint32_t *tables, cudaStream_t stream)
{
    typedef typename EngineOf<ENG>::type E;
    constexpr int n = E::NBITS, NW = n / 32;
    k_build_T<ENG><<<(n + 127) / 128, 128, 0, stream>>>(tables);
    count_launch();
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    if constexpr (NW <= 8) {
        k_square_chain<NW><<<1, n, 0, stream>>>(tables);
        count_launch();
        return cudaGetLastError();
    } else {
        const size_t mat = (size_t)n * NW;
        for (int k = 0; k + 1 < n && err == cudaSuccess; ++k) {
            k_square_step<NW><<<n / 128, 128, 0, stream>>>(tables + k * mat, tables + (k + 1) * mat);
            count_launch();
            err = cudaGetLastError();
        }
        return err;
    }
}

cudaError_t launch_build_tables(int engine, uint32_t *tables, cudaStream_t stream)
{
    switch (engine) {
    case ENG_XOSHIRO256: return build_tables_e<ENG_XOSHIRO256>(tables, stream);
    case ENG_XOROSHIRO128: return build_tables_e<ENG_XOROSHIRO128>(tables, stream);
    case ENG_XOROSHIRO128PP: return build_tables_e<ENG_XOROSHIRO128PP>(tables, stream);
    case ENG_XOSHIRO128: return build_tables_e<ENG_XOSHIRO128>(tables, stream);
    case ENG_XOROSHIRO64: return build_tables_e<ENG_XOROSHIRO64>(tables, stream);
    case ENG_XOSHIRO512: return build_tables_e<ENG_XOSHIRO512>(tables, stream);
    case ENG_XOROSHIRO1024: return build_tables_e<ENG_XOROSHIRO1024>(tables, stream);
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------- apply powers


template <int NW>
__global__ void __launch_bounds__(128)
    k_apply_pow(const u32 *__restrict__ tables, KList ks, u32 *states, size_t count)
{
    constexpr int n = NW * 32;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    u32 v[NW], r[NW];
    load_vec<NW>(v, states + i * NW);
    for (int t = 0; t < ks.n; ++t) {
        const u32 *M = tables + (size_t)ks.k[t] * n * NW;
        f2_matvec<NW, false>(M, v, r);
#pragma unroll
        for (int j = 0; j < NW; ++j) v[j] = r[j];
    }
    store_vec<NW>(v, states + i * NW);
}

cudaError_t launch_apply_pow(int engine, const uint32_t *tables, const KList &ks, void *states,
                             size_t count, cudaStream_t stream)
{
    if (count == 0 || ks.n == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((count + 127) / 128);
    switch (engine_bits(engine)) {
    case 1024: k_apply_pow<32><<<grid, 128, 0, stream>>>(tables, ks, (u32 *)states, count); break;
    case 512: k_apply_pow<16><<<grid, 128, 0, stream>>>(tables, ks, (u32 *)states, count); break;
    case 256: k_apply_pow<8><<<grid, 128, 0, stream>>>(tables, ks, (u32 *)states, count); break;
    case 128: k_apply_pow<4><<<grid, 128, 0, stream>>>(tables, ks, (u32 *)states, count); break;
    default: k_apply_pow<2><<<grid, 128, 0, stream>>>(tables, ks, (u32 *)states, count); break;
    }
    count_launch();
    return cudaGetLastError();
}

// out = (T^(2^d))^e base by one warp: the start state of a range of streams
// that does not begin at stream 0.
template <int NW>
__global__ void __launch_bounds__(32)
    k_warp_jump(const u32 *__restrict__ psets_d, const u32 *__restrict__ tables, int d, const u32 *base, u32 *out,
                u64 e)
{
    const int lane = threadIdx.x;
    u32 v[NW];
    load_vec<NW>(v, base);
    warp_advance<NW>(psets_d, tables, d, v, e, lane);
    if (lane == 0) store_vec<NW>(v, out);
}

cudaError_t launch_warp_jump(int engine, const uint32_t *psets_d, const uint32_t *tables, int d, const void *base,
                             void *out, uint64_t e, cudaStream_t stream)
{
    const u32 *P = (const u32 *)psets_d, *T = (const u32 *)tables, *b = (const u32 *)base;
    switch (engine_bits(engine)) {
    case 256: k_warp_jump<8><<<1, 32, 0, stream>>>(P, T, d, b, (u32 *)out, e); break;
    case 128: k_warp_jump<4><<<1, 32, 0, stream>>>(P, T, d, b, (u32 *)out, e); break;
    case 64: k_warp_jump<2><<<1, 32, 0, stream>>>(P, T, d, b, (u32 *)out, e); break;
    default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- doubling tree

// Levels L while 2^L < min(S, 2 * blockDim): one CTA, the level matrix staged
// in shared memory, a barrier between levels.
// The level matrix is staged in shared memory for states up to 512 bits;
// the 1024-bit one (128 KiB) is read through the read-only cache instead.
template <int NW>
struct TreeStage {
    static constexpr bool on = NW <= 16;
    static constexpr int words = on ? NW * 32 * NW : 4;
};

template <int NW>
__global__ void __launch_bounds__(256)
    k_tree_small(const u32 *__restrict__ tables, int kbase, u32 *states, size_t S, int levels)
{
    constexpr int n = NW * 32;
    __shared__ __align__(16) u32 M[TreeStage<NW>::words];
    for (int L = 0; L < levels; ++L) {
        const u32 *src = tables + (size_t)((kbase + L) % n) * n * NW;
        if (TreeStage<NW>::on) {
            for (int t = threadIdx.x; t < n * NW / 4; t += blockDim.x)
                reinterpret_cast<uint4 *>(M)[t] = reinterpret_cast<const uint4 *>(src)[t];
        }
        __syncthreads();
        const size_t half = (size_t)1 << L;
        const size_t idx = threadIdx.x;
        if (idx < half && half + idx < S) {
            u32 v[NW], r[NW];
            load_vec<NW>(v, states + idx * NW);
            if (TreeStage<NW>::on) f2_matvec<NW, true>(M, v, r);
            else f2_matvec<NW, false>(src, v, r);
            store_vec<NW>(r, states + (half + idx) * NW);
        }
        __syncthreads();
    }
}

// One level: states[half + idx] = M states[idx] for idx < min(half, S - half).
template <int NW>
__global__ void __launch_bounds__(256)
    k_tree_level(const u32 *__restrict__ Mg, u32 *states, size_t half, size_t S)
{
    constexpr int n = NW * 32;
    __shared__ __align__(16) u32 M[TreeStage<NW>::words];
    if (TreeStage<NW>::on) {
        for (int t = threadIdx.x; t < n * NW / 4; t += blockDim.x)
            reinterpret_cast<uint4 *>(M)[t] = reinterpret_cast<const uint4 *>(Mg)[t];
    }
    __syncthreads();
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= half || half + idx >= S) return;
    u32 v[NW], r[NW];
    load_vec<NW>(v, states + idx * NW);
    if (TreeStage<NW>::on) f2_matvec<NW, true>(M, v, r);
    else f2_matvec<NW, false>(Mg, v, r);
    store_vec<NW>(r, states + (half + idx) * NW);
}

template <int NW>
static cudaError_t tree_nw(const uint32_t *tables, int kbase, void *states, size_t S,
                           cudaStream_t stream)
{
    constexpr int n = NW * 32;
    if (S <= 1) return cudaSuccess;
    int small = 0;
    while (small < 9 && ((size_t)1 << small) < S) ++small;  // 2^L <= 256 threads
    k_tree_small<NW><<<1, 256, 0, stream>>>(tables, kbase, (u32 *)states, S, small);
    count_launch();
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    for (int L = small; ((size_t)1 << L) < S; ++L) {
        const size_t half = (size_t)1 << L;
        const size_t work = (S - half) < half ? (S - half) : half;
        const unsigned grid = (unsigned)((work + 255) / 256);
        const uint32_t *M = tables + (size_t)((kbase + L) % n) * n * NW;
        k_tree_level<NW><<<grid, 256, 0, stream>>>(M, (u32 *)states, half, S);
        count_launch();
        err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

cudaError_t launch_tree(int engine, const uint32_t *tables, int kbase, void *states, size_t S,
                        cudaStream_t stream)
{
    switch (engine_bits(engine)) {
    case 1024: return tree_nw<32>(tables, kbase, states, S, stream);
    case 512: return tree_nw<16>(tables, kbase, states, S, stream);
    case 256: return tree_nw<8>(tables, kbase, states, S, stream);
    case 128: return tree_nw<4>(tables, kbase, states, S, stream);
    default: return tree_nw<2>(tables, kbase, states, S, stream);
    }
}

// ---------------------------------------------------------------- power sets
//
// Stream starts in three levels instead of a tree of depth log2(S).  For a
// jump distance 2^d and level l = 0, 1, 2 the context keeps the power set
//   P_l[j] = (T^(2^(d + 9 l)))^j,   j = 0 .. 511,
// built once by doubling: P_l[0] = I and, for j in [2^L, 2^(L+1)),
// P_l[j] = T^(2^(d + 9 l + L)) P_l[j - 2^L], the multiplier being a jump-table
// entry.  Writing the stream index in base 512, i = p * 512^(l+1) + j * 512^l,
// stream i is P_l[j] applied to stream p * 512^(l+1), which an earlier (higher)
// level wrote; so the states array itself holds every intermediate level and
// each level is one launch reading only entries it does not write.

template <int NW>
__global__ void __launch_bounds__(NW * 32) k_pset_identity(u32 *sets)
{
    constexpr int n = NW * 32;
    const int c = threadIdx.x;
    u32 *col = sets + (size_t)blockIdx.x * PSET_SIZE * n * NW + (size_t)c * NW;
#pragma unroll
    for (int w = 0; w < NW; ++w) col[w] = (w == c / 32) ? (1u << (c % 32)) : 0u;
}

// Level L of the doubling: P[j] = T^(2^k) P[j - 2^L], j = 2^L + blockIdx.x,
// set blockIdx.y, column threadIdx.x; k = (kfirst[set] + L) mod n.
template <int NW>
__global__ void __launch_bounds__(NW * 32)
    k_pset_level(const u32 *__restrict__ tables, u32 *sets, KList kfirst, int L)
{
    constexpr int n = NW * 32;
    __shared__ __align__(16) u32 M[n * NW];
    const int set = blockIdx.y, c = threadIdx.x;
    const int j = (1 << L) + blockIdx.x;
    const u32 *src = tables + (size_t)((kfirst.k[set] + L) % n) * n * NW;
    for (int t = c; t < n * NW / 4; t += n)
        reinterpret_cast<uint4 *>(M)[t] = reinterpret_cast<const uint4 *>(src)[t];
    __syncthreads();
    u32 *P = sets + (size_t)set * PSET_SIZE * n * NW;
    u32 v[NW], r[NW];
    load_vec<NW>(v, P + (size_t)(j - (1 << L)) * n * NW + (size_t)c * NW);
    f2_matvec<NW, true>(M, v, r);
    store_vec<NW>(r, P + (size_t)j * n * NW + (size_t)c * NW);
}

cudaError_t launch_build_power_sets(int engine, const uint32_t *tables, const int *dists, int ndist,
                                    uint32_t *sets, cudaStream_t stream)
{
    const int n = engine_bits(engine);
    KList kf;
    kf.n = ndist * PSET_LEVELS;
    for (int di = 0; di < ndist; ++di)
        for (int l = 0; l < PSET_LEVELS; ++l) kf.k[di * PSET_LEVELS + l] = (dists[di] + PSET_BITS * l) % n;
    const int nsets = kf.n;
    if (n == 256) k_pset_identity<8><<<nsets, 256, 0, stream>>>((u32 *)sets);
    else if (n == 128) k_pset_identity<4><<<nsets, 128, 0, stream>>>((u32 *)sets);
    else k_pset_identity<2><<<nsets, 64, 0, stream>>>((u32 *)sets);
    count_launch();
    cudaError_t err = cudaGetLastError();
    for (int L = 0; L < PSET_BITS && err == cudaSuccess; ++L) {
        const dim3 grid(1u << L, (unsigned)nsets);
        if (n == 256) k_pset_level<8><<<grid, 256, 0, stream>>>(tables, (u32 *)sets, kf, L);
        else if (n == 128) k_pset_level<4><<<grid, 128, 0, stream>>>(tables, (u32 *)sets, kf, L);
        else k_pset_level<2><<<grid, 64, 0, stream>>>(tables, (u32 *)sets, kf, L);
        count_launch();
        err = cudaGetLastError();
    }
    return err;
}

// One level: for every parent p (index p * 512 * stride) and j in 1 .. 511,
// states[p * 512 * stride + j * stride] = P[j] states[p * 512 * stride].  The
// CTA shares j (blockIdx.y + 1), builds the Four-Russians tables of P[j] in
// shared memory and handles two parents per thread.
constexpr int STREAMS_PER_THREAD = 2;

template <int NW>
__global__ void __launch_bounds__(256)
    k_streams_level(const u32 *__restrict__ P, u32 *states, size_t S, size_t stride, size_t nparents)
{
    typedef Russians<NW> RT;
    __shared__ __align__(16) u32 T[RT::WORDS];
    const int j = blockIdx.y + 1;
    russians_build<NW>(P + (size_t)j * RT::n * NW, T);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < STREAMS_PER_THREAD; ++k) {
        const size_t p = ((size_t)blockIdx.x * STREAMS_PER_THREAD + k) * blockDim.x + threadIdx.x;
        if (p >= nparents) return;
        const size_t parent = p * PSET_SIZE * stride;
        const size_t child = parent + (size_t)j * stride;
        if (child >= S) continue;
        u32 v[NW], r[NW];
        load_vec<NW>(v, states + parent * NW);
        russians_matvec<NW>(T, v, r);
        store_vec<NW>(r, states + child * NW);
    }
}

// Children of a chunk whose first P streams (the parents) are in place:
// states[p + P j] = Q_j states[p] for j = 1 .. 511, with Q_j = T^(2^d P j) the
// level-0 power set of the distance 2^d P.  The CTA shares j (its tables in
// shared memory) and its lanes take consecutive parents, so the parent loads
// and the child stores of a warp are contiguous.
template <int NW>
__global__ void __launch_bounds__(256) k_streams_jmajor(const u32 *__restrict__ Q, u32 *states, size_t P)
{
    typedef Russians<NW> RT;
    __shared__ __align__(16) u32 T[RT::WORDS];
    const int j = blockIdx.y + 1;
    russians_build<NW>(Q + (size_t)j * RT::n * NW, T);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < STREAMS_PER_THREAD; ++k) {
        const size_t p = ((size_t)blockIdx.x * STREAMS_PER_THREAD + k) * blockDim.x + threadIdx.x;
        if (p >= P) return;
        u32 v[NW], r[NW];
        load_vec<NW>(v, states + p * NW);
        russians_matvec<NW>(T, v, r);
        store_vec<NW>(r, states + (p + P * (size_t)j) * NW);
    }
}

cudaError_t launch_streams_jmajor(int engine, const uint32_t *Q, void *states, size_t P, cudaStream_t stream)
{
    const size_t per_cta = (size_t)256 * STREAMS_PER_THREAD;
    const dim3 grid((unsigned)((P + per_cta - 1) / per_cta), PSET_SIZE - 1);
    switch (engine_bits(engine)) {
    case 256: k_streams_jmajor<8><<<grid, 256, 0, stream>>>(Q, (u32 *)states, P); break;
    case 128: k_streams_jmajor<4><<<grid, 256, 0, stream>>>(Q, (u32 *)states, P); break;
    case 64: k_streams_jmajor<2><<<grid, 256, 0, stream>>>(Q, (u32 *)states, P); break;
    default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_streams_psets(int engine, const uint32_t *sets3, void *states, size_t S,
                                 cudaStream_t stream)
{
    const int n = engine_bits(engine);
    if (S <= 1) return cudaSuccess;
    const size_t set_words = (size_t)PSET_SIZE * n * (n / 32);
    int top = 0;
    while (top + 1 < PSET_LEVELS && S > ((size_t)1 << (PSET_BITS * (top + 1)))) ++top;
    for (int l = top; l >= 0; --l) {
        const size_t stride = (size_t)1 << (PSET_BITS * l);
        const size_t span = stride * PSET_SIZE;
        const size_t nparents = (S + span - 1) / span;
        const size_t per_cta = (size_t)256 * STREAMS_PER_THREAD;
        // children j of parent 0 stop below S (only the top level has fewer than 511)
        const size_t maxj = std::min<size_t>(PSET_SIZE - 1, (S + stride - 1) / stride - 1);
        const dim3 grid((unsigned)((nparents + per_cta - 1) / per_cta), (unsigned)maxj);
        const uint32_t *P = sets3 + (size_t)l * set_words;
        if (n == 256) k_streams_level<8><<<grid, 256, 0, stream>>>(P, (u32 *)states, S, stride, nparents);
        else if (n == 128) k_streams_level<4><<<grid, 256, 0, stream>>>(P, (u32 *)states, S, stride, nparents);
        else k_streams_level<2><<<grid, 256, 0, stream>>>(P, (u32 *)states, S, stride, nparents);
        count_launch();
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------- seeding

// WORDBYTES = 8: state word j = output j.  WORDBYTES = 4: output t gives words
// 2t (low half) and 2t + 1 (high half).
template <int WORDBYTES, int K>
__global__ void k_seed(const u64 *__restrict__ seeds, u64 seed1, size_t count, u32 *states,
                       int *status)
{
    constexpr int NW = WORDBYTES * K / 4;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    u64 x = seeds ? seeds[i] : seed1;
    u32 w[NW];
    if (WORDBYTES == 8) {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const u64 z = splitmix64_next(x);
            w[2 * j] = (u32)z;
            w[2 * j + 1] = (u32)(z >> 32);
        }
    } else {
#pragma unroll
        for (int j = 0; j < K; j += 2) {
            const u64 z = splitmix64_next(x);
            w[j] = (u32)z;
            w[j + 1] = (u32)(z >> 32);
        }
    }
    u32 any = 0;
#pragma unroll
    for (int j = 0; j < NW; ++j) any |= w[j];
    if (!any) atomicCAS(status, 0, XR_EZERO_STATE);
    store_vec<NW>(w, states + i * NW);
}

cudaError_t launch_seed(int variant, const uint64_t *d_seeds, uint64_t seed, size_t count,
                        void *states, int *status, cudaStream_t stream)
{
    if (count == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((count + 127) / 128);
    const int eng = engine_of(variant);
    const u64 *sp = (const u64 *)d_seeds;
    switch (eng) {
    case ENG_XOSHIRO256: k_seed<8, 4><<<grid, 128, 0, stream>>>(sp, seed, count, (u32 *)states, status); break;
    case ENG_XOSHIRO128: k_seed<4, 4><<<grid, 128, 0, stream>>>(sp, seed, count, (u32 *)states, status); break;
    case ENG_XOROSHIRO64: k_seed<4, 2><<<grid, 128, 0, stream>>>(sp, seed, count, (u32 *)states, status); break;
    case ENG_XOSHIRO512: k_seed<8, 8><<<grid, 128, 0, stream>>>(sp, seed, count, (u32 *)states, status); break;
    case ENG_XOROSHIRO1024: k_seed<8, 16><<<grid, 128, 0, stream>>>(sp, seed, count, (u32 *)states, status); break;
    default: k_seed<8, 2><<<grid, 128, 0, stream>>>(sp, seed, count, (u32 *)states, status); break;
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace xr
