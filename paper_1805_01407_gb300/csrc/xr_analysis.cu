// xr_analysis.cu -- the paper's analysis workloads on the device: escaping
// zeroland and linear complexity.
//
// Escaping zeroland (Sec. 8): starting from each of the n states with
// exactly one bit set, how fast do the outputs reach half ones?  One thread
// per one-bit state keeps a running count of one bits over a window of
// `window` consecutive outputs and adds it to counts[t] for every window start
// t; the curve in the paper is counts[t] / (n * window * w).
#include <algorithm>
#include <vector>

#include "xr_device.cuh"
#include "xr_f2.cuh"
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
//
// Berlekamp-Massey over F2 (Sec. 9.3; the paper computes Table 13's lowest
// values this way) on bit `bit` of the first N outputs of a sequence, for many
// sequences at once: one CTA per sequence, or a cluster of CTAs per sequence
// when a call has few.  The bits are stored reversed and packed (bit j of
// rev = s_{N-1-j}), so the window s_n, s_{n-1}, ..., s_{n-L} lines up with the
// connection polynomial's coefficients c_0 .. c_L starting at bit N-1-n.

static constexpr u32 LC_REV_PAD = 20;  // zero words after a sequence

struct LcJob {
    const void *state;        // device, 16-byte aligned
    u32 *rev;                 // rev_words(N) + LC_REV_PAD words, zeroed
    unsigned long long *out;  // L, or ~0 when the prefix cannot decide it
    u32 N, W, chunk, bit;
};
static_assert(XR_LC_MAX_BITS / 64 + 5 <= 12 * 1024, "12 words per thread cover every prefix in 1024 threads");
static_assert(sizeof(LcJob) == 40, "the scratch size formula of xr.h assumes 40-byte job records");

__host__ __device__ static inline u32 lc_rev_words(size_t N) { return (u32)((N + 31) / 32 + 2); }
static inline u32 lc_words(size_t N) { return (u32)(N / 64 + 5); }

// Thread p of job j produces outputs p * chunk .. (p + 1) * chunk - 1: it
// jumps its copy of the state by T^(p * chunk) with the context's tables of
// T^(2^k) (one F2 matrix-vector product per set bit), then steps.  Words
// shared with the neighbouring chunks are merged with atomicOr.
template <int V>
__global__ void __launch_bounds__(128) k_lc_bits(const u32 *__restrict__ tables, const LcJob *__restrict__ jobs)
{
    typedef Gen<V> G;
    typedef typename G::E E;
    constexpr int n = E::NBITS, NW = n / 32;
    const LcJob job = jobs[blockIdx.y];
    const size_t N = job.N;
    const size_t t0 = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * job.chunk;
    if (t0 >= N) return;
    E e;
    load_state(e, job.state);
    u32 v[NW], r[NW];
    to_words(e, v);
    for (int k = 0; (t0 >> k) != 0; ++k) {
        if (!((t0 >> k) & 1)) continue;
        f2_matvec<NW, false>(tables + (size_t)k * n * NW, v, r);
#pragma unroll
        for (int j = 0; j < NW; ++j) v[j] = r[j];
    }
    from_words(e, v);
    const size_t t1 = t0 + job.chunk < N ? t0 + job.chunk : N;
    const int bit = (int)job.bit;
    u32 acc = 0u;
    for (size_t t = t0; t < t1; ++t) {
        const size_t pos = N - 1 - t;
        acc |= (u32)((G::out(e) >> bit) & 1u) << (pos & 31);
        e.step();
        if ((pos & 31) == 0 || t + 1 == t1) {
            atomicOr(job.rev + (pos >> 5), acc);
            acc = 0u;
        }
    }
}

// The same bits for runs of many sequences of one generator: lane l of a warp
// is sequence 32 blockIdx.y + l of the run and the warp shares its chunk index
// p, so every jump product is the same matrix for all lanes (broadcast column
// loads, no divergence).  Chunks are 2^lg outputs; with the power sets of that
// distance (P_l[j] = T^(2^lg j 512^l)) thread p starts at P_1[p >> 9] P_0[p & 511]
// (p < 2048), else at the product of the tables T^(2^k) over the set bits of
// p 2^lg.
template <int V>
__global__ void __launch_bounds__(128) k_lc_bits_many(const u32 *__restrict__ tables, const u32 *__restrict__ psets,
                                                     const LcJob *__restrict__ jobs, unsigned count, u32 lg)
{
    typedef Gen<V> G;
    typedef typename G::E E;
    constexpr int n = E::NBITS, NW = n / 32;
    const unsigned jx = blockIdx.y * 32 + (threadIdx.x & 31);
    const size_t p = (size_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (jx >= count) return;
    const LcJob job = jobs[jx];
    const size_t N = job.N, t0 = p << lg;
    if (t0 >= N) return;
    E e;
    load_state(e, job.state);
    u32 v[NW], r[NW];
    to_words(e, v);
    if (psets) {
        const u32 j0 = (u32)p & (PSET_SIZE - 1), j1 = (u32)(p >> PSET_BITS);
        if (j0) {
            f2_matvec<NW, false>(psets + (size_t)j0 * n * NW, v, r);
#pragma unroll
            for (int w = 0; w < NW; ++w) v[w] = r[w];
        }
        if (j1) {
            f2_matvec<NW, false>(psets + ((size_t)PSET_SIZE + j1) * n * NW, v, r);
#pragma unroll
            for (int w = 0; w < NW; ++w) v[w] = r[w];
        }
    } else {
        for (int k = 0; (t0 >> k) != 0; ++k) {
            if (!((t0 >> k) & 1)) continue;
            f2_matvec<NW, false>(tables + (size_t)k * n * NW, v, r);
#pragma unroll
            for (int w = 0; w < NW; ++w) v[w] = r[w];
        }
    }
    from_words(e, v);
    const size_t t1 = t0 + ((size_t)1 << lg) < N ? t0 + ((size_t)1 << lg) : N;
    const int bit = (int)job.bit;
    u32 acc = 0u;
    for (size_t t = t0; t < t1; ++t) {
        const size_t pos = N - 1 - t;
        acc |= (u32)((G::out(e) >> bit) & 1u) << (pos & 31);
        e.step();
        if ((pos & 31) == 0 || t + 1 == t1) {
            atomicOr(job.rev + (pos >> 5), acc);
            acc = 0u;
        }
    }
}

// One CTA per job, blocked Berlekamp-Massey: a barrier per block of (up to)
// 32 sequence bits instead of one per bit.  Notation of the bit-serial
// algorithm: C_n the connection polynomial, L_n its length, and
// X_n = x^m B, B being C before the last length change; step n with
// discrepancy d_n = sum_t C_t s_{n-t} sets C_{n+1} = C_n + d_n X_n and
// X_{n+1} = x C_n when the length changes (d_n = 1 and 2 L_n <= n, then
// L_{n+1} = n + 1 - L_n), else x X_n.  Over one block n .. n+k-1 every
// C_{n+u} is a C_n + b X_n with polynomials a, b of degree <= u, so each
// d_{n+u} follows from the 2k lookahead parities
//   e_C(u) = sum_t (C_n)_t s_{n+u-t},   e_X(u) = sum_t (X_n)_t s_{n+u-t}:
//   d_{n+u} = sum_j a_j e_C(u-j) + b_j e_X(u-j).
// A block is then:
//   1. lookahead: each thread ANDs its words of C_n and X_n with the 32
//      windows s_{n+u-32w-31 .. n+u-32w}, read straight from the packed
//      reversed sequence (one funnel shift per word and u), and folds the
//      parities into two 32-bit masks; a warp XORs its lanes' masks by
//      shuffles, and the warps' masks meet in shared memory at the block's
//      first barrier;
//   2. the k steps on the 2x2 polynomial matrix, by warp 0 alone (scalar,
//      branch-free): the steps with d = 1 and the length changes as two bit
//      masks, and the new L, go to shared memory; a second barrier publishes
//      them;
//   3. replay on the words, visiting only the steps with d = 1.  X is held
//      lazily as x^(u - tau) Y (Y = X_n at first, Y = C_{n+tau} after a
//      length change at step tau), so such a step costs one funnel shift and
//      one XOR per word, and the block ends with one shift of Y.
// Thread t holds words tR .. tR+R-1 of C and Y.  A shift brings in bits of
// the word below, owned by the lane below or by the previous warp's lane 31.
// Instead of exchanging them every step, a thread replays a shadow of that
// word from its value at the block's start (by shuffle, or from shared memory
// written at the end of the previous block) with zeros shifted in below: after
// shifts totalling u bits only its lowest u bits can be wrong, and a shift
// that ends at step u <= 32 reads only bits at or above u, so a block of
// k <= 32 steps needs no exchange.
//
// deg C_n <= L_n and deg X_n <= n + 1 - L_n, so words above
// max(L, n+1-L) / 32 are zero at the block's start (no lookahead) and stay
// zero above (max + 32) / 32 through the block (no replay).  Bits shifted
// past the last word are never needed: X is added to C only when its degree
// is below the new L, which is checked against 32 W first (a larger
// complexity stores ~0 instead of a result).
//
// Blocks end on sequence positions N - 32 j, so each block's windows start on
// a word boundary of the packed reversed sequence (bit i of rev = s_{N-1-i});
// the first block takes the remaining ((N - 1) mod 32) + 1 steps.
template <int R, bool FULL>
__device__ __forceinline__ void bm_lookahead(const u32 *__restrict__ rev, u32 k, const u32 (&c)[R],
                                             const u32 (&y)[R], u32 &eC, u32 &eX)
{
    u32 rv[R + 1];
#pragma unroll
    for (int i = 0; i <= R; ++i) rv[i] = __ldg(rev + i);
#pragma unroll
    for (int u = 0; u < 32; ++u) {
        if (!FULL && (u32)u >= k) break;
        const u32 s = FULL ? (u32)(31 - u) : k - 1 - (u32)u;
        u32 ac = 0u, ax = 0u;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const u32 t = __funnelshift_r(rv[j], rv[j + 1], s);  // window word j at step n + u
            ac ^= c[j] & t;
            ax ^= y[j] & t;
        }
        eC |= (u32)(__popc(ac) & 1) << u;
        eX |= (u32)(__popc(ax) & 1) << u;
    }
}

template <int R>
__global__ void __launch_bounds__(1024) k_berlekamp_massey(const LcJob *__restrict__ jobs)
{
    __shared__ uint2 masks[2][32];  // [slot][warp]: the warp's e_C, e_X masks
    __shared__ uint2 tops[2][32];   // [slot][warp]: top words of C, Y of the warp's lane 31
    __shared__ uint4 steps[2];      // [slot]: d mask, length-change mask, L, overflow
    const LcJob job = jobs[blockIdx.x];
    const u32 N = job.N, W = job.W;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const u32 w0 = (u32)tid * R;
    for (int i = tid; i < 2 * 32; i += blockDim.x) (&tops[0][0])[i] = make_uint2(0u, 0u);
    u32 c[R], y[R];
#pragma unroll
    for (int j = 0; j < R; ++j) c[j] = y[j] = 0u;
    if (tid == 0) {
        c[0] = 1u;  // C = 1
        y[0] = 2u;  // X = x^1 B, B = 1
    }
    u32 L = 0, n = 0;
    int slot = 0;
    __syncthreads();
    while (n < N) {
        const u32 k = ((N - 1 - n) & 31u) + 1u;
        const u32 q = (N - 1 - n - (k - 1)) >> 5;  // rev word of window word 0 at step n + k - 1
        const u32 D = L > n + 1 - L ? L : n + 1 - L;
        u32 eC = 0u, eX = 0u;
        if (w0 <= D / 32) {
            if (k == 32) bm_lookahead<R, true>(job.rev + q + w0, k, c, y, eC, eX);
            else bm_lookahead<R, false>(job.rev + q + w0, k, c, y, eC, eX);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            eC ^= __shfl_xor_sync(0xffffffffu, eC, o);
            eX ^= __shfl_xor_sync(0xffffffffu, eX, o);
        }
        u32 sC = __shfl_up_sync(0xffffffffu, c[R - 1], 1);
        u32 sY = __shfl_up_sync(0xffffffffu, y[R - 1], 1);
        if (lane == 0) masks[slot][warp] = make_uint2(eC, eX);
        __syncthreads();
        if (lane == 0) {
            if (warp == 0) {
                sC = sY = 0u;
            } else {
                const uint2 t = tops[slot][warp - 1];
                sC = t.x;
                sY = t.y;
            }
        }
        if (warp == 0) {
            eC = eX = 0u;
            for (int w = 0; w < nwarps; ++w) {
                const uint2 t = masks[slot][w];
                eC ^= t.x;
                eX ^= t.y;
            }
            // a, b (C_{n+u} = a C_n + b X_n) and a', b' (X_{n+u} = a' C_n +
            // b' X_n), each aligned to bit 31 - u, so that with E = brev(e)
            // (bit 31 - v = e(v)) the discrepancy is parity((A & E_C) ^ (B & E_X)).
            const u32 EC = __brev(eC), EX = __brev(eX);
            u32 A = 0x80000000u, B = 0u, A2 = 0u, B2 = 0x80000000u, dm = 0u, gm = 0u, over = 0u;
            for (u32 u = 0; u < k; ++u) {
                const u32 dmask = 0u - (u32)(__popc((A & EC) ^ (B & EX)) & 1);
                const u32 gmask = dmask & (0u - (u32)(2 * L <= n + u));
                const u32 Lg = n + u + 1 - L;
                over |= gmask & (0u - (u32)(Lg >= W * 32));
                const u32 nA = A ^ (A2 & dmask), nB = B ^ (B2 & dmask);
                A2 = (A & gmask) | (A2 & ~gmask);
                B2 = (B & gmask) | (B2 & ~gmask);
                A = nA >> 1;
                B = nB >> 1;
                L = gmask ? Lg : L;
                dm |= (dmask & 1u) << u;
                gm |= (gmask & 1u) << u;
            }
            if (lane == 0) steps[slot] = make_uint4(dm, gm, L, over);
        }
        __syncthreads();
        const uint4 sd = steps[slot];
        if (sd.w) {  // uniform
            if (tid == 0) *job.out = ~0ull;
            return;
        }
        L = sd.z;
        if (w0 <= (D + 32) / 32) {
            u32 ev = sd.x, tau = 0u;
            while (ev) {
                const u32 u = (u32)__ffs(ev) - 1u;
                ev &= ev - 1u;
                const u32 dl = u - tau;  // X_{n+u} = x^dl Y, dl < 32
                const u32 sx = sY << dl;
                if ((sd.y >> u) & 1u) {  // length change: Y = C_{n+u}, tau = u
#pragma unroll
                    for (int j = R - 1; j >= 0; --j) {
                        const u32 xw = __funnelshift_l(j ? y[j - 1] : sY, y[j], dl);
                        y[j] = c[j];
                        c[j] ^= xw;
                    }
                    const u32 t = sC;
                    sC ^= sx;
                    sY = t;
                    tau = u;
                } else {
#pragma unroll
                    for (int j = R - 1; j >= 0; --j) c[j] ^= __funnelshift_l(j ? y[j - 1] : sY, y[j], dl);
                    sC ^= sx;
                }
            }
            const u32 sh = k - tau;  // X_{n+k} = x^sh Y, 1 <= sh <= 32
#pragma unroll
            for (int j = R - 1; j >= 0; --j) y[j] = __funnelshift_lc(j ? y[j - 1] : sY, y[j], sh);
        }
        n += k;
        if (lane == 31) tops[slot ^ 1][warp] = make_uint2(c[R - 1], y[R - 1]);
        slot ^= 1;
    }
    if (tid == 0) *job.out = (unsigned long long)L;
}

// Words per thread (at most 1024 threads per sequence): the fewest of 1, 2,
// 4, 8 that fit one warp; otherwise 8 when at least one sequence per SM is
// running (448 sequences of 2^16 bits: R = 4, 8, 12 took 12.0, 11.9, 12.5 ms
// on GB300), and 4 for fewer sequences, which then have an SM each (one
// 65,992-bit sequence: 6.7, 7.8, 8.6 ms); 12 where 8 does not fit (above
// about 524,000 bits).
static int lc_r(u32 W, bool many)
{
    for (int r : {1, 2, 4, 8})
        if ((W + r - 1) / r <= 32) return r;
    if (!many && (W + 3) / 4 <= 1024) return 4;
    return (W + 7) / 8 <= 1024 ? 8 : 12;
}

template <int R>
static cudaError_t launch_bm_r(const LcJob *d_jobs, unsigned count, u32 Wmax, cudaStream_t st)
{
    const unsigned threads = (unsigned)(((Wmax + R - 1) / R + 31) / 32 * 32);
    k_berlekamp_massey<R><<<count, threads, 0, st>>>(d_jobs);
    count_launch();
    return cudaGetLastError();
}

static cudaError_t launch_bm(int R, const LcJob *d_jobs, unsigned count, u32 Wmax, cudaStream_t st)
{
    switch (R) {
    case 1: return launch_bm_r<1>(d_jobs, count, Wmax, st);
    case 2: return launch_bm_r<2>(d_jobs, count, Wmax, st);
    case 4: return launch_bm_r<4>(d_jobs, count, Wmax, st);
    case 8: return launch_bm_r<8>(d_jobs, count, Wmax, st);
    default: return launch_bm_r<12>(d_jobs, count, Wmax, st);
    }
}

// ---------------------------------------------------------------- one sequence on a cluster of CTAs
//
// The same blocked algorithm for calls with few sequences, which would leave
// most SMs idle with one CTA each: a cluster of 16 or 8 CTAs (one per SM)
// shares a sequence, global thread g = rank * blockDim + tid holding words
// gR .. gR+R-1.  Per block, every warp sends its lookahead masks to every
// CTA of the cluster with st.async, which lands them in that CTA's shared
// memory and counts their bytes on its mbarrier; the CTA before this one sends
// its last thread's top words (the shadow of this CTA's first thread) the same
// way.  Only warp 0 of each CTA waits, on its own mbarrier, then runs the
// block recurrence; all CTAs see the same masks, so they take the same
// decisions and exit on overflow at the same block.  A CTA sends block b + 2's
// masks only after receiving everyone's block b + 1 masks, which each CTA
// sent after reading its block b masks, so two slots suffice and an mbarrier
// phase never receives bytes of the next one.  Cluster barriers come only
// before the first remote store (every mbarrier initialised) and before exit
// (no CTA leaves while another may still store into it).  A wait that runs out
// (LC_WAIT_TRIES polls) makes its CTA report ~1, which the call turns into an
// error, and return.
constexpr unsigned LC_CLUSTER = 8, LC_CLUSTER_MAX = 16;

__device__ __forceinline__ u32 cluster_ctarank()
{
    u32 r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ u32 cluster_nctarank()
{
    u32 r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// v into the same shared-memory variable of CTA `rank` of the cluster
__device__ __forceinline__ void st_cluster(const uint2 *local, u32 rank, uint2 v)
{
    const u32 a = (u32)__cvta_generic_to_shared(local);
    u32 ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("st.shared::cluster.v2.u32 [%0], {%1, %2};" ::"r"(ra), "r"(v.x), "r"(v.y) : "memory");
}

__device__ __forceinline__ u32 smem_addr32(const void *p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ u32 mapa32(u32 a, u32 rank)
{
    u32 r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

// 8 bytes into shared memory of another CTA of the cluster, counted on that
// CTA's mbarrier (transaction bytes)
__device__ __forceinline__ void st_async8(u32 raddr, uint2 v, u32 rmbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.u32 [%0], {%1, %2}, [%3];" ::"r"(raddr),
                 "r"(v.x), "r"(v.y), "r"(rmbar)
                 : "memory");
}

__device__ __forceinline__ void mbar_init(u32 a, u32 count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(u32 a, u32 bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}

__device__ __forceinline__ u32 mbar_try_wait(u32 a, u32 parity)
{
    u32 ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok;
}

constexpr u32 LC_WAIT_TRIES = 1u << 24;

template <int R>
__global__ void __launch_bounds__(1024) k_berlekamp_massey_cluster(const LcJob *__restrict__ jobs)
{
    __shared__ uint2 parts[2][LC_CLUSTER_MAX * 32];  // [slot][rank * nwarps + warp]: every warp's e_C, e_X
    __shared__ uint2 tops[2][32];                // [slot][warp]: top words of C, Y of the warp's lane 31
    __shared__ uint2 ctop[2];                    // [slot]: top words of the previous CTA's last thread
    __shared__ uint4 steps[2];                   // [slot]: d mask, length-change mask, L, overflow / timeout
    __shared__ __align__(8) unsigned long long mbar[2];  // [slot]: parts and ctop of the block arrived
    const u32 rank = cluster_ctarank(), ncta = cluster_nctarank();
    const LcJob job = jobs[blockIdx.x / ncta];
    const u32 N = job.N, W = job.W;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const u32 g = rank * blockDim.x + (u32)tid, w0 = g * R;
    for (int i = tid; i < 2 * 32; i += blockDim.x) (&tops[0][0])[i] = make_uint2(0u, 0u);
    if (tid < 2) ctop[tid] = make_uint2(0u, 0u);
    if (tid == 0) {
        mbar_init(smem_addr32(&mbar[0]), 1);
        mbar_init(smem_addr32(&mbar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    u32 c[R], y[R];
#pragma unroll
    for (int j = 0; j < R; ++j) c[j] = y[j] = 0u;
    if (g == 0) {
        c[0] = 1u;
        y[0] = 2u;
    }
    u32 L = 0, n = 0, parity = 0u;  // parity: bit s = phase parity of mbar[s]
    int slot = 0;
    const u32 tx = ncta * (u32)nwarps * 8u + (rank ? 8u : 0u);
    cluster_barrier();  // every CTA initialised before the first remote store
    while (n < N) {
        const u32 k = ((N - 1 - n) & 31u) + 1u;
        const u32 q = (N - 1 - n - (k - 1)) >> 5;
        const u32 D = L > n + 1 - L ? L : n + 1 - L;
        u32 eC = 0u, eX = 0u;
        if (w0 <= D / 32) {
            if (k == 32) bm_lookahead<R, true>(job.rev + q + w0, k, c, y, eC, eX);
            else bm_lookahead<R, false>(job.rev + q + w0, k, c, y, eC, eX);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            eC ^= __shfl_xor_sync(0xffffffffu, eC, o);
            eX ^= __shfl_xor_sync(0xffffffffu, eX, o);
        }
        u32 sC = __shfl_up_sync(0xffffffffu, c[R - 1], 1);
        u32 sY = __shfl_up_sync(0xffffffffu, y[R - 1], 1);
        const u32 mb = smem_addr32(&mbar[slot]);
        if ((u32)lane < ncta)
            st_async8(mapa32(smem_addr32(&parts[slot][rank * nwarps + warp]), (u32)lane), make_uint2(eC, eX),
                      mapa32(mb, (u32)lane));
        if (tid == (int)blockDim.x - 1 && rank + 1 < ncta)
            st_async8(mapa32(smem_addr32(&ctop[slot]), rank + 1), make_uint2(c[R - 1], y[R - 1]), mapa32(mb, rank + 1));
        if (warp == 0) {
            u32 ok = 1u;
            if (lane == 0) {
                mbar_arrive_expect_tx(mb, tx);
                ok = 0u;
                for (u32 i = 0; i < LC_WAIT_TRIES && !ok; ++i) ok = mbar_try_wait(mb, (parity >> slot) & 1u);
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            __syncwarp();
            if (lane == 0) {
                const uint2 t = ctop[slot];  // stays zero in CTA 0
                sC = t.x;
                sY = t.y;
            }
            eC = eX = 0u;
            for (u32 i = (u32)lane; i < ncta * (u32)nwarps; i += 32) {
                const uint2 t = parts[slot][i];
                eC ^= t.x;
                eX ^= t.y;
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                eC ^= __shfl_xor_sync(0xffffffffu, eC, o);
                eX ^= __shfl_xor_sync(0xffffffffu, eX, o);
            }
            const u32 EC = __brev(eC), EX = __brev(eX);
            u32 A = 0x80000000u, B = 0u, A2 = 0u, B2 = 0x80000000u, dm = 0u, gm = 0u, over = 0u;
            for (u32 u = 0; u < k; ++u) {
                const u32 dmask = 0u - (u32)(__popc((A & EC) ^ (B & EX)) & 1);
                const u32 gmask = dmask & (0u - (u32)(2 * L <= n + u));
                const u32 Lg = n + u + 1 - L;
                over |= gmask & (0u - (u32)(Lg >= W * 32));
                const u32 nA = A ^ (A2 & dmask), nB = B ^ (B2 & dmask);
                A2 = (A & gmask) | (A2 & ~gmask);
                B2 = (B & gmask) | (B2 & ~gmask);
                A = nA >> 1;
                B = nB >> 1;
                L = gmask ? Lg : L;
                dm |= (dmask & 1u) << u;
                gm |= (gmask & 1u) << u;
            }
            if (lane == 0) steps[slot] = make_uint4(dm, gm, L, ok ? (over ? 1u : 0u) : 2u);
        }
        parity ^= 1u << slot;
        __syncthreads();
        if (warp > 0 && lane == 0) {  // written by the previous warp's lane 31 before this barrier
            const uint2 t = tops[slot][warp - 1];
            sC = t.x;
            sY = t.y;
        }
        const uint4 sd = steps[slot];
        if (sd.w) {  // overflow: uniform across the cluster; timeout: this CTA gives up
            if (g == 0 || sd.w == 2u) *job.out = sd.w == 2u ? ~1ull : ~0ull;
            return;
        }
        L = sd.z;
        if (w0 <= (D + 32) / 32) {
            u32 ev = sd.x, tau = 0u;
            while (ev) {
                const u32 u = (u32)__ffs(ev) - 1u;
                ev &= ev - 1u;
                const u32 dl = u - tau;
                const u32 sx = sY << dl;
                if ((sd.y >> u) & 1u) {
#pragma unroll
                    for (int j = R - 1; j >= 0; --j) {
                        const u32 xw = __funnelshift_l(j ? y[j - 1] : sY, y[j], dl);
                        y[j] = c[j];
                        c[j] ^= xw;
                    }
                    const u32 t = sC;
                    sC ^= sx;
                    sY = t;
                    tau = u;
                } else {
#pragma unroll
                    for (int j = R - 1; j >= 0; --j) c[j] ^= __funnelshift_l(j ? y[j - 1] : sY, y[j], dl);
                    sC ^= sx;
                }
            }
            const u32 sh = k - tau;
#pragma unroll
            for (int j = R - 1; j >= 0; --j) y[j] = __funnelshift_lc(j ? y[j - 1] : sY, y[j], sh);
        }
        n += k;
        if (lane == 31) tops[slot ^ 1][warp] = make_uint2(c[R - 1], y[R - 1]);
        slot ^= 1;
    }
    cluster_barrier();  // no CTA leaves while another may still store into it
    if (g == 0) *job.out = (unsigned long long)L;
}

// Clusters of LC_CLUSTER_MAX CTAs (a non-portable size, allowed per kernel)
// where the device takes them and the call has few enough sequences, else
// LC_CLUSTER.  Words
// per thread: 2 on 16 CTAs; on 8, 2 up to 2048 words (about 131,000 bits),
// else 4.  Measured on GB300: one 699,464-bit sequence 92.8 ms on 8 CTAs (R = 4;
// 102.7 at R = 2), 77.7 ms on 16 (R = 2; 80.2 at R = 4, 98.0 at R = 1), 191.8 ms
// on one CTA; one 65,992-bit sequence 5.8 ms on 8 or 16 CTAs (R = 2; 6.4 and
// 6.9 ms at R = 1 and 4 on 8).
static int lc_r_cluster(u32 W, unsigned ncta) { return ncta >= 16 || W <= 2048 ? 2 : 4; }

static unsigned lc_cluster_threads(u32 Wmax, int R, unsigned ncta)
{
    return (unsigned)(((Wmax + R * ncta - 1) / (R * ncta) + 31) / 32 * 32);
}

static cudaLaunchConfig_t lc_cluster_config(unsigned count, unsigned threads, unsigned ncta, cudaStream_t st,
                                            cudaLaunchAttribute *attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(count * ncta);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ncta;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// Whether clusters of ncta CTAs of `threads` threads fit this device (one
// resident at least); sizes above 8 are first allowed for the kernel.
template <int R>
static bool cluster_fits(unsigned threads, unsigned ncta)
{
    if (ncta > 8 &&
        cudaFuncSetAttribute(k_berlekamp_massey_cluster<R>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = lc_cluster_config(1, threads, ncta, nullptr, attr);
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k_berlekamp_massey_cluster<R>, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return nc >= 1;
}

template <int R>
static cudaError_t launch_bm_cluster_r(const LcJob *d_jobs, unsigned count, u32 Wmax, unsigned ncta,
                                       cudaStream_t st)
{
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = lc_cluster_config(count, lc_cluster_threads(Wmax, R, ncta), ncta, st, attr);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k_berlekamp_massey_cluster<R>, d_jobs);
    count_launch();
    return e != cudaSuccess ? e : cudaGetLastError();
}

// Launches the jobs on clusters when some size fits (first LC_CLUSTER_MAX if
// count allows, then LC_CLUSTER); *launched = false when none does.
static cudaError_t launch_bm_cluster(const LcJob *d_jobs, unsigned count, u32 Wmax, int sms, cudaStream_t st,
                                     bool *launched)
{
    *launched = false;
    for (unsigned ncta : {LC_CLUSTER_MAX, LC_CLUSTER}) {
        if ((size_t)count * ncta > (size_t)sms) continue;
        const int R = lc_r_cluster(Wmax, ncta);
        const unsigned threads = lc_cluster_threads(Wmax, R, ncta);
        const bool fits = R == 2 ? cluster_fits<2>(threads, ncta) : cluster_fits<4>(threads, ncta);
        if (!fits) continue;
        *launched = true;
        return R == 2 ? launch_bm_cluster_r<2>(d_jobs, count, Wmax, ncta, st)
                      : launch_bm_cluster_r<4>(d_jobs, count, Wmax, ncta, st);
    }
    return cudaSuccess;
}

template <int V>
static cudaError_t lc_bits_v(const u32 *tables, const LcJob *d_jobs, unsigned count, size_t max_threads,
                             cudaStream_t st)
{
    const dim3 grid((unsigned)((max_threads + 127) / 128), count);
    k_lc_bits<V><<<grid, 128, 0, st>>>(tables, d_jobs);
    count_launch();
    return cudaGetLastError();
}

template <int V>
static cudaError_t lc_bits_many_v(const u32 *tables, const u32 *psets, const LcJob *d_jobs, unsigned count, u32 lg,
                                  size_t nchunks, cudaStream_t st)
{
    const dim3 grid((unsigned)((nchunks + 3) / 4), (count + 31) / 32);
    k_lc_bits_many<V><<<grid, 128, 0, st>>>(tables, psets, d_jobs, count, lg);
    count_launch();
    return cudaGetLastError();
}

static cudaError_t launch_lc_bits_many(int variant, const u32 *tables, const u32 *psets, const LcJob *d_jobs,
                                       unsigned count, u32 lg, size_t nchunks, cudaStream_t st)
{
    switch (variant) {
#define XR_LC_CASE(V) \
    case V: return lc_bits_many_v<V>(tables, psets, d_jobs, count, lg, nchunks, st);
    XR_LC_CASE(0) XR_LC_CASE(1) XR_LC_CASE(2) XR_LC_CASE(3) XR_LC_CASE(4) XR_LC_CASE(5)
    XR_LC_CASE(6) XR_LC_CASE(7) XR_LC_CASE(8) XR_LC_CASE(9) XR_LC_CASE(10) XR_LC_CASE(11)
    XR_LC_CASE(12) XR_LC_CASE(13) XR_LC_CASE(14) XR_LC_CASE(15) XR_LC_CASE(16) XR_LC_CASE(17)
#undef XR_LC_CASE
    default: return cudaErrorInvalidValue;
    }
}

static cudaError_t launch_lc_bits(int variant, const u32 *tables, const LcJob *d_jobs, unsigned count,
                                  size_t max_threads, cudaStream_t st)
{
    switch (variant) {
#define XR_LC_CASE(V) \
    case V: return lc_bits_v<V>(tables, d_jobs, count, max_threads, st);
    XR_LC_CASE(0) XR_LC_CASE(1) XR_LC_CASE(2) XR_LC_CASE(3) XR_LC_CASE(4) XR_LC_CASE(5)
    XR_LC_CASE(6) XR_LC_CASE(7) XR_LC_CASE(8) XR_LC_CASE(9) XR_LC_CASE(10) XR_LC_CASE(11)
    XR_LC_CASE(12) XR_LC_CASE(13) XR_LC_CASE(14) XR_LC_CASE(15) XR_LC_CASE(16) XR_LC_CASE(17)
#undef XR_LC_CASE
    default: return cudaErrorInvalidValue;
    }
}

static int lc_engine_of(int variant)
{
    switch (variant) {
#define XR_LC_ENG(V) \
    case V: return Gen<V>::engine;
    XR_LC_ENG(0) XR_LC_ENG(1) XR_LC_ENG(2) XR_LC_ENG(3) XR_LC_ENG(4) XR_LC_ENG(5)
    XR_LC_ENG(6) XR_LC_ENG(7) XR_LC_ENG(8) XR_LC_ENG(9) XR_LC_ENG(10) XR_LC_ENG(11)
    XR_LC_ENG(12) XR_LC_ENG(13) XR_LC_ENG(14) XR_LC_ENG(15) XR_LC_ENG(16) XR_LC_ENG(17)
#undef XR_LC_ENG
    default: return -1;
    }
}

static size_t lc_round16(size_t x) { return (x + 15) & ~(size_t)15; }

// Scratch: the job table, the results, then each job's packed sequence.
static size_t lc_scratch_layout(const xr_lc_job *jobs, size_t njobs, size_t *rev_off)
{
    size_t off = lc_round16(njobs * sizeof(LcJob)) + lc_round16(njobs * 8);
    if (rev_off) *rev_off = off;
    for (size_t j = 0; j < njobs; ++j) off += lc_round16((size_t)(lc_rev_words(jobs[j].N) + LC_REV_PAD) * 4);
    return off;
}

static int lc_check(const xr_lc_job &j)
{
    if (j.variant < 0 || j.variant >= XR_NUM_VARIANTS) return XR_EINVAL;
    if (j.bit < 0 || j.bit >= xr_word_bits(j.variant) || j.N < 2 || j.N > XR_LC_MAX_BITS) return XR_EINVAL;
    return XR_OK;
}

static int lc_run(xr_ctx *ctx, const xr_lc_job *jobs, size_t njobs, const void *d_states, size_t stride,
                  void *d_scratch, size_t scratch_bytes, uint64_t *h_lc, cudaStream_t st)
{
    if (njobs == 0) return XR_OK;
    size_t rev_off = 0;
    const size_t need = lc_scratch_layout(jobs, njobs, &rev_off);
    if (scratch_bytes < need) return XR_EINVAL;
    for (size_t j = 0; j < njobs; ++j) {
        const int eng = lc_engine_of(jobs[j].variant);
        const int rc = ensure_engine(ctx, eng);
        if (rc != XR_OK) return rc;
    }
    // jobs ordered by (launch group, variant): one Berlekamp-Massey launch per
    // group, one bit-generation launch per variant run
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) return XR_ECUDA;
    const bool many = njobs >= (size_t)sms;
    // launch group of a job: its words per thread on one CTA, or 100 for a
    // cluster per sequence (few sequences, each longer than one warp's 256
    // words; the cluster size and words per thread are chosen at launch)
    const bool clustered = njobs * LC_CLUSTER <= (size_t)sms;
    auto group = [&](u32 W) { return clustered && W > 256 ? 100 : lc_r(W, many); };
    std::vector<size_t> order(njobs);
    for (size_t j = 0; j < njobs; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        const int ra = group(lc_words(jobs[a].N)), rb = group(lc_words(jobs[b].N));
        return ra != rb ? ra < rb : jobs[a].variant < jobs[b].variant;
    });
    char *base = (char *)d_scratch;
    LcJob *d_jobs = (LcJob *)base;
    unsigned long long *d_out = (unsigned long long *)(base + lc_round16(njobs * sizeof(LcJob)));
    std::vector<LcJob> h_jobs(njobs);
    std::vector<size_t> rev_at(njobs);
    {
        size_t off = rev_off;
        for (size_t j = 0; j < njobs; ++j) {
            rev_at[j] = off;
            off += lc_round16((size_t)(lc_rev_words(jobs[j].N) + LC_REV_PAD) * 4);
        }
    }
    for (size_t i = 0; i < njobs; ++i) {
        const size_t j = order[i];
        const size_t N = jobs[j].N;
        size_t chunk = (N + 2047) / 2048;
        chunk = chunk < 256 ? 256 : (chunk + 31) / 32 * 32;
        h_jobs[i].state = (const char *)d_states + j * stride;
        h_jobs[i].rev = (u32 *)(base + rev_at[j]);
        h_jobs[i].out = d_out + j;
        h_jobs[i].N = (u32)N;
        h_jobs[i].W = lc_words(N);
        h_jobs[i].chunk = (u32)chunk;
        h_jobs[i].bit = (u32)jobs[j].bit;
    }
    cudaError_t err = cudaMemsetAsync(base + rev_off, 0, need - rev_off, st);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(d_jobs, h_jobs.data(), njobs * sizeof(LcJob), cudaMemcpyHostToDevice, st);
    for (size_t i = 0; err == cudaSuccess && i < njobs;) {  // one launch per variant run
        size_t e = i, max_threads = 0;
        while (e < njobs && jobs[order[e]].variant == jobs[order[i]].variant &&
               group(h_jobs[e].W) == group(h_jobs[i].W)) {
            max_threads = std::max(max_threads, ((size_t)h_jobs[e].N + h_jobs[e].chunk - 1) / h_jobs[e].chunk);
            ++e;
        }
        const int v = jobs[order[i]].variant;
        const int eng = lc_engine_of(v);
        if (e - i >= 32) {  // a run of many sequences: one sequence per lane
            size_t Nmax = 0;
            for (size_t k = i; k < e; ++k) Nmax = std::max(Nmax, (size_t)h_jobs[k].N);
            u32 lg = 8;  // chunks of 2^lg >= 256 outputs, at most 2048 per sequence
            while ((Nmax + ((size_t)1 << lg) - 1) >> lg > 2048) ++lg;
            const u32 *ps = eng < NUM_PSET_ENGINES ? dist_sets(ctx, eng, (int)lg) : nullptr;
            err = launch_lc_bits_many(v, ctx->tables[eng], ps, d_jobs + i, (unsigned)(e - i), lg,
                                      (Nmax + ((size_t)1 << lg) - 1) >> lg, st);
        } else {
            err = launch_lc_bits(v, ctx->tables[eng], d_jobs + i, (unsigned)(e - i), max_threads, st);
        }
        i = e;
    }
    for (size_t i = 0; err == cudaSuccess && i < njobs;) {  // one launch per words-per-thread group
        const int G = group(h_jobs[i].W);
        size_t e = i;
        u32 Wmax = 0;
        while (e < njobs && group(h_jobs[e].W) == G) {
            Wmax = std::max(Wmax, h_jobs[e].W);
            ++e;
        }
        bool on_clusters = false;
        if (G >= 100) err = launch_bm_cluster(d_jobs + i, (unsigned)(e - i), Wmax, sms, st, &on_clusters);
        if (err == cudaSuccess && !on_clusters)
            err = launch_bm(lc_r(Wmax, many), d_jobs + i, (unsigned)(e - i), Wmax, st);
        i = e;
    }
    std::vector<unsigned long long> res(njobs);
    if (err == cudaSuccess) err = cudaMemcpyAsync(res.data(), d_out, njobs * 8, cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return XR_ECUDA;
    for (size_t j = 0; j < njobs; ++j)
        if (res[j] == ~1ull) return XR_ECUDA;  // a cluster's wait ran out
    for (size_t j = 0; j < njobs; ++j) h_lc[j] = res[j];
    return XR_OK;
}

}  // namespace xr

using namespace xr;

extern "C" size_t xr_lc_scratch_bytes(const xr_lc_job *jobs, size_t njobs)
{
    if (!jobs && njobs) return 0;
    return lc_scratch_layout(jobs, njobs, nullptr);
}

extern "C" int xr_linear_complexity_many(xr_ctx *ctx, const xr_lc_job *jobs, size_t njobs, const void *d_states,
                                         size_t state_stride, void *d_scratch, size_t scratch_bytes,
                                         uint64_t *h_lc, void *stream)
{
    if (!ctx || (njobs && (!jobs || !d_states || !d_scratch || !h_lc))) return XR_EINVAL;
    DeviceScope dscope(ctx->device);
    NvtxRange nvtx("xr_linear_complexity_many");
    if (njobs > (1u << 20) || ((uintptr_t)d_states % 16) || (state_stride % 16) ||
        ((uintptr_t)d_scratch % 16))
        return XR_EINVAL;
    for (size_t j = 0; j < njobs; ++j) {
        if (lc_check(jobs[j]) != XR_OK) return XR_EINVAL;
        if (njobs > 1 && state_stride < (size_t)xr_state_bytes(jobs[j].variant)) return XR_EINVAL;
    }
    return lc_run(ctx, jobs, njobs, d_states, state_stride, d_scratch, scratch_bytes, h_lc,
                  (cudaStream_t)stream);
}

extern "C" int xr_linear_complexity(xr_ctx *ctx, int variant, int bit, size_t N, const void *d_state,
                                    void *d_scratch, size_t scratch_bytes, uint64_t *h_lc, void *stream)
{
    if (!ctx || !d_state || !h_lc || !d_scratch) return XR_EINVAL;
    DeviceScope dscope(ctx->device);
    NvtxRange nvtx("xr_linear_complexity");
    xr_lc_job job;
    job.variant = variant;
    job.bit = bit;
    job.N = N;
    if (lc_check(job) != XR_OK) return XR_EINVAL;
    if (((uintptr_t)d_state % 16) || ((uintptr_t)d_scratch % 16)) return XR_EINVAL;
    uint64_t L = 0;
    const int rc = lc_run(ctx, &job, 1, d_state, 0, d_scratch, scratch_bytes, &L, (cudaStream_t)stream);
    if (rc != XR_OK) return rc;
    if (L == ~(uint64_t)0) return XR_EUNSUPPORTED;
    *h_lc = L;
    return XR_OK;
}

extern "C" int xr_zeroland(xr_ctx *ctx, int variant, size_t nout, size_t window, uint64_t *d_counts, void *stream)
{
    if (!ctx || variant < 0 || variant >= XR_NUM_VARIANTS || !d_counts) return XR_EINVAL;
    DeviceScope dscope(ctx->device);
    NvtxRange nvtx("xr_zeroland");
    if (window < 1 || window > 64 || nout < window || nout > ((size_t)1 << 32)) return XR_EINVAL;
    if ((uintptr_t)d_counts % 8) return XR_EINVAL;
    const cudaStream_t st = (cudaStream_t)stream;
    cudaError_t err = cudaMemsetAsync(d_counts, 0, (nout - window + 1) * sizeof(uint64_t), st);
    if (err == cudaSuccess)
        err = launch_zeroland(variant, nout, (int)window, reinterpret_cast<unsigned long long *>(d_counts), st);
    return err == cudaSuccess ? XR_OK : XR_ECUDA;
}
