// xr_analysis.cu -- the paper's analysis workloads on the device.
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
// sequences at once: one CTA per sequence.  The bits are stored reversed and
// packed (bit j of rev = s_{N-1-j}), so the window s_n, s_{n-1}, ..., s_{n-L}
// lines up with the connection polynomial's coefficients c_0 .. c_L starting
// at bit N-1-n.

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

// One CTA per job, everything in registers.  Thread t holds words t R ..
// t R + R - 1 of three bit strings:
//   c   = C, the connection polynomial;
//   xb  = x^m B, B being C before the last length change;
//   win = the window, bit i = s_{n-i} (zero for i > n).
// Step n (d_n known): C_{n+1} = C_n + d_n x^m B; x^m B moves to x^(m+1) B, or
// to x C_n when the length changes (B = C_n, m = 1); the window moves up one
// bit and takes s_{n+1} at bit 0.  Each is a shift by one bit, so a word only
// needs the top word of the word below it: from the lane below by shuffle, or
// for lane 0 from the previous warp's lane 31, which publishes its top words
// in shared memory before every barrier.  Then d_{n+1} = parity(c & win).
//
// deg C <= L, deg x^m B <= n + 2 and deg win <= n + 1 after step n, so a
// thread whose first word is above (n + 2) / 32 + 1 holds zeros and skips the
// step.  Bits shifted past the last word are never needed: an update uses
// x^m B only when its degree is below the new L, which is checked against
// 32 W first (a larger complexity stores ~0 instead of a result).
//
// One barrier per sequence bit, which also reduces the parity: d_{n+1} is
// the parity of the number of threads whose partial sum is odd
// (__syncthreads_count).  The carry slots alternate, so a slot is rewritten
// two barriers after it was read.
template <int R>
__global__ void __launch_bounds__(1024) k_berlekamp_massey(const LcJob *__restrict__ jobs)
{
    __shared__ uint4 carry[2][32];  // [slot][warp]: top words of c, xb, win
    const LcJob job = jobs[blockIdx.x];
    const u32 N = job.N, W = job.W;
    const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const u32 *rev = job.rev;
    const u32 w0 = (u32)tid * R;
    for (int i = tid; i < 2 * 32; i += nth) (&carry[0][0])[i] = make_uint4(0u, 0u, 0u, 0u);
    u32 c[R], xb[R], win[R];
#pragma unroll
    for (int k = 0; k < R; ++k) c[k] = xb[k] = win[k] = 0u;
    // bit j of the packed sequence is s_{N-1-j}
    const u32 s0 = (__ldg(rev + ((N - 1) >> 5)) >> ((N - 1) & 31)) & 1u;
    if (tid == 0) {
        c[0] = 1u;   // C = 1
        xb[0] = 2u;  // x^1 B, B = 1
        win[0] = s0;
    }
    int d = (int)s0;
    u32 sword = 0u;  // thread 0: the packed word holding s_{n+1}
    u32 L = 0;
    __syncthreads();
    for (u32 n = 0; n < N; ++n) {
        const bool grow = d && 2 * L <= n;
        const u32 Lnew = grow ? n + 1 - L : L;
        if (d && Lnew >= W * 32) {  // uniform
            if (tid == 0) *job.out = ~0ull;
            return;
        }
        const int slot = (int)(n & 1);
        u32 cc = __shfl_up_sync(0xffffffffu, c[R - 1], 1);
        u32 cx = __shfl_up_sync(0xffffffffu, xb[R - 1], 1);
        u32 cw = __shfl_up_sync(0xffffffffu, win[R - 1], 1);
        if (lane == 0) {
            if (warp == 0) {
                cc = cx = cw = 0u;
                if (n + 1 < N) {
                    const u32 j = N - 2 - n;
                    if (n == 0 || (j & 31) == 31) sword = __ldg(rev + (j >> 5));
                    cw = ((sword >> (j & 31)) & 1u) << 31;
                }
            } else {
                const uint4 t = carry[slot][warp - 1];
                cc = t.x;
                cx = t.y;
                cw = t.z;
            }
        }
        u32 acc = 0u;
        if (w0 <= (n + 2) / 32 + 1) {
            if (grow) {
#pragma unroll
                for (int k = R - 1; k >= 0; --k) {
                    const u32 nx = __funnelshift_l(k ? c[k - 1] : cc, c[k], 1);
                    c[k] ^= xb[k];
                    xb[k] = nx;
                }
            } else if (d) {
#pragma unroll
                for (int k = R - 1; k >= 0; --k) {
                    c[k] ^= xb[k];
                    xb[k] = __funnelshift_l(k ? xb[k - 1] : cx, xb[k], 1);
                }
            } else {
#pragma unroll
                for (int k = R - 1; k >= 0; --k) xb[k] = __funnelshift_l(k ? xb[k - 1] : cx, xb[k], 1);
            }
#pragma unroll
            for (int k = R - 1; k >= 0; --k) {
                win[k] = __funnelshift_l(k ? win[k - 1] : cw, win[k], 1);
                acc ^= c[k] & win[k];
            }
        }
        L = Lnew;
        if (lane == 31) carry[slot ^ 1][warp] = make_uint4(c[R - 1], xb[R - 1], win[R - 1], 0u);
        d = __syncthreads_count((int)(__popc(acc) & 1)) & 1;
    }
    if (tid == 0) *job.out = (unsigned long long)L;
}

// Words per thread: 12 (measured best on GB300 from one to 448 sequences of
// 2^16 to 7 10^5 bits: enough words per warp to outweigh the per-step
// shuffles, carry exchange and barrier, few enough registers for 1024
// threads), or the fewest that fit one warp for sequences under 12 288 bits.
static int lc_r(u32 W)
{
    for (int r : {1, 2, 4, 8})
        if ((W + r - 1) / r <= 32) return r;
    return 12;
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

template <int V>
static cudaError_t lc_bits_v(const u32 *tables, const LcJob *d_jobs, unsigned count, size_t max_threads,
                             cudaStream_t st)
{
    const dim3 grid((unsigned)((max_threads + 127) / 128), count);
    k_lc_bits<V><<<grid, 128, 0, st>>>(tables, d_jobs);
    count_launch();
    return cudaGetLastError();
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
    // jobs ordered by (words per thread, variant): one Berlekamp-Massey launch
    // per words-per-thread group, one bit-generation launch per variant run
    std::vector<size_t> order(njobs);
    for (size_t j = 0; j < njobs; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        const int ra = lc_r(lc_words(jobs[a].N)), rb = lc_r(lc_words(jobs[b].N));
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
               lc_r(h_jobs[e].W) == lc_r(h_jobs[i].W)) {
            max_threads = std::max(max_threads, ((size_t)h_jobs[e].N + h_jobs[e].chunk - 1) / h_jobs[e].chunk);
            ++e;
        }
        const int v = jobs[order[i]].variant;
        err = launch_lc_bits(v, ctx->tables[lc_engine_of(v)], d_jobs + i, (unsigned)(e - i), max_threads, st);
        i = e;
    }
    for (size_t i = 0; err == cudaSuccess && i < njobs;) {  // one launch per words-per-thread group
        const int R = lc_r(h_jobs[i].W);
        size_t e = i;
        u32 Wmax = 0;
        while (e < njobs && lc_r(h_jobs[e].W) == R) {
            Wmax = std::max(Wmax, h_jobs[e].W);
            ++e;
        }
        err = launch_bm(R, d_jobs + i, (unsigned)(e - i), Wmax, st);
        i = e;
    }
    std::vector<unsigned long long> res(njobs);
    if (err == cudaSuccess) err = cudaMemcpyAsync(res.data(), d_out, njobs * 8, cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return XR_ECUDA;
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
