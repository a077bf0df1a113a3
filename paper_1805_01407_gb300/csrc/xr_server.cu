// xr_server.cu -- continuous batching of generation requests from many
// clients (declared in include/xr.h).
//
// The server keeps one generator state per client on the device.  A
// scheduler thread admits pending requests in arrival order while a round slot
// and arena space are free.  Admission runs a small kernel on one serialized
// admit stream: each admitted request receives the client's current state in
// a private slot, and the client's state jumps ahead by the request's n
// (T^n by the bits of n), so requests of one client continue a single
// sequence in submission order no matter how rounds overlap.  A round is a
// batch plan (xr_batch_plan.h) run on its own stream after its admit step;
// several rounds are in flight at once, so new arrivals overlap the tail of
// earlier rounds.  Plain mode runs one xr_fill_seq per request on one stream.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "xr_batch_plan.h"
#include "xr_device.cuh"
#include "xr_f2.cuh"
#include "xr_internal.h"

namespace xr {

struct AdmitClient {
    u32 client, first, count, engine;
};
struct AdmitReq {
    u64 n, slot;
};
// Jump tables of every engine (T^(2^k)), and the single-step power sets of
// the engines that have them (null for xoshiro512 and xoroshiro1024).
struct Tables4 {
    const u32 *t[NUM_ENGINES_H];
};

// Client state slots of sw words <- SplitMix64(seed): one 64-bit output per 8
// state bytes (32-bit words take each output's low half first); words past
// the state are zero.
__global__ void k_server_seed(const int *variants, const u64 *seeds, u32 nclients, u32 sw, u32 *cstates)
{
    const u32 c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nclients) return;
    u64 x = seeds[c];
    const int v = variants[c];
    const int sb = v <= 2 ? 32 : v <= 9 ? 16 : v <= 11 ? 8 : v <= 14 ? 64 : 128;
    uint4 *d = reinterpret_cast<uint4 *>(cstates + (size_t)c * sw);
    for (u32 k = 0; k < sw / 4; ++k) {
        u32 w[4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const u64 z = (int)(16 * k + 8 * h) < sb ? splitmix64_next(x) : 0ull;
            w[2 * h] = (u32)z;
            w[2 * h + 1] = (u32)(z >> 32);
        }
        d[k] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// v <- T^e v by one warp from the jump tables alone (one product per set bit
// of e), for the engines without power sets.
template <int NW>
__device__ void warp_advance_tables(const u32 *tables, u32 (&v)[NW], u64 e, int lane)
{
    constexpr int n = NW * 32;
    while (e) {
        const int k = __ffsll((long long)e) - 1;
        e &= e - 1;
        warp_matvec<NW>(tables + (size_t)k * n * NW, v, lane);
    }
}

// One client's admitted requests in order, by one warp: each request gets the
// current state in its destination of sw words (req.slot indexes `rslots`: a
// round's segment states, at the request's first segment, or a plain slot),
// then the state advances by the request's n.
template <int NW>
__device__ void admit_chain(const u32 *psets0, const u32 *tables, u32 *cstate, const AdmitReq *reqs, u32 first,
                            u32 count, unsigned char *rslots, u32 sw, int lane)
{
    constexpr int W = NW < 8 ? 8 : NW;  // words written: the state, zero-padded to 32 bytes
    u32 v[NW];
#pragma unroll
    for (int j = 0; j < NW; ++j) v[j] = cstate[j];
    for (u32 i = 0; i < count; ++i) {
        const AdmitReq q = reqs[first + i];
        if (lane == 0) {
            u32 *d = reinterpret_cast<u32 *>(rslots + q.slot * sw * 4u);
#pragma unroll
            for (int w = 0; w < W; ++w) d[w] = w < NW ? v[w % NW] : 0u;
        }
        if (psets0) warp_advance<NW>(psets0, tables, 0, v, q.n, lane);
        else warp_advance_tables<NW>(tables, v, q.n, lane);
    }
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < NW; ++j) cstate[j] = v[j];
    }
}

__device__ __forceinline__ void admit_engine(const Tables4 &T, const Tables4 &P0, u32 engine, u32 *cs,
                                             const AdmitReq *reqs, u32 first, u32 count, unsigned char *rslots,
                                             u32 sw, int lane)
{
    switch (engine) {
    case ENG_XOSHIRO256: admit_chain<8>(P0.t[0], T.t[0], cs, reqs, first, count, rslots, sw, lane); break;
    case ENG_XOROSHIRO64:
        admit_chain<2>(P0.t[engine], T.t[engine], cs, reqs, first, count, rslots, sw, lane);
        break;
    case ENG_XOSHIRO512: admit_chain<16>(nullptr, T.t[engine], cs, reqs, first, count, rslots, sw, lane); break;
    case ENG_XOROSHIRO1024:
        admit_chain<32>(nullptr, T.t[engine], cs, reqs, first, count, rslots, sw, lane);
        break;
    default: admit_chain<4>(P0.t[engine], T.t[engine], cs, reqs, first, count, rslots, sw, lane); break;
    }
}

// One warp per client of the round.
__global__ void k_admit(Tables4 T, Tables4 P0, const AdmitClient *clients, u32 nclients, const AdmitReq *reqs,
                        u32 *cstates, unsigned char *rslots, u32 sw)
{
    const u32 i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= nclients) return;
    const AdmitClient c = clients[i];
    admit_engine(T, P0, c.engine, cstates + (size_t)c.client * sw, reqs, c.first, c.count, rslots, sw, lane);
}

// The admit step of one request, arguments by value (plain mode); one warp.
__global__ void k_admit_one(Tables4 T, Tables4 P0, u32 client, u32 engine, u64 n, u32 *cstates, unsigned char *slot,
                            u32 sw)
{
    const AdmitReq q{n, 0};
    const int lane = threadIdx.x & 31;
    admit_engine(T, P0, engine, cstates + (size_t)client * sw, &q, 0, 1, slot, sw, lane);
}

}  // namespace xr

using namespace xr;

namespace {

double now_us()
{
    using namespace std::chrono;
    return (double)duration_cast<nanoseconds>(steady_clock::now().time_since_epoch()).count() * 1e-3;
}

enum { S_PENDING = 0, S_ADMITTED = 1, S_DONE = 2, S_RELEASED = 3, S_FAILED = 4 };

struct SReq {
    u32 client;
    u64 n;
    int dtype;
    u64 off, bytes;
    double t_sub, t_done;
    double t_start = 0, t_launched = 0;  // round launch begun / enqueued (host clock)
    int state;
    bool auto_release;
};

// First-fit allocator over the arena, 8 KiB granules (a request starts on a
// row of 1024 outputs, which lets its full segments use tile stores).
struct Arena {
    static constexpr u64 G = 8192;
    std::map<u64, u64> free_;  // offset -> bytes
    u64 in_use = 0, peak = 0;
    void init(u64 total) { free_[0] = total / G * G; }
    bool alloc(u64 bytes, u64 *off)
    {
        bytes = std::max<u64>(G, (bytes + G - 1) / G * G);
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes) {
                *off = it->first;
                const u64 rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                in_use += bytes;
                peak = std::max(peak, in_use);
                return true;
            }
        return false;
    }
    void release(u64 off, u64 bytes)
    {
        bytes = std::max<u64>(G, (bytes + G - 1) / G * G);
        in_use -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Round {
    HostPlan plan;
    DevPlan dev;
    std::vector<u64> tickets;
    std::vector<u32> clients;  // client of each request (copied under the lock)
    std::vector<xr_request> reqs;
    std::vector<AdmitClient> aclients;
    std::vector<AdmitReq> areqs;
    unsigned char *d_slots = nullptr;
    unsigned char *h_admit = nullptr;
    size_t admit_cap = 0;
    cudaStream_t st = nullptr;
    cudaEvent_t admitted = nullptr, done = nullptr;
};

struct PlainUnit {
    u64 ticket;
    int ev;
};

constexpr int PLAIN_DEPTH = 64;

int es_of_dtype(int dt) { return (dt == XR_U64 || dt == XR_F64) ? 8 : 4; }

}  // namespace

struct xr_server {
    xr_ctx *ctx = nullptr;
    xr_server_config cfg{};
    std::vector<int> cvar;
    u32 *d_cstates = nullptr;
    u32 sw = 8;  // words per client state, segment state and request slot (the largest client state)
    unsigned char *arena = nullptr;
    Arena alloc;
    std::mutex mu;
    std::condition_variable cv;
    std::unordered_map<u64, SReq> reqs;
    std::deque<u64> pending;
    u64 next_ticket = 1;
    std::vector<Round> rounds;
    std::deque<int> inflight;
    std::vector<int> free_rounds;
    cudaStream_t admit_st = nullptr, plain_st = nullptr;
    std::deque<PlainUnit> plain_inflight;
    std::vector<cudaEvent_t> plain_events;
    std::vector<int> free_plain;
    unsigned char *d_plain_slots = nullptr;
    std::thread th;
    std::atomic<bool> stop{false};
    xr_serve_stats stats{};
    int error = XR_OK;
};

static int sst(cudaError_t e)
{
    if (e == cudaSuccess) return XR_OK;
    if (e == cudaErrorMemoryAllocation) return XR_ENOMEM;
    return XR_ECUDA;
}

static Tables4 tables_of(xr_ctx *ctx)
{
    Tables4 T;
    for (int e = 0; e < NUM_ENGINES_H; ++e) T.t[e] = ctx->tables[e];
    return T;
}

// The single-step power sets (distance 2^0) of every engine that has them.
static Tables4 steps_of(xr_ctx *ctx)
{
    Tables4 T;
    for (int e = 0; e < NUM_ENGINES_H; ++e) T.t[e] = e < NUM_PSET_ENGINES ? pset_sets(ctx, e, pset_index(e, 0)) : nullptr;
    return T;
}

// Complete finished rounds / plain units (lock held by the caller).
static bool complete_finished(xr_server *s)
{
    bool progress = false;
    const double t = now_us();
    auto finish = [&](u64 tk) {
        SReq &q = s->reqs[tk];
        q.state = S_DONE;
        q.t_done = t;
        s->stats.queue_ns += (u64)(1e3 * (q.t_start - q.t_sub));
        s->stats.launch_ns += (u64)(1e3 * (q.t_launched - q.t_start));
        s->stats.device_ns += (u64)(1e3 * (q.t_done - q.t_launched));
        s->stats.completed++;
        s->stats.bytes += q.n * (u64)es_of_dtype(q.dtype);
        if (q.auto_release) {
            s->alloc.release(q.off, q.bytes);
            q.state = S_RELEASED;
            s->stats.released++;
        }
    };
    while (!s->inflight.empty()) {
        Round &R = s->rounds[s->inflight.front()];
        const cudaError_t e = cudaEventQuery(R.done);
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) {
            s->error = XR_ECUDA;
            for (u64 tk : R.tickets) s->reqs[tk].state = S_FAILED;
        } else {
            for (u64 tk : R.tickets) finish(tk);
        }
        s->free_rounds.push_back(s->inflight.front());
        s->inflight.pop_front();
        progress = true;
    }
    while (!s->plain_inflight.empty()) {
        const PlainUnit u = s->plain_inflight.front();
        const cudaError_t e = cudaEventQuery(s->plain_events[u.ev]);
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) {
            s->error = XR_ECUDA;
            s->reqs[u.ticket].state = S_FAILED;
        } else {
            finish(u.ticket);
        }
        s->free_plain.push_back(u.ev);
        s->plain_inflight.pop_front();
        progress = true;
    }
    return progress;
}

static cudaError_t launch_round(xr_server *s, Round &R)
{
    NvtxRange nvtx("xr_server round");
    // The plan first: admission writes each request's start state straight
    // into its first segment state (seg_base), so the round needs no seed step.
    build_plan(R.reqs.data(), R.reqs.size(), R.plan);
    R.plan.slot_words = s->sw;  // admission writes segment states at the server's stride
    // admit arrays, grouped by client in submission order
    R.aclients.clear();
    R.areqs.clear();
    std::vector<std::pair<u32, u32>> byc(R.reqs.size());  // (client, request)
    for (u32 i = 0; i < (u32)R.reqs.size(); ++i) byc[i] = {R.clients[i], i};
    std::stable_sort(byc.begin(), byc.end(),
                     [](const std::pair<u32, u32> &x, const std::pair<u32, u32> &y) { return x.first < y.first; });
    for (size_t k = 0; k < byc.size();) {
        size_t e = k;
        AdmitClient c;
        c.client = byc[k].first;
        c.first = (u32)R.areqs.size();
        c.engine = (u32)engine_of(s->cvar[c.client]);
        for (; e < byc.size() && byc[e].first == c.client; ++e)
            R.areqs.push_back({R.reqs[byc[e].second].n, R.plan.reqs[byc[e].second].seg_base});
        c.count = (u32)(e - k);
        R.aclients.push_back(c);
        k = e;
    }
    const size_t ca = R.aclients.size() * sizeof(AdmitClient), ra = R.areqs.size() * sizeof(AdmitReq);
    const size_t roff = (ca + 255) & ~(size_t)255;
    if (roff + ra > R.admit_cap) return cudaErrorInvalidValue;  // sized for the largest round at creation
    memcpy(R.h_admit, R.aclients.data(), ca);
    memcpy(R.h_admit + roff, R.areqs.data(), ra);
    // plan + admission records + a zero task counter: one copy, on the
    // admission stream, which orders the rounds' admissions
    cudaError_t err = upload_plan(R.plan, R.dev, s->admit_st, R.h_admit, roff + ra);
    if (err != cudaSuccess) return err;
    const unsigned char *recs = R.dev.blob + R.dev.off_extra;
    const u32 nc = (u32)R.aclients.size();
    k_admit<<<(nc + 3) / 4, 128, 0, s->admit_st>>>(tables_of(s->ctx), steps_of(s->ctx), (const AdmitClient *)recs,
                                                   nc, (const AdmitReq *)(recs + roff), s->d_cstates,
                                                   (unsigned char *)R.dev.segstates, s->sw);
    count_launch();
    err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaEventRecord(R.admitted, s->admit_st);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(R.st, R.admitted, 0);
    const int opt = s->cfg.outputs_per_row ? s->cfg.outputs_per_row : 32;
    const int block = s->cfg.block ? s->cfg.block : 128;
    if (err == cudaSuccess)
        err = enqueue_plan(s->ctx, R.plan, R.dev, nullptr, R.d_slots, s->arena, s->cfg.arena_bytes, opt, block, R.st,
                           true);
    if (err == cudaSuccess) err = cudaEventRecord(R.done, R.st);
    return err;
}

// One plain request: its admit step, then xr_fill_seq from its private slot.
// `q` is a copy taken under the lock.
static cudaError_t launch_plain(xr_server *s, const SReq &q, int ev, int slot)
{
    unsigned char *sl = s->d_plain_slots + (size_t)slot * s->sw * 4;
    k_admit_one<<<1, 32, 0, s->plain_st>>>(tables_of(s->ctx), steps_of(s->ctx), q.client,
                                            (u32)engine_of(s->cvar[q.client]), q.n, s->d_cstates, sl, s->sw);
    count_launch();
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess) {
        const int rc = xr_fill_seq(s->ctx, s->cvar[q.client], sl, q.n, q.dtype, s->arena + q.off, s->plain_st);
        if (rc != XR_OK) err = cudaErrorUnknown;
    }
    if (err == cudaSuccess) err = cudaEventRecord(s->plain_events[ev], s->plain_st);
    return err;
}

static void scheduler(xr_server *s)
{
    cudaSetDevice(s->ctx->device);
    u64 plain_seq = 0;
    while (!s->stop.load(std::memory_order_acquire)) {
        bool progress = false;
        std::unique_lock<std::mutex> lk(s->mu);
        if (complete_finished(s)) {
            progress = true;
            s->cv.notify_all();
        }
        if (s->cfg.mode == XR_SERVE_BATCHED) {
            if (!s->free_rounds.empty() && !s->pending.empty()) {
                const int ri = s->free_rounds.back();
                Round &R = s->rounds[ri];
                R.tickets.clear();
                R.clients.clear();
                R.reqs.clear();
                // A round takes at most its share of the arena, so the rounds in
                // flight divide the memory and the next one is admitted while
                // the current one runs (a larger request still goes alone).
                const u64 share = s->cfg.arena_bytes / s->cfg.max_rounds;
                u64 round_bytes = 0;
                while (!s->pending.empty() && R.tickets.size() < s->cfg.max_round_requests) {
                    SReq &q = s->reqs[s->pending.front()];
                    if (!R.tickets.empty() && round_bytes + q.bytes > share) break;
                    u64 off;
                    if (!s->alloc.alloc(q.bytes, &off)) break;  // arrival order: wait for memory
                    round_bytes += q.bytes;
                    q.off = off;
                    q.state = S_ADMITTED;
                    const u32 i = (u32)R.tickets.size();
                    R.tickets.push_back(s->pending.front());
                    R.clients.push_back(q.client);
                    R.reqs.push_back(xr_request{s->cvar[q.client], q.dtype, q.n, (uint64_t)i, off});
                    s->pending.pop_front();
                }
                if (!R.tickets.empty()) {
                    s->free_rounds.pop_back();
                    s->stats.rounds++;
                    s->stats.arena_in_use = s->alloc.in_use;
                    s->stats.arena_peak = s->alloc.peak;
                    const double t_start = now_us();
                    for (u64 tk : R.tickets) s->reqs[tk].t_start = t_start;
                    lk.unlock();
                    const cudaError_t err = launch_round(s, R);
                    const double t_launched = now_us();
                    lk.lock();
                    for (u64 tk : R.tickets) s->reqs[tk].t_launched = t_launched;
                    if (err != cudaSuccess) s->error = sst(err);
                    s->inflight.push_back(ri);
                    progress = true;
                }
            }
        } else {
            while (!s->pending.empty() && !s->free_plain.empty()) {
                SReq &q = s->reqs[s->pending.front()];
                u64 off;
                if (!s->alloc.alloc(q.bytes, &off)) break;
                q.off = off;
                q.state = S_ADMITTED;
                const u64 tk = s->pending.front();
                s->pending.pop_front();
                const int ev = s->free_plain.back();
                s->free_plain.pop_back();
                s->stats.arena_in_use = s->alloc.in_use;
                s->stats.arena_peak = s->alloc.peak;
                const int slot = (int)(plain_seq++ % PLAIN_DEPTH);
                q.t_start = now_us();
                const SReq qc = q;
                lk.unlock();
                const cudaError_t err = launch_plain(s, qc, ev, slot);
                const double t_launched = now_us();
                lk.lock();
                s->reqs[tk].t_launched = t_launched;
                if (err != cudaSuccess) s->error = sst(err);
                s->plain_inflight.push_back({tk, ev});
                progress = true;
            }
        }
        lk.unlock();
        if (!progress) std::this_thread::yield();
    }
}

extern "C" int xr_server_destroy(xr_server *s)
{
    if (!s) return XR_OK;
    if (s->th.joinable()) {
        // stop admitting (requests still pending are dropped), let admitted
        // work finish
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->pending.clear();
        }
        for (;;) {
            std::unique_lock<std::mutex> lk(s->mu);
            if ((s->inflight.empty() && s->plain_inflight.empty()) || s->error != XR_OK) break;
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(200));
        }
        s->stop.store(true, std::memory_order_release);
        s->th.join();
    }
    DeviceScope dscope(s->ctx->device);
    cudaDeviceSynchronize();
    for (Round &R : s->rounds) {
        free_devplan(R.dev);
        cudaFree(R.d_slots);
        cudaFreeHost(R.h_admit);
        if (R.st) cudaStreamDestroy(R.st);
        if (R.admitted) cudaEventDestroy(R.admitted);
        if (R.done) cudaEventDestroy(R.done);
    }
    for (cudaEvent_t e : s->plain_events) cudaEventDestroy(e);
    if (s->admit_st) cudaStreamDestroy(s->admit_st);
    if (s->plain_st) cudaStreamDestroy(s->plain_st);
    cudaFree(s->d_cstates);
    cudaFree(s->arena);
    cudaFree(s->d_plain_slots);
    delete s;
    return XR_OK;
}

extern "C" int xr_server_create(xr_ctx *ctx, const xr_server_config *cfg, const int *h_client_variants,
                                const uint64_t *h_client_seeds, xr_server **out)
{
    if (!ctx || !cfg || !out || !h_client_variants || !h_client_seeds) return XR_EINVAL;
    *out = nullptr;
    if (cfg->nclients == 0 || cfg->arena_bytes < 8192 || cfg->max_rounds == 0 || cfg->max_round_requests == 0)
        return XR_EINVAL;
    if (cfg->mode != XR_SERVE_BATCHED && cfg->mode != XR_SERVE_PLAIN) return XR_EINVAL;
    if (cfg->outputs_per_row && batch_smem_bytes(cfg->outputs_per_row, cfg->block ? cfg->block : 128) > 227 * 1024)
        return XR_EINVAL;
    u32 sw = 8;
    for (u32 c = 0; c < cfg->nclients; ++c) {
        if (h_client_variants[c] < 0 || h_client_variants[c] >= XR_NUM_VARIANTS) return XR_EINVAL;
        sw = std::max(sw, slot_words_of(h_client_variants[c]));
    }
    DeviceScope dscope(ctx->device);
    for (u32 c = 0; c < cfg->nclients; ++c) {  // the large engines' tables are built on first use
        const int erc = ensure_engine(ctx, engine_of(h_client_variants[c]));
        if (erc != XR_OK) return erc;
    }
    xr_server *s = new xr_server();
    s->ctx = ctx;
    s->cfg = *cfg;
    s->sw = sw;
    s->cvar.assign(h_client_variants, h_client_variants + cfg->nclients);
    s->alloc.init(cfg->arena_bytes);
    cudaError_t err = cudaSuccess;
    int *d_var = nullptr;
    u64 *d_seed = nullptr;
    if (err == cudaSuccess) err = cudaMalloc((void **)&s->d_cstates, (size_t)cfg->nclients * sw * 4);
    if (err == cudaSuccess) err = cudaMalloc((void **)&s->arena, cfg->arena_bytes);
    if (err == cudaSuccess) err = cudaMalloc((void **)&d_var, (size_t)cfg->nclients * sizeof(int));
    if (err == cudaSuccess) err = cudaMalloc((void **)&d_seed, (size_t)cfg->nclients * sizeof(u64));
    if (err == cudaSuccess)
        err = cudaMemcpy(d_var, h_client_variants, (size_t)cfg->nclients * sizeof(int), cudaMemcpyHostToDevice);
    if (err == cudaSuccess)
        err = cudaMemcpy(d_seed, h_client_seeds, (size_t)cfg->nclients * sizeof(u64), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) {
        k_server_seed<<<(cfg->nclients + 127) / 128, 128>>>(d_var, d_seed, cfg->nclients, sw, s->d_cstates);
        count_launch();
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaDeviceSynchronize();
    cudaFree(d_var);
    cudaFree(d_seed);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&s->admit_st, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&s->plain_st, cudaStreamNonBlocking);
    if (cfg->mode == XR_SERVE_BATCHED) {
        s->rounds.resize(cfg->max_rounds);
        const u64 segcap = cfg->arena_bytes / 4096 + cfg->max_round_requests + 64;
        for (u32 i = 0; i < cfg->max_rounds && err == cudaSuccess; ++i) {
            Round &R = s->rounds[i];
            err = cudaStreamCreateWithFlags(&R.st, cudaStreamNonBlocking);
            if (err == cudaSuccess) err = cudaEventCreateWithFlags(&R.admitted, cudaEventDisableTiming);
            if (err == cudaSuccess) err = cudaEventCreateWithFlags(&R.done, cudaEventDisableTiming);
            if (err == cudaSuccess) err = cudaMalloc((void **)&R.d_slots, (size_t)cfg->max_round_requests * sw * 4);
            // host staging of the admission records for the largest round (a
            // round has at most as many clients as requests); they travel to
            // the device inside the plan upload
            if (err == cudaSuccess) {
                const size_t ca = (size_t)cfg->max_round_requests * sizeof(AdmitClient);
                R.admit_cap = ((ca + 255) & ~(size_t)255) + (size_t)cfg->max_round_requests * sizeof(AdmitReq) + 256;
                err = cudaMallocHost((void **)&R.h_admit, R.admit_cap);
            }
            // size the plan buffers for the largest round up front
            if (err == cudaSuccess) {
                R.dev.seg_cap = segcap * sw * 4;
                err = cudaMalloc((void **)&R.dev.segstates, R.dev.seg_cap);
            }
            if (err == cudaSuccess) {
                // + tree items of the large engines: one per request and level
                R.dev.blob_cap = (size_t)cfg->max_round_requests * (sw > 8 ? 160 + 24 * sizeof(BTreeItem) : 160) +
                                 segcap / 32 * 8 * 2 + R.admit_cap + (1 << 20);
                err = cudaMalloc((void **)&R.dev.blob, R.dev.blob_cap);
                if (err == cudaSuccess) err = cudaMallocHost((void **)&R.dev.pinned, R.dev.blob_cap);
            }
            s->free_rounds.push_back((int)i);
        }
    } else {
        s->plain_events.resize(PLAIN_DEPTH);
        for (int i = 0; i < PLAIN_DEPTH && err == cudaSuccess; ++i) {
            err = cudaEventCreateWithFlags(&s->plain_events[i], cudaEventDisableTiming);
            s->free_plain.push_back(i);
        }
        if (err == cudaSuccess) err = cudaMalloc((void **)&s->d_plain_slots, (size_t)PLAIN_DEPTH * sw * 4);
    }
    if (err != cudaSuccess) {
        xr_server_destroy(s);
        return sst(err);
    }
    s->th = std::thread(scheduler, s);
    *out = s;
    return XR_OK;
}

static int submit(xr_server *s, uint32_t client, uint64_t n, int dtype, bool auto_release, uint64_t *ticket)
{
    if (!s || client >= s->cfg.nclients) return XR_EINVAL;
    const int v = s->cvar[client];
    const bool w32 = xr_word_bits(v) == 32;
    const bool ok = dtype == XR_F64 || dtype == XR_F32 || (dtype == XR_U64 && !w32) || (dtype == XR_U32 && w32);
    if (!ok) return XR_EINVAL;
    const u64 bytes = n * (u64)es_of_dtype(dtype);
    if (n == 0 || bytes + Arena::G > s->cfg.arena_bytes) return XR_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    const u64 tk = s->next_ticket++;
    SReq q;
    q.client = client;
    q.n = n;
    q.dtype = dtype;
    q.off = 0;
    q.bytes = bytes;
    q.t_sub = now_us();
    q.t_done = 0;
    q.state = S_PENDING;
    q.auto_release = auto_release;
    s->reqs[tk] = q;
    s->pending.push_back(tk);
    s->stats.submitted++;
    if (ticket) *ticket = tk;
    return XR_OK;
}

extern "C" int xr_server_submit(xr_server *s, uint32_t client, uint64_t n, int dtype, uint64_t *ticket)
{
    return submit(s, client, n, dtype, false, ticket);
}

extern "C" int xr_server_wait(xr_server *s, uint64_t ticket, uint64_t *out_offset, double *latency_us)
{
    if (!s) return XR_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return XR_EINVAL;
    s->cv.wait(lk, [&] { return it->second.state >= S_DONE || s->error != XR_OK; });
    if (it->second.state == S_FAILED || it->second.state < S_DONE) return s->error != XR_OK ? s->error : XR_ECUDA;
    if (out_offset) *out_offset = it->second.off;
    if (latency_us) *latency_us = it->second.t_done - it->second.t_sub;
    return XR_OK;
}

extern "C" int xr_server_wait_for(xr_server *s, uint64_t ticket, double timeout_us, uint64_t *out_offset,
                                  double *latency_us)
{
    if (!s || !(timeout_us >= 0.0)) return XR_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return XR_EINVAL;
    auto ready = [&] { return it->second.state >= S_DONE || s->error != XR_OK; };
    if (timeout_us >= 1e15) {  // over 30 years: an unbounded wait (and no clock overflow)
        s->cv.wait(lk, ready);
    } else if (!s->cv.wait_for(lk, std::chrono::duration<double, std::micro>(timeout_us), ready)) {
        return XR_ETIMEOUT;
    }
    if (it->second.state == S_FAILED || it->second.state < S_DONE) return s->error != XR_OK ? s->error : XR_ECUDA;
    if (out_offset) *out_offset = it->second.off;
    if (latency_us) *latency_us = it->second.t_done - it->second.t_sub;
    return XR_OK;
}

extern "C" int xr_server_release(xr_server *s, uint64_t ticket)
{
    if (!s) return XR_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end() || it->second.state != S_DONE) return XR_EINVAL;
    s->alloc.release(it->second.off, it->second.bytes);
    s->stats.released++;
    s->reqs.erase(it);
    return XR_OK;
}

extern "C" void *xr_server_arena(xr_server *s) { return s ? s->arena : nullptr; }

extern "C" int xr_server_read(xr_server *s, uint64_t offset, uint64_t bytes, void *dst, void *stream)
{
    if (!s || (bytes && !dst) || offset + bytes > s->cfg.arena_bytes) return XR_EINVAL;
    DeviceScope dscope(s->ctx->device);
    cudaError_t err = cudaMemcpyAsync(dst, s->arena + offset, bytes, cudaMemcpyDefault, (cudaStream_t)stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize((cudaStream_t)stream);
    return sst(err);
}

extern "C" int xr_server_client_state(xr_server *s, uint32_t client, void *h_words)
{
    if (!s || !h_words || client >= s->cfg.nclients) return XR_EINVAL;
    DeviceScope dscope(s->ctx->device);
    cudaError_t err = cudaStreamSynchronize(s->admit_st);
    unsigned char buf[XR_MAX_STATE_BYTES];
    if (err == cudaSuccess)
        err = cudaMemcpy(buf, s->d_cstates + (size_t)client * s->sw, (size_t)xr_state_bytes(s->cvar[client]),
                         cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) return sst(err);
    memcpy(h_words, buf, (size_t)xr_state_bytes(s->cvar[client]));
    return XR_OK;
}

extern "C" int xr_server_stats(xr_server *s, xr_serve_stats *out)
{
    if (!s || !out) return XR_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->arena_in_use = s->alloc.in_use;
    out->arena_peak = s->alloc.peak;
    return XR_OK;
}

extern "C" int xr_server_replay(xr_server *s, const double *arrival_us, const uint32_t *clients, const uint64_t *ns,
                                const int *dtypes, size_t nreq, double *latency_us, double *wall_us)
{
    if (!s || (nreq && (!arrival_us || !clients || !ns || !dtypes))) return XR_EINVAL;
    std::vector<u64> tk(nreq);
    const double t0 = now_us();
    for (size_t i = 0; i < nreq; ++i) {
        while (now_us() - t0 < arrival_us[i]) {
        }
        uint64_t t = 0;
        const int rc = submit(s, clients[i], ns[i], dtypes[i], true, &t);
        tk[i] = t;
        if (rc != XR_OK) return rc;
    }
    double last = t0;
    std::unique_lock<std::mutex> lk(s->mu);
    for (size_t i = 0; i < nreq; ++i) {
        auto it = s->reqs.find(tk[i]);
        s->cv.wait(lk, [&] { return it->second.state >= S_DONE || s->error != XR_OK; });
        if (it->second.state == S_FAILED || it->second.state < S_DONE) return s->error != XR_OK ? s->error : XR_ECUDA;
        if (latency_us) latency_us[i] = it->second.t_done - it->second.t_sub;
        last = std::max(last, it->second.t_done);
        s->reqs.erase(it);
    }
    if (wall_us) *wall_us = last - (t0 + (nreq ? arrival_us[0] : 0.0));
    return XR_OK;
}
