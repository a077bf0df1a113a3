/*
 * xr.h -- C ABI of libxr: bulk output generation from many independent
 * scrambled linear generators on one GB300 GPU (sm_103a).
 *
 * The generators are those of Blackman & Vigna, "Scrambled Linear Pseudorandom
 * Number Generators" (ACM TOMS; arXiv 1805.01407):
 *   - linear engines xoshiro256 (Sec. 3.2, matrix S_4w, Table 4: A=17, B=45),
 *     xoroshiro128 (Sec. 3.1, matrix X_2w, Table 4: (24,16,37), and (49,21,28)
 *     for the ++ scrambler) and the 32-bit xoshiro128 (Table 7: A=9, B=11);
 *   - scramblers + (Sec. 4.1), ++ (Sec. 4.3), ** (Sec. 4.4), parameters from
 *     Tables 5 and 8; the output is computed from the current state before the
 *     engine step (Sec. 2);
 *   - seeding with SplitMix64 (Sec. 5.3);
 *   - jumps: every engine is F2-linear, so advancing by J steps is the matrix
 *     power T^J (Sec. 5, Sec. 6).  The paper prints no jump distances; this
 *     library uses 2^(n/2) for a jump and 2^(3n/4) for a long jump of an n-bit
 *     state (2^128 and 2^192 for xoshiro256, 2^64 and 2^96 otherwise);
 *   - doubles in [0,1) from the upper 53 bits: (x >> 11) * 2^-53 (Sec. 5.3).
 *
 * Conventions for every call:
 *   - Pointers named d_* are device memory owned by the caller (e.g. torch
 *     tensors); h_* are host memory owned by the caller.  The library never
 *     allocates or frees caller buffers.  The context owns its jump tables, a
 *     status word and scratch for segment start states.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Every call that takes a stream only enqueues work on it and returns
 *     without waiting, unless its comment says otherwise.
 *   - A state is stored as its words in order, little-endian: 4 x uint64 (32 B)
 *     for xoshiro256, 2 x uint64 (16 B) for xoroshiro128, 4 x uint32 (16 B) for
 *     xoshiro128, 2 x uint32 (8 B) for xoroshiro64, 8 x uint64 (64 B) for
 *     xoshiro512, 16 x uint64 (128 B, the word that the paper's cyclic index p
 *     points past first) for xoroshiro1024.  Arrays of states are contiguous,
 *     state i at byte i * state bytes.  A state must not be all zero (captions
 *     of Figs. 1 to 4).
 *   - The jump tables of the 512- and 1024-bit engines (16 and 128 MiB) are
 *     built on the first call that needs them (a one-off wait of some ms).
 *   - Every call returns an xr status code.  Host-side argument errors return
 *     XR_EINVAL before any work is enqueued.  A failed CUDA launch or copy
 *     returns XR_ECUDA.  Errors found by kernels (an all-zero state) are
 *     recorded in a sticky device status word read by xr_status().
 *   - Device pointers must be aligned to the element size.  Output pointers
 *     aligned to 16 bytes with rows (m * element bytes) a multiple of 16 bytes
 *     take the fast path (TMA tile stores); other shapes take a plain-store
 *     path that gives the same values more slowly.
 */
#ifndef XR_H
#define XR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define XR_OK 0
#define XR_EINVAL 1        /* bad argument (variant, dtype, size, pointer, kind) */
#define XR_EZERO_STATE 2   /* an all-zero generator state was given or seen */
#define XR_ENOMEM 3        /* the context could not allocate its own memory */
#define XR_ECUDA 4         /* a CUDA call failed */
#define XR_ETIMEOUT 5      /* a bounded wait (xr_server_wait_for) ran out */
#define XR_EUNSUPPORTED 6  /* valid request this build does not implement */

/* ---- enums ------------------------------------------------------------- */
/* Generator = linear engine + scrambler (Tables 4, 5, 7, 8). */
enum xr_variant {
    XR_XOSHIRO256_PLUS = 0,       /* s0 + s3 */
    XR_XOSHIRO256_PLUSPLUS = 1,   /* rotl(s0 + s3, 23) + s0 */
    XR_XOSHIRO256_STARSTAR = 2,   /* rotl(s1 * 5, 7) * 9 */
    XR_XOROSHIRO128_PLUS = 3,     /* s0 + s1, engine (24,16,37) */
    XR_XOROSHIRO128_PLUSPLUS = 4, /* rotl(s0 + s1, 17) + s0, engine (49,21,28) */
    XR_XOROSHIRO128_STARSTAR = 5, /* rotl(s0 * 5, 7) * 9, engine (24,16,37) */
    XR_XOSHIRO128_PLUSPLUS = 6,   /* 32-bit: rotl(s0 + s3, 7) + s0 */
    XR_XOSHIRO128_STARSTAR = 7,   /* 32-bit: rotl(s1 * 5, 7) * 9 */
    XR_XOSHIRO128_PLUS = 8,       /* 32-bit: s0 + s3 */
    /* further generators of Sec. 5 (Tables 4, 5, 7, 8; Figs. 1, 2, 4) */
    XR_XOROSHIRO128_STAR = 9,     /* s0 * 0x9e3779b97f4a7c13, engine (24,16,37) */
    XR_XOROSHIRO64_STAR = 10,     /* 32-bit, engine (26,9,13): s0 * 0x9E3779BB */
    XR_XOROSHIRO64_STARSTAR = 11, /* 32-bit: rotl(s0 * 0x9E3779BB, 5) * 5 */
    XR_XOSHIRO512_PLUS = 12,      /* engine S_8w (11,21): s0 + s2 */
    XR_XOSHIRO512_PLUSPLUS = 13,  /* rotl(s0 + s2, 17) + s2 */
    XR_XOSHIRO512_STARSTAR = 14,  /* rotl(s1 * 5, 7) * 9 */
    XR_XOROSHIRO1024_STAR = 15,   /* engine X_kw, k = 16 (25,27,36): s0 * 0x9e3779b97f4a7c13 */
    XR_XOROSHIRO1024_PLUSPLUS = 16, /* rotl(s0 + s15, 23) + s15 */
    XR_XOROSHIRO1024_STARSTAR = 17, /* rotl(s0 * 5, 7) * 9 */
    XR_NUM_VARIANTS = 18
};

/* Value type of the outputs. */
enum xr_dtype {
    XR_U64 = 0,  /* raw 64-bit output; 64-bit generators only */
    XR_U32 = 1,  /* raw 32-bit output; 32-bit generators only */
    XR_F64 = 2,  /* double in [0,1): (x >> 11) * 2^-53, or x * 2^-32 for 32-bit words */
    XR_F32 = 3   /* float in [0,1): upper 24 bits * 2^-24 */
};

/* Placement of the S x m outputs of xr_fill. */
enum xr_layout {
    XR_STREAM_MAJOR = 0, /* out[i * m + j] = output j of stream i */
    XR_INTERLEAVED = 1   /* out[j * S + i] = output j of stream i */
};

enum xr_jump_kind {
    XR_JUMP = 0,      /* advance 2^(n/2) steps */
    XR_LONG_JUMP = 1  /* advance 2^(3n/4) steps */
};

typedef struct xr_ctx xr_ctx;

/* ---- context ----------------------------------------------------------- */

/* Create a context on `device` (made current on the calling thread).  Builds
 * the jump tables T^(2^k), k = 0 .. n-1, of the 64- to 256-bit engines on the
 * device by stepping unit states (column j of T is the step of e_j, Sec. 3)
 * and repeated squaring, and their power sets for stream starts; waits for
 * them.  About 90 MiB of device memory; the xoshiro512 and xoroshiro1024
 * tables (16 MiB and 128 MiB) are built on their first use.  Returns
 * XR_ENOMEM / XR_ECUDA on failure, with *out = NULL.
 *
 * Every later call that takes a context, or a batch or server made from one,
 * runs on the context's device: it makes that device current for the call and
 * restores the caller's current device before returning. */
int xr_ctx_create(int device, xr_ctx **out);

/* Free everything the context owns.  Waits for the device first.  NULL is
 * accepted. */
int xr_ctx_destroy(xr_ctx *ctx);

/* ---- properties (pure host functions, no GPU needed) --------------------
 * State size k words of w bits (n = k w) of each engine, from its definition:
 * Sec. 3.1 (xoroshiro, k = 2 or 16), Sec. 3.2 (xoshiro, k = 4 or 8), Table 4
 * (w = 64) and Table 7 (w = 32). */
int xr_state_words(int variant);      /* 2 .. 16; -1 for a bad variant */
int xr_word_bits(int variant);        /* 64 or 32; -1 for a bad variant */
int xr_state_bytes(int variant);      /* 8 .. 128; -1 for a bad variant */
int xr_state_bits(int variant);       /* n = 64 .. 1024; -1 for a bad variant */
/* Bytes of one output value: 8, 4, 8, 4 for u64, u32, f64, f32 (Sec. 5.3
 * for the floating-point values); -1 for a bad dtype. */
int xr_dtype_bytes(int dtype);
/* Name of a generator as in Tables 5 and 8, e.g. "xoshiro256**"; NULL if bad. */
const char *xr_variant_name(int variant);
const char *xr_error_string(int status);   /* never NULL; no counterpart in the paper */
/* log2 of the jump distance of `kind` for `variant`; -1 if bad.  Sec. 5
 * offers jumps but prints no distance; this library takes 2^(n/2) (jump) and
 * 2^(3n/4) (long jump) for an n-bit state. */
int xr_jump_log2(int variant, int kind);

/* ---- seeding (Sec. 5.3) ---------------------------------------------------
 * SplitMix64 initialized with the seed fills the state: consecutive 64-bit
 * outputs for 64-bit words; for 32-bit words each output gives two words, low
 * half first.  xr_seed writes one state to d_state; xr_seed_many writes
 * count states, state i from d_seeds[i] (device array of uint64). */
int xr_seed(xr_ctx *ctx, int variant, uint64_t seed, void *d_state, void *stream);
int xr_seed_many(xr_ctx *ctx, int variant, const uint64_t *d_seeds, size_t count,
                 void *d_states, void *stream);

/* ---- state transfer ------------------------------------------------------
 * The generator state is the whole checkpoint of a sequence; the captions of
 * Figs. 1 to 4 require it not to be all zeros (the zero state is the one
 * fixed point of a linear engine, Sec. 6).
 * xr_set_state copies one state from host words (h_words: state bytes, layout
 * as above) to d_state; rejects the all-zero state with XR_EZERO_STATE.
 * xr_get_state copies one state from d_state to h_words and waits on stream. */
int xr_set_state(xr_ctx *ctx, int variant, const void *h_words, void *d_state, void *stream);
int xr_get_state(xr_ctx *ctx, int variant, const void *d_state, void *h_words, void *stream);

/* ---- jumps (Sec. 5, Sec. 6) ----------------------------------------------
 * xr_jump: each of the `count` states in d_states is replaced by T^(times*J) s,
 * the state after `times` successive jumps of the given kind.
 * xr_advance: each state is replaced by T^nsteps s (nsteps next() calls).
 * Both are F2 matrix-vector products with the powers T^(2^k) selected by the
 * bits of the exponent. */
int xr_jump(xr_ctx *ctx, int variant, int kind, void *d_states, size_t count, uint64_t times,
            void *stream);
int xr_advance(xr_ctx *ctx, int variant, void *d_states, size_t count, uint64_t nsteps,
               void *stream);

/* xr_make_streams (Sec. 5, jumps; Sec. 6, jumping is a product with the
 * matrix power T^J): start states of S independent streams,
 *   d_states_out[i] = J^(first + i)(d_base),  i = 0 .. S-1,
 * where J is the jump (or long jump): stream 0 is the base after `first`
 * jumps, each next stream one jump further.  d_base (one state) is read only;
 * it may not overlap d_states_out.
 *   - For S of at least 512 x 32 streams (engines of at most 256 bits) the
 *     first call that needs the power set of a new distance 2^J P (P the
 *     largest power of two with 512 P <= S) builds and keeps it in the context
 *     (cudaMalloc, 12 MiB for 256-bit states) and waits for the device once;
 *     under stream capture it is not built and the call takes a slower path
 *     with the same results. */
int xr_make_streams(xr_ctx *ctx, int variant, int kind, const void *d_base, uint64_t first,
                    size_t S, void *d_states_out, void *stream);

/* ---- generation ------------------------------------------------------------
 * xr_fill: S streams x m outputs.  Stream i starts at d_states[i] and emits
 * m outputs of next() (Sec. 2: the output is the scrambler, Sec. 4, applied
 * to the current state, then the engine of Sec. 3 steps the state; doubles
 * and floats as in Sec. 5.3), converted to dtype, placed by
 * layout into d_out (S * m elements of dtype).  With write_back != 0 the
 * state after the m steps is written back to d_states[i], so a later call
 * continues each sequence.  S = 0 or m = 0 is a valid no-op (apart from
 * write-back, which then leaves the states unchanged). */
int xr_fill(xr_ctx *ctx, int variant, void *d_states, size_t S, size_t m, int dtype, int layout,
            void *d_out, int write_back, void *stream);

/* xr_fill_streams: xr_make_streams followed by xr_fill.  Stream
 * i = J^(first + i)(d_base) for i < S (the jump or long jump, Sec. 5; jumps
 * as products with T^J, Sec. 6) emits m outputs of next(), converted to
 * dtype, at d_out[i * m .. i * m + m - 1] (stream-major).  For short rows
 * one kernel computes each stream's start state in the thread that then
 * generates it, with no state table in global memory: in chunks of 512 P
 * streams (P a power of two, at least 32), stream p + P j of a chunk starts
 * at (T^J)^(P j) applied to stream p.  The states are not written back (use
 * xr_make_streams and xr_fill with write_back to continue sequences).
 *   - d_base: one state (device), read only; d_out: S * m elements of dtype
 *     (device, aligned to the element size).
 *   - The fused kernel takes rows of at most 512 bytes (m * element size a
 *     multiple of 16, d_out 16-byte aligned), engines of at most 256 bits,
 *     and chunks while at least 512 x 32 streams are left.  Everything else
 *     (longer rows, where it measured slower, the rest below 512 x 32 streams,
 *     the 512- and 1024-bit generators) goes through a state table, with the
 *     same results.
 *   - The first call that needs the power set of a new distance 2^J P builds
 *     and keeps it in the context (3 x 512 matrices: 12 MiB for 256-bit
 *     states, with cudaMalloc) and waits for the device once; under stream
 *     capture it is not built and those streams take the state table.  A call
 *     that grows the scratch waits for the device too: make first calls
 *     outside stream capture.
 *   - Uses the context scratch (grown with cudaMalloc when too small: P
 *     states for a chunk, S states on the state-table path); not safe to call
 *     concurrently with xr_fill_seq or another xr_fill_streams on the same
 *     context.
 *   - XR_EINVAL for bad arguments, and when the last stream index
 *     first + S - 1 does not fit in 64 bits; S = 0 or m = 0 is a valid
 *     no-op. */
int xr_fill_streams(xr_ctx *ctx, int variant, int kind, const void *d_base, uint64_t first, size_t S, size_t m,
                    int dtype, void *d_out, void *stream);

/* xr_fill_seq: the first n outputs of one sequence starting at d_state, into
 * d_out (n elements of dtype); d_state is then advanced by n steps (the n
 * calls of next() of Sec. 2).  The
 * sequence is split into segments of 2^10 outputs whose start states are
 * T^(p * 2^10) s (jump-ahead as a matrix power, Sec. 6), kept in the
 * context's scratch memory, so the
 * whole GPU works on one sequence.  Not safe to call concurrently on two
 * streams with the same context (shared scratch). */
int xr_fill_seq(xr_ctx *ctx, int variant, void *d_state, size_t n, int dtype, void *d_out,
                void *stream);

/* xr_fill_seq_noalloc: xr_fill_seq for callers that cannot allocate device
 * memory during the call -- for example code that runs while the application
 * owns all device memory through its own pool, or inside a real-time or
 * callback path where cudaMalloc/cudaFree would block, synchronize the device
 * or fail.  (The paper has no counterpart: this is a property of the
 * library, not of the method.)  The outputs and the advanced state are the
 * ones xr_fill_seq gives.
 *   - Allocates nothing: the segment start states (one state per 1024
 *     outputs) live in one static device array of XR_NOALLOC_SCRATCH_BYTES
 *     (2 MiB) that every GPU loading the library holds until the process
 *     exits.  The context (created earlier) supplies the jump tables.
 *   - The largest n is XR_NOALLOC_MAX_OUTPUTS_FOR(state bytes): 2^26 outputs
 *     for states of up to 32 bytes, 2^25 for xoshiro512 (64-byte states) and
 *     2^24 for xoroshiro1024 (128-byte states).  A larger n returns XR_EINVAL
 *     and enqueues nothing.
 *   - The jump tables of xoshiro512 and xoroshiro1024 are built on first use,
 *     which allocates; this call does not build them and returns
 *     XR_EUNSUPPORTED until an earlier call on the same context has (any
 *     call on that generator that jumps: xr_fill_seq, xr_jump, xr_advance,
 *     xr_make_streams, xr_jump_table).
 *   - The first call on a device looks up the array's device address (with
 *     that device current, cudaGetSymbolAddress); make that first call
 *     before any stream capture.
 *   - All calls in the process share the array, which keeps the last call's
 *     contents; nothing in it needs to start at zero, since every slot a call
 *     reads is written earlier in the same call.  Calls that overlap on the
 *     GPU (different streams, or different threads without ordering) race on
 *     the array and give wrong outputs: serialize them. */
#define XR_NOALLOC_SCRATCH_BYTES ((size_t)2 << 20)
#define XR_NOALLOC_MAX_OUTPUTS ((size_t)1 << 26)
#define XR_NOALLOC_MAX_OUTPUTS_FOR(state_bytes)                                  \
    ((size_t)(state_bytes) <= 32 ? XR_NOALLOC_MAX_OUTPUTS                        \
                                 : (XR_NOALLOC_SCRATCH_BYTES / (size_t)(state_bytes)) << 10)
int xr_fill_seq_noalloc(xr_ctx *ctx, int variant, void *d_state, size_t n, int dtype, void *d_out,
                        void *stream);

/* xr_fill_host: end-to-end call with host memory.  Copies one base state from
 * h_base (host), makes S streams J^(first + i)(base), generates S x m outputs
 * (stream-major) and copies them to h_out (host, S * m elements of dtype;
 * page-locked memory gives full copy speed).  Generation and device-to-host
 * copies overlap through two staging buffers the context owns.  Blocks until
 * h_out is complete.  XR_EINVAL for bad arguments and when the last stream
 * index first + S - 1 does not fit in 64 bits. */
int xr_fill_host(xr_ctx *ctx, int variant, int kind, const void *h_base, uint64_t first,
                 size_t S, size_t m, int dtype, void *h_out, void *stream);

/* ---- batching: many uneven requests in one persistent launch ---------------
 * A request asks for the first n outputs of one sequence (as xr_fill_seq),
 * starting from the state in slot `slot` of a caller-owned state table, and
 * writes them at byte offset `out_offset` (a multiple of 16) of a
 * caller-owned output arena.  Slots are xr_batch_slot_bytes(b) bytes: 32
 * when every request's state fits (smaller states use the start of a slot),
 * 64 when the batch holds xoshiro512 requests and 128 with xoroshiro1024
 * requests (Sec. 3: 512- and 1024-bit states).  When
 * the batch runs, every request's slot is advanced by its n steps, so the
 * next batch continues each sequence.  Two requests of one batch must not
 * share a slot.  Optionally each slot is first seeded with SplitMix64 from a
 * per-request seed (Sec. 5.3).
 *
 * The plan groups requests by (variant, dtype), cuts them into segments of
 * 1024 outputs whose start states come from jump-ahead (power sets, three
 * launches for the whole batch; a doubling tree for xoshiro512 and
 * xoroshiro1024), and packs 32 segments per warp task.  One persistent kernel
 * pulls tasks from a device queue (a second one serves the 512- and
 * 1024-bit generators); each lane writes its rows with its own bulk copies,
 * so segments of different requests share a warp.  Results equal
 * xr_fill_seq on each request alone, bit for bit. */
typedef struct {
    int variant;          /* xr_variant */
    int dtype;            /* xr_dtype valid for the variant */
    uint64_t n;           /* outputs (0 allowed: only seeding, if any) */
    uint64_t slot;        /* state slot index */
    uint64_t out_offset;  /* byte offset in the output arena, multiple of 16 */
} xr_request;

typedef struct xr_batch xr_batch;

/* Plan a batch: checks the requests (XR_EINVAL on a bad variant/dtype, an
 * unaligned offset or a slot used twice), builds the jump tables of the
 * 512- and 1024-bit engines if a request needs them and the context has
 * none yet, copies the plan to device memory owned by the batch and sizes
 * its scratch.  h_reqs is read during the call only.  The batch keeps using
 * ctx (which must outlive it). */
int xr_batch_create(xr_ctx *ctx, const xr_request *h_reqs, size_t nreq, xr_batch **out);
int xr_batch_destroy(xr_batch *b);

/* Bytes of output arena the batch writes (max of out_offset + n * element
 * size over requests), the number of warp tasks, and the bytes of one state
 * slot (32, 64 or 128: the largest state among the requests, at least 32). */
uint64_t xr_batch_arena_bytes(const xr_batch *b);
uint64_t xr_batch_tasks(const xr_batch *b);
uint64_t xr_batch_slot_bytes(const xr_batch *b);

/* Run the batch on `stream`: d_seeds (device, one uint64 per request, or
 * NULL to use the slots as they are), d_slots (device state table), d_out
 * (device arena, 16-byte aligned).  With use_graph != 0 the launches are
 * captured into a CUDA graph on the first run with these pointers and the
 * graph is replayed on later runs (a different pointer set recaptures). */
int xr_batch_run(xr_batch *b, const uint64_t *d_seeds, void *d_slots, void *d_out, int use_graph,
                 void *stream);

/* Launch configuration of the persistent kernel: outputs per staged row
 * (4, 8, 16, 32 or 64) and threads per block (128, 256 or 512). */
int xr_batch_set_config(xr_batch *b, int outputs_per_row, int block);
int xr_batch_get_config(const xr_batch *b, int *outputs_per_row, int *block);

/* Autotune: time every (outputs_per_row, block) pair that fits in shared
 * memory on this batch (each trial restores d_slots first), keep the
 * fastest, restore d_slots and report the best time in *best_ms.  Blocks
 * on `stream`. */
int xr_batch_tune(xr_batch *b, const uint64_t *d_seeds, void *d_slots, void *d_out, void *stream,
                  float *best_ms);

/* ---- serving: continuous batching for many clients -------------------------
 * A server owns, on the device, one generator state per client (seeded with
 * SplitMix64 from a per-client seed; any of the 18 generators, the jump
 * tables of the 512- and 1024-bit engines built at creation when a client
 * needs them) and an output arena of a fixed budget.
 * Clients submit requests "the next n outputs of my sequence as dtype" at any
 * time, from any thread.  A scheduler thread admits pending requests in
 * arrival order while arena space (and a round slot) is free; at admission a
 * small kernel gives each request its own start state (the client's state,
 * after which the client's state jumps ahead by n), so a client's requests
 * continue one sequence in submission order whatever runs concurrently.
 * Admitted requests run as rounds of the batched kernels of xr_batch_*;
 * up to max_rounds rounds are in flight on separate streams, so requests that
 * arrive while others run are admitted and overlap on the device.  A round
 * takes at most arena_bytes / max_rounds bytes of outputs (a single larger
 * request forms a round alone), so under load the next round is admitted
 * while the current one runs.  Outputs
 * stay in the arena until released.  Plain mode instead runs one
 * xr_fill_seq per request, in arrival order, on one stream (for comparison). */
#define XR_SERVE_BATCHED 0
#define XR_SERVE_PLAIN 1

typedef struct {
    uint64_t arena_bytes;          /* output budget (device memory the server allocates) */
    uint32_t nclients;
    uint32_t max_rounds;           /* rounds in flight (batched mode), >= 1 */
    uint32_t max_round_requests;   /* requests per round (batched mode), >= 1 */
    int mode;                      /* XR_SERVE_BATCHED or XR_SERVE_PLAIN */
    int outputs_per_row, block;    /* batched kernel configuration; 0 = 32, 128 */
} xr_server_config;

/* Counters since creation.  For completed requests, summed over requests:
 * queue_ns from submission to the start of its round's launch, launch_ns the
 * host time launching that round (admission, plan upload, kernel launches),
 * device_ns from the end of that launch to the observed completion. */
typedef struct {
    uint64_t submitted, completed, released, rounds, bytes;
    uint64_t arena_in_use, arena_peak;
    uint64_t queue_ns, launch_ns, device_ns;
} xr_serve_stats;

typedef struct xr_server xr_server;

/* Create a server: h_client_variants / h_client_seeds have nclients entries
 * (host).  Starts the scheduler thread.  XR_EINVAL on a bad config. */
int xr_server_create(xr_ctx *ctx, const xr_server_config *cfg, const int *h_client_variants,
                     const uint64_t *h_client_seeds, xr_server **out);
/* Drop requests not yet admitted, wait for admitted ones, stop the
 * scheduler and free everything. */
int xr_server_destroy(xr_server *s);
/* Queue a request (non-blocking).  XR_EINVAL for a bad client/dtype or a
 * request larger than the whole arena. */
int xr_server_submit(xr_server *s, uint32_t client, uint64_t n, int dtype, uint64_t *ticket);
/* Block until the request is complete: its outputs are at byte *out_offset
 * of the arena (xr_server_arena) until released; *latency_us is the time from
 * submission to observed completion. */
int xr_server_wait(xr_server *s, uint64_t ticket, uint64_t *out_offset, double *latency_us);

/* As xr_server_wait, but gives up after timeout_us microseconds of host time
 * (0 polls once) and returns XR_ETIMEOUT, with the request still queued or
 * running: a caller can bound its wait and detect a stalled server without
 * any device-side wait.  A later wait on the same ticket is allowed. */
int xr_server_wait_for(xr_server *s, uint64_t ticket, double timeout_us, uint64_t *out_offset, double *latency_us);
/* Free a completed request's arena space (its outputs become invalid). */
int xr_server_release(xr_server *s, uint64_t ticket);
void *xr_server_arena(xr_server *s);
/* Copy `bytes` of the arena at `offset` to dst (host or device memory, any
 * kind) on `stream` and wait for the copy. */
int xr_server_read(xr_server *s, uint64_t offset, uint64_t bytes, void *dst, void *stream);
/* Current state of a client after every admitted request (waits for them);
 * h_words receives the state's bytes (up to 128). */
int xr_server_client_state(xr_server *s, uint32_t client, void *h_words);
int xr_server_stats(xr_server *s, xr_serve_stats *out);
/* Load replay: submit request i at arrival_us[i] microseconds after the call
 * starts (from the calling thread), release every output as soon as it
 * completes, wait for all, and return each request's latency (us) and the
 * wall time from the first arrival to the last completion. */
int xr_server_replay(xr_server *s, const double *arrival_us, const uint32_t *clients, const uint64_t *ns,
                     const int *dtypes, size_t nreq, double *latency_us, double *wall_us);

/* ---- analysis workloads of the paper ---------------------------------------
 * Escaping zeroland (Sec. 8): for each of the n states with exactly one bit
 * set, the first nout outputs are generated; d_counts[t] (device, nout -
 * window + 1 uint64) receives the number of one bits in outputs t .. t +
 * window - 1 summed over the n states.  The paper's curve (window 4, 1000
 * outputs) is d_counts[t] / (n * window * word bits).  window <= 64.
 * XR_EINVAL on bad sizes. */
int xr_zeroland(xr_ctx *ctx, int variant, size_t nout, size_t window, uint64_t *d_counts, void *stream);

/* Linear complexity of one output bit (Sec. 9.3, Table 13): Berlekamp-Massey
 * over F2 on bit `bit` (0 = least significant) of the first N outputs of the
 * sequence starting at d_state (device, 16-byte aligned, read only, not
 * advanced).  d_scratch (device, caller-owned, 16-byte aligned) must hold
 * XR_LC_SCRATCH_BYTES(N) bytes.  Writes the linear complexity of the N-bit
 * prefix to *h_lc and waits for the device; it is the sequence's linear
 * complexity when N >= 2 L.  XR_EINVAL for bad arguments or N outside
 * 2 .. XR_LC_MAX_BITS.  A prefix complexity of 32 (floor(N / 64) + 5) or more
 * (above N / 2 + 127, so not decided by an N-bit prefix) returns
 * XR_EUNSUPPORTED.  The polynomials stay in registers; the algorithm takes
 * blocks of 32 sequence bits per synchronisation.  A sequence of 16,128 bits
 * or more runs on a thread-block cluster of 16 CTAs (16 SMs; 8 where the
 * device does not take 16), a shorter one on one CTA; XR_ECUDA also covers a
 * cluster whose internal exchange did not complete (not expected).  Calls on
 * different streams run concurrently. */
#define XR_LC_MAX_BITS ((size_t)786000)
#define XR_LC_SCRATCH_BYTES(N) (64 + ((((N) + 31) / 32 + 22) * 4 + 15) / 16 * 16)
int xr_linear_complexity(xr_ctx *ctx, int variant, int bit, size_t N, const void *d_state, void *d_scratch,
                         size_t scratch_bytes, uint64_t *h_lc, void *stream);

/* Many linear complexities in one call: job j takes the state at d_states +
 * j * state_stride (device, 16-byte aligned; the stride a multiple of 16 and
 * at least the largest state) and gives h_lc[j] (host): the complexity, or
 * UINT64_MAX where xr_linear_complexity would return XR_EUNSUPPORTED.  With
 * at most (SMs / 8) jobs each sequence of 16,128 bits or more runs on a
 * cluster of 8 CTAs (16 with at most SMs / 16 jobs); otherwise one CTA per
 * job, so up to a few hundred jobs run at once.  d_scratch (device, 16-byte
 * aligned) must hold xr_lc_scratch_bytes(jobs, njobs) bytes.  Any bad job
 * makes the call return XR_EINVAL before work is enqueued.  Waits for the
 * device. */
typedef struct xr_lc_job {
    int32_t variant;
    int32_t bit;
    uint64_t N;
} xr_lc_job;
size_t xr_lc_scratch_bytes(const xr_lc_job *jobs, size_t njobs);
int xr_linear_complexity_many(xr_ctx *ctx, const xr_lc_job *jobs, size_t njobs, const void *d_states,
                              size_t state_stride, void *d_scratch, size_t scratch_bytes, uint64_t *h_lc,
                              void *stream);

/* ---- status and inspection ------------------------------------------------ */

/* Sticky device status: XR_OK, or the first error a kernel recorded
 * (XR_EZERO_STATE: a kernel met the all-zero state, which a full-period
 * linear engine never leaves or reaches from a nonzero state, Sec. 6).
 * Waits for the device.  reset != 0 clears it. */
int xr_status(xr_ctx *ctx, int reset);

/* Copy the jump table entry T^(2^k) of variant's engine (the F2 transition
 * matrix T of Sec. 3 raised to 2^k, Sec. 6) to h_out (host):
 * n columns, column c = T^(2^k) e_c as n/32 uint32 words (bit r of the column
 * is bit r % 32 of word r / 32); n * n / 8 bytes.  Waits for the copy. */
int xr_jump_table(xr_ctx *ctx, int variant, int k, void *h_out);

/* Number of kernels this process has launched through libxr so far (all
 * contexts; a host-side counter, no GPU needed; no counterpart in the paper).  Lets a caller count the
 * launches inside a timed region. */
uint64_t xr_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* XR_H */
