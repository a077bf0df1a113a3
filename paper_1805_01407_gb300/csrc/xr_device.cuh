// xr_device.cuh -- device-side building blocks of libxr (sm_103a).
//
// Linear engines (Sec. 3), scramblers (Sec. 4), exact output conversions
// (Sec. 5.3), F2 matrix-vector products for jumps (Sec. 5, 6), and inline-PTX
// wrappers for the Blackwell bulk-tensor (TMA) stores used by the fill kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace xr {

typedef unsigned long long u64;
typedef unsigned int u32;

// ---------------------------------------------------------------- word ops
__device__ __forceinline__ u64 rotl(u64 x, int r) { return (x << r) | (x >> (64 - r)); }
__device__ __forceinline__ u32 rotl(u32 x, int r) { return __funnelshift_l(x, x, r); }

// ---------------------------------------------------------------- engines
// xoshiro with four words (Sec. 3.2): the new words are the columns of S_4w,
//   s0' = s0 ^ s1 ^ s3          s1' = s0 ^ s1 ^ s2
//   s2' = s0 ^ s2 ^ (s1 << A)   s3' = rotl(s1 ^ s3, B)
template <typename W, int A, int B>
struct Xoshiro4 {
    typedef W word;
    static constexpr int K = 4;
    static constexpr int NBITS = 4 * 8 * (int)sizeof(W);
    W s[4];
    __device__ __forceinline__ void step()
    {
        const W x02 = s[0] ^ s[2];
        const W x13 = s[1] ^ s[3];
        const W n2 = x02 ^ (s[1] << A);
        s[1] = s[1] ^ x02;
        s[0] = s[0] ^ x13;
        s[2] = n2;
        s[3] = rotl(x13, B);
    }
};

// xoroshiro with two words (Sec. 3.1), the columns of X_2w:
//   t = s0 ^ s1;  s0' = rotl(s0, A) ^ t ^ (t << B);  s1' = rotl(t, C)
template <typename W, int A, int B, int C>
struct Xoroshiro2 {
    typedef W word;
    static constexpr int K = 2;
    static constexpr int NBITS = 2 * 8 * (int)sizeof(W);
    W s[2];
    __device__ __forceinline__ void step()
    {
        const W t = s[0] ^ s[1];
        s[0] = rotl(s[0], A) ^ t ^ (t << B);
        s[1] = rotl(t, C);
    }
};

// xoshiro with eight words (Sec. 3.2), the columns of S_8w:
//   s0' = s0 ^ s6          s1' = s0 ^ s1 ^ s2     s2' = s0 ^ s2        s3' = s3 ^ s4
//   s4' = s1 ^ s4 ^ s5     s5' = s1 ^ s5          s6' = (s1 << A) ^ s3 ^ s6 ^ s7
//   s7' = rotl(s3 ^ s7, B)
template <typename W, int A, int B>
struct Xoshiro8 {
    typedef W word;
    static constexpr int K = 8;
    static constexpr int NBITS = 8 * 8 * (int)sizeof(W);
    W s[8];
    __device__ __forceinline__ void step()
    {
        const W n0 = s[0] ^ s[6], n1 = s[0] ^ s[1] ^ s[2], n2 = s[0] ^ s[2], n3 = s[3] ^ s[4];
        const W n4 = s[1] ^ s[4] ^ s[5], n5 = s[1] ^ s[5], n6 = (s[1] << A) ^ s[3] ^ s[6] ^ s[7];
        const W n7 = rotl(s[3] ^ s[7], B);
        s[0] = n0; s[1] = n1; s[2] = n2; s[3] = n3; s[4] = n4; s[5] = n5; s[6] = n6; s[7] = n7;
    }
};

// xoroshiro with sixteen words (Eq. (M), X_kw with k = 16), written with the
// words shifting down one place per step (the figure's cyclic index becomes
// register renaming once 16 steps are unrolled):
//   t = s0 ^ s15;  s_j' = s_{j+1} (j <= 13);  s14' = rotl(s0, A) ^ t ^ (t << B);
//   s15' = rotl(t, C)
template <typename W, int A, int B, int C>
struct Xoroshiro16 {
    typedef W word;
    static constexpr int K = 16;
    static constexpr int NBITS = 16 * 8 * (int)sizeof(W);
    W s[16];
    __device__ __forceinline__ void step()
    {
        const W t = s[0] ^ s[15];
        const W n14 = rotl(s[0], A) ^ t ^ (t << B);
        const W n15 = rotl(t, C);
#pragma unroll
        for (int j = 0; j < 14; ++j) s[j] = s[j + 1];
        s[14] = n14;
        s[15] = n15;
    }
};

// Engine ids used for the jump tables.
enum { ENG_XOSHIRO256 = 0, ENG_XOROSHIRO128 = 1, ENG_XOROSHIRO128PP = 2, ENG_XOSHIRO128 = 3,
       ENG_XOROSHIRO64 = 4, ENG_XOSHIRO512 = 5, ENG_XOROSHIRO1024 = 6, NUM_ENGINES = 7 };

template <int ENG> struct EngineOf;
template <> struct EngineOf<ENG_XOSHIRO256> { typedef Xoshiro4<u64, 17, 45> type; };      // Table 4
template <> struct EngineOf<ENG_XOROSHIRO128> { typedef Xoroshiro2<u64, 24, 16, 37> type; };  // Table 4
template <> struct EngineOf<ENG_XOROSHIRO128PP> { typedef Xoroshiro2<u64, 49, 21, 28> type; };// Table 4
template <> struct EngineOf<ENG_XOSHIRO128> { typedef Xoshiro4<u32, 9, 11> type; };        // Table 7
template <> struct EngineOf<ENG_XOROSHIRO64> { typedef Xoroshiro2<u32, 26, 9, 13> type; };  // Table 7
template <> struct EngineOf<ENG_XOSHIRO512> { typedef Xoshiro8<u64, 11, 21> type; };       // Table 4
template <> struct EngineOf<ENG_XOROSHIRO1024> { typedef Xoroshiro16<u64, 25, 27, 36> type; };  // Table 4

// ---------------------------------------------------------------- generators
// Scrambler applied to the current state (Sec. 2), parameters of Tables 5, 8.
template <int V> struct Gen;

#define XR_GEN(V, ENG, BODY)                                                    \
    template <> struct Gen<V> {                                                 \
        static constexpr int engine = ENG;                                      \
        typedef typename EngineOf<ENG>::type E;                                 \
        typedef typename E::word word;                                          \
        __device__ __forceinline__ static word out(const E &e) { BODY }         \
    };

XR_GEN(0, ENG_XOSHIRO256, return e.s[0] + e.s[3];)                              // xoshiro256+
XR_GEN(1, ENG_XOSHIRO256, return rotl(e.s[0] + e.s[3], 23) + e.s[0];)          // xoshiro256++
XR_GEN(2, ENG_XOSHIRO256, return rotl(e.s[1] * 5ull, 7) * 9ull;)               // xoshiro256**
XR_GEN(3, ENG_XOROSHIRO128, return e.s[0] + e.s[1];)                            // xoroshiro128+
XR_GEN(4, ENG_XOROSHIRO128PP, return rotl(e.s[0] + e.s[1], 17) + e.s[0];)      // xoroshiro128++
XR_GEN(5, ENG_XOROSHIRO128, return rotl(e.s[0] * 5ull, 7) * 9ull;)             // xoroshiro128**
XR_GEN(6, ENG_XOSHIRO128, return rotl(e.s[0] + e.s[3], 7) + e.s[0];)           // xoshiro128++
XR_GEN(7, ENG_XOSHIRO128, return rotl(e.s[1] * 5u, 7) * 9u;)                   // xoshiro128**
XR_GEN(8, ENG_XOSHIRO128, return e.s[0] + e.s[3];)                              // xoshiro128+
XR_GEN(9, ENG_XOROSHIRO128, return e.s[0] * 0x9e3779b97f4a7c13ull;)             // xoroshiro128*
XR_GEN(10, ENG_XOROSHIRO64, return e.s[0] * 0x9E3779BBu;)                       // xoroshiro64*
XR_GEN(11, ENG_XOROSHIRO64, return rotl(e.s[0] * 0x9E3779BBu, 5) * 5u;)         // xoroshiro64**
XR_GEN(12, ENG_XOSHIRO512, return e.s[0] + e.s[2];)                             // xoshiro512+
XR_GEN(13, ENG_XOSHIRO512, return rotl(e.s[0] + e.s[2], 17) + e.s[2];)         // xoshiro512++
XR_GEN(14, ENG_XOSHIRO512, return rotl(e.s[1] * 5ull, 7) * 9ull;)              // xoshiro512**
XR_GEN(15, ENG_XOROSHIRO1024, return e.s[0] * 0x9e3779b97f4a7c13ull;)           // xoroshiro1024*
XR_GEN(16, ENG_XOROSHIRO1024, return rotl(e.s[0] + e.s[15], 23) + e.s[15];)    // xoroshiro1024++
XR_GEN(17, ENG_XOROSHIRO1024, return rotl(e.s[0] * 5ull, 7) * 9ull;)           // xoroshiro1024**
#undef XR_GEN

// ---------------------------------------------------------------- state I/O
// A state in memory is its words in order, little-endian: 8 to 128 bytes,
// aligned to its size (16 bytes at most).
template <typename E>
__device__ __forceinline__ void load_state(E &e, const void *p)
{
    constexpr int B = (int)sizeof(e.s);
    u32 w[B / 4];
    if constexpr (B >= 16) {
#pragma unroll
        for (int q = 0; q < B / 16; ++q) {
            const uint4 a = reinterpret_cast<const uint4 *>(p)[q];
            w[4 * q] = a.x; w[4 * q + 1] = a.y; w[4 * q + 2] = a.z; w[4 * q + 3] = a.w;
        }
    } else {
        const uint2 a = reinterpret_cast<const uint2 *>(p)[0];
        w[0] = a.x; w[1] = a.y;
    }
    if constexpr (sizeof(typename E::word) == 8) {
#pragma unroll
        for (int j = 0; j < E::K; ++j) e.s[j] = (u64)w[2 * j] | ((u64)w[2 * j + 1] << 32);
    } else {
#pragma unroll
        for (int j = 0; j < E::K; ++j) e.s[j] = w[j];
    }
}

template <typename E>
__device__ __forceinline__ void store_state(const E &e, void *p)
{
    constexpr int B = (int)sizeof(e.s);
    u32 w[B / 4];
    if constexpr (sizeof(typename E::word) == 8) {
#pragma unroll
        for (int j = 0; j < E::K; ++j) {
            w[2 * j] = (u32)e.s[j];
            w[2 * j + 1] = (u32)(e.s[j] >> 32);
        }
    } else {
#pragma unroll
        for (int j = 0; j < E::K; ++j) w[j] = e.s[j];
    }
    if constexpr (B >= 16) {
#pragma unroll
        for (int q = 0; q < B / 16; ++q)
            reinterpret_cast<uint4 *>(p)[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
    } else {
        reinterpret_cast<uint2 *>(p)[0] = make_uint2(w[0], w[1]);
    }
}

// State <-> its n / 32 little-endian u32 words held in registers.
template <typename E, int NW>
__device__ __forceinline__ void from_words(E &e, const u32 (&w)[NW])
{
    if constexpr (sizeof(typename E::word) == 8) {
#pragma unroll
        for (int j = 0; j < E::K; ++j) e.s[j] = (u64)w[2 * j] | ((u64)w[2 * j + 1] << 32);
    } else {
#pragma unroll
        for (int j = 0; j < E::K; ++j) e.s[j] = w[j];
    }
}

template <typename E, int NW>
__device__ __forceinline__ void to_words(const E &e, u32 (&w)[NW])
{
    if constexpr (sizeof(typename E::word) == 8) {
#pragma unroll
        for (int j = 0; j < E::K; ++j) {
            w[2 * j] = (u32)e.s[j];
            w[2 * j + 1] = (u32)(e.s[j] >> 32);
        }
    } else {
#pragma unroll
        for (int j = 0; j < E::K; ++j) w[j] = e.s[j];
    }
}

template <typename E>
__device__ __forceinline__ bool state_is_zero(const E &e)
{
    typename E::word acc = 0;
#pragma unroll
    for (int j = 0; j < E::K; ++j) acc |= e.s[j];
    return acc == 0;
}

// ---------------------------------------------------------------- conversions
// Output element codes (match xr_dtype).
enum { DT_U64 = 0, DT_U32 = 1, DT_F64 = 2, DT_F32 = 3 };

// (x >> 11) * 2^-53 as binary64 bits, built with integer operations only.
//
// Rare path, x < 2^32: v = x >> 11 < 2^21; with its leading one at bit p the
// value is 1.f * 2^(p - 53): biased exponent p + 970, fraction v << (52 - p)
// without the leading one; v = 0 gives +0.0.
static __device__ __noinline__ u64 unit_f64_bits_small(u64 x)
{
    const u32 v = (u32)(x >> 11);
    if (v == 0u) return 0ull;
    const int p = 31 - __clz(v);
    const u64 frac = ((u64)v << (52 - p)) & ((1ull << 52) - 1);
    return ((u64)(p + 970) << 52) | frac;
}

// Common path, high word hi != 0 with lz = clz(hi) <= 31: v = x >> 11 has its
// leading one at bit 52 - lz, so v << lz puts it at bit 52 (bit 20 of the high
// word) and its low 52 bits are the fraction.  The value is 1.f * 2^(-1 - lz):
// biased exponent 1022 - lz, and since the leading one already adds one to the
// exponent field, adding (1021 - lz) << 20 to the high word completes the
// encoding.  Seven integer operations; the rare x < 2^32 branches out of line.
__device__ __forceinline__ u64 unit_f64_bits(u64 x)
{
    u32 lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(x));
    if (__builtin_expect(hi == 0u, 0)) return unit_f64_bits_small(x);
    const u32 vl = __funnelshift_r(lo, hi, 11);
    const u32 vh = hi >> 11;
    const int lz = __clz(hi);
    const u32 mh = __funnelshift_l(vl, vh, lz) + ((u32)(1021 - lz) << 20);
    const u32 ml = vl << lz;
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(ml), "r"(mh));
    return r;
}

// x * 2^-32 as binary64 bits for a 32-bit word: leading one at bit p = 31 - lz,
// value 1.f * 2^(p - 32), biased exponent p + 991:
// bits = (x << (21 + lz)) + ((1021 - lz) << 52).
__device__ __forceinline__ u64 unit_f64_bits(u32 x)
{
    const int lz = __clz(x);
    const u64 bits = ((u64)x << ((21 + lz) & 63)) + ((u64)(1021 - lz) << 52);
    return x ? bits : 0ull;
}

// Upper 24 bits times 2^-24 as binary32 bits (exact: a 24-bit integer converts
// exactly and the scaling is a power of two).
__device__ __forceinline__ u32 unit_f32_bits(u64 x) { return __float_as_uint(__uint2float_rn((u32)(x >> 40)) * 0x1p-24f); }
__device__ __forceinline__ u32 unit_f32_bits(u32 x) { return __float_as_uint(__uint2float_rn(x >> 8) * 0x1p-24f); }

template <int DT> struct OutElem { typedef u64 type; };
template <> struct OutElem<DT_U32> { typedef u32 type; };
template <> struct OutElem<DT_F32> { typedef u32 type; };

template <int DT, typename W>
__device__ __forceinline__ typename OutElem<DT>::type convert(W x)
{
    if (DT == DT_U64 || DT == DT_U32) return (typename OutElem<DT>::type)x;
    if (DT == DT_F64) return (typename OutElem<DT>::type)unit_f64_bits(x);
    return (typename OutElem<DT>::type)unit_f32_bits(x);
}

// ---------------------------------------------------------------- output words
// Next 16 bytes of output elements (2 x 8 B or 4 x 4 B), stepping the engine.
template <typename G, int DT>
__device__ __forceinline__ void gen16(typename G::E &e, u32 (&w)[4])
{
    typedef typename OutElem<DT>::type OT;
    if (sizeof(OT) == 8) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const u64 o = (u64)convert<DT>(G::out(e));
            e.step();
            w[2 * q] = (u32)o;
            w[2 * q + 1] = (u32)(o >> 32);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            w[q] = (u32)convert<DT>(G::out(e));
            e.step();
        }
    }
}

// Same for the last, partial tile: only `cnt` more outputs are taken.
template <typename G, int DT>
__device__ __forceinline__ void gen16_partial(typename G::E &e, u32 (&w)[4], int cnt)
{
    typedef typename OutElem<DT>::type OT;
    constexpr int PER = 16 / (int)sizeof(OT);
    w[0] = w[1] = w[2] = w[3] = 0u;
    for (int q = 0; q < PER && q < cnt; ++q) {
        const u64 o = (u64)convert<DT>(G::out(e));
        e.step();
        if (sizeof(OT) == 8) {
            w[2 * q] = (u32)o;
            w[2 * q + 1] = (u32)(o >> 32);
        } else {
            w[q] = (u32)o;
        }
    }
}

// ---------------------------------------------------------------- seeding
// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014; Sec. 5.3): Weyl sequence with
// increment 0x9e3779b97f4a7c15, then the 64-bit mixer (shifts 30, 27, 31;
// multipliers 0xbf58476d1ce4e5b9, 0x94d049bb133111eb).
__device__ __forceinline__ u64 splitmix64_next(u64 &x)
{
    x += 0x9e3779b97f4a7c15ull;
    u64 z = x;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ u32 smem_addr(const void *p)
{
    return (u32)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void st_shared_v4(u32 addr, u32 a, u32 b, u32 c, u32 d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
                 "r"(d)
                 : "memory");
}

// Order this thread's generic-proxy shared-memory writes before later
// async-proxy (TMA) reads of the same memory.
__device__ __forceinline__ void fence_proxy_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 2D tile store shared -> global through the tensor map (cp.async.bulk.tensor).
// Elements outside the tensor's extent are not written.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, u32 src, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(src), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Wait until at most N committed bulk groups still read shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

// Wait until at most N committed bulk groups are still in flight (writes done).
template <int N>
__device__ __forceinline__ void bulk_wait_all()
{
    asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace xr
