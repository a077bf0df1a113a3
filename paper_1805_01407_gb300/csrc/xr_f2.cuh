// xr_f2.cuh -- F2 linear algebra on the device: matrix-vector products with
// the jump matrices T^(2^k) and the power sets built from them (Sec. 5, 6):
// per-thread masked products, Four-Russians tables shared by a CTA, and
// warp-cooperative products for a single state.
#pragma once

#include "xr_device.cuh"
#include "xr_internal.h"

namespace xr {

// ---------------------------------------------------------------- vectors
// A state as NW u32 words, moved with 16-byte (8-byte for NW = 2) accesses.

template <int NW>
__device__ __forceinline__ void load_vec(u32 (&v)[NW], const u32 *p)
{
    if constexpr (NW >= 4) {
#pragma unroll
        for (int q = 0; q < NW / 4; ++q) {
            const uint4 a = reinterpret_cast<const uint4 *>(p)[q];
            v[4 * q] = a.x; v[4 * q + 1] = a.y; v[4 * q + 2] = a.z; v[4 * q + 3] = a.w;
        }
    } else {
        const uint2 a = reinterpret_cast<const uint2 *>(p)[0];
        v[0] = a.x; v[1] = a.y;
    }
}

template <int NW>
__device__ __forceinline__ void store_vec(const u32 (&v)[NW], u32 *p)
{
    if constexpr (NW >= 4) {
#pragma unroll
        for (int q = 0; q < NW / 4; ++q)
            reinterpret_cast<uint4 *>(p)[q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
        reinterpret_cast<uint2 *>(p)[0] = make_uint2(v[0], v[1]);
    }
}

// ---------------------------------------------------------------- F2 algebra
// A state is a column vector of n bits; bit c is bit c % 32 of u32 word c / 32
// of the state in memory.  A matrix is stored by columns: column c (the image
// of the unit state e_c) is NW = n / 32 consecutive u32 words.
//
// r = M v as the XOR of the columns selected by the set bits of v.  Every
// thread of a warp walks the columns in the same order, so the column loads are
// warp-uniform (one broadcast per load) whatever the vectors are.
template <int NW, bool SHARED>
__device__ __forceinline__ void f2_matvec(const u32 *__restrict__ M, const u32 (&v)[NW],
                                          u32 (&r)[NW])
{
    u32 acc[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) acc[w] = 0u;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const u32 bits = v[w];
#pragma unroll 8
        for (int b = 0; b < 32; ++b) {
            const u32 mask = (u32)((int)(bits << (31 - b)) >> 31);
            const uint4 *col = reinterpret_cast<const uint4 *>(M + (size_t)(w * 32 + b) * NW);
            if constexpr (NW >= 4) {
#pragma unroll
                for (int q = 0; q < NW / 4; ++q) {
                    uint4 c;
                    if (SHARED) c = col[q];
                    else c = __ldg(col + q);
                    acc[4 * q + 0] ^= c.x & mask;
                    acc[4 * q + 1] ^= c.y & mask;
                    acc[4 * q + 2] ^= c.z & mask;
                    acc[4 * q + 3] ^= c.w & mask;
                }
            } else {
                const uint2 *col2 = reinterpret_cast<const uint2 *>(col);
                uint2 c;
                if (SHARED) c = col2[0];
                else c = __ldg(col2);
                acc[0] ^= c.x & mask;
                acc[1] ^= c.y & mask;
            }
        }
    }
#pragma unroll
    for (int w = 0; w < NW; ++w) r[w] = acc[w];
}

// Four-Russians tables of one F2 matrix (n columns of NW words): for each
// group of four consecutive columns 4g .. 4g+3, the XOR of every subset (16
// entries), so a matrix-vector product is n/4 table reads instead of n
// masked XORs.  An entry is split into 16-byte pieces (8-byte for NW = 2).
// Piece h of entry e of group g sits at slot (e H + h) G + g, so the bank of
// a read depends on the group alone; lane l visits the groups in the order
// l, l+1, ... (mod G), which puts the 8 lanes of a quarter-warp (16 of a
// half-warp for 8-byte pieces) on distinct banks whatever their entries.
template <int NW>
struct Russians {
    static constexpr int n = NW * 32;
    static constexpr int G = n / 4;             // groups of four columns
    static constexpr int Q = NW >= 4 ? 4 : NW;  // words per piece
    static constexpr int H = NW / Q;            // pieces per entry
    static constexpr int WORDS = 16 * G * NW;
};

// Thread task (h, g, q) builds word q of piece h for the 16 entries of group
// g, each from a smaller entry and one column: T[e] = T[e - b] ^ col(4g + k)
// for b = 2^k the top bit of e.  The matrix is read once.
template <int NW>
__device__ __forceinline__ void russians_build(const u32 *__restrict__ M, u32 *T)
{
    typedef Russians<NW> RT;
    for (int i = threadIdx.x; i < RT::G * NW; i += blockDim.x) {
        const int q = i % RT::Q, g = (i / RT::Q) % RT::G, h = i / (RT::Q * RT::G);
        const int word = h * RT::Q + q;
        u32 c[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] = __ldg(M + (size_t)(4 * g + k) * NW + word);
        u32 x[16];
        x[0] = 0u;
#pragma unroll
        for (int e = 1; e < 16; ++e) {
            const int k = e >= 8 ? 3 : (e >= 4 ? 2 : (e >= 2 ? 1 : 0));
            x[e] = x[e - (1 << k)] ^ c[k];
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) T[((e * RT::H + h) * RT::G + g) * RT::Q + q] = x[e];
    }
}

// r = M v from the tables.  The vector is first rotated right by 4 lane bits
// (mod n), so step s reads the fixed bits 4s .. 4s+3 of the rotated vector,
// which are group (s + lane) mod G of v.
template <int NW>
__device__ __forceinline__ void russians_matvec(const u32 *T, const u32 (&v)[NW], u32 (&r)[NW])
{
    typedef Russians<NW> RT;
    const int lane = (int)(threadIdx.x & 31u);
    const int rot = (4 * lane) & (RT::n - 1);  // bits; below 128
    u32 u[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) u[w] = v[w];
    // whole words first (1 and 2 words), then the bits within a word
#pragma unroll
    for (int st = 1; st <= 2; st <<= 1) {
        if (st < NW && ((rot >> 5) & st)) {
            u32 t[NW];
#pragma unroll
            for (int w = 0; w < NW; ++w) t[w] = u[(w + st) % NW];
#pragma unroll
            for (int w = 0; w < NW; ++w) u[w] = t[w];
        }
    }
    const int bs = rot & 31;
    {
        u32 t[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) t[w] = __funnelshift_r(u[w], u[(w + 1) % NW], bs);
#pragma unroll
        for (int w = 0; w < NW; ++w) u[w] = t[w];
    }
#pragma unroll
    for (int w = 0; w < NW; ++w) r[w] = 0u;
#pragma unroll
    for (int s = 0; s < RT::G; ++s) {
        const u32 e = (u[(4 * s) >> 5] >> ((4 * s) & 31)) & 15u;
        const u32 g = (u32)(s + lane) & (u32)(RT::G - 1);
#pragma unroll
        for (int h = 0; h < RT::H; ++h) {
            const u32 slot = (e * RT::H + (u32)h) * RT::G + g;
            if constexpr (RT::Q == 4) {
                const uint4 t = reinterpret_cast<const uint4 *>(T)[slot];
                r[4 * h] ^= t.x; r[4 * h + 1] ^= t.y; r[4 * h + 2] ^= t.z; r[4 * h + 3] ^= t.w;
            } else {
                const uint2 t = reinterpret_cast<const uint2 *>(T)[slot];
                r[0] ^= t.x; r[1] ^= t.y;
            }
        }
    }
}

// r = M v by one warp for a warp-uniform v: lane l owns columns k*32 + l, so
// the column loads of the warp are contiguous, and the partial sums are
// XOR-reduced across the lanes.
template <int NW>
__device__ __forceinline__ void warp_matvec(const u32 *__restrict__ M, u32 (&v)[NW], int lane)
{
    u32 acc[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) acc[w] = 0u;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        const u32 mask = 0u - ((v[k] >> lane) & 1u);
        const u32 *colp = M + (size_t)(k * 32 + lane) * NW;
        if constexpr (NW >= 4) {
            const uint4 *col = reinterpret_cast<const uint4 *>(colp);
#pragma unroll
            for (int q = 0; q < NW / 4; ++q) {
                const uint4 c = __ldg(col + q);
                acc[4 * q] ^= c.x & mask;
                acc[4 * q + 1] ^= c.y & mask;
                acc[4 * q + 2] ^= c.z & mask;
                acc[4 * q + 3] ^= c.w & mask;
            }
        } else {
            const uint2 c = __ldg(reinterpret_cast<const uint2 *>(colp));
            acc[0] ^= c.x & mask;
            acc[1] ^= c.y & mask;
        }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1)
#pragma unroll
        for (int w = 0; w < NW; ++w) acc[w] ^= __shfl_xor_sync(0xffffffffu, acc[w], off);
#pragma unroll
    for (int w = 0; w < NW; ++w) v[w] = acc[w];
}

// v <- (T^(2^d))^e v by one warp, with psets_d the three power sets of the
// distance 2^d (P_l[j] = T^(2^d j 512^l)): the low 27 bits of e take three
// products at most, higher bits one T^(2^(d + k)) each (exponents mod n).
template <int NW>
__device__ void warp_advance(const u32 *psets_d, const u32 *tables, int d, u32 (&v)[NW], u64 e, int lane)
{
    constexpr int n = NW * 32;
    const size_t set_words = (size_t)PSET_SIZE * n * NW;
    for (int l = 0; l < PSET_LEVELS; ++l) {
        const u32 j = (u32)(e >> (PSET_BITS * l)) & (PSET_SIZE - 1);
        if (j) warp_matvec<NW>(psets_d + l * set_words + (size_t)j * n * NW, v, lane);
    }
    u64 hi = e >> (PSET_BITS * PSET_LEVELS);
    while (hi) {
        const int k = __ffsll((long long)hi) - 1;
        hi &= hi - 1;
        warp_matvec<NW>(tables + (size_t)((d + PSET_BITS * PSET_LEVELS + k) % n) * n * NW, v, lane);
    }
}

}  // namespace xr
