/*
 * Plain CPU oracle for the scrambled linear generators of Blackman & Vigna,
 * "Scrambled Linear Pseudorandom Number Generators" (ACM TOMS, arXiv 1805.01407).
 *
 * TEST INFRASTRUCTURE ONLY.  The library never links, loads or calls this file.
 * Only the tests, the smoke check of the build entry and the benchmark's CPU
 * legs (the baseline beside the device numbers and the reference arm) may
 * load it.  It shares no code, header, table or constant with
 * the CUDA path: every parameter below is typed here from the paper's tables.
 *
 * Everything is the plain definition, computed one value at a time:
 *   - engines: the block matrices X_kw (Sec. 3.1, Eq. (M)), S_4w and S_8w
 *     (Sec. 3.2), written word by word as "new word j = XOR over rows i of
 *     s_i times block (i, j)";
 *   - scramblers: Sec. 4 (+ Sec. 4.1, * Sec. 4.2, ++ Sec. 4.3, ** Sec. 4.4),
 *     applied to the current state before the update (Sec. 2);
 *   - parameters: Table 4 (64-bit engines), Table 5 (64-bit scramblers),
 *     Table 7 (32-bit engines), Table 8 (32-bit scramblers); word choices from
 *     the code figures of Sec. 3 and the remark in Sec. 5.2 that the 32-bit
 *     xoshiro128 uses the words of xoshiro256;
 *   - seeding with SplitMix64 (Sec. 5.3; the paper cites Steele, Lea and
 *     Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014,
 *     and prints no definition: the Weyl increment is the odd integer nearest
 *     2^64 / phi and the finalizer Stafford's variant 13, both pinned by the
 *     tests against values derived or implemented independently of this file);
 *   - doubles from the upper 53 bits (Sec. 5.3, "(x >> 11) * 2^-53");
 *   - F2 matrices T (transition as a map on column vectors of state bits), the
 *     characteristic polynomial (Sec. 6), Berlekamp-Massey (Sec. 6, Sec. 9.3),
 *     polynomial arithmetic over F2 and jumps as T^J s = sum_i c_i T^i s with
 *     x^J mod p(x) = sum_i c_i x^i (Sec. 6, Cayley-Hamilton);
 *   - the escaping-zeroland counts of Sec. 8 (one bits in windows of outputs
 *     from every state with one bit set).
 *
 * Bit convention.  A state of k words of w bits is the column vector whose bit
 * index is word * w + b, where b is the machine bit (b = 0 is the least
 * significant).  The paper writes row vectors with position 0 leftmost, so its
 * position p in a word is machine bit w - 1 - p; with that reading its S (ones
 * on the principal subdiagonal) is "x << 1" and R is "rotate left by 1".
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t u64;

/* ------------------------------------------------------------------------ */
/* Generator descriptions                                                   */
/* ------------------------------------------------------------------------ */

enum { ENG_XOROSHIRO = 1, ENG_XOSHIRO4 = 2, ENG_XOSHIRO8 = 3, ENG_XORSHIFT = 4 };
enum { SCR_NONE = 0, SCR_PLUS = 1, SCR_PLUSPLUS = 2, SCR_STAR = 3, SCR_STARSTAR = 4 };

typedef struct {
    const char *name;
    int eng;          /* engine family */
    int w, k;         /* word size, number of words */
    int a, b, c;      /* engine parameters (letters as in Tables 4 and 7) */
    int scr;          /* scrambler */
    int p, q;         /* + : s_p + s_q ; ++ : rotl(s_p + s_q, r) + s_p ; * and ** read s_p */
    u64 mul1;         /* * multiplier, or first ** multiplier (Tables 5 and 8, column S) */
    int rot;          /* ++ or ** rotation (column R) */
    u64 mul2;         /* second ** multiplier (column T) */
} gen_t;

#define PHI64 0x9e3779b97f4a7c13ull /* Table 5, row "*" */
#define PHI32 0x9E3779BBull         /* Table 8, rows xoroshiro64* and xoroshiro64** */

static const gen_t GENS[] = {
    /* xoshiro256: Table 4 (A=17 shift, B=45 rotate); Fig. 3 word choices; Table 5 */
    {"xoshiro256+",    ENG_XOSHIRO4, 64, 4, 17, 45, 0, SCR_PLUS,     0, 3, 0, 0, 0},
    {"xoshiro256++",   ENG_XOSHIRO4, 64, 4, 17, 45, 0, SCR_PLUSPLUS, 0, 3, 0, 23, 0},
    {"xoshiro256**",   ENG_XOSHIRO4, 64, 4, 17, 45, 0, SCR_STARSTAR, 1, 1, 5, 7, 9},
    /* xoroshiro128: Table 4 rows xoroshiro128 (24,16,37) and xoroshiro128++ (49,21,28);
       Fig. 1 word choices; Table 5 */
    {"xoroshiro128+",  ENG_XOROSHIRO, 64, 2, 24, 16, 37, SCR_PLUS,     0, 1, 0, 0, 0},
    {"xoroshiro128++", ENG_XOROSHIRO, 64, 2, 49, 21, 28, SCR_PLUSPLUS, 0, 1, 0, 17, 0},
    {"xoroshiro128**", ENG_XOROSHIRO, 64, 2, 24, 16, 37, SCR_STARSTAR, 0, 0, 5, 7, 9},
    /* xoshiro128 (32-bit): Table 7 (A=9, B=11); words of xoshiro256 (Sec. 5.2); Table 8 */
    {"xoshiro128++",   ENG_XOSHIRO4, 32, 4, 9, 11, 0, SCR_PLUSPLUS, 0, 3, 0, 7, 0},
    {"xoshiro128**",   ENG_XOSHIRO4, 32, 4, 9, 11, 0, SCR_STARSTAR, 1, 1, 5, 7, 9},
    {"xoshiro128+",    ENG_XOSHIRO4, 32, 4, 9, 11, 0, SCR_PLUS,     0, 3, 0, 0, 0},
    /* further generators of Sec. 5 (Tables 4, 5, 7, 8; Figs. 1, 2, 4) */
    {"xoroshiro128*",  ENG_XOROSHIRO, 64, 2, 24, 16, 37, SCR_STAR, 0, 0, PHI64, 0, 0},
    {"xoshiro512+",    ENG_XOSHIRO8, 64, 8, 11, 21, 0, SCR_PLUS,     0, 2, 0, 0, 0},
    {"xoshiro512++",   ENG_XOSHIRO8, 64, 8, 11, 21, 0, SCR_PLUSPLUS, 2, 0, 0, 17, 0},
    {"xoshiro512**",   ENG_XOSHIRO8, 64, 8, 11, 21, 0, SCR_STARSTAR, 1, 1, 5, 7, 9},
    {"xoroshiro1024*", ENG_XOROSHIRO, 64, 16, 25, 27, 36, SCR_STAR,     0, 0, PHI64, 0, 0},
    {"xoroshiro1024++",ENG_XOROSHIRO, 64, 16, 25, 27, 36, SCR_PLUSPLUS, 15, 0, 0, 23, 0},
    {"xoroshiro1024**",ENG_XOROSHIRO, 64, 16, 25, 27, 36, SCR_STARSTAR, 0, 0, 5, 7, 9},
    {"xoroshiro64*",   ENG_XOROSHIRO, 32, 2, 26, 9, 13, SCR_STAR,     0, 0, PHI32, 0, 0},
    {"xoroshiro64**",  ENG_XOROSHIRO, 32, 2, 26, 9, 13, SCR_STARSTAR, 0, 0, PHI32, 5, 5},
    /* tiny engines named in Sec. 7 (equidistribution counterexamples) and the
       xorshift example of Sec. 9; their scramblers use the same word choices */
    {"xoroshiro10+",   ENG_XOROSHIRO, 5, 2, 1, 3, 1, SCR_PLUS, 0, 1, 0, 0, 0},
    {"xoroshiro16x4+", ENG_XOROSHIRO, 4, 4, 3, 1, 2, SCR_PLUS, 0, 3, 0, 0, 0},
    {"xoshiro8+",      ENG_XOSHIRO4, 2, 4, 1, 1, 0, SCR_PLUS, 0, 3, 0, 0, 0},
    {"xoshiro40+",     ENG_XOSHIRO8, 5, 8, 2, 3, 0, SCR_PLUS, 0, 2, 0, 0, 0},
    {"xorshift6+",     ENG_XORSHIFT, 3, 2, 1, 2, 1, SCR_PLUS, 0, 1, 0, 0, 0},
    {"xoshiro8++",     ENG_XOSHIRO4, 2, 4, 1, 1, 0, SCR_PLUSPLUS, 0, 3, 0, 1, 0},
    /* linear engines with the + scrambler on the first and last word: bit 0 of
       the output is a linear function of the state, so Berlekamp-Massey on it
       returns the engine's characteristic polynomial (Sec. 4.1, Sec. 6) */
    {"engine/xoshiro256",     ENG_XOSHIRO4, 64, 4, 17, 45, 0, SCR_PLUS, 0, 3, 0, 0, 0},
    {"engine/xoroshiro128",   ENG_XOROSHIRO, 64, 2, 24, 16, 37, SCR_PLUS, 0, 1, 0, 0, 0},
    {"engine/xoroshiro128pp", ENG_XOROSHIRO, 64, 2, 49, 21, 28, SCR_PLUS, 0, 1, 0, 0, 0},
    {"engine/xoshiro128",     ENG_XOSHIRO4, 32, 4, 9, 11, 0, SCR_PLUS, 0, 3, 0, 0, 0},
    {"engine/xoshiro512",     ENG_XOSHIRO8, 64, 8, 11, 21, 0, SCR_PLUS, 0, 7, 0, 0, 0},
    {"engine/xoroshiro1024",  ENG_XOROSHIRO, 64, 16, 25, 27, 36, SCR_PLUS, 0, 15, 0, 0, 0},
    {"engine/xoroshiro64",    ENG_XOROSHIRO, 32, 2, 26, 9, 13, SCR_PLUS, 0, 1, 0, 0, 0},
};
#define NGENS ((int)(sizeof(GENS) / sizeof(GENS[0])))

static const gen_t *gen(int gi) { return (gi >= 0 && gi < NGENS) ? &GENS[gi] : NULL; }

int orc_num_generators(void) { return NGENS; }
const char *orc_generator_name(int gi) { return gen(gi) ? gen(gi)->name : NULL; }
int orc_word_bits(int gi) { return gen(gi) ? gen(gi)->w : -1; }
int orc_state_words(int gi) { return gen(gi) ? gen(gi)->k : -1; }
int orc_state_bits(int gi) { return gen(gi) ? gen(gi)->k * gen(gi)->w : -1; }

/* ------------------------------------------------------------------------ */
/* w-bit word operations (Sec. 3: S = shift left by one, R = rotate left)   */
/* ------------------------------------------------------------------------ */

static u64 wmask(int w) { return w >= 64 ? ~0ull : ((1ull << w) - 1); }
static u64 shl_w(u64 x, int a, int w) { return a >= w ? 0 : (x << a) & wmask(w); }
static u64 shr_w(u64 x, int a, int w) { return a >= w ? 0 : (x & wmask(w)) >> a; }
static u64 rotl_w(u64 x, int r, int w)
{
    x &= wmask(w);
    r %= w;
    if (r == 0) return x;
    return ((x << r) | (x >> (w - r))) & wmask(w);
}

/* ------------------------------------------------------------------------ */
/* One engine step: new state = s * M for the paper's matrix M              */
/* ------------------------------------------------------------------------ */

static void engine_step(const gen_t *g, u64 *s)
{
    const int w = g->w, k = g->k;
    u64 n[16];
    switch (g->eng) {
    case ENG_XOROSHIRO: {
        /* X_kw (Eq. (M)): out[j] = s[j+1] for j <= k-3;
           out[k-2] = s0 (R^a + S^b + I) + s_{k-1} (S^b + I);
           out[k-1] = (s0 + s_{k-1}) R^c.  For k = 2 this is X_2w. */
        const u64 t = s[0] ^ s[k - 1];
        for (int j = 0; j + 1 <= k - 2; j++) n[j] = s[j + 1];
        n[k - 2] = rotl_w(s[0], g->a, w) ^ t ^ shl_w(t, g->b, w);
        n[k - 1] = rotl_w(t, g->c, w);
        break;
    }
    case ENG_XOSHIRO4:
        /* S_4w, block rows (I I I 0), (I I S^a R^b), (0 I I 0), (I 0 0 R^b) */
        n[0] = s[0] ^ s[1] ^ s[3];
        n[1] = s[0] ^ s[1] ^ s[2];
        n[2] = s[0] ^ shl_w(s[1], g->a, w) ^ s[2];
        n[3] = rotl_w(s[1] ^ s[3], g->b, w);
        break;
    case ENG_XOSHIRO8:
        /* S_8w, read column by column */
        n[0] = s[0] ^ s[6];
        n[1] = s[0] ^ s[1] ^ s[2];
        n[2] = s[0] ^ s[2];
        n[3] = s[3] ^ s[4];
        n[4] = s[1] ^ s[4] ^ s[5];
        n[5] = s[1] ^ s[5];
        n[6] = shl_w(s[1], g->a, w) ^ s[3] ^ s[6] ^ s[7];
        n[7] = rotl_w(s[3] ^ s[7], g->b, w);
        break;
    case ENG_XORSHIFT: {
        /* the xorshift example of Sec. 9 (a left shift, b and c right shifts):
           the old second word becomes the first; the new second word is
           t ^ u ^ (t >> b) ^ (u >> c) with t = s0 ^ (s0 << a), u = s1 */
        const u64 t = s[0] ^ shl_w(s[0], g->a, w);
        const u64 u = s[1];
        n[0] = u;
        n[1] = t ^ u ^ shr_w(t, g->b, w) ^ shr_w(u, g->c, w);
        break;
    }
    default:
        return;
    }
    for (int j = 0; j < k; j++) s[j] = n[j] & wmask(w);
}

/* ------------------------------------------------------------------------ */
/* Scramblers (Sec. 4), applied to the current state                        */
/* ------------------------------------------------------------------------ */

static u64 scramble(const gen_t *g, const u64 *s)
{
    const int w = g->w;
    const u64 m = wmask(w);
    switch (g->scr) {
    case SCR_PLUS:     /* Sec. 4.1: sum of two words mod 2^w */
        return (s[g->p] + s[g->q]) & m;
    case SCR_PLUSPLUS: /* Sec. 4.3: sum, rotate left by r, add the first word */
        return (rotl_w((s[g->p] + s[g->q]) & m, g->rot, w) + s[g->p]) & m;
    case SCR_STAR:     /* Sec. 4.2: product by an odd constant */
        return (s[g->p] * g->mul1) & m;
    case SCR_STARSTAR: /* Sec. 4.4: multiply, rotate, multiply */
        return (rotl_w((s[g->p] * g->mul1) & m, g->rot, w) * g->mul2) & m;
    default:           /* raw linear engine: first word */
        return s[0] & m;
    }
}

/* next(): output from the current state, then one engine step (Sec. 2). */
static u64 next_output(const gen_t *g, u64 *s)
{
    const u64 r = scramble(g, s);
    engine_step(g, s);
    return r;
}

int orc_generate(int gi, u64 *state, size_t n, u64 *out)
{
    const gen_t *g = gen(gi);
    if (!g) return -1;
    for (size_t i = 0; i < n; i++) out[i] = next_output(g, state);
    return 0;
}

int orc_step(int gi, u64 *state, u64 nsteps)
{
    const gen_t *g = gen(gi);
    if (!g) return -1;
    for (u64 i = 0; i < nsteps; i++) engine_step(g, state);
    return 0;
}

int orc_scramble(int gi, const u64 *state, u64 *out)
{
    const gen_t *g = gen(gi);
    if (!g) return -1;
    *out = scramble(g, state);
    return 0;
}

/* Stream-major fill from explicit start states: out[i*m + j] = output j of
   stream i.  The start states are left untouched. */
int orc_fill_streams(int gi, const u64 *starts, size_t S, size_t m, u64 *out)
{
    const gen_t *g = gen(gi);
    if (!g) return -1;
    u64 s[16];
    for (size_t i = 0; i < S; i++) {
        memcpy(s, starts + i * (size_t)g->k, sizeof(u64) * (size_t)g->k);
        for (size_t j = 0; j < m; j++) out[i * m + j] = next_output(g, s);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Seeding (Sec. 5.3) with SplitMix64                                       */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): a Weyl sequence with the odd
   increment 0x9e3779b97f4a7c15 followed by the 64-bit mixer with shifts 30, 27,
   31 and multipliers 0xbf58476d1ce4e5b9, 0x94d049bb133111eb. */
static u64 splitmix64_next(u64 *x)
{
    *x += 0x9e3779b97f4a7c15ull;
    u64 z = *x;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

int orc_splitmix64(u64 seed, size_t n, u64 *out)
{
    u64 x = seed;
    for (size_t i = 0; i < n; i++) out[i] = splitmix64_next(&x);
    return 0;
}

/* Fill a state from a 64-bit seed.  64-bit words: consecutive SplitMix64
   outputs.  32-bit words: each SplitMix64 output gives two words, low half
   first.  Returns 1 when the result is the all-zero state (which the paper
   notes cannot happen for SplitMix64's equidistributed output), else 0. */
int orc_seed(int gi, u64 seed, u64 *state)
{
    const gen_t *g = gen(gi);
    if (!g) return -1;
    u64 x = seed;
    if (g->w == 64) {
        for (int j = 0; j < g->k; j++) state[j] = splitmix64_next(&x);
    } else if (g->w == 32) {
        for (int j = 0; j < g->k; j += 2) {
            const u64 z = splitmix64_next(&x);
            state[j] = z & 0xffffffffull;
            if (j + 1 < g->k) state[j + 1] = z >> 32;
        }
    } else {
        for (int j = 0; j < g->k; j++) state[j] = splitmix64_next(&x) & wmask(g->w);
    }
    u64 any = 0;
    for (int j = 0; j < g->k; j++) any |= state[j];
    return any ? 0 : 1;
}

/* ------------------------------------------------------------------------ */
/* Conversions (Sec. 5.3)                                                    */
/* ------------------------------------------------------------------------ */

/* double in [0,1): upper 53 bits times 2^-53 for 64-bit words; a 32-bit word
   times 2^-32 for 32-bit generators.  Both are exact in binary64. */
int orc_to_f64(int w, const u64 *x, size_t n, double *out)
{
    for (size_t i = 0; i < n; i++) {
        if (w == 64)
            out[i] = (double)(x[i] >> 11) * 0x1p-53;
        else
            out[i] = (double)(x[i] & 0xffffffffull) * 0x1p-32;
    }
    return 0;
}

/* float in [0,1): upper 24 bits times 2^-24 (exact in binary32). */
int orc_to_f32(int w, const u64 *x, size_t n, float *out)
{
    for (size_t i = 0; i < n; i++) {
        const u64 top24 = (w == 64) ? (x[i] >> 40) : ((x[i] & 0xffffffffull) >> 8);
        out[i] = (float)top24 * 0x1p-24f;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* F2 bit matrices: n x n, row-major, nw = ceil(n/64) words per row;         */
/* entry (r, c) is bit (c % 64) of word c / 64 of row r.                     */
/* ------------------------------------------------------------------------ */

static int words_for(int n) { return (n + 63) / 64; }
static int getbit(const u64 *v, int i) { return (int)((v[i >> 6] >> (i & 63)) & 1u); }
static void setbit(u64 *v, int i) { v[i >> 6] |= 1ull << (i & 63); }
static void flipbit(u64 *v, int i) { v[i >> 6] ^= 1ull << (i & 63); }

int orc_state_to_bits(int gi, const u64 *state, u64 *bits)
{
    const gen_t *g = gen(gi);
    if (!g) return -1;
    const int n = g->k * g->w;
    memset(bits, 0, sizeof(u64) * (size_t)words_for(n));
    for (int j = 0; j < g->k; j++)
        for (int b = 0; b < g->w; b++)
            if ((state[j] >> b) & 1u) setbit(bits, j * g->w + b);
    return 0;
}

int orc_bits_to_state(int gi, const u64 *bits, u64 *state)
{
    const gen_t *g = gen(gi);
    if (!g) return -1;
    for (int j = 0; j < g->k; j++) {
        state[j] = 0;
        for (int b = 0; b < g->w; b++)
            if (getbit(bits, j * g->w + b)) state[j] |= 1ull << b;
    }
    return 0;
}

/* T from the step: column c is the state reached from the unit state e_c. */
int orc_matrix_from_step(int gi, u64 *T)
{
    const gen_t *g = gen(gi);
    if (!g) return -1;
    const int n = g->k * g->w, nw = words_for(n);
    memset(T, 0, sizeof(u64) * (size_t)n * (size_t)nw);
    u64 e[16 * 64 / 64 + 1];
    u64 s[16];
    for (int c = 0; c < n; c++) {
        memset(e, 0, sizeof(e));
        setbit(e, c);
        orc_bits_to_state(gi, e, s);
        engine_step(g, s);
        orc_state_to_bits(gi, s, e);
        for (int r = 0; r < n; r++)
            if (getbit(e, r)) setbit(T + (size_t)r * nw, c);
    }
    return 0;
}

/* w x w blocks in the paper's indexing (position 0 leftmost).  kind: 0 = zero,
   bit 1 = I, bit 2 = S^e1, bit 4 = R^e2 (a sum of those terms). */
typedef struct { int terms; int sp; int rp; } block_t;

static void wmat_identity(int w, unsigned char *A)
{
    memset(A, 0, (size_t)w * w);
    for (int i = 0; i < w; i++) A[i * w + i] = 1;
}

static void wmat_mul(int w, const unsigned char *A, const unsigned char *B, unsigned char *C)
{
    unsigned char tmp[64 * 64];
    for (int i = 0; i < w; i++)
        for (int j = 0; j < w; j++) {
            int x = 0;
            for (int t = 0; t < w; t++) x ^= A[i * w + t] & B[t * w + j];
            tmp[i * w + j] = (unsigned char)x;
        }
    memcpy(C, tmp, (size_t)w * w);
}

/* S: ones on the principal subdiagonal; R: S plus a one in the upper right corner. */
static void wmat_power(int w, int which_R, int e, unsigned char *out)
{
    unsigned char base[64 * 64];
    memset(base, 0, (size_t)w * w);
    for (int i = 1; i < w; i++) base[i * w + (i - 1)] = 1;
    if (which_R) base[0 * w + (w - 1)] = 1;
    wmat_identity(w, out);
    for (int t = 0; t < e; t++) wmat_mul(w, out, base, out);
}

static block_t engine_block(const gen_t *g, int bi, int bj)
{
    block_t z = {0, 0, 0};
    const int k = g->k;
    switch (g->eng) {
    case ENG_XOROSHIRO:
        if (bi == 0 && bj == k - 2) { z.terms = 1 | 2 | 4; z.sp = g->b; z.rp = g->a; }
        else if (bi == 0 && bj == k - 1) { z.terms = 4; z.rp = g->c; }
        else if (bi == k - 1 && bj == k - 2) { z.terms = 1 | 2; z.sp = g->b; }
        else if (bi == k - 1 && bj == k - 1) { z.terms = 4; z.rp = g->c; }
        else if (bi >= 1 && bi <= k - 2 && bj == bi - 1) { z.terms = 1; }
        break;
    case ENG_XOSHIRO4: {
        /* S_4w as printed in Sec. 3.2; 'I' identity, 'S' = S^a, 'R' = R^b */
        static const char *rows[4] = {"III0", "IISR", "0II0", "I00R"};
        const char ch = rows[bi][bj];
        if (ch == 'I') z.terms = 1;
        else if (ch == 'S') { z.terms = 2; z.sp = g->a; }
        else if (ch == 'R') { z.terms = 4; z.rp = g->b; }
        break;
    }
    case ENG_XOSHIRO8: {
        static const char *rows[8] = {"III00000", "0I00IIS0", "0II00000", "000I00IR",
                                      "000II000", "0000II00", "I00000I0", "000000IR"};
        const char ch = rows[bi][bj];
        if (ch == 'I') z.terms = 1;
        else if (ch == 'S') { z.terms = 2; z.sp = g->a; }
        else if (ch == 'R') { z.terms = 4; z.rp = g->b; }
        break;
    }
    default:
        z.terms = -1;
    }
    return z;
}

/* T from the paper's block formula: M (row-vector convention, paper bit
   positions) is assembled from its blocks, then T[(bj, w-1-j)][(bi, w-1-i)] =
   M[(bi, i)][(bj, j)]. Returns -2 for engines without a printed matrix. */
int orc_matrix_from_blocks(int gi, u64 *T)
{
    const gen_t *g = gen(gi);
    if (!g) return -1;
    const int w = g->w, k = g->k, n = k * w, nw = words_for(n);
    memset(T, 0, sizeof(u64) * (size_t)n * (size_t)nw);
    unsigned char blk[64 * 64], tmp[64 * 64];
    for (int bi = 0; bi < k; bi++)
        for (int bj = 0; bj < k; bj++) {
            const block_t b = engine_block(g, bi, bj);
            if (b.terms < 0) return -2;
            memset(blk, 0, sizeof(blk));
            if (b.terms & 1) { wmat_identity(w, tmp); for (int t = 0; t < w * w; t++) blk[t] ^= tmp[t]; }
            if (b.terms & 2) { wmat_power(w, 0, b.sp, tmp); for (int t = 0; t < w * w; t++) blk[t] ^= tmp[t]; }
            if (b.terms & 4) { wmat_power(w, 1, b.rp, tmp); for (int t = 0; t < w * w; t++) blk[t] ^= tmp[t]; }
            for (int i = 0; i < w; i++)
                for (int j = 0; j < w; j++)
                    if (blk[i * w + j]) {
                        const int r = bj * w + (w - 1 - j);
                        const int c = bi * w + (w - 1 - i);
                        setbit(T + (size_t)r * nw, c);
                    }
        }
    return 0;
}

/* C = A * B over F2 (plain triple loop on bits). */
int orc_mat_mul(int n, const u64 *A, const u64 *B, u64 *C)
{
    const int nw = words_for(n);
    u64 *out = (u64 *)calloc((size_t)n * nw, sizeof(u64));
    if (!out) return -1;
    for (int r = 0; r < n; r++)
        for (int t = 0; t < n; t++)
            if (getbit(A + (size_t)r * nw, t))
                for (int x = 0; x < nw; x++) out[(size_t)r * nw + x] ^= B[(size_t)t * nw + x];
    memcpy(C, out, sizeof(u64) * (size_t)n * nw);
    free(out);
    return 0;
}

/* out = A v: bit r is the parity of row r AND v. */
int orc_mat_vec(int n, const u64 *A, const u64 *v, u64 *out)
{
    const int nw = words_for(n);
    u64 res[32];
    memset(res, 0, sizeof(res));
    for (int r = 0; r < n; r++) {
        int par = 0;
        for (int x = 0; x < nw; x++) par ^= __builtin_parityll(A[(size_t)r * nw + x] & v[x]);
        if (par) setbit(res, r);
    }
    memcpy(out, res, sizeof(u64) * (size_t)nw);
    return 0;
}

/* Rank over F2 by Gaussian elimination on a copy. */
int orc_mat_rank(int n, const u64 *A)
{
    const int nw = words_for(n);
    u64 *M = (u64 *)malloc(sizeof(u64) * (size_t)n * nw);
    if (!M) return -1;
    memcpy(M, A, sizeof(u64) * (size_t)n * nw);
    int rank = 0;
    for (int c = 0; c < n && rank < n; c++) {
        int piv = -1;
        for (int r = rank; r < n; r++)
            if (getbit(M + (size_t)r * nw, c)) { piv = r; break; }
        if (piv < 0) continue;
        if (piv != rank)
            for (int x = 0; x < nw; x++) {
                u64 t = M[(size_t)piv * nw + x];
                M[(size_t)piv * nw + x] = M[(size_t)rank * nw + x];
                M[(size_t)rank * nw + x] = t;
            }
        for (int r = 0; r < n; r++)
            if (r != rank && getbit(M + (size_t)r * nw, c))
                for (int x = 0; x < nw; x++) M[(size_t)r * nw + x] ^= M[(size_t)rank * nw + x];
        rank++;
    }
    free(M);
    return rank;
}

/* ------------------------------------------------------------------------ */
/* Polynomials over F2: bit i of the array is the coefficient of x^i.        */
/* ------------------------------------------------------------------------ */

#define PW 40 /* words of a polynomial buffer: degrees below 2560 */

static int pdeg(const u64 *a, int nw)
{
    for (int x = nw - 1; x >= 0; x--)
        if (a[x]) return x * 64 + 63 - __builtin_clzll(a[x]);
    return -1;
}

/* dst ^= src << sh (multi-word shift of a polynomial). */
static void xor_shifted(u64 *dst, int dstw, const u64 *src, int srcw, int sh)
{
    const int ws = sh / 64, bs = sh % 64;
    for (int x = 0; x < srcw; x++) {
        const u64 v = src[x];
        if (!v) continue;
        if (x + ws < dstw) dst[x + ws] ^= v << bs;
        if (bs && x + ws + 1 < dstw) dst[x + ws + 1] ^= v >> (64 - bs);
    }
}

/* r = a * b mod p, with deg p = d and deg a, deg b < d: schoolbook product,
   then the remainder by cancelling the top coefficients with shifted p. */
static void pmulmod(const u64 *a, const u64 *b, const u64 *p, int d, u64 *r)
{
    u64 prod[2 * PW];
    memset(prod, 0, sizeof(prod));
    const int dw = words_for(d), pwords = words_for(d + 1);
    for (int i = 0; i < d; i++)
        if (getbit(b, i)) xor_shifted(prod, 2 * PW, a, dw, i);
    for (int i = 2 * d - 2; i >= d; i--)
        if (getbit(prod, i)) xor_shifted(prod, 2 * PW, p, pwords, i - d);
    memset(r, 0, sizeof(u64) * PW);
    memcpy(r, prod, sizeof(u64) * (size_t)dw);
    if (d % 64) r[dw - 1] &= (1ull << (d % 64)) - 1;
}

/* r = x^e mod p.  e is given as nbytes little-endian bytes. */
int orc_poly_xpow(const u64 *p, int pw, const unsigned char *e, size_t nbytes, u64 *r)
{
    u64 pp[PW];
    if (pw > PW) return -1;
    memset(pp, 0, sizeof(pp));
    memcpy(pp, p, sizeof(u64) * (size_t)pw);
    const int d = pdeg(pp, PW);
    if (d < 1) return -1;
    u64 acc[PW], sq[PW];
    memset(acc, 0, sizeof(acc));
    acc[0] = 1; /* x^0 */
    for (long bit = (long)nbytes * 8 - 1; bit >= 0; bit--) {
        pmulmod(acc, acc, pp, d, sq);
        memcpy(acc, sq, sizeof(acc));
        if ((e[bit >> 3] >> (bit & 7)) & 1) {
            /* multiply by x: shift left by one, reduce if degree d appears */
            for (int x = PW - 1; x > 0; x--) acc[x] = (acc[x] << 1) | (acc[x - 1] >> 63);
            acc[0] <<= 1;
            if (getbit(acc, d))
                for (int j = 0; j <= d; j++)
                    if (getbit(pp, j)) flipbit(acc, j);
        }
    }
    memcpy(r, acc, sizeof(u64) * (size_t)pw);
    return 0;
}

/* r = a * b mod p (public wrapper). */
int orc_poly_mulmod(const u64 *a, const u64 *b, const u64 *p, int pw, u64 *r)
{
    u64 aa[PW], bb[PW], pp[PW], rr[PW];
    if (pw > PW) return -1;
    memset(aa, 0, sizeof(aa)); memset(bb, 0, sizeof(bb)); memset(pp, 0, sizeof(pp));
    memcpy(aa, a, sizeof(u64) * (size_t)pw);
    memcpy(bb, b, sizeof(u64) * (size_t)pw);
    memcpy(pp, p, sizeof(u64) * (size_t)pw);
    const int d = pdeg(pp, PW);
    if (d < 1) return -1;
    pmulmod(aa, bb, pp, d, rr);
    memcpy(r, rr, sizeof(u64) * (size_t)pw);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Berlekamp-Massey over F2 (Massey 1969), used in Sec. 6 and Sec. 9.3.     */
/* ------------------------------------------------------------------------ */

/* seq: N bits, bit t of the sequence is bit (t % 64) of word t / 64.
   On return conn (capacity cap words) holds C(x) = 1 + c_1 x + ... + c_L x^L,
   the connection polynomial of the shortest LFSR: s_t = sum_i c_i s_{t-i}.
   Returns L, or -1 when cap is too small. */
long orc_berlekamp_massey(const u64 *seq, size_t N, u64 *conn, size_t cap)
{
    const size_t W = N / 64 + 2;
    if (cap < W) return -1;
    u64 *rev = (u64 *)calloc(W + 1, sizeof(u64));
    u64 *C = (u64 *)calloc(W, sizeof(u64));
    u64 *B = (u64 *)calloc(W, sizeof(u64));
    u64 *Tm = (u64 *)calloc(W, sizeof(u64));
    if (!rev || !C || !B || !Tm) { free(rev); free(C); free(B); free(Tm); return -1; }
    /* rev[j] = s_{N-1-j}: the window s_n, s_{n-1}, ..., s_{n-L} then starts at
       bit N-1-n of rev and lines up with the coefficients c_0, ..., c_L. */
    for (size_t t = 0; t < N; t++)
        if ((seq[t >> 6] >> (t & 63)) & 1u) rev[(N - 1 - t) >> 6] |= 1ull << ((N - 1 - t) & 63);
    C[0] = 1; B[0] = 1;
    long L = 0;
    size_t m = 1;
    for (size_t n = 0; n < N; n++) {
        /* discrepancy d = sum_{i=0..L} c_i s_{n-i} */
        const size_t off = N - 1 - n;
        const size_t nwords = (size_t)L / 64 + 1;
        u64 acc = 0;
        for (size_t x = 0; x < nwords; x++) {
            const size_t bitpos = off + 64 * x;
            const size_t wi = bitpos >> 6, sh = bitpos & 63;
            u64 win = rev[wi] >> sh;
            if (sh && wi + 1 <= W) win |= rev[wi + 1] << (64 - sh);
            acc ^= C[x] & win;
        }
        /* only bits 0..L of C are set, so higher window bits do not matter */
        if (!__builtin_parityll(acc)) { m++; continue; }
        /* C <- C + x^m B (B has degree below W*64 - m by construction) */
        if (2 * L <= (long)n) {
            memcpy(Tm, C, sizeof(u64) * W);
            const size_t ws = m / 64, bs = m % 64;
            for (size_t x = W; x-- > ws;) {
                u64 v = B[x - ws] << bs;
                if (bs && x > ws) v |= B[x - ws - 1] >> (64 - bs);
                C[x] ^= v;
            }
            L = (long)n + 1 - L;
            memcpy(B, Tm, sizeof(u64) * W);
            m = 1;
        } else {
            const size_t ws = m / 64, bs = m % 64;
            for (size_t x = W; x-- > ws;) {
                u64 v = B[x - ws] << bs;
                if (bs && x > ws) v |= B[x - ws - 1] >> (64 - bs);
                C[x] ^= v;
            }
            m++;
        }
    }
    memset(conn, 0, sizeof(u64) * cap);
    memcpy(conn, C, sizeof(u64) * W);
    free(rev); free(C); free(B); free(Tm);
    return L;
}

/* Bit b of successive outputs of a generator (starting from state, which is
   advanced), packed as for orc_berlekamp_massey. */
int orc_output_bits(int gi, u64 *state, int b, size_t N, u64 *seq)
{
    const gen_t *g = gen(gi);
    if (!g) return -1;
    memset(seq, 0, sizeof(u64) * (N / 64 + 1));
    for (size_t t = 0; t < N; t++)
        if ((next_output(g, state) >> b) & 1u) seq[t >> 6] |= 1ull << (t & 63);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Jumps by polynomial (Cayley-Hamilton, Sec. 6): T^J s = sum_i c_i T^i s    */
/* where x^J mod p(x) = sum_i c_i x^i.                                       */
/* ------------------------------------------------------------------------ */

int orc_apply_poly(int gi, const u64 *coef, int ncoef, u64 *state)
{
    const gen_t *g = gen(gi);
    if (!g) return -1;
    u64 acc[16] = {0}, s[16];
    memcpy(s, state, sizeof(u64) * (size_t)g->k);
    for (int i = 0; i < ncoef; i++) {
        if (getbit(coef, i))
            for (int j = 0; j < g->k; j++) acc[j] ^= s[j];
        engine_step(g, s);
    }
    memcpy(state, acc, sizeof(u64) * (size_t)g->k);
    return 0;
}

/* Start states of S streams: out[i] = J^(i) (base), J applied by
   orc_apply_poly with the given jump polynomial, one jump after another. */
int orc_sequential_jumps(int gi, const u64 *coef, int ncoef, const u64 *base, size_t S, u64 *out)
{
    const gen_t *g = gen(gi);
    if (!g) return -1;
    u64 s[16];
    memcpy(s, base, sizeof(u64) * (size_t)g->k);
    for (size_t i = 0; i < S; i++) {
        memcpy(out + i * (size_t)g->k, s, sizeof(u64) * (size_t)g->k);
        if (i + 1 < S) orc_apply_poly(gi, coef, ncoef, s);
    }
    return 0;
}

/* Whole bulk fill as the plain definition: stream i starts at J^i(base) and
   emits m outputs.  Same as orc_sequential_jumps followed by orc_fill_streams,
   without keeping the start table. */
int orc_bulk_fill(int gi, const u64 *coef, int ncoef, const u64 *base, size_t first_jumps,
                  size_t S, size_t m, u64 *out)
{
    const gen_t *g = gen(gi);
    if (!g) return -1;
    u64 s[16], t[16];
    memcpy(s, base, sizeof(u64) * (size_t)g->k);
    for (size_t i = 0; i < first_jumps; i++) orc_apply_poly(gi, coef, ncoef, s);
    for (size_t i = 0; i < S; i++) {
        memcpy(t, s, sizeof(u64) * (size_t)g->k);
        for (size_t j = 0; j < m; j++) out[i * m + j] = next_output(g, t);
        if (i + 1 < S) orc_apply_poly(gi, coef, ncoef, s);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Escaping zeroland (Sec. 8): for each of the n states with exactly one bit */
/* set, the first nout outputs; counts[t] = number of one bits in outputs    */
/* t .. t + window - 1, summed over the n states.                            */
/* ------------------------------------------------------------------------ */

int orc_zeroland(int gi, size_t nout, size_t window, u64 *counts)
{
    const gen_t *g = gen(gi);
    if (!g || window == 0 || window > nout) return -1;
    const int n = g->k * g->w;
    const size_t T = nout - window + 1;
    memset(counts, 0, sizeof(u64) * T);
    u64 *ones = (u64 *)malloc(sizeof(u64) * nout);
    if (!ones) return -1;
    for (int j = 0; j < n; j++) {
        u64 s[16] = {0};
        s[j / g->w] = 1ull << (j % g->w);
        for (size_t i = 0; i < nout; i++) ones[i] = (u64)__builtin_popcountll(next_output(g, s));
        for (size_t t = 0; t < T; t++)
            for (size_t i = t; i < t + window; i++) counts[t] += ones[i];
    }
    free(ones);
    return 0;
}
