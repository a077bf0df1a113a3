"""Pins of the CPU oracle against what the paper fixes.  No GPU needed.

Each test checks the oracle against something other than itself: the paper's
printed block matrices (Sec. 3), the weights of Tables 4 and 7, the linear
complexities of Table 13, the worked xorshift example of Sec. 9, the
equidistribution statements on tiny engines of Sec. 7, primitivity (Sec. 6),
the prose restatements of the scrambler parameters (Sec. 10), and exact
rational arithmetic for the doubles (Sec. 5.3).
"""
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

# Generators whose engine has a printed block matrix (Sec. 3.1 Eq. (M), Sec. 3.2).
MATRIX_GENERATORS = [
    "xoshiro256+", "xoroshiro128+", "xoroshiro128++", "xoshiro128++", "xoshiro512+",
    "xoroshiro1024++", "xoroshiro64*", "xoroshiro10+", "xoshiro8+", "xoroshiro16x4+",
    "xoshiro40+",
]
ENGINES_256_128 = ["xoshiro256**", "xoroshiro128+", "xoroshiro128++", "xoshiro128**"]


def rand_state(name, rng):
    w, k = O.word_bits(name), O.state_words(name)
    while True:
        s = np.array([rng.getrandbits(w) for _ in range(k)], dtype=np.uint64)
        if s.any():
            return s


# --------------------------------------------------------------- P1: one step = T s

@pytest.mark.parametrize("name", MATRIX_GENERATORS)
def test_step_equals_paper_block_matrix(name):
    """The code step equals the paper's block matrix (X_kw, S_4w, S_8w) read with
    S = shift left, R = rotate left, acting on random states."""
    T = O.matrix_from_blocks(name)
    assert (T == O.matrix_from_step(name)).all()
    rng = random.Random(1)
    for _ in range(300):
        s = rand_state(name, rng)
        via_matrix = O.bits_to_state(name, O.mat_vec(T, O.state_to_bits(name, s)))
        assert (via_matrix == O.step(name, s)).all()


def test_block_matrix_detects_a_wrong_parameter():
    """Negative control: the block formula with the xoroshiro128++ parameters is
    not the xoroshiro128 matrix (the two rows of Table 4 differ)."""
    assert not (O.matrix_from_blocks("xoroshiro128+") == O.matrix_from_blocks("xoroshiro128++")).all()


# --------------------------------------------------------------- P2: T^k s = k steps

@pytest.mark.parametrize("name", ENGINES_256_128)
def test_matrix_power_equals_sequential_steps(name):
    T = O.matrix_from_step(name)
    rng = random.Random(2)
    s = rand_state(name, rng)
    for k in (0, 1, 2, 3, 17, 100, 999, 1000):
        Tk = O.mat_pow(T, k)
        via_matrix = O.bits_to_state(name, O.mat_vec(Tk, O.state_to_bits(name, s)))
        assert (via_matrix == O.step(name, s, k)).all(), k


# --------------------------------------------------------------- P3: jump two ways

@pytest.mark.parametrize("name", ENGINES_256_128)
@pytest.mark.parametrize("kind", ["jump", "long"])
def test_jump_polynomial_equals_repeated_squaring(name, kind):
    """T^(2^d) by d matrix squarings equals sum c_i T^i with x^(2^d) mod p(x)."""
    d = O.jump_log2(name, kind)
    assert d == {("jump", 256): 128, ("long", 256): 192,
                 ("jump", 128): 64, ("long", 128): 96}[(kind, O.state_bits(name))]
    M = O.mat_pow2(O.matrix_from_step(name), d)
    rng = random.Random(3)
    for _ in range(8):
        s = rand_state(name, rng)
        via_matrix = O.bits_to_state(name, O.mat_vec(M, O.state_to_bits(name, s)))
        assert (via_matrix == O.jump(name, kind, s)).all()


@pytest.mark.parametrize("name", ["xoshiro256++", "xoroshiro128**", "xoshiro128++"])
def test_successive_jumps_equal_one_power(name):
    s = O.seed(name, 11)
    st = O.streams(name, "jump", s, 40)
    d = O.jump_log2(name, "jump")
    for i in (0, 1, 2, 7, 39):
        assert (st[i] == O.jump_pow(name, d, i, s)).all()
        assert (st[i] == O.jump(name, "jump", s, i)).all()
    # first > 0 continues the same sequence of streams
    assert (O.streams(name, "jump", s, 10, first=30) == st[30:40]).all()


@pytest.mark.parametrize("name", ["xoshiro256++", "xoroshiro128**", "xoroshiro128++", "xoshiro128**", "xoroshiro64*"])
@pytest.mark.parametrize("kind", ["jump", "long"])
def test_chunk_decomposition_of_streams(name, kind):
    """Stream p + P j of a range equals j jumps of distance 2^(J + log2 P)
    applied to stream p (P a power of two): the reading behind chunks of 512 P
    streams, whose streams are taken from P parents with the power set of
    that distance.  Distances past the state size wrap (T^(2^n) = T)."""
    s = O.seed(name, 13)
    d = O.jump_log2(name, kind)
    n = O.state_bits(name)
    for k in (5, 6, 15, 70):
        P = 1 << k
        for p, j in ((0, 1), (3, 2), (P - 1, 511), (17 % P, 300)):
            stream = O.jump_pow(name, d, p + P * j, s)
            parent = O.jump_pow(name, d, p, s)
            assert (stream == O.jump_pow(name, (d + k) % n, j, parent)).all(), (k, p, j)


def test_long_jump_is_a_power_of_the_jump():
    """2^192 = 2^64 * 2^128 and 2^96 = 2^32 * 2^64."""
    for name, ratio in (("xoshiro256**", 2**64), ("xoroshiro128++", 2**32)):
        s = O.seed(name, 5)
        d = O.jump_log2(name, "jump")
        assert (O.jump(name, "long", s) == O.jump_pow(name, d, ratio, s)).all()


# --------------------------------------------------------------- P4: char. polynomial

def test_char_poly_degree_and_weight(golden):
    """Berlekamp-Massey on bit 0 of the + output returns a polynomial of degree n
    whose weight is the one printed in Tables 4 and 7."""
    for eng, deg, weight in golden("char_poly_weights.txt"):
        p = O.char_poly(eng)
        assert p.bit_length() - 1 == int(deg), eng
        assert O.poly_weight(p) == int(weight), eng


@pytest.mark.parametrize("name", ENGINES_256_128 + ["xoshiro512+", "xoroshiro64*"])
def test_char_poly_annihilates_T(name):
    """Cayley-Hamilton: p(T) s = 0 for every state s."""
    p = O.char_poly(name)
    rng = random.Random(4)
    for _ in range(4):
        assert not O.apply_poly(name, p, rand_state(name, rng)).any()
    # negative control: dropping the constant term no longer annihilates
    assert O.apply_poly(name, p ^ 1, rand_state(name, rng)).any()


# Fermat numbers F_i = 2^(2^i) + 1 with their published prime factorizations
# (Euler 1732 for F5, Landry 1880 for F6, Morrison and Brillhart 1975 for F7);
# 2^(2^m) - 1 = F_0 F_1 ... F_{m-1}.  The test below re-checks products and primality.
FERMAT_FACTORS = {
    0: [3], 1: [5], 2: [17], 3: [257], 4: [65537],
    5: [641, 6700417],
    6: [274177, 67280421310721],
    7: [59649589127497217, 5704689200685129054721],
}


def is_probable_prime(n):
    """Miller-Rabin with the first 13 primes as bases (deterministic below 3.3e24)."""
    if n < 2:
        return False
    small = [2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41]
    for q in small:
        if n % q == 0:
            return n == q
    d, r = n - 1, 0
    while d % 2 == 0:
        d //= 2
        r += 1
    for a in small:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(r - 1):
            x = pow(x, 2, n)
            if x == n - 1:
                break
        else:
            return False
    return True


def prime_factors_of_2n_minus_1(n):
    if n & (n - 1) == 0 and n >= 2:
        fs = [f for i in range(n.bit_length() - 1) for f in FERMAT_FACTORS[i]]
    else:
        fs, m, q = [], 2**n - 1, 2
        while q * q <= m:
            while m % q == 0:
                fs.append(q)
                m //= q
            q += 1
        if m > 1:
            fs.append(m)
    prod = 1
    for f in fs:
        prod *= f
        assert is_probable_prime(f), f
    assert prod == 2**n - 1
    return sorted(set(fs))


def is_primitive(p, n):
    """x has order exactly 2^n - 1 modulo p(x)."""
    if O.poly_xpow(p, 2**n) != 0b10:
        return False
    return all(O.poly_xpow(p, (2**n - 1) // q) != 1 for q in prime_factors_of_2n_minus_1(n))


@pytest.mark.parametrize("name,n", [("engine/xoshiro256", 256), ("engine/xoroshiro128", 128),
                                    ("engine/xoroshiro128pp", 128), ("engine/xoshiro128", 128),
                                    ("engine/xoroshiro64", 64), ("xoshiro40+", 40),
                                    ("xoroshiro16x4+", 16), ("xoroshiro10+", 10), ("xoshiro8+", 8)])
def test_char_poly_is_primitive(name, n):
    """Sec. 6: full period 2^n - 1 iff p(x) is primitive; the engines of Tables 4
    and 7 and the tiny full-period engines of Sec. 7 all have full period."""
    p = O.char_poly(name)
    assert p.bit_length() - 1 == n
    assert is_primitive(p, n)


def test_primitivity_check_rejects_non_primitive():
    assert not is_primitive(0b10001, 4)          # x^4 + 1 = (x + 1)^4
    assert not is_primitive(0b11111, 4)          # x^4+x^3+x^2+x+1: irreducible, order 5
    assert is_primitive(0b10011, 4)              # x^4 + x + 1
    p = O.char_poly("engine/xoroshiro128")
    assert not is_primitive(p ^ 0b110, 128)


# --------------------------------------------------------------- P5: Table 13

def _lc_rows(golden, slow):
    rows = [(g, int(b), int(lc)) for g, b, lc in golden("plus_linear_complexity.txt")]
    return [r for r in rows if (r[2] > 200000) == slow]


def test_plus_low_bits_linear_complexity(golden):
    for g, b, lc in _lc_rows(golden, slow=False):
        assert O.linear_complexity(g, b, 2 * lc + 200) == lc, (g, b)


@pytest.mark.slow
def test_plus_bit2_linear_complexity_128(golden):
    for g, b, lc in _lc_rows(golden, slow=True):
        assert O.linear_complexity(g, b, 2 * lc + 200) == lc, (g, b)


def test_table13_values_are_the_ub_bound(golden):
    """Table 13's values are U(n, b+1) = sum_{j=1}^{b+1} C(n, j) (Eq. (ub))."""
    from math import comb
    for g, b, lc in golden("plus_linear_complexity.txt"):
        n = O.state_bits(g)
        assert int(lc) == sum(comb(n, j) for j in range(1, int(b) + 2)), (g, b)


# --------------------------------------------------------------- P6: zero state, periods

@pytest.mark.parametrize("name", ENGINES_256_128 + ["xoshiro512+", "xoroshiro1024++"])
def test_transition_is_invertible(name):
    assert O.mat_rank(O.matrix_from_step(name)) == O.state_bits(name)


def full_cycle(name):
    """Outputs and states along one orbit from state (1, 0, ...)."""
    k = O.state_words(name)
    s0 = np.zeros(k, np.uint64)
    s0[0] = 1
    n = O.state_bits(name)
    period = 2**n - 1
    out, end = O.generate(name, s0, period)
    assert (end == s0).all()
    return out


@pytest.mark.parametrize("name,period", [("xoroshiro10+", 1023), ("xoshiro8+", 255),
                                         ("xoroshiro16x4+", 65535)])
def test_tiny_engine_full_period(name, period):
    """Sec. 7: these tiny engines have full period: every nonzero state lies on one
    orbit of length 2^n - 1, so no nonzero state ever reaches zero."""
    k = O.state_words(name)
    s = np.zeros(k, np.uint64)
    s[0] = 1
    seen = set()
    for _ in range(period):
        key = tuple(int(x) for x in s)
        assert key not in seen and any(key)
        seen.add(key)
        s = O.step(name, s)
    assert tuple(int(x) for x in s) == (1,) + (0,) * (k - 1)
    assert len(seen) == period


def tuple_counts(values, d):
    P = len(values)
    ext = np.concatenate([values, values[: d - 1]])
    counts = {}
    for t in range(P):
        key = tuple(int(x) for x in ext[t:t + d])
        counts[key] = counts.get(key, 0) + 1
    return counts


def equidistributed(values, w, k, d):
    """Every d-tuple appears 2^(w(k-d)) times, the zero tuple once less (Sec. 7)."""
    c = tuple_counts(values, d)
    full = 2 ** (w * (k - d))
    for key in np.ndindex(*([2**w] * d)):
        want = full - 1 if not any(key) else full
        if c.get(tuple(key), 0) != want:
            return False
    return True


def test_xoroshiro10_equidistribution():
    """Sec. 7: the 5-bit xoroshiro with 10 bits of state (a, b, c) = (1, 3, 1) is
    2-dimensionally equidistributed as an engine (every word), while xoroshiro+
    on it is 1- but not 2-dimensionally equidistributed (Prop. on xoroshiro+)."""
    out = full_cycle("xoroshiro10+")
    assert equidistributed(out, 5, 2, 1)
    assert not equidistributed(out, 5, 2, 2)
    k, s = 2, np.array([1, 0], np.uint64)
    words = [[], []]
    for _ in range(1023):
        words[0].append(int(s[0]))
        words[1].append(int(s[1]))
        s = O.step("xoroshiro10+", s)
    for j in range(k):
        assert equidistributed(np.array(words[j], np.uint64), 5, 2, 2)


def test_xoshiro8_equidistribution():
    """Sec. 7: the only 2-bit xoshiro (8 bits of state) has full period; xoshiro+
    on the first and last word is 3- but not 4-dimensionally equidistributed, and
    xoshiro++ is 3-dimensionally equidistributed."""
    out = full_cycle("xoshiro8+")
    assert equidistributed(out, 2, 4, 3)
    assert not equidistributed(out, 2, 4, 4)
    assert equidistributed(full_cycle("xoshiro8++"), 2, 4, 3)


def test_xoroshiro16x4_plus_equidistribution():
    """Sec. 7: xoroshiro+ with k words on the first and last word is
    (k-1)-dimensionally equidistributed; here w = 4, k = 4, (a, b, c) = (3, 1, 2)."""
    out = full_cycle("xoroshiro16x4+")
    assert equidistributed(out, 4, 4, 3)


def test_seeded_states_are_nonzero():
    for name in O.VARIANTS:
        for sv in list(range(64)) + [2**64 - 1, 0x0123456789ABCDEF]:
            assert O.seed(name, sv).any()


# --------------------------------------------------------------- P7: xorshift example

def test_xorshift_example_of_section_9(golden):
    rows = {r[0]: [int(x) for x in r[1:]] for r in golden("xorshift6_example.txt")}
    poly = lambda exps: sum(1 << e for e in exps)
    assert O.char_poly("xorshift6+") == poly(rows["char_poly"])
    for b in range(3):
        for sv in (1, 2, 99):
            L, C = O.berlekamp_massey(O.output_bits("xorshift6+", O.seed("xorshift6+", sv), b, 300), 300)
            assert L == rows["lc_bit%d" % b][0]
            # the connection polynomial is the denominator of the generating function
            assert C == poly(rows["denominator_bit%d" % b])


# --------------------------------------------------------------- P8: doubles

@pytest.mark.parametrize("name", ["xoshiro256**", "xoshiro128++"])
def test_doubles_are_exact(name):
    w = O.word_bits(name)
    rng = random.Random(8)
    xs = [0, 1, 2**w - 1, 2**(w - 1), 2**11 - 1, 2**11] + [rng.getrandbits(w) for _ in range(5000)]
    got = O.to_f64(name, np.array(xs, dtype=np.uint64))
    for x, g in zip(xs, got):
        want = Fraction(x >> 11, 2**53) if w == 64 else Fraction(x, 2**32)
        assert Fraction(float(g)) == want
        assert 0.0 <= g < 1.0
    if w == 64:
        assert got[2] == 1.0 - 2.0**-53 and got[0] == 0.0
    else:
        assert got[2] == 1.0 - 2.0**-32


def test_floats_are_exact():
    rng = random.Random(9)
    for name, w in (("xoshiro128+", 32), ("xoshiro256+", 64)):
        xs = [0, 2**w - 1] + [rng.getrandbits(w) for _ in range(2000)]
        got = O.to_f32(name, np.array(xs, dtype=np.uint64))
        for x, g in zip(xs, got):
            assert Fraction(float(g)) == Fraction(x >> (w - 24), 2**24)


# --------------------------------------------------------------- scramblers (Sec. 4, 10)

def test_starstar_parameters_from_section_10():
    """Sec. 10.4 chooses s = 2, t = 3, r = 7: multipliers 2^2+1 = 5 and 2^3+1 = 9.
    Its stated consequence: the min(r, t) lowest bits of z = rotl(x(2^s+1), r)(2^t+1)
    come from the highest bits of x(2^s+1).  Read exactly: rotl by r brings bits
    w-r .. w-1 down to 0 .. r-1, and the multiplier 2^t+1 leaves the t lowest bits
    alone, so bits 0 .. t-1 of z are bits w-r .. w-r+t-1 of x(2^s+1)."""
    rng = random.Random(10)
    for name, w, word in (("xoshiro256**", 64, 1), ("xoroshiro128**", 64, 0), ("xoshiro128**", 32, 1),
                          ("xoshiro512**", 64, 1), ("xoroshiro1024**", 64, 0)):
        for _ in range(2000):
            s = rand_state(name, rng)
            z = O.scramble(name, s)
            y = (int(s[word]) * 5) % 2**w
            assert z & 0b111 == (y >> (w - 7)) & 0b111
            # bit 3 of z is bit 3 xor bit 0 of the rotated word (multiplier 2^3 + 1)
            rot = ((y << 7) | (y >> (w - 7))) % 2**w
            assert (z >> 3) & 1 == ((rot >> 3) ^ rot) & 1


def test_xoroshiro64_starstar_parameters():
    """Sec. 10.4: at 32 bits the first multiplier is the * constant and the second
    is 2^t + 1 with bit t not set in the first constant, and r = 2t + 1."""
    first = 0x9E3779BB
    t = 2
    assert not (first >> t) & 1 and 2 * t + 1 == 5
    rng = random.Random(12)
    for _ in range(1000):
        s = rand_state("xoroshiro64**", rng)
        y = (int(s[0]) * first) % 2**32
        z = O.scramble("xoroshiro64**", s)
        rot = ((y << 5) | (y >> 27)) % 2**32
        assert z == (rot * (2**t + 1)) % 2**32


def test_plusplus_low_bit():
    """Sec. 4.3 / 10.3: z = rotl(x + y, r) + x; bit 0 of z is bit (w - r) of x + y
    xor bit 0 of x (rotations 23, 17, 7 from Tables 5 and 8; xoshiro512++ adds
    s2 after the rotation, xoroshiro1024++ the last word s15)."""
    rng = random.Random(13)
    for name, w, r, (p, q) in (("xoshiro256++", 64, 23, (0, 3)), ("xoroshiro128++", 64, 17, (0, 1)),
                               ("xoshiro128++", 32, 7, (0, 3)), ("xoshiro512++", 64, 17, (2, 0)),
                               ("xoroshiro1024++", 64, 23, (15, 0))):
        for _ in range(2000):
            s = rand_state(name, rng)
            z = O.scramble(name, s)
            sm = (int(s[p]) + int(s[q])) % 2**w
            assert z & 1 == ((sm >> (w - r)) ^ int(s[p])) & 1


def test_plus_sums_the_plusplus_pair():
    """Sec. 4.1 and 4.3: the + and ++ scramblers of an engine sum the same two
    words (the code figures of Sec. 3), ++ then rotating and adding one of
    them.  So the + output is rotr(z++ - x, r) on the same state, which ties
    the + word pair to the ++ one pinned by the low-bit test above."""
    rng = random.Random(15)
    for plus, pp, w, r, p in (("xoshiro256+", "xoshiro256++", 64, 23, 0), ("xoroshiro128+", "xoroshiro128++", 64, 17, 0),
                              ("xoshiro128+", "xoshiro128++", 32, 7, 0), ("xoshiro512+", "xoshiro512++", 64, 17, 2)):
        M = 2**w - 1
        for _ in range(1000):
            s = rand_state(plus, rng)
            y = (O.scramble(pp, s) - int(s[p])) & M
            assert O.scramble(plus, s) == ((y >> r) | (y << (w - r))) & M, plus


def test_star_low_bits():
    """Sec. 4.2: with the second-lowest set bit of the multiplier at position b,
    the lowest b output bits are unmodified and bit b is bit 0 xor bit b; the
    64-bit constant has bit 1 set (b = 1)."""
    m = 0x9e3779b97f4a7c13
    assert m & 1 and (m >> 1) & 1
    rng = random.Random(14)
    for _ in range(1000):
        s = rand_state("xoroshiro128*", rng)
        z = O.scramble("xoroshiro128*", s)
        x = int(s[0])
        assert z & 1 == x & 1 and (z >> 1) & 1 == ((x >> 1) ^ x) & 1


def test_star_multipliers_from_the_golden_ratio():
    """Sec. 4.2: the * multiplier is close to phi 2^w mod 2^w = 2^w / phi (phi
    the golden ratio), its low bits adjusted so that bit 1 is set.  With the
    scrambled word equal to 1 the * output is the multiplier itself, so the
    oracle's constant is read back and compared with 2^w / phi computed from
    an exact integer square root (within the few units the adjustment of the
    lowest bits allows), with bits 0 and 1 set, and with the values printed in
    Tables 5 and 8.  A wrong digit anywhere fails."""
    import math
    for name, w, k, printed in (("xoroshiro128*", 64, 2, 0x9e3779b97f4a7c13),
                                ("xoroshiro1024*", 64, 16, 0x9e3779b97f4a7c13),
                                ("xoroshiro64*", 32, 2, 0x9E3779BB)):
        # 2^w / phi = (sqrt(5) - 1) 2^(w-1), scaled by 2^(w+1) to stay an integer: exact to < 1 unit
        golden_x = math.isqrt(5 << (4 * w)) - (1 << (2 * w))
        # the scrambled word is word 0 of the state in the oracle's order
        s = np.zeros(k, np.uint64)
        s[0] = 1
        m = O.scramble(name, s)
        assert m == printed, (name, hex(m))
        assert m & 3 == 3, name
        assert abs(m * 2 ** (w + 1) - golden_x) < 4 * 2 ** (w + 1), (name, hex(m))
    # xoroshiro64** takes the same first multiplier (Table 8)
    s = np.zeros(2, np.uint64)
    s[0] = 1
    assert O.scramble("xoroshiro64**", s) == (((0x9E3779BB << 5) | (0x9E3779BB >> 27)) & 0xffffffff) * 5 % 2**32


def test_output_precedes_update():
    """Sec. 2: the scrambler reads the current state, before the engine step."""
    for name in O.VARIANTS:
        s = O.seed(name, 3)
        out, after = O.generate(name, s, 2)
        assert int(out[0]) == O.scramble(name, s)
        assert int(out[1]) == O.scramble(name, O.step(name, s))
        assert (after == O.step(name, s, 2)).all()


# --------------------------------------------------------------- SplitMix64 seeding (Sec. 5.3)

def test_splitmix64_properties():
    """Word layout of the seeding (Sec. 5.3): 32-bit states take the low half of
    each SplitMix64 output first, 64-bit states take consecutive outputs, and
    the outputs of a seed are distinct (the mixer is a bijection of a Weyl
    sequence).  The constants are pinned by the next test."""
    z = O.splitmix64(42, 2)
    s = O.seed("xoshiro128++", 42)
    assert [int(x) for x in s] == [int(z[0]) & 0xffffffff, int(z[0]) >> 32,
                                   int(z[1]) & 0xffffffff, int(z[1]) >> 32]
    assert (O.seed("xoshiro256**", 42) == O.splitmix64(42, 4)).all()
    assert (O.seed("xoroshiro128+", 42) == O.splitmix64(42, 2)).all()
    many = O.splitmix64(0, 1 << 16)
    assert len(set(int(x) for x in many)) == 1 << 16


def _golden_gamma():
    """The odd 64-bit integer nearest 2^64 / phi, phi the golden ratio, from an
    exact integer square root: 2^64 (sqrt 5 - 1) / 2 = (sqrt(5 * 2^256) - 2^128) / 2^65."""
    import math
    x = (math.isqrt(5 << 256) - (1 << 128)) >> 65     # floor(2^64 / phi)
    return x if x & 1 else x + 1


def _independent_mix64(tmp_path):
    """The 64-bit SplitMix finalizer as an independent project defines it:
    pybind11 carries it in pybind11/detail/internals.h as `mix64` (its comment
    names it David Stafford's variant 13 of the MurmurHash3 finalizer, the
    one SplitMix popularized).  The header is compiled into a one-function
    shared object and called; nothing of it is copied here."""
    import ctypes
    import shutil
    import subprocess
    import sysconfig
    try:
        import pybind11
        inc = pybind11.get_include()
    except ImportError:
        pytest.skip("pybind11 headers not installed")
    pyinc = sysconfig.get_paths()["include"]
    gxx = shutil.which("g++")
    if not gxx or not os.path.exists(os.path.join(inc, "pybind11", "detail", "internals.h")) \
            or not os.path.exists(os.path.join(pyinc, "Python.h")):
        pytest.skip("g++, pybind11's internals.h or Python.h missing")
    src = tmp_path / "mix.cpp"
    src.write_text('#include <pybind11/detail/internals.h>\n'
                   'extern "C" unsigned long long ext_mix64(unsigned long long z)\n'
                   '{ return pybind11::detail::mix64(z); }\n')
    so = tmp_path / "mix.so"
    subprocess.run([gxx, "-O1", "-std=c++17", "-fPIC", "-shared", "-w", "-I" + inc, "-I" + pyinc, str(src),
                    "-o", str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    lib.ext_mix64.restype = ctypes.c_ulonglong
    lib.ext_mix64.argtypes = [ctypes.c_ulonglong]
    return lib.ext_mix64


def test_splitmix64_against_golden_gamma_and_independent_mixer(tmp_path):
    """Sec. 5.3 names SplitMix but does not define it.  Output i of the oracle's
    SplitMix64(seed) must be the finalizer applied to seed + (i + 1) gamma
    (mod 2^64): a Weyl sequence whose increment is the golden-ratio gamma,
    derived here from phi, and whose outputs go through the variant-13
    finalizer, taken from an independent implementation in this environment.
    A changed multiplier, shift or increment, or mixing before the increment,
    fails this test."""
    gamma = _golden_gamma()
    assert gamma == 0x9E3779B97F4A7C15
    mix64 = _independent_mix64(tmp_path)
    rng = random.Random(55)
    M = (1 << 64) - 1
    seeds = [0, 1, 42, 0x0123456789ABCDEF, M, 1 << 63] + [rng.getrandbits(64) for _ in range(200)]
    for seed in seeds:
        got = [int(x) for x in O.splitmix64(seed, 6)]
        want = [mix64((seed + (i + 1) * gamma) & M) for i in range(6)]
        assert got == want, hex(seed)
    # the seeding of every word size follows those outputs
    for name in ("xoshiro256**", "xoroshiro128++", "xoshiro512+", "xoroshiro1024**"):
        k = O.state_words(name)
        assert [int(x) for x in O.seed(name, 42)] == [mix64((42 + (i + 1) * gamma) & M) for i in range(k)]
    z = [mix64((42 + (i + 1) * gamma) & M) for i in range(2)]
    assert [int(x) for x in O.seed("xoshiro128**", 42)] == [z[0] & 0xffffffff, z[0] >> 32,
                                                            z[1] & 0xffffffff, z[1] >> 32]
    assert [int(x) for x in O.seed("xoroshiro64*", 42)] == [z[0] & 0xffffffff, z[0] >> 32]


def test_bulk_fill_equals_streams_then_fill():
    name = "xoshiro256**"
    base = O.seed(name, 0x0123456789ABCDEF)
    st = O.streams(name, "jump", base, 33)
    a = O.fill_streams(name, st, 17)
    b = O.bulk_fill(name, "jump", base, 33, 17)
    assert (a == b).all()
    assert (st[0] == base).all()


# --------------------------------------------------------------- P9: escaping zeroland (Sec. 8)

# One bits of the first output, summed over the n states with one bit set.
# Derived by hand from the scramblers' definitions (Sec. 4):
#   +  : the sum of two words of which at most one is nonzero has one bit for
#        the states with the bit in a summed word, none otherwise;
#   ++ : rotl(a + b, r) + a has 2 bits for a bit in a (distinct positions, no
#        carry), 1 for a bit in b;
#   ** : rotl(5 s, 7) * 9.  5 * 2^b has bits b, b + 2 (one bit when b + 2 >= w);
#        * 9 adds those bits shifted by 3 and never carries (the two pairs
#        cannot overlap), dropping the shifted bits that reach w.  For w = 64
#        that gives 62 * 2 + 59 + 59 + 2 + 2 = 246, for w = 32 30 * 2 + 27 + 27
#        + 2 + 2 = 118.
ZEROLAND_FIRST_OUTPUT = {
    "xoroshiro128+": 128, "xoshiro256+": 128, "xoshiro128+": 64,
    "xoshiro256++": 192, "xoroshiro128++": 192, "xoshiro128++": 96,
    "xoshiro256**": 246, "xoroshiro128**": 246, "xoshiro128**": 118,
}


@pytest.mark.parametrize("name", sorted(ZEROLAND_FIRST_OUTPUT))
def test_zeroland_first_output_closed_form(name):
    assert int(O.zeroland(name, 3, 1)[0]) == ZEROLAND_FIRST_OUTPUT[name]


def test_zeroland_windows_add_up():
    """A window's count is the sum of the single-output counts it covers."""
    for name in ("xoshiro256++", "xoroshiro64**", "xoshiro512**"):
        one = O.zeroland(name, 300, 1).astype(np.int64)
        for window in (2, 4, 17, 64):
            w = O.zeroland(name, 300, window).astype(np.int64)
            want = np.convolve(one, np.ones(window, np.int64), mode="valid")
            assert (w == want).all(), (name, window)


@pytest.mark.parametrize("name", ["xoshiro256**", "xoroshiro128+", "xoshiro128++", "xoroshiro1024*"])
def test_zeroland_escapes_to_one_half(name):
    """Sec. 8: starting near the zero state the outputs hold few ones; after a
    number of steps depending on the engine's diffusion they look random (one
    half ones).  The last 200 windows of 1000 outputs are within 0.02 of 1/2."""
    n, w, window = O.state_bits(name), O.word_bits(name), 4
    ratio = O.zeroland(name, 1000, window) / float(n * window * w)
    assert ratio[0] < 0.2
    assert abs(ratio[-200:].mean() - 0.5) < 0.02
