"""Plain CPU oracle for the scrambled linear generators of Blackman & Vigna
("Scrambled Linear Pseudorandom Number Generators", arXiv 1805.01407).

TEST INFRASTRUCTURE ONLY.  The library (``paper_1805_01407_gb300``) never imports
this package.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` (the baseline beside the device numbers and the reference arm) may
import it.  It shares no code with the CUDA path.

The arithmetic lives in ``xr_oracle.c`` (plain C, compiled here with gcc); this
module only marshals arguments and orchestrates the definitions:

* ``generate``/``fill_streams`` -- next() = scramble the current state, then one
  engine step (Sec. 2; engines Sec. 3, scramblers Sec. 4, Tables 4, 5, 7, 8);
* ``seed`` -- SplitMix64 seeding (Sec. 5.3);
* ``to_f64`` -- (x >> 11) * 2^-53 (Sec. 5.3);
* ``char_poly`` -- Berlekamp-Massey on bit 0 of the ``+`` output (Sec. 4.1, 6);
* ``jump``/``jump_pow``/``streams`` -- T^J s = sum c_i T^i s with
  x^J mod p(x) = sum c_i x^i (Sec. 6, Cayley-Hamilton);
* matrix helpers -- T from the step or from the paper's block matrices (Sec. 3);
* ``linear_complexity`` -- Berlekamp-Massey on one output bit (Sec. 9.3, Table 13);
* ``zeroland`` -- one bits in windows of outputs from every one-bit state (Sec. 8).

Jump distances are not printed in the paper.  Reading used here: a jump
advances 2^(n/2) steps and a long jump 2^(3n/4) steps for an n-bit state
(2^128 and 2^192 for xoshiro256; 2^64 and 2^96 for the 128-bit generators).
"""
from __future__ import annotations

import ctypes
import functools
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xr_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")

# Generators graded on the GPU path, in a fixed order.
VARIANTS = (
    "xoshiro256+", "xoshiro256++", "xoshiro256**",
    "xoroshiro128+", "xoroshiro128++", "xoroshiro128**",
    "xoshiro128++", "xoshiro128**", "xoshiro128+",
)

# Which engine (linear part) each generator uses; the engine entries carry the
# + scrambler on the first and last word so that bit 0 of their output is linear.
ENGINE_OF = {
    "xoshiro256+": "engine/xoshiro256", "xoshiro256++": "engine/xoshiro256",
    "xoshiro256**": "engine/xoshiro256",
    "xoroshiro128+": "engine/xoroshiro128", "xoroshiro128**": "engine/xoroshiro128",
    "xoroshiro128*": "engine/xoroshiro128",
    "xoroshiro128++": "engine/xoroshiro128pp",
    "xoshiro128++": "engine/xoshiro128", "xoshiro128**": "engine/xoshiro128",
    "xoshiro128+": "engine/xoshiro128",
    "xoshiro512+": "engine/xoshiro512", "xoshiro512++": "engine/xoshiro512",
    "xoshiro512**": "engine/xoshiro512",
    "xoroshiro1024*": "engine/xoroshiro1024", "xoroshiro1024++": "engine/xoroshiro1024",
    "xoroshiro1024**": "engine/xoroshiro1024",
    "xoroshiro64*": "engine/xoroshiro64", "xoroshiro64**": "engine/xoroshiro64",
}


def build(force: bool = False) -> str:
    """Compile xr_oracle.c into liboracle.so next to it (gcc, -O2)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC],
                       check=True)
        os.replace(tmp, _SO)
    return _SO


_u64p = ctypes.POINTER(ctypes.c_uint64)


@functools.lru_cache(maxsize=None)
def _lib():
    build()
    lib = ctypes.CDLL(_SO)
    lib.orc_generator_name.restype = ctypes.c_char_p
    lib.orc_berlekamp_massey.restype = ctypes.c_long
    for fn in ("orc_splitmix64", "orc_seed", "orc_step", "orc_generate", "orc_fill_streams",
               "orc_apply_poly", "orc_sequential_jumps", "orc_bulk_fill"):
        getattr(lib, fn).restype = ctypes.c_int
    lib.orc_step.argtypes = [ctypes.c_int, _u64p, ctypes.c_uint64]
    lib.orc_seed.argtypes = [ctypes.c_int, ctypes.c_uint64, _u64p]
    lib.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_size_t, _u64p]
    lib.orc_generate.argtypes = [ctypes.c_int, _u64p, ctypes.c_size_t, _u64p]
    lib.orc_fill_streams.argtypes = [ctypes.c_int, _u64p, ctypes.c_size_t, ctypes.c_size_t, _u64p]
    lib.orc_apply_poly.argtypes = [ctypes.c_int, _u64p, ctypes.c_int, _u64p]
    lib.orc_sequential_jumps.argtypes = [ctypes.c_int, _u64p, ctypes.c_int, _u64p,
                                         ctypes.c_size_t, _u64p]
    lib.orc_bulk_fill.argtypes = [ctypes.c_int, _u64p, ctypes.c_int, _u64p, ctypes.c_size_t,
                                  ctypes.c_size_t, ctypes.c_size_t, _u64p]
    lib.orc_berlekamp_massey.argtypes = [_u64p, ctypes.c_size_t, _u64p, ctypes.c_size_t]
    lib.orc_output_bits.argtypes = [ctypes.c_int, _u64p, ctypes.c_int, ctypes.c_size_t, _u64p]
    lib.orc_poly_xpow.argtypes = [_u64p, ctypes.c_int, ctypes.c_char_p, ctypes.c_size_t, _u64p]
    lib.orc_poly_mulmod.argtypes = [_u64p, _u64p, _u64p, ctypes.c_int, _u64p]
    lib.orc_to_f64.argtypes = [ctypes.c_int, _u64p, ctypes.c_size_t,
                               ctypes.POINTER(ctypes.c_double)]
    lib.orc_to_f32.argtypes = [ctypes.c_int, _u64p, ctypes.c_size_t,
                               ctypes.POINTER(ctypes.c_float)]
    for fn in ("orc_matrix_from_step", "orc_matrix_from_blocks"):
        getattr(lib, fn).argtypes = [ctypes.c_int, _u64p]
    lib.orc_mat_mul.argtypes = [ctypes.c_int, _u64p, _u64p, _u64p]
    lib.orc_mat_vec.argtypes = [ctypes.c_int, _u64p, _u64p, _u64p]
    lib.orc_mat_rank.argtypes = [ctypes.c_int, _u64p]
    lib.orc_state_to_bits.argtypes = [ctypes.c_int, _u64p, _u64p]
    lib.orc_bits_to_state.argtypes = [ctypes.c_int, _u64p, _u64p]
    lib.orc_scramble.argtypes = [ctypes.c_int, _u64p, _u64p]
    lib.orc_zeroland.argtypes = [ctypes.c_int, ctypes.c_size_t, ctypes.c_size_t, _u64p]
    return lib


def _p(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_u64p)


@functools.lru_cache(maxsize=None)
def _index(name: str) -> int:
    lib = _lib()
    for i in range(lib.orc_num_generators()):
        if lib.orc_generator_name(i).decode() == name:
            return i
    raise KeyError(name)


def generator_names():
    lib = _lib()
    return [lib.orc_generator_name(i).decode() for i in range(lib.orc_num_generators())]


def word_bits(name: str) -> int:
    return _lib().orc_word_bits(_index(name))


def state_words(name: str) -> int:
    return _lib().orc_state_words(_index(name))


def state_bits(name: str) -> int:
    return _lib().orc_state_bits(_index(name))


def _nw(n: int) -> int:
    return (n + 63) // 64


# ---------------------------------------------------------------- generation

def splitmix64(seed: int, n: int) -> np.ndarray:
    out = np.zeros(n, np.uint64)
    _lib().orc_splitmix64(ctypes.c_uint64(seed & (2**64 - 1)), n, _p(out))
    return out


def seed(name: str, seed_value: int) -> np.ndarray:
    """State words of ``name`` filled from SplitMix64(seed) (Sec. 5.3)."""
    st = np.zeros(state_words(name), np.uint64)
    rc = _lib().orc_seed(_index(name), ctypes.c_uint64(seed_value & (2**64 - 1)), _p(st))
    if rc != 0:
        raise ValueError("all-zero state")
    return st


def generate(name: str, state: np.ndarray, n: int):
    """First ``n`` outputs from ``state``; returns (outputs, state after n steps)."""
    st = np.array(state, dtype=np.uint64, copy=True)
    out = np.zeros(n, np.uint64)
    _lib().orc_generate(_index(name), _p(st), n, _p(out))
    return out, st


def step(name: str, state: np.ndarray, nsteps: int = 1) -> np.ndarray:
    st = np.array(state, dtype=np.uint64, copy=True)
    _lib().orc_step(_index(name), _p(st), ctypes.c_uint64(nsteps))
    return st


def scramble(name: str, state: np.ndarray) -> int:
    st = np.ascontiguousarray(state, dtype=np.uint64)
    out = np.zeros(1, np.uint64)
    _lib().orc_scramble(_index(name), _p(st), _p(out))
    return int(out[0])


def fill_streams(name: str, starts: np.ndarray, m: int) -> np.ndarray:
    """out[i*m + j] = output j of the stream that starts at starts[i]."""
    st = np.ascontiguousarray(starts, dtype=np.uint64).reshape(-1, state_words(name))
    S = st.shape[0]
    out = np.zeros(S * m, np.uint64)
    _lib().orc_fill_streams(_index(name), _p(st), S, m, _p(out))
    return out


def to_f64(name: str, x: np.ndarray) -> np.ndarray:
    xx = np.ascontiguousarray(x, dtype=np.uint64)
    out = np.zeros(xx.size, np.float64)
    _lib().orc_to_f64(word_bits(name), _p(xx), xx.size,
                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def to_f32(name: str, x: np.ndarray) -> np.ndarray:
    xx = np.ascontiguousarray(x, dtype=np.uint64)
    out = np.zeros(xx.size, np.float32)
    _lib().orc_to_f32(word_bits(name), _p(xx), xx.size,
                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    return out


def convert(name: str, raw: np.ndarray, dtype: str) -> np.ndarray:
    """Raw outputs as the requested value type: 'native' (uint64 or uint32),
    'f64' or 'f32'."""
    if dtype == "native":
        return raw.astype(np.uint32) if word_bits(name) == 32 else raw
    if dtype == "f64":
        return to_f64(name, raw)
    if dtype == "f32":
        return to_f32(name, raw)
    raise ValueError(dtype)


# ---------------------------------------------------------------- F2 matrices

def matrix_from_step(name: str) -> np.ndarray:
    n = state_bits(name)
    T = np.zeros((n, _nw(n)), np.uint64)
    _lib().orc_matrix_from_step(_index(name), _p(T))
    return T


def matrix_from_blocks(name: str) -> np.ndarray:
    n = state_bits(name)
    T = np.zeros((n, _nw(n)), np.uint64)
    rc = _lib().orc_matrix_from_blocks(_index(name), _p(T))
    if rc != 0:
        raise ValueError("no printed block matrix for %s" % name)
    return T


def mat_mul(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    n = A.shape[0]
    C = np.zeros_like(A)
    _lib().orc_mat_mul(n, _p(np.ascontiguousarray(A)), _p(np.ascontiguousarray(B)), _p(C))
    return C


def mat_vec(A: np.ndarray, v: np.ndarray) -> np.ndarray:
    n = A.shape[0]
    out = np.zeros(_nw(n), np.uint64)
    _lib().orc_mat_vec(n, _p(np.ascontiguousarray(A)), _p(np.ascontiguousarray(v)), _p(out))
    return out


def mat_rank(A: np.ndarray) -> int:
    return _lib().orc_mat_rank(A.shape[0], _p(np.ascontiguousarray(A)))


def mat_identity(n: int) -> np.ndarray:
    Id = np.zeros((n, _nw(n)), np.uint64)
    for r in range(n):
        Id[r, r // 64] |= np.uint64(1 << (r % 64))
    return Id


def mat_pow(T: np.ndarray, e: int) -> np.ndarray:
    """T^e by binary powering."""
    R = mat_identity(T.shape[0])
    B = T.copy()
    while e:
        if e & 1:
            R = mat_mul(R, B)
        e >>= 1
        if e:
            B = mat_mul(B, B)
    return R


def mat_pow2(T: np.ndarray, k: int) -> np.ndarray:
    """T^(2^k) by k squarings."""
    B = T.copy()
    for _ in range(k):
        B = mat_mul(B, B)
    return B


def state_to_bits(name: str, state: np.ndarray) -> np.ndarray:
    v = np.zeros(_nw(state_bits(name)), np.uint64)
    _lib().orc_state_to_bits(_index(name), _p(np.ascontiguousarray(state, dtype=np.uint64)), _p(v))
    return v


def bits_to_state(name: str, v: np.ndarray) -> np.ndarray:
    st = np.zeros(state_words(name), np.uint64)
    _lib().orc_bits_to_state(_index(name), _p(np.ascontiguousarray(v, dtype=np.uint64)), _p(st))
    return st


# ---------------------------------------------------------------- polynomials

def _int_to_words(x: int, nw: int) -> np.ndarray:
    return np.array([(x >> (64 * i)) & (2**64 - 1) for i in range(nw)], dtype=np.uint64)


def _words_to_int(a: np.ndarray) -> int:
    return sum(int(v) << (64 * i) for i, v in enumerate(a))


_PW = 40  # words of a polynomial buffer in xr_oracle.c


def poly_xpow(p: int, e: int) -> int:
    """x^e mod p(x) over F2; polynomials are Python ints (bit i = coeff of x^i)."""
    nb = max(1, (e.bit_length() + 7) // 8)
    r = np.zeros(_PW, np.uint64)
    rc = _lib().orc_poly_xpow(_p(_int_to_words(p, _PW)), _PW, e.to_bytes(nb, "little"), nb, _p(r))
    if rc != 0:
        raise ValueError("bad modulus")
    return _words_to_int(r)


def poly_mulmod(a: int, b: int, p: int) -> int:
    r = np.zeros(_PW, np.uint64)
    _lib().orc_poly_mulmod(_p(_int_to_words(a, _PW)), _p(_int_to_words(b, _PW)),
                           _p(_int_to_words(p, _PW)), _PW, _p(r))
    return _words_to_int(r)


def output_bits(name: str, state: np.ndarray, bit: int, N: int) -> np.ndarray:
    st = np.array(state, dtype=np.uint64, copy=True)
    seq = np.zeros(N // 64 + 1, np.uint64)
    _lib().orc_output_bits(_index(name), _p(st), bit, N, _p(seq))
    return seq


def berlekamp_massey(seq: np.ndarray, N: int):
    """(L, C) with C(x) = 1 + c_1 x + ... + c_L x^L the shortest LFSR's
    connection polynomial (Python int)."""
    cap = N // 64 + 2
    conn = np.zeros(cap, np.uint64)
    L = _lib().orc_berlekamp_massey(_p(np.ascontiguousarray(seq, dtype=np.uint64)), N,
                                    _p(conn), cap)
    if L < 0:
        raise RuntimeError("berlekamp_massey failed")
    return int(L), _words_to_int(conn)


def linear_complexity(name: str, bit: int, N: int, seed_value: int = 1) -> int:
    seq = output_bits(name, seed(name, seed_value), bit, N)
    return berlekamp_massey(seq, N)[0]


def reciprocal(C: int, L: int) -> int:
    """x^L C(1/x): the characteristic polynomial of the recurrence."""
    return sum(1 << (L - i) for i in range(L + 1) if (C >> i) & 1)


@functools.lru_cache(maxsize=None)
def char_poly(name: str) -> int:
    """Characteristic polynomial of the engine of ``name`` by Berlekamp-Massey
    on bit 0 of the + output (Sec. 4.1 and Sec. 6)."""
    eng = ENGINE_OF.get(name, name)
    n = state_bits(eng)
    N = 2 * n + 64
    L, C = berlekamp_massey(output_bits(eng, seed(eng, 1), 0, N), N)
    return reciprocal(C, L)


def poly_weight(p: int) -> int:
    return bin(p).count("1")


# ---------------------------------------------------------------- jumps

def jump_log2(name: str, kind: str) -> int:
    """log2 of the jump distance: 2^(n/2) for 'jump', 2^(3n/4) for 'long'."""
    n = state_bits(ENGINE_OF.get(name, name))
    return {"jump": n // 2, "long": 3 * n // 4}[kind]


@functools.lru_cache(maxsize=None)
def jump_poly(name: str, log2_distance: int) -> int:
    """x^(2^d) mod p(x)."""
    return poly_xpow(char_poly(name), 1 << log2_distance)


def apply_poly(name: str, poly: int, state: np.ndarray) -> np.ndarray:
    """sum_i c_i T^i state, stepping the engine (Cayley-Hamilton jump)."""
    n = state_bits(ENGINE_OF.get(name, name))
    ncoef = max(n, poly.bit_length())
    coef = _int_to_words(poly, _nw(ncoef) + 1)
    st = np.array(state, dtype=np.uint64, copy=True)
    _lib().orc_apply_poly(_index(name), _p(coef), ncoef, _p(st))
    return st


def jump_pow(name: str, log2_distance: int, e: int, state: np.ndarray) -> np.ndarray:
    """T^(e * 2^d) state through x^(e * 2^d) mod p(x)."""
    if e == 0:
        return np.array(state, dtype=np.uint64, copy=True)
    return apply_poly(name, poly_xpow(char_poly(name), e << log2_distance), state)


def jump(name: str, kind: str, state: np.ndarray, times: int = 1) -> np.ndarray:
    """``times`` successive jumps (or long jumps), one after another."""
    d = jump_log2(name, kind)
    poly = jump_poly(name, d)
    st = np.array(state, dtype=np.uint64, copy=True)
    for _ in range(times):
        st = apply_poly(name, poly, st)
    return st


def advance(name: str, state: np.ndarray, nsteps: int) -> np.ndarray:
    return step(name, state, nsteps)


def streams(name: str, kind: str, base: np.ndarray, S: int, first: int = 0) -> np.ndarray:
    """Start states of S streams: row i = J^(first + i)(base), computed by one
    jump after another (after ``first`` jumps taken through x^(first * J))."""
    k = state_words(name)
    d = jump_log2(name, kind)
    b = jump_pow(name, d, first, base) if first else np.array(base, dtype=np.uint64)
    n = state_bits(ENGINE_OF.get(name, name))
    coef = _int_to_words(jump_poly(name, d), _nw(n) + 1)
    out = np.zeros((S, k), np.uint64)
    if S:
        _lib().orc_sequential_jumps(_index(name), _p(coef), n, _p(np.ascontiguousarray(b)), S,
                                    _p(out))
    return out


def bulk_fill(name: str, kind: str, base: np.ndarray, S: int, m: int, first: int = 0) -> np.ndarray:
    """Raw outputs of S streams x m values, stream i started at J^(first+i)(base)."""
    d = jump_log2(name, kind)
    b = jump_pow(name, d, first, base) if first else np.array(base, dtype=np.uint64)
    n = state_bits(ENGINE_OF.get(name, name))
    coef = _int_to_words(jump_poly(name, d), _nw(n) + 1)
    out = np.zeros(S * m, np.uint64)
    _lib().orc_bulk_fill(_index(name), _p(coef), n, _p(np.ascontiguousarray(b)), 0, S, m, _p(out))
    return out


def zeroland(name: str, nout: int = 1000, window: int = 4) -> np.ndarray:
    """Sec. 8: counts[t] = one bits in outputs t .. t+window-1, summed over the
    n states with exactly one bit set; the paper plots counts / (n window w)."""
    counts = np.zeros(nout - window + 1, np.uint64)
    if _lib().orc_zeroland(_index(name), nout, window, _p(counts)) != 0:
        raise ValueError("bad window")
    return counts
