"""A plain-Python model of the blocked Berlekamp-Massey kernel (Sec. 9.3;
csrc/xr_analysis.cu, k_berlekamp_massey), checked on the CPU against the
oracle's bit-serial Berlekamp-Massey.

The model keeps the kernel's data layout and shortcuts, so a flaw in them
fails here without a GPU: R contiguous words per thread, the lookahead read
from the packed reversed sequence at the kernel's indices (each index checked
against the buffer the kernel gets: the packed words plus 20 zero words), the
block recurrence on aligned 32-bit polynomials, the replay of the steps with
d = 1 only with X held as x^(u - tau) Y, one shadow word per thread started
from the word below at the block's start with zeros shifted in, and the live
bounds (asserted: every word above them is zero).  Sequences: random, an LFSR
of known length, all zero, a single one at either end, half zeros; lengths
that give partial first blocks, one and several warps."""
import random

import numpy as np
import pytest

import oracle as O

M32 = 0xFFFFFFFF
REV_PAD = 20


def _fsr(lo, hi, s):    # funnel shift right of hi:lo, s < 32
    return (((hi << 32) | lo) >> s) & M32


def _fsl(lo, hi, s):    # funnel shift left of hi:lo, s clamped to 32
    return ((((hi << 32) | lo) << min(s, 32)) >> 32) & M32


def _parity(x):
    return bin(x).count("1") & 1


def _brev(x):
    return int(format(x, "032b")[::-1], 2)


def blocked_bm(s, R):
    """L for the bits s (list of 0/1), or None where the kernel reports that the
    prefix cannot decide it (L reaching 32 W)."""
    N = len(s)
    W = N // 64 + 5
    rev = [0] * ((N + 31) // 32 + 2 + REV_PAD)
    for j in range(N):
        if s[N - 1 - j]:
            rev[j >> 5] |= 1 << (j & 31)
    T = ((W + R - 1) // R + 31) // 32 * 32
    nwords = T * R
    C = [0] * nwords
    Y = [0] * nwords
    C[0], Y[0] = 1, 2
    L = n = 0
    while n < N:
        k = ((N - 1 - n) & 31) + 1
        assert (N - 1 - n - (k - 1)) % 32 == 0
        q = (N - 1 - n - (k - 1)) >> 5
        D = max(L, n + 1 - L)
        assert all(C[w] == 0 and Y[w] == 0 for w in range(D // 32 + 1, nwords))
        eC = eX = 0
        for t in range(T):
            w0 = t * R
            if w0 > D // 32:
                continue
            assert q + w0 + R < len(rev)
            rv = rev[q + w0: q + w0 + R + 1]
            for u in range(k):
                ac = ax = 0
                for j in range(R):
                    win = _fsr(rv[j], rv[j + 1], k - 1 - u)
                    ac ^= C[w0 + j] & win
                    ax ^= Y[w0 + j] & win
                eC ^= _parity(ac) << u
                eX ^= _parity(ax) << u
        EC, EX = _brev(eC), _brev(eX)
        A, B, A2, B2 = 1 << 31, 0, 0, 1 << 31
        dm = gm = over = 0
        for u in range(k):
            dmask = M32 if _parity((A & EC) ^ (B & EX)) else 0
            gmask = dmask if 2 * L <= n + u else 0
            Lg = n + u + 1 - L
            over |= gmask and Lg >= 32 * W
            nA, nB = A ^ (A2 & dmask), B ^ (B2 & dmask)
            A2 = (A & gmask) | (A2 & ~gmask & M32)
            B2 = (B & gmask) | (B2 & ~gmask & M32)
            A, B = nA >> 1, nB >> 1
            if gmask:
                L = Lg
            dm |= (dmask & 1) << u
            gm |= (gmask & 1) << u
        if over:
            return None
        start = [(C[t * R - 1], Y[t * R - 1]) if t else (0, 0) for t in range(T)]
        for t in range(T):
            w0 = t * R
            if w0 > (D + 32) // 32:
                continue
            sC, sY = start[t]
            c, y = C[w0:w0 + R], Y[w0:w0 + R]
            ev, tau = dm, 0
            while ev:
                u = (ev & -ev).bit_length() - 1
                ev &= ev - 1
                dl = u - tau
                assert 0 <= dl < 32
                xw = [_fsl(y[j - 1] if j else sY, y[j], dl) for j in range(R)]
                sx = (sY << dl) & M32
                if (gm >> u) & 1:
                    y = c[:]
                    sC, sY = sC ^ sx, sC
                    tau = u
                else:
                    sC ^= sx
                c = [c[j] ^ xw[j] for j in range(R)]
            y = [_fsl(y[j - 1] if j else sY, y[j], k - tau) for j in range(R)]
            C[w0:w0 + R], Y[w0:w0 + R] = c, y
        n += k
    return L


def _oracle_L(s):
    N = len(s)
    words = np.zeros(N // 64 + 1, np.uint64)
    for i, b in enumerate(s):
        if b:
            words[i // 64] |= np.uint64(1) << np.uint64(i % 64)
    return O.berlekamp_massey(words, N)[0]


def _sequences(N, rnd):
    d = max(1, N // 3)
    lfsr = [rnd.getrandbits(1) for _ in range(d)]
    taps = sorted({0, d // 2, d - 1})
    while len(lfsr) < N:
        bit = 0
        for tp in taps:
            bit ^= lfsr[-d + tp]
        lfsr.append(bit)
    return {"random": [rnd.getrandbits(1) for _ in range(N)], "lfsr": lfsr[:N], "zeros": [0] * N,
            "last_one": [0] * (N - 1) + [1], "first_one": [1] + [0] * (N - 1),
            "half_zeros": [0] * (N // 2) + [rnd.getrandbits(1) for _ in range(N - N // 2)]}


@pytest.mark.parametrize("R,N", [(1, 2), (1, 3), (12, 33), (12, 64), (2, 200), (8, 777), (12, 1031),
                                 (1, 2500), (2, 4500)])
def test_blocked_model_matches_bit_serial(R, N):
    rnd = random.Random(1000 * R + N)
    W = N // 64 + 5
    for kind, s in _sequences(N, rnd).items():
        want = _oracle_L(s)
        got = blocked_bm(s, R)
        if want >= 32 * W:
            assert got is None, (kind, R, N, want, got)
        else:
            assert got == want, (kind, R, N, want, got)


def test_model_covers_several_warps():
    """The (1, 2500) and (2, 4500) cases span two warps (W / R > 32), so the
    shadow of a warp's first lane comes from the previous warp."""
    for R, N in ((1, 2500), (2, 4500)):
        W = N // 64 + 5
        assert (W + R - 1) // R > 32
