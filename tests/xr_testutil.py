"""Helpers for the GPU parity tests: moving generator states and outputs
between the CUDA path (byte tensors on the device) and the oracle (uint64
word arrays), and bit-exact comparison."""
import numpy as np

import oracle as O


def word_dtype(name):
    return np.uint32 if O.word_bits(name) == 32 else np.uint64


def states_to_bytes(name, states):
    """oracle words [count, k] (uint64) -> the library's state bytes."""
    a = np.ascontiguousarray(np.asarray(states, dtype=np.uint64).reshape(-1, O.state_words(name)))
    return a.astype(word_dtype(name)).tobytes()


def bytes_to_states(name, b):
    return np.frombuffer(b, dtype=word_dtype(name)).astype(np.uint64).reshape(-1, O.state_words(name))


def states_to_device(name, states, device="cuda"):
    import torch
    b = states_to_bytes(name, states)
    return torch.frombuffer(bytearray(b), dtype=torch.uint8).to(device)


def states_from_device(name, t):
    return bytes_to_states(name, t.cpu().numpy().tobytes())


NP_OF = {"u64": np.uint64, "u32": np.uint32, "f64": np.float64, "f32": np.float32}


def out_to_numpy(t, dtype):
    return t.cpu().numpy().view(NP_OF[dtype])


def oracle_dtype(dtype):
    return "native" if dtype in ("u64", "u32") else dtype


def expected(name, raw, dtype):
    return np.asarray(O.convert(name, raw, oracle_dtype(dtype)), dtype=NP_OF[dtype])


def assert_bits_equal(got, want, what=""):
    got = np.ascontiguousarray(got)
    want = np.ascontiguousarray(want)
    assert got.shape == want.shape, (what, got.shape, want.shape)
    ib = {1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}[got.dtype.itemsize]
    g, w = got.view(ib), want.view(ib)
    bad = np.nonzero(g != w)[0]
    assert bad.size == 0, "%s: %d of %d differ; first at %d: got %r want %r" % (
        what, bad.size, g.size, bad[0], got[bad[0]], want[bad[0]])


def dense_from_oracle_rows(T):
    """oracle packed rows (bit c of row r) -> dense uint8 [n, n]."""
    n = T.shape[0]
    return np.unpackbits(T.view(np.uint8).reshape(n, -1), axis=1, bitorder="little")[:, :n]


def dense_from_library_columns(buf, n):
    """library column table (bit r of column c) -> dense uint8 [n, n] (row r, col c)."""
    cols = np.frombuffer(buf, dtype=np.uint8).reshape(n, n // 8)
    return np.unpackbits(cols, axis=1, bitorder="little")[:, :n].T.copy()
