"""Bulk generation from scrambled linear pseudorandom generators on GB300.

Thin Python binding of libxr (C ABI in include/xr.h).  Every computation runs
in the library's CUDA kernels; this module only marshals torch tensors
(device memory), CUDA streams and sizes into the C calls, checks that every
buffer is large enough for the call, and turns status codes into exceptions.
There is no CPU fallback: if libxr.so is missing the import of the native
library fails loudly.

Generators (Blackman & Vigna, arXiv 1805.01407): xoshiro256+/++/**,
xoroshiro128+/++/**/*, xoshiro512+/++/**, xoroshiro1024*/++/** (64-bit words),
xoshiro128++/**/+ and xoroshiro64*/** (32-bit words).
"""
from __future__ import annotations

import ctypes
import os
import struct

__all__ = ["Context", "XRError", "VARIANTS", "DTYPES", "state_words", "word_bits", "state_bytes",
           "state_bits", "jump_log2", "lib", "library_path"]

_PKG = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_PKG, "libxr.so")

VARIANTS = {
    "xoshiro256+": 0, "xoshiro256++": 1, "xoshiro256**": 2,
    "xoroshiro128+": 3, "xoroshiro128++": 4, "xoroshiro128**": 5,
    "xoshiro128++": 6, "xoshiro128**": 7, "xoshiro128+": 8,
    "xoroshiro128*": 9, "xoroshiro64*": 10, "xoroshiro64**": 11,
    "xoshiro512+": 12, "xoshiro512++": 13, "xoshiro512**": 14,
    "xoroshiro1024*": 15, "xoroshiro1024++": 16, "xoroshiro1024**": 17,
}
DTYPES = {"u64": 0, "u32": 1, "f64": 2, "f32": 3}
LAYOUTS = {"stream": 0, "interleaved": 1}
KINDS = {"jump": 0, "long": 1}

XR_OK, XR_EINVAL, XR_EZERO_STATE, XR_ENOMEM, XR_ECUDA, XR_ETIMEOUT, XR_EUNSUPPORTED = range(7)
XR_LC_MAX_BITS = 786000  # longest prefix xr_linear_complexity accepts

_lib = None


class ServerConfig(ctypes.Structure):
    """xr_server_config of include/xr.h."""
    _fields_ = [("arena_bytes", ctypes.c_uint64), ("nclients", ctypes.c_uint32),
                ("max_rounds", ctypes.c_uint32), ("max_round_requests", ctypes.c_uint32),
                ("mode", ctypes.c_int), ("outputs_per_row", ctypes.c_int), ("block", ctypes.c_int)]


class ServeStats(ctypes.Structure):
    """xr_serve_stats of include/xr.h."""
    _fields_ = [(f, ctypes.c_uint64) for f in ("submitted", "completed", "released", "rounds", "bytes",
                                                "arena_in_use", "arena_peak", "queue_ns", "launch_ns", "device_ns")]


class Request(ctypes.Structure):
    """xr_request of include/xr.h."""
    _fields_ = [("variant", ctypes.c_int), ("dtype", ctypes.c_int), ("n", ctypes.c_uint64),
                ("slot", ctypes.c_uint64), ("out_offset", ctypes.c_uint64)]


class LcJob(ctypes.Structure):
    """xr_lc_job of include/xr.h."""
    _fields_ = [("variant", ctypes.c_int32), ("bit", ctypes.c_int32), ("N", ctypes.c_uint64)]


_LC_RECORD = struct.Struct("<iiQ")  # one LcJob
assert _LC_RECORD.size == ctypes.sizeof(LcJob)


class XRError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, _err(status), status))


def _err(status):
    return lib().xr_error_string(status).decode()


def lib():
    """The loaded libxr.so (built by __graft_entry__.build() or
    `python -m paper_1805_01407_gb300.build`)."""
    global _lib
    if _lib is None:
        if not os.path.exists(library_path):
            raise ImportError("libxr.so is not built (%s); run `python -m paper_1805_01407_gb300.build`"
                              % library_path)
        L = ctypes.CDLL(library_path)
        vp, sz, u64, i = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_int
        sigs = {
            "xr_ctx_create": [i, ctypes.POINTER(vp)],
            "xr_ctx_destroy": [vp],
            "xr_state_words": [i], "xr_word_bits": [i], "xr_state_bytes": [i], "xr_state_bits": [i],
            "xr_dtype_bytes": [i], "xr_variant_name": [i], "xr_error_string": [i],
            "xr_jump_log2": [i, i],
            "xr_seed": [vp, i, u64, vp, vp],
            "xr_seed_many": [vp, i, vp, sz, vp, vp],
            "xr_set_state": [vp, i, vp, vp, vp],
            "xr_get_state": [vp, i, vp, vp, vp],
            "xr_jump": [vp, i, i, vp, sz, u64, vp],
            "xr_advance": [vp, i, vp, sz, u64, vp],
            "xr_make_streams": [vp, i, i, vp, u64, sz, vp, vp],
            "xr_fill": [vp, i, vp, sz, sz, i, i, vp, i, vp],
            "xr_fill_seq": [vp, i, vp, sz, i, vp, vp],
            "xr_fill_streams": [vp, i, i, vp, u64, sz, sz, i, vp, vp],
            "xr_fill_host": [vp, i, i, vp, u64, sz, sz, i, vp, vp],
            "xr_status": [vp, i],
            "xr_jump_table": [vp, i, i, vp],
            "xr_probe_store": [vp, sz, i, vp],
            "xr_probe_memset": [vp, sz, vp],
            "xr_probe_alu": [vp, i, i, vp],
            "xr_probe_tile_store": [vp, sz, sz, i, vp],
        }
        L.xr_launch_count.argtypes = []
        L.xr_launch_count.restype = ctypes.c_uint64
        L.xr_batch_create.argtypes = [vp, ctypes.POINTER(Request), sz, ctypes.POINTER(vp)]
        L.xr_batch_create.restype = i
        L.xr_batch_destroy.argtypes = [vp]
        L.xr_batch_destroy.restype = i
        L.xr_batch_arena_bytes.argtypes = [vp]
        L.xr_batch_arena_bytes.restype = ctypes.c_uint64
        L.xr_batch_tasks.argtypes = [vp]
        L.xr_batch_tasks.restype = ctypes.c_uint64
        L.xr_batch_slot_bytes.argtypes = [vp]
        L.xr_batch_slot_bytes.restype = ctypes.c_uint64
        L.xr_batch_run.argtypes = [vp, vp, vp, vp, i, vp]
        L.xr_batch_run.restype = i
        L.xr_batch_set_config.argtypes = [vp, i, i]
        L.xr_batch_set_config.restype = i
        L.xr_batch_get_config.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.xr_batch_get_config.restype = i
        L.xr_batch_tune.argtypes = [vp, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_float)]
        L.xr_batch_tune.restype = i
        dp = ctypes.POINTER(ctypes.c_double)
        L.xr_server_create.argtypes = [vp, ctypes.POINTER(ServerConfig), ctypes.POINTER(i),
                                       ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(vp)]
        L.xr_server_destroy.argtypes = [vp]
        L.xr_server_submit.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint64, i, ctypes.POINTER(ctypes.c_uint64)]
        L.xr_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), dp]
        L.xr_server_wait_for.argtypes = [vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_uint64), dp]
        L.xr_server_release.argtypes = [vp, ctypes.c_uint64]
        L.xr_server_arena.argtypes = [vp]
        L.xr_server_arena.restype = vp
        L.xr_server_read.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64, vp, vp]
        L.xr_server_client_state.argtypes = [vp, ctypes.c_uint32, vp]
        L.xr_server_stats.argtypes = [vp, ctypes.POINTER(ServeStats)]
        L.xr_server_replay.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64),
                                       ctypes.POINTER(i), sz, dp, dp]
        L.xr_zeroland.argtypes = [vp, i, sz, sz, vp, vp]
        L.xr_zeroland.restype = i
        L.xr_linear_complexity.argtypes = [vp, i, i, sz, vp, vp, sz, ctypes.POINTER(ctypes.c_uint64), vp]
        L.xr_linear_complexity.restype = i
        L.xr_lc_scratch_bytes.argtypes = [ctypes.POINTER(LcJob), sz]
        L.xr_lc_scratch_bytes.restype = sz
        L.xr_linear_complexity_many.argtypes = [vp, ctypes.POINTER(LcJob), sz, vp, sz, vp, sz,
                                                ctypes.POINTER(ctypes.c_uint64), vp]
        L.xr_linear_complexity_many.restype = i
        for fn in ("xr_server_create", "xr_server_destroy", "xr_server_submit", "xr_server_wait", "xr_server_wait_for",
                   "xr_server_release", "xr_server_read", "xr_server_client_state", "xr_server_stats",
                   "xr_server_replay"):
            getattr(L, fn).restype = i
        for name, args in sigs.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = i
        L.xr_variant_name.restype = ctypes.c_char_p
        L.xr_error_string.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _v(variant):
    if isinstance(variant, str):
        return VARIANTS[variant]
    return int(variant)


_PROPERTIES = {}


def _property(name, variant):
    """A pure property of a generator from libxr, asked once per (property,
    variant): the per-job checks of a call with hundreds of jobs would
    otherwise cost a foreign call each."""
    key = (name, _v(variant))
    value = _PROPERTIES.get(key)
    if value is None:
        value = _PROPERTIES[key] = getattr(lib(), name)(key[1])
    return value


def state_words(variant):
    return _property("xr_state_words", variant)


def word_bits(variant):
    return _property("xr_word_bits", variant)


def state_bytes(variant):
    return _property("xr_state_bytes", variant)


def state_bits(variant):
    return _property("xr_state_bits", variant)


def jump_log2(variant, kind="jump"):
    return lib().xr_jump_log2(_v(variant), KINDS[kind])


def launch_count():
    """Kernels launched through libxr by this process so far."""
    return lib().xr_launch_count()


def probe_store(d_buf, ctas_per_sm=0, stream=None):
    """Store-only kernel over all of d_buf (include/xr_probe.h)."""
    _need(d_buf, 16, "d_buf")
    _check(lib().xr_probe_store(d_buf.data_ptr(), _nbytes(d_buf) // 16 * 16, ctas_per_sm, _stream(stream)),
           "xr_probe_store")


def probe_tile_store(d_buf, rows, row_bytes, config=0, stream=None):
    """The fill's tile-store pattern over rows x row_bytes of d_buf, nothing
    generated (include/xr_probe.h); config 0, 1, 2 = 2 warps x 6 tiles,
    1 x 8, 1 x 3."""
    _need(d_buf, rows * row_bytes, "d_buf")
    _check(lib().xr_probe_tile_store(d_buf.data_ptr(), rows, row_bytes, config, _stream(stream)),
           "xr_probe_tile_store")


def probe_memset(d_buf, stream=None):
    """cudaMemsetAsync over all of d_buf (include/xr_probe.h)."""
    _need(d_buf, 1, "d_buf")
    _check(lib().xr_probe_memset(d_buf.data_ptr(), _nbytes(d_buf), _stream(stream)), "xr_probe_memset")


def probe_alu(d_sink, blocks, iters, stream=None):
    """blocks x 256 threads x iters x 16 lop3 lane operations (include/xr_probe.h)."""
    _need(d_sink, 4, "d_sink")
    _check(lib().xr_probe_alu(d_sink.data_ptr(), blocks, iters, _stream(stream)), "xr_probe_alu")


def dtype_bytes(dtype):
    return lib().xr_dtype_bytes(DTYPES[dtype])


def native_dtype(variant):
    return "u64" if word_bits(variant) == 64 else "u32"


def _check(rc, what):
    if rc != XR_OK:
        raise XRError(rc, what)


def _nbytes(t):
    return t.numel() * t.element_size()


def _need(t, nbytes, what):
    """The tensor must be contiguous, on the GPU, and hold `nbytes`."""
    if nbytes == 0:
        return
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % what)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    if _nbytes(t) < nbytes:
        raise ValueError("%s holds %d bytes, the call needs %d" % (what, _nbytes(t), nbytes))


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def torch_dtype(dtype):
    import torch
    return {"u64": torch.int64, "u32": torch.int32, "f64": torch.float64, "f32": torch.float32}[dtype]


class Context:
    """A libxr context on one device: jump tables, status word, scratch.

    Method names follow the C ABI (xr_seed -> seed, xr_fill -> fill, ...).
    States are uint8/int32/int64 CUDA tensors holding `state_bytes(variant)`
    bytes per state; outputs are CUDA tensors of the dtype's width (u64 as
    torch.int64 bit patterns, u32 as torch.int32, f64, f32).
    """

    def __init__(self, device=0):
        import torch
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        torch.cuda.set_device(self.device)
        h = ctypes.c_void_p()
        _check(lib().xr_ctx_create(self.device.index or 0, ctypes.byref(h)), "xr_ctx_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().xr_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    # -------------------------------------------------------------- helpers
    def empty_states(self, variant, count):
        import torch
        return torch.zeros(count * state_bytes(variant), dtype=torch.uint8, device=self.device)

    def empty_output(self, count, dtype):
        import torch
        return torch.empty(count, dtype=torch_dtype(dtype), device=self.device)

    # -------------------------------------------------------------- C calls
    def seed(self, variant, seed, d_state, stream=None):
        _need(d_state, state_bytes(variant), "d_state")
        _check(lib().xr_seed(self._h, _v(variant), seed & (2**64 - 1), d_state.data_ptr(),
                             _stream(stream)), "xr_seed")

    def seed_many(self, variant, d_seeds, d_states, stream=None):
        count = d_seeds.numel()
        _need(d_seeds, count * 8, "d_seeds")
        _need(d_states, count * state_bytes(variant), "d_states")
        _check(lib().xr_seed_many(self._h, _v(variant), d_seeds.data_ptr(), count,
                                  d_states.data_ptr(), _stream(stream)), "xr_seed_many")

    def set_state(self, variant, words, d_state, stream=None):
        """words: bytes-like holding one state (little-endian words)."""
        b = bytes(words)
        if len(b) != state_bytes(variant):
            raise ValueError("state must be %d bytes" % state_bytes(variant))
        _need(d_state, len(b), "d_state")
        buf = ctypes.create_string_buffer(b, len(b))
        _check(lib().xr_set_state(self._h, _v(variant), buf, d_state.data_ptr(), _stream(stream)),
               "xr_set_state")

    def get_state(self, variant, d_state, stream=None) -> bytes:
        n = state_bytes(variant)
        _need(d_state, n, "d_state")
        buf = ctypes.create_string_buffer(n)
        _check(lib().xr_get_state(self._h, _v(variant), d_state.data_ptr(), buf, _stream(stream)),
               "xr_get_state")
        return buf.raw

    def jump(self, variant, kind, d_states, count, times=1, stream=None):
        _need(d_states, count * state_bytes(variant), "d_states")
        _check(lib().xr_jump(self._h, _v(variant), KINDS[kind], d_states.data_ptr(), count, times,
                             _stream(stream)), "xr_jump")

    def advance(self, variant, d_states, count, nsteps, stream=None):
        _need(d_states, count * state_bytes(variant), "d_states")
        _check(lib().xr_advance(self._h, _v(variant), d_states.data_ptr(), count, nsteps,
                                _stream(stream)), "xr_advance")

    def make_streams(self, variant, kind, d_base, first, S, d_states_out, stream=None):
        _need(d_base, state_bytes(variant), "d_base")
        _need(d_states_out, S * state_bytes(variant), "d_states_out")
        _check(lib().xr_make_streams(self._h, _v(variant), KINDS[kind], d_base.data_ptr(), first, S,
                                     d_states_out.data_ptr(), _stream(stream)), "xr_make_streams")

    def fill(self, variant, d_states, S, m, dtype, d_out, layout="stream", write_back=False,
             stream=None):
        _need(d_states, S * state_bytes(variant), "d_states")
        _need(d_out, S * m * dtype_bytes(dtype), "d_out")
        _check(lib().xr_fill(self._h, _v(variant), d_states.data_ptr(), S, m, DTYPES[dtype],
                             LAYOUTS[layout], d_out.data_ptr(), int(bool(write_back)),
                             _stream(stream)), "xr_fill")

    def fill_streams(self, variant, kind, d_base, first, S, m, dtype, d_out, stream=None):
        _need(d_base, state_bytes(variant), "d_base")
        _need(d_out, S * m * dtype_bytes(dtype), "d_out")
        _check(lib().xr_fill_streams(self._h, _v(variant), KINDS[kind], d_base.data_ptr(), first, S, m,
                                     DTYPES[dtype], d_out.data_ptr(), _stream(stream)), "xr_fill_streams")

    def fill_seq(self, variant, d_state, n, dtype, d_out, stream=None):
        _need(d_state, state_bytes(variant), "d_state")
        _need(d_out, n * dtype_bytes(dtype), "d_out")
        _check(lib().xr_fill_seq(self._h, _v(variant), d_state.data_ptr(), n, DTYPES[dtype],
                                 d_out.data_ptr(), _stream(stream)), "xr_fill_seq")

    def fill_host(self, variant, kind, base_words, first, S, m, dtype, h_out, stream=None):
        """h_out: a CPU tensor (pinned for full speed) of >= S*m elements."""
        b = bytes(base_words)
        if len(b) != state_bytes(variant):
            raise ValueError("state must be %d bytes" % state_bytes(variant))
        if h_out.is_cuda or not h_out.is_contiguous() or _nbytes(h_out) < S * m * dtype_bytes(dtype):
            raise ValueError("h_out must be a contiguous host tensor of S*m elements")
        buf = ctypes.create_string_buffer(b, len(b))
        _check(lib().xr_fill_host(self._h, _v(variant), KINDS[kind], buf, first, S, m, DTYPES[dtype],
                                  h_out.data_ptr(), _stream(stream)), "xr_fill_host")

    def zeroland(self, variant, nout=1000, window=4, stream=None):
        """Sec. 8 escaping-zeroland counts (a CUDA int64 tensor of nout-window+1
        entries, one bits per window summed over all one-bit states)."""
        import torch
        out = torch.empty(nout - window + 1, dtype=torch.int64, device=self.device)
        _check(lib().xr_zeroland(self._h, _v(variant), nout, window, out.data_ptr(), _stream(stream)),
               "xr_zeroland")
        return out

    def linear_complexity(self, variant, bit, N, d_state, stream=None):
        """Sec. 9.3 linear complexity (Berlekamp-Massey over F2) of bit `bit`
        of the first N outputs from the state in d_state (not advanced)."""
        import torch
        _need(d_state, state_bytes(variant), "d_state")
        job = LcJob(_v(variant), bit, N)
        nbytes = lib().xr_lc_scratch_bytes(ctypes.byref(job), 1)
        scratch = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=self.device)
        L = ctypes.c_uint64(0)
        _check(lib().xr_linear_complexity(self._h, _v(variant), bit, N, d_state.data_ptr(), scratch.data_ptr(),
                                          nbytes, ctypes.byref(L), _stream(stream)), "xr_linear_complexity")
        return L.value

    def linear_complexity_many(self, jobs, d_states, state_stride=128, stream=None):
        """Linear complexities of many (variant, bit, N) jobs in one call; job
        j reads its state at byte j * state_stride of d_states.  Returns a list
        of ints, None where N bits cannot decide the complexity."""
        import torch
        # the records packed in one pass (xr_lc_job: int32 variant, int32 bit, uint64 N)
        arr = (LcJob * max(len(jobs), 1)).from_buffer_copy(
            b"".join([_LC_RECORD.pack(_v(v), b, n) for (v, b, n) in jobs]) or bytes(ctypes.sizeof(LcJob)))
        sb = {v: state_bytes(v) for v in {v for (v, _, _) in jobs}}
        if state_stride % 16 or any(state_stride < sb[v] for v in {v for (v, _, _) in jobs[:-1]}):
            raise ValueError("state_stride must be a multiple of 16 and hold every state")
        # every state but the last fits its stride, so the last one ends furthest
        _need(d_states, (len(jobs) - 1) * state_stride + sb[jobs[-1][0]] if jobs else 0, "d_states")
        nbytes = lib().xr_lc_scratch_bytes(arr, len(jobs))
        scratch = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=self.device)
        out = (ctypes.c_uint64 * max(len(jobs), 1))()
        _check(lib().xr_linear_complexity_many(self._h, arr, len(jobs), d_states.data_ptr(), state_stride,
                                               scratch.data_ptr(), nbytes, out, _stream(stream)),
               "xr_linear_complexity_many")
        return [None if out[j] == 2**64 - 1 else int(out[j]) for j in range(len(jobs))]

    def status(self, reset=False):
        return lib().xr_status(self._h, int(bool(reset)))

    def jump_table(self, variant, k) -> bytes:
        n = state_bits(variant)
        buf = ctypes.create_string_buffer(n * n // 8)
        _check(lib().xr_jump_table(self._h, _v(variant), k, buf), "xr_jump_table")
        return buf.raw


def pack_requests(specs, align=None):
    """Lay out requests in one output arena.

    specs: iterable of (variant, dtype, n[, slot]); slot defaults to the
    request's index.  Returns (list of Request, list of byte offsets, arena
    bytes).  By default every request starts on a boundary of 1024 of its
    elements, which lets the batch write whole 1024-output segments with
    tile stores; `align` (a multiple of 16) overrides that."""
    reqs, offs, off = [], [], 0
    for r, spec in enumerate(specs):
        v, dt, n = spec[0], spec[1], int(spec[2])
        slot = int(spec[3]) if len(spec) > 3 else r
        a = align or 1024 * dtype_bytes(dt)
        off = (off + a - 1) // a * a
        reqs.append(Request(_v(v), DTYPES[dt], n, slot, off))
        offs.append(off)
        off += n * dtype_bytes(dt)
    a = align or 8192
    return reqs, offs, (off + a - 1) // a * a


class Batch:
    """Many uneven requests in one persistent launch (xr_batch_*)."""

    def __init__(self, ctx, requests):
        self.ctx = ctx
        arr = (Request * len(requests))(*requests)
        h = ctypes.c_void_p()
        _check(lib().xr_batch_create(ctx.handle, arr, len(requests), ctypes.byref(h)), "xr_batch_create")
        self._h = h
        self.nreq = len(requests)
        self.max_slot = max((r.slot for r in requests), default=0)

    @property
    def arena_bytes(self):
        return lib().xr_batch_arena_bytes(self._h)

    @property
    def tasks(self):
        return lib().xr_batch_tasks(self._h)

    @property
    def slot_bytes(self):
        """Bytes per state slot: 32, or 64 / 128 with xoshiro512 / xoroshiro1024 requests."""
        return lib().xr_batch_slot_bytes(self._h)

    def _args(self, d_seeds, d_slots, d_out):
        if d_seeds is not None:
            _need(d_seeds, self.nreq * 8, "d_seeds")
        _need(d_slots, (self.max_slot + 1) * self.slot_bytes, "d_slots")
        if self.arena_bytes:
            _need(d_out, self.arena_bytes, "d_out")
        return (ctypes.c_void_p(d_seeds.data_ptr() if d_seeds is not None else None),
                ctypes.c_void_p(d_slots.data_ptr()), ctypes.c_void_p(d_out.data_ptr() if d_out is not None else None))

    def run(self, d_seeds, d_slots, d_out, use_graph=False, stream=None):
        a = self._args(d_seeds, d_slots, d_out)
        _check(lib().xr_batch_run(self._h, *a, int(bool(use_graph)), _stream(stream)), "xr_batch_run")

    def tune(self, d_seeds, d_slots, d_out, stream=None):
        a = self._args(d_seeds, d_slots, d_out)
        ms = ctypes.c_float()
        _check(lib().xr_batch_tune(self._h, *a, _stream(stream), ctypes.byref(ms)), "xr_batch_tune")
        return ms.value

    def set_config(self, outputs_per_row, block):
        _check(lib().xr_batch_set_config(self._h, outputs_per_row, block), "xr_batch_set_config")

    def get_config(self):
        o, b = ctypes.c_int(), ctypes.c_int()
        _check(lib().xr_batch_get_config(self._h, ctypes.byref(o), ctypes.byref(b)), "xr_batch_get_config")
        return o.value, b.value

    def close(self):
        if getattr(self, "_h", None):
            lib().xr_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SERVE_MODES = {"batched": 0, "plain": 1}


class Server:
    """Continuous batching for many clients with device-resident states
    (xr_server_*).  client_variants / client_seeds: one entry per client."""

    def __init__(self, ctx, client_variants, client_seeds, arena_bytes, mode="batched", max_rounds=3,
                 max_round_requests=4096, outputs_per_row=0, block=0):
        n = len(client_variants)
        cfg = ServerConfig(arena_bytes, n, max_rounds, max_round_requests, SERVE_MODES[mode], outputs_per_row,
                           block)
        var = (ctypes.c_int * n)(*[_v(v) for v in client_variants])
        seeds = (ctypes.c_uint64 * n)(*[int(x) & (2**64 - 1) for x in client_seeds])
        h = ctypes.c_void_p()
        _check(lib().xr_server_create(ctx.handle, ctypes.byref(cfg), var, seeds, ctypes.byref(h)),
               "xr_server_create")
        self._h = h
        self.ctx = ctx
        self.client_variants = list(client_variants)

    def submit(self, client, n, dtype):
        t = ctypes.c_uint64()
        _check(lib().xr_server_submit(self._h, client, n, DTYPES[dtype], ctypes.byref(t)), "xr_server_submit")
        return t.value

    def wait(self, ticket, timeout_us=None):
        """(arena offset, latency in us) once the request is complete; with
        timeout_us, None when it is not complete within that host time."""
        off, lat = ctypes.c_uint64(), ctypes.c_double()
        if timeout_us is None:
            _check(lib().xr_server_wait(self._h, ticket, ctypes.byref(off), ctypes.byref(lat)), "xr_server_wait")
            return off.value, lat.value
        rc = lib().xr_server_wait_for(self._h, ticket, float(timeout_us), ctypes.byref(off), ctypes.byref(lat))
        if rc == XR_ETIMEOUT:
            return None
        _check(rc, "xr_server_wait_for")
        return off.value, lat.value

    def release(self, ticket):
        _check(lib().xr_server_release(self._h, ticket), "xr_server_release")

    def read(self, offset, nbytes, dst, stream=None):
        """Copy arena bytes into a tensor (host or device) of >= nbytes."""
        if _nbytes(dst) < nbytes or not dst.is_contiguous():
            raise ValueError("dst too small")
        _check(lib().xr_server_read(self._h, offset, nbytes, dst.data_ptr(), _stream(stream)), "xr_server_read")

    def client_state(self, client):
        nb = state_bytes(self.client_variants[client])
        buf = ctypes.create_string_buffer(max(nb, 32))
        _check(lib().xr_server_client_state(self._h, client, buf), "xr_server_client_state")
        return buf.raw[:nb]

    def stats(self):
        st = ServeStats()
        _check(lib().xr_server_stats(self._h, ctypes.byref(st)), "xr_server_stats")
        return {f: getattr(st, f) for f, _ in ServeStats._fields_}

    def replay(self, arrival_us, clients, ns, dtypes):
        """Submit request i at arrival_us[i] (us after the call starts), release
        each output on completion; returns (latencies in us, wall time in us)."""
        import numpy as np
        n = len(ns)
        arr = np.ascontiguousarray(arrival_us, dtype=np.float64)
        cl = np.ascontiguousarray(clients, dtype=np.uint32)
        nn = np.ascontiguousarray(ns, dtype=np.uint64)
        dt = np.ascontiguousarray([DTYPES[d] if isinstance(d, str) else int(d) for d in dtypes], dtype=np.int32)
        lat = np.zeros(n, dtype=np.float64)
        wall = ctypes.c_double()
        dp = ctypes.POINTER(ctypes.c_double)
        _check(lib().xr_server_replay(self._h, arr.ctypes.data_as(dp), cl.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                      nn.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                      dt.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), n, lat.ctypes.data_as(dp),
                                      ctypes.byref(wall)), "xr_server_replay")
        return lat, wall.value

    def close(self):
        if getattr(self, "_h", None):
            lib().xr_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
