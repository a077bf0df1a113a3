"""libxr.so builds here (nvcc cross-compiles sm_103a), loads without a GPU and
exports every entry point include/xr.h declares; the pure host functions and
the argument checks work without a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libxr():
    from paper_1805_01407_gb300 import build
    build.build()
    import paper_1805_01407_gb300 as xr
    return xr.lib()


def header_functions():
    """Every function declared in include/*.h."""
    names = set()
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            text = open(os.path.join(inc, h)).read()
            names |= set(re.findall(r"^\s*(?:int|uint64_t|size_t|void \*|const char \*)\s*(xr_\w+)\s*\(", text, re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("xr_ctx_create", "xr_ctx_destroy", "xr_seed", "xr_set_state", "xr_get_state",
                     "xr_jump", "xr_advance", "xr_make_streams", "xr_fill", "xr_fill_seq",
                     "xr_fill_host", "xr_status", "xr_error_string"):
        assert required in names


def test_binding_constants_match_the_header():
    import paper_1805_01407_gb300 as xr
    text = open(os.path.join(ROOT, "include", "xr.h")).read()
    assert int(re.search(r"#define XR_LC_MAX_BITS \(\(size_t\)(\d+)\)", text).group(1)) == xr.XR_LC_MAX_BITS
    assert int(re.search(r"XR_NUM_VARIANTS\s*=\s*(\d+)", text).group(1)) == len(xr.VARIANTS)


def test_lc_scratch_macro_matches_the_library(libxr):
    """XR_LC_SCRATCH_BYTES(N) (header) is what xr_lc_scratch_bytes gives for one job."""
    import paper_1805_01407_gb300 as xr
    text = open(os.path.join(ROOT, "include", "xr.h")).read()
    expr = re.search(r"#define XR_LC_SCRATCH_BYTES\(N\) (.+)", text).group(1).replace("/", "//")
    for N in (2, 31, 32, 33, 1000, 65992, 699464, 786000):
        job = xr.LcJob(0, 0, N)
        assert libxr.xr_lc_scratch_bytes(ctypes.byref(job), 1) == eval(expr.replace("(N)", "(%d)" % N))
    jobs = (xr.LcJob * 3)(xr.LcJob(0, 0, 100), xr.LcJob(3, 1, 5000), xr.LcJob(7, 2, 77))
    one = [libxr.xr_lc_scratch_bytes(ctypes.byref(jobs[k]), 1) for k in range(3)]
    assert libxr.xr_lc_scratch_bytes(jobs, 3) > max(one)


def test_every_declared_symbol_is_exported(libxr):
    for name in header_functions():
        assert hasattr(libxr, name), name


def test_properties(libxr):
    import paper_1805_01407_gb300 as xr
    expect = {  # (state words, word bits, state bits)
        "xoshiro256+": (4, 64, 256), "xoshiro256++": (4, 64, 256), "xoshiro256**": (4, 64, 256),
        "xoroshiro128+": (2, 64, 128), "xoroshiro128++": (2, 64, 128), "xoroshiro128**": (2, 64, 128),
        "xoshiro128++": (4, 32, 128), "xoshiro128**": (4, 32, 128), "xoshiro128+": (4, 32, 128),
        "xoroshiro128*": (2, 64, 128), "xoroshiro64*": (2, 32, 64), "xoroshiro64**": (2, 32, 64),
        "xoshiro512+": (8, 64, 512), "xoshiro512++": (8, 64, 512), "xoshiro512**": (8, 64, 512),
        "xoroshiro1024*": (16, 64, 1024), "xoroshiro1024++": (16, 64, 1024), "xoroshiro1024**": (16, 64, 1024),
    }
    for name, v in xr.VARIANTS.items():
        assert libxr.xr_variant_name(v).decode() == name
        assert (xr.state_words(name), xr.word_bits(name), xr.state_bits(name)) == expect[name]
        assert xr.state_bytes(name) == expect[name][0] * expect[name][1] // 8
        n = expect[name][2]
        assert xr.jump_log2(name, "jump") == n // 2 and xr.jump_log2(name, "long") == 3 * n // 4
    assert libxr.xr_state_words(99) == -1 and libxr.xr_variant_name(-1) is None
    assert [libxr.xr_dtype_bytes(d) for d in range(4)] == [8, 4, 8, 4]
    for s in range(8):
        assert libxr.xr_error_string(s)


def test_argument_checks_need_no_device(libxr):
    import paper_1805_01407_gb300 as xr
    vp = ctypes.c_void_p
    # a NULL context is rejected before anything reaches CUDA
    assert libxr.xr_fill(None, 0, vp(16), 1, 1, 0, 0, vp(16), 0, None) == xr.XR_EINVAL
    assert libxr.xr_seed(None, 0, 1, vp(16), None) == xr.XR_EINVAL
    assert libxr.xr_status(None, 0) == xr.XR_EINVAL
    assert libxr.xr_ctx_create(0, None) == xr.XR_EINVAL
    L = ctypes.c_uint64(0)
    assert libxr.xr_zeroland(None, 0, 1000, 4, vp(16), None) == xr.XR_EINVAL
    assert libxr.xr_linear_complexity(None, 0, 0, 100, vp(16), vp(16), 1 << 12, ctypes.byref(L), None) \
        == xr.XR_EINVAL
    job = xr.LcJob(0, 0, 100)
    assert libxr.xr_linear_complexity_many(None, ctypes.byref(job), 1, vp(16), 128, vp(16), 1 << 12,
                                           ctypes.byref(L), None) == xr.XR_EINVAL


def test_context_creation_fails_cleanly_without_gpu(libxr):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = libxr.xr_ctx_create(0, ctypes.byref(h))
    assert rc != 0 and not h.value
