"""The C boundary from C: include/xr.h and include/xr_probe.h compile as strict
C11 (-Wall -Wextra -pedantic -Werror), a C program links against libxr.so and
calls the pure property functions and an argument check without a GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include "xr.h"
#include "xr_probe.h"

int main(void)
{
    int v;
    for (v = 0; v < XR_NUM_VARIANTS; ++v)
        printf("%s %d %d %d %d %d %d\n", xr_variant_name(v), xr_state_words(v), xr_word_bits(v),
               xr_state_bytes(v), xr_state_bits(v), xr_jump_log2(v, XR_JUMP), xr_jump_log2(v, XR_LONG_JUMP));
    printf("bad %d %d %s\n", xr_state_words(XR_NUM_VARIANTS), xr_dtype_bytes(7), xr_error_string(XR_EINVAL));
    /* argument checks answer before any device work */
    printf("null %d %d\n", xr_fill(NULL, 0, NULL, 1, 1, XR_U64, XR_STREAM_MAJOR, NULL, 0, NULL),
           xr_probe_store(NULL, 16, 0, NULL));
    printf("noalloc %lu %lu %lu\n", (unsigned long)XR_NOALLOC_MAX_OUTPUTS_FOR(16),
           (unsigned long)XR_NOALLOC_MAX_OUTPUTS_FOR(64), (unsigned long)XR_NOALLOC_MAX_OUTPUTS_FOR(128));
    return 0;
}
"""


@pytest.fixture(scope="module")
def libdir():
    from paper_1805_01407_gb300 import build
    build.build()
    return os.path.join(ROOT, "paper_1805_01407_gb300")


def test_c_program_uses_the_boundary(tmp_path, libdir):
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc missing")
    src = tmp_path / "use_xr.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "use_xr"
    subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I" + os.path.join(ROOT, "include"),
                    str(src), "-L" + libdir, "-lxr", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    rows = {line.split()[0]: line.split()[1:] for line in out}
    assert rows["xoshiro256**"] == ["4", "64", "32", "256", "128", "192"]
    assert rows["xoroshiro128++"] == ["2", "64", "16", "128", "64", "96"]
    assert rows["xoshiro128+"] == ["4", "32", "16", "128", "64", "96"]
    assert rows["xoroshiro64*"] == ["2", "32", "8", "64", "32", "48"]
    assert rows["xoshiro512**"] == ["8", "64", "64", "512", "256", "384"]
    assert rows["xoroshiro1024++"] == ["16", "64", "128", "1024", "512", "768"]
    assert rows["bad"][:2] == ["-1", "-1"] and " ".join(rows["bad"][2:]) == "invalid argument"
    assert rows["null"] == ["1", "1"]                       # XR_EINVAL from both, no device touched
    assert rows["noalloc"] == [str(1 << 26), str(1 << 25), str(1 << 24)]
