"""The C ABI library builds, loads and exports every function include/ams.h declares
(host-only calls; no GPU needed)."""
import ctypes
import os
import subprocess

import pytest

import paper_1410_6754_gb300 as ams
from paper_1410_6754_gb300 import build as B


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_header_declares_the_boundary():
    syms = ams.header_symbols()
    for name in ["ams_sort_keys", "ams_sort_pairs", "ams_sort_segmented", "ams_sort_keys_into",
                 "ams_sort_pairs_into", "ams_sort_host", "ams_context_create",
                 "ams_context_destroy", "ams_sort_request", "ams_context_sync", "ams_get_stats",
                 "ams_step_sample", "ams_step_rank_sort", "ams_step_splitters",
                 "ams_step_classify", "ams_step_bin_pack", "ams_step_partition", "ams_step_partition_arrival",
                 "ams_step_base_case", "ams_status_string", "ams_version"]:
        assert name in syms


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [s for s in ams.header_symbols() if s not in exported]
    assert not missing, missing
    # nothing else is exported under the ams_ prefix by accident
    extra = sorted(s for s in exported if s.startswith("ams_") and s not in ams.header_symbols())
    assert not extra, extra


def test_python_binding_covers_header(libpath):
    assert set(ams.header_symbols()) <= set(ams._SIGS)
    L = ams.lib()
    for name in ams.header_symbols():
        assert hasattr(L, name)


def test_host_only_calls(libpath):
    L = ams.lib()
    assert L.ams_version().decode().count(".") == 2
    for st in range(7):
        assert L.ams_status_string(st)
    assert L.ams_status_string(99) == b"unknown status"
    assert ams.default_basecase_cap(ams.U32) == 16384
    assert ams.default_basecase_cap(ams.U64) == 8192
    assert ams.default_basecase_cap(ams.F32, pairs=True) == 8192


def test_struct_layouts_match_header(tmp_path):
    """ctypes structures against the C compiler's view of include/ams.h (host gcc)."""
    fields = {
        "ams_options": (ams.Options, ["oversample_a", "overpartition_b", "basecase_cap", "flags"]),
        "ams_request": (ams.Request, ["keys_in", "keys_out", "vals_in", "vals_out", "d_offsets", "nseg",
                                      "n", "kt", "levels", "buckets_per_level", "seed", "opt"]),
        "ams_stats": (ams.Stats, ["levels_planned", "kernel_launches", "segments", "basecase_items",
                                  "device_status", "kernel_ms", "kernel_calls", "kernel_elems"]),
        "ams_tuned": (ams.Tuned, ["levels", "buckets_per_level", "overpartition_b", "candidates", "ms",
                                  "oversample_a", "basecase_cap"]),
        "ams_segment_info": (ams.SegmentInfo, ["begin", "end", "a", "S", "L", "ngroups", "npieces",
                                               "nbucket_ids"]),
    }
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ams.h"', "int main(void) {"]
    for st, (_, names) in fields.items():
        lines.append(f'  printf("{st} size %zu\\n", sizeof({st}));')
        for f in names:
            lines.append(f'  printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(ams.HEADER), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        parts = ln.split()
        got[tuple(parts[:-1])] = int(parts[-1])
    for st, (cls, names) in fields.items():
        assert got[(st, "size")] == ctypes.sizeof(cls), st
        for f in names:
            assert got[(st, f)] == getattr(cls, f).offset, (st, f)


def test_built_for_sm103a(libpath):
    # the fat binary carries sm_103a code (cuobjdump is not used; the build flags are checked)
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)
    assert os.path.getsize(libpath) > 100_000


def test_noalloc_refuses_misaligned_views_on_the_host(libpath):
    """ams_sort_small_noalloc checks alignment before any CUDA call: a 64-bit key view
    at a 4-byte offset, or a payload pointer that is not 8-byte aligned, returns
    AMS_ERR_INVALID (these addresses are never dereferenced)."""
    L = ams.lib()
    p = ctypes.c_void_p
    assert L.ams_sort_small_noalloc(p(0x10004), None, 10, ams.U64, None) == ams.ERR_INVALID
    assert L.ams_sort_small_noalloc(p(0x10002), None, 10, ams.U32, None) == ams.ERR_INVALID
    assert L.ams_sort_small_noalloc(p(0x10000), p(0x20004), 10, ams.U32, None) == ams.ERR_INVALID
    assert L.ams_sort_small_noalloc(p(0x10000), None, ams.NOALLOC_MAX_KEYS + 1, ams.U32, None) \
        == ams.ERR_INVALID
    assert L.ams_sort_small_noalloc(p(0x10000), None, 10, 7, None) == ams.ERR_INVALID
    assert L.ams_sort_small_noalloc(None, None, 0, ams.U32, None) == ams.OK


def test_host_async_checks_arguments_on_the_host(libpath):
    """ams_sort_host_async returns AMS_ERR_INVALID for a null key array with n > 0, and
    AMS_OK for n = 0, before it touches a context or the GPU."""
    L = ams.lib()
    bk = (ctypes.c_uint32 * 2)(16, 16)
    assert L.ams_sort_host_async(None, None, None, 10, ams.U64, 2, bk, 0, None, None) == ams.ERR_INVALID
    assert L.ams_sort_host_async(None, None, None, 0, ams.U64, 2, bk, 0, None, None) == ams.OK


def test_server_admission_rule(libpath):
    """The serving loop's admission decision (a pure function; no GPU): by the budget of
    scratch in flight, and by the device's free memory when a worker context must grow."""
    L = ams.lib()
    GiB, MiB = 1 << 30, 1 << 20
    adm = L.ams_server_admits
    assert adm(0, 100 * GiB, 64 * GiB, 50 * GiB, 0) == 1          # nothing in flight: runs alone
    assert adm(10 * GiB, 50 * GiB, 64 * GiB, 0, 0) == 1           # within budget, no growth
    assert adm(10 * GiB, 55 * GiB, 64 * GiB, 0, 0) == 0           # over budget
    assert adm(10 * GiB, 55 * GiB, 0, 0, 0) == 1                  # no budget set
    assert adm(10 * GiB, 1 * GiB, 64 * GiB, 1 * GiB, 2 * GiB) == 1  # growth fits in free memory
    assert adm(10 * GiB, 1 * GiB, 64 * GiB, 1 * GiB, 1 * GiB + 255 * MiB) == 0  # not with the spare
    assert adm(10 * GiB, 1 * GiB, 64 * GiB, 1 * GiB, 1 * GiB + 256 * MiB) == 1
