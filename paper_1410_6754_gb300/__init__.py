"""AMS-sort on one GB300: Python binding of libams (include/ams.h).

The functions below marshal arguments for the C ABI and nothing else: every step of
the sort runs in the CUDA kernels of ``libams.so``.  Tensors are torch CUDA tensors
(device memory and streams come from PyTorch); the current torch stream is used
unless ``stream`` is given.  Integer tensors are sorted as unsigned bit patterns:
int32/uint32 -> 32-bit keys, int64/uint64 -> 64-bit keys; float32 tensors are sorted
in float order (with -0.0 before +0.0).  Payloads are 64-bit.

If the library has not been built the first call raises; there is no fallback.
Build it with ``python -m paper_1410_6754_gb300.build``.
"""
from __future__ import annotations

import ctypes
import os
import re

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libams.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "ams.h")

U32, U64, F32 = 0, 1, 2
OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_INTERNAL = range(7)
FLAG_PHASE_TIMERS = 1
FLAG_TREE_CLASSIFIER = 2
FLAG_GRAPH = 4
KERNEL_KINDS = ("init", "setup", "sample_sort", "cross_rank", "splitters", "classify", "scan",
                "binpack", "scatter", "basecase", "table")

_lib = None


class AmsError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = _lib.ams_status_string(status).decode() if _lib else str(status)
        super().__init__(f"{what}: {msg} (status {status})")


class Options(ctypes.Structure):
    _fields_ = [("oversample_a", ctypes.c_uint32), ("overpartition_b", ctypes.c_uint32),
                ("basecase_cap", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class Request(ctypes.Structure):
    _fields_ = [("keys_in", ctypes.c_void_p), ("keys_out", ctypes.c_void_p),
                ("vals_in", ctypes.c_void_p), ("vals_out", ctypes.c_void_p),
                ("d_offsets", ctypes.c_void_p), ("nseg", ctypes.c_uint64),
                ("n", ctypes.c_uint64), ("kt", ctypes.c_int), ("levels", ctypes.c_int),
                ("buckets_per_level", ctypes.POINTER(ctypes.c_uint32)),
                ("seed", ctypes.c_uint64), ("opt", Options)]


class SegmentInfo(ctypes.Structure):
    _fields_ = [("begin", ctypes.c_uint32), ("end", ctypes.c_uint32), ("a", ctypes.c_uint32),
                ("S", ctypes.c_uint32), ("L", ctypes.c_uint32), ("ngroups", ctypes.c_uint32),
                ("npieces", ctypes.c_uint32), ("nbucket_ids", ctypes.c_uint32)]


class Tuned(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("buckets_per_level", ctypes.c_uint32 * 8),
                ("overpartition_b", ctypes.c_uint32), ("candidates", ctypes.c_uint32),
                ("ms", ctypes.c_float), ("oversample_a", ctypes.c_uint32), ("basecase_cap", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [("levels_planned", ctypes.c_uint32), ("kernel_launches", ctypes.c_uint32),
                ("segments", ctypes.c_uint32 * 8), ("basecase_items", ctypes.c_uint32 * 9),
                ("device_status", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("kernel_ms", ctypes.c_float * 11), ("kernel_calls", ctypes.c_uint32 * 11),
                ("kernel_elems", ctypes.c_uint64 * 11)]

    def as_dict(self):
        return {
            "levels_planned": self.levels_planned,
            "kernel_launches": self.kernel_launches,
            "segments": list(self.segments),
            "basecase_items": list(self.basecase_items),
            "device_status": self.device_status,
            "kernel_ms": dict(zip(KERNEL_KINDS, list(self.kernel_ms))),
            "kernel_calls": dict(zip(KERNEL_KINDS, list(self.kernel_calls))),
            "kernel_elems": dict(zip(KERNEL_KINDS, list(self.kernel_elems))),
        }


_P, _U32, _U64, _I, _ST = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_int
_PU32 = ctypes.POINTER(ctypes.c_uint32)
_SIGS = {
    "ams_sort_keys": (_ST, [_P, _U64, _I, _I, _PU32, _U64, _P, _P]),
    "ams_sort_pairs": (_ST, [_P, _P, _U64, _I, _I, _PU32, _U64, _P, _P]),
    "ams_sort_segmented": (_ST, [_P, _P, _P, _U64, _U64, _I, _I, _PU32, _U64, _P, _P]),
    "ams_sort_keys_into": (_ST, [_P, _P, _U64, _I, _I, _PU32, _U64, _P, _P]),
    "ams_sort_pairs_into": (_ST, [_P, _P, _P, _P, _U64, _I, _I, _PU32, _U64, _P, _P]),
    "ams_sort_host": (_ST, [_P, _P, _U64, _I, _I, _PU32, _U64, _P, _P]),
    "ams_sort_host_async": (_ST, [_P, _P, _P, _U64, _I, _I, _PU32, _U64, _P, _P]),
    "ams_context_create": (_ST, [_U64, ctypes.POINTER(ctypes.c_void_p)]),
    "ams_context_destroy": (_ST, [_P]),
    "ams_sort_request": (_ST, [_P, ctypes.POINTER(Request), _P]),
    "ams_context_sync": (_ST, [_P]),
    "ams_context_scratch_bytes": (_U64, [_P]),
    "ams_request_scratch_bytes": (_U64, [ctypes.POINTER(Request)]),
    "ams_context_reserve": (_ST, [_P, _U64]),
    "ams_get_stats": (_ST, [_P, ctypes.POINTER(Stats)]),
    "ams_get_level_segments": (_ST, [_P, _I, _PU32, ctypes.POINTER(SegmentInfo), _U32]),
    "ams_get_segment_tables": (_ST, [_P, _I, _U32, _P, _P, _P]),
    "ams_step_sample": (_ST, [_P, _U64, _I, _U32, _U64, _U32, _U64, _P, _P]),
    "ams_step_rank_sort": (_ST, [_P, _U32, _I, _P, _P]),
    "ams_step_splitters": (_ST, [_P, _U32, _U32, _I, _P, _P]),
    "ams_step_classify": (_ST, [_P, _U64, _I, _P, _U32, _P, _P, _P]),
    "ams_step_bin_pack": (_ST, [_P, _U32, _U32, _P, _P, _P, _P]),
    "ams_step_partition": (_ST, [_P, _P, _P, _P, _U64, _I, _P, _U32, _P]),
    "ams_step_partition_arrival": (_ST, [_P, _P, _U64, _I, _P, _U32, _P]),
    "ams_step_base_case": (_ST, [_P, _P, _U64, _I, _P]),
    "ams_sort_small_noalloc": (_ST, [_P, _P, _U64, _I, _P]),
    "ams_rlm_sort": (_ST, [_P, _P, _P, _P, _P, _U64, _I, _U32, _I, _PU32, _U64, _P]),
    "ams_tune": (_ST, [_P, _U64, _I, _I, _P, ctypes.POINTER(Tuned)]),
    "ams_server_create": (_ST, [_U64, _I, _U64, ctypes.POINTER(ctypes.c_void_p)]),
    "ams_server_reserve": (_ST, [_P, ctypes.POINTER(Request)]),
    "ams_server_admits": (ctypes.c_int, [_U64, _U64, _U64, _U64, _U64]),
    "ams_server_submit": (_ST, [_P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "ams_server_wait": (_ST, [_P, _U64, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "ams_server_done": (ctypes.c_int, [_P, _U64]),
    "ams_server_counters": (_ST, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
    "ams_server_destroy": (_ST, [_P]),
    "ams_status_string": (ctypes.c_char_p, [_ST]),
    "ams_default_basecase_cap": (_U32, [_I, _I]),
    "ams_version": (ctypes.c_char_p, []),
}


def header_symbols():
    """Names of the functions include/ams.h declares."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"AMS_API\s+[\w\s\*]+?\b(ams_\w+)\s*\(", text)))


def lib():
    """The loaded libams (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1410_6754_gb300.build` (no fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(st, what):
    if st != OK:
        raise AmsError(st, what)


def _torch():
    import torch
    return torch


def key_type(t, kt=None):
    if kt is not None:
        return kt
    torch = _torch()
    if t.dtype == torch.float32:
        return F32
    if t.element_size() == 4:
        return U32
    if t.element_size() == 8:
        return U64
    raise TypeError(f"unsupported key dtype {t.dtype}")


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _opts(a=0, b=0, cap=0, flags=0):
    return Options(a, b, cap, flags)


def _buckets(buckets):
    arr = (ctypes.c_uint32 * len(buckets))(*[int(x) for x in buckets])
    return arr


def _dev(t):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def sort_keys(keys, levels=2, buckets=(256, 256), seed=0, a=0, b=0, cap=0, flags=0, kt=None,
              stream=None):
    """Sort a CUDA tensor in place (Section 6 AMS-sort)."""
    L = lib()
    bk = _buckets(buckets)
    o = _opts(a, b, cap, flags)
    _check(L.ams_sort_keys(_dev(keys), keys.numel(), key_type(keys, kt), levels, bk, seed,
                           ctypes.byref(o), _stream(stream)), "ams_sort_keys")
    return keys


def sort_pairs(keys, vals, levels=2, buckets=(256, 256), seed=0, a=0, b=0, cap=0, flags=0,
               kt=None, stream=None):
    L = lib()
    assert vals.numel() == keys.numel() and vals.element_size() == 8
    bk = _buckets(buckets)
    o = _opts(a, b, cap, flags)
    _check(L.ams_sort_pairs(_dev(keys), _dev(vals), keys.numel(), key_type(keys, kt), levels, bk,
                            seed, ctypes.byref(o), _stream(stream)), "ams_sort_pairs")
    return keys, vals


def sort_segmented(keys, offsets, vals=None, levels=2, buckets=(256, 256), seed=0, a=0, b=0,
                   cap=0, flags=0, kt=None, stream=None):
    """offsets: int64 CUDA tensor of nseg+1 entries."""
    L = lib()
    bk = _buckets(buckets)
    o = _opts(a, b, cap, flags)
    _check(L.ams_sort_segmented(_dev(keys), _dev(vals) if vals is not None else None, _dev(offsets),
                                offsets.numel() - 1, keys.numel(), key_type(keys, kt), levels, bk,
                                seed, ctypes.byref(o), _stream(stream)), "ams_sort_segmented")
    return keys if vals is None else (keys, vals)


def sort_keys_into(src, dst, levels=2, buckets=(256, 256), seed=0, a=0, b=0, cap=0, flags=0,
                   kt=None, stream=None):
    L = lib()
    bk = _buckets(buckets)
    o = _opts(a, b, cap, flags)
    _check(L.ams_sort_keys_into(_dev(src), _dev(dst), src.numel(), key_type(src, kt), levels, bk,
                                seed, ctypes.byref(o), _stream(stream)), "ams_sort_keys_into")
    return dst


def sort_pairs_into(ksrc, kdst, vsrc, vdst, levels=2, buckets=(256, 256), seed=0, a=0, b=0,
                    cap=0, flags=0, kt=None, stream=None):
    L = lib()
    bk = _buckets(buckets)
    o = _opts(a, b, cap, flags)
    _check(L.ams_sort_pairs_into(_dev(ksrc), _dev(kdst), _dev(vsrc), _dev(vdst), ksrc.numel(),
                                 key_type(ksrc, kt), levels, bk, seed, ctypes.byref(o),
                                 _stream(stream)), "ams_sort_pairs_into")
    return kdst, vdst


def sort_host(keys, vals=None, levels=2, buckets=(256, 256), seed=0, a=0, b=0, cap=0, flags=0,
              kt=None, stream=None):
    """Sort host arrays (numpy or CPU tensors) through the device; synchronous."""
    import numpy as np
    L = lib()
    if isinstance(keys, np.ndarray):
        assert keys.flags["C_CONTIGUOUS"]
        kptr = keys.ctypes.data_as(ctypes.c_void_p)
        n = keys.size
        if kt is None:
            kt = F32 if keys.dtype == np.float32 else (U32 if keys.itemsize == 4 else U64)
        vptr = vals.ctypes.data_as(ctypes.c_void_p) if vals is not None else None
    else:
        kptr = ctypes.c_void_p(keys.data_ptr())
        n = keys.numel()
        kt = key_type(keys, kt)
        vptr = ctypes.c_void_p(vals.data_ptr()) if vals is not None else None
    bk = _buckets(buckets)
    o = _opts(a, b, cap, flags)
    _check(L.ams_sort_host(kptr, vptr, n, kt, levels, bk, seed, ctypes.byref(o), _stream(stream)),
           "ams_sort_host")
    return keys if vals is None else (keys, vals)


def sort_host_async(keys, vals=None, levels=2, buckets=(256, 256), seed=0, a=0, b=0, cap=0, flags=0,
                    kt=None, ctx=None, stream=None):
    """Sort page-locked CPU tensors through the device without waiting
    (ams_sort_host_async): the copies in, the sort and the copies back are enqueued on
    `stream` with the scratch of `ctx`; the tensors hold the result once the stream has
    passed the call (ctx.sync() / stream synchronize)."""
    assert not keys.is_cuda and keys.is_contiguous()
    if vals is not None:
        assert not vals.is_cuda and vals.is_contiguous() and vals.numel() == keys.numel()
        assert vals.element_size() == 8
    h = ctx.handle if ctx is not None else None
    _check(lib().ams_sort_host_async(h, ctypes.c_void_p(keys.data_ptr()),
                                     ctypes.c_void_p(vals.data_ptr()) if vals is not None else None,
                                     keys.numel(), key_type(keys, kt), levels, _buckets(buckets), seed,
                                     ctypes.byref(_opts(a, b, cap, flags)), _stream(stream)),
           "ams_sort_host_async")
    return keys if vals is None else (keys, vals)


def sync(ctx=None):
    _check(lib().ams_context_sync(ctx), "ams_context_sync")


def stats(ctx=None) -> dict:
    s = Stats()
    _check(lib().ams_get_stats(ctx, ctypes.byref(s)), "ams_get_stats")
    return s.as_dict()


def default_basecase_cap(kt, pairs=False) -> int:
    return int(lib().ams_default_basecase_cap(kt, 1 if pairs else 0))


class Context:
    """A scratch-memory context (one per concurrent stream)."""

    def __init__(self, hbm_budget_bytes=0):
        self.handle = ctypes.c_void_p()
        _check(lib().ams_context_create(hbm_budget_bytes, ctypes.byref(self.handle)),
               "ams_context_create")

    def sort(self, keys_in, keys_out=None, vals_in=None, vals_out=None, offsets=None,
             levels=2, buckets=(256, 256), seed=0, a=0, b=0, cap=0, flags=0, kt=None,
             stream=None):
        keys_out = keys_in if keys_out is None else keys_out
        if vals_in is not None and vals_out is None:
            vals_out = vals_in
        bk = _buckets(buckets)
        rq = Request()
        rq.keys_in = keys_in.data_ptr()
        rq.keys_out = keys_out.data_ptr()
        rq.vals_in = vals_in.data_ptr() if vals_in is not None else None
        rq.vals_out = vals_out.data_ptr() if vals_out is not None else None
        rq.d_offsets = offsets.data_ptr() if offsets is not None else None
        rq.nseg = (offsets.numel() - 1) if offsets is not None else 1
        rq.n = keys_in.numel()
        rq.kt = key_type(keys_in, kt)
        rq.levels = levels
        rq.buckets_per_level = ctypes.cast(bk, ctypes.POINTER(ctypes.c_uint32))
        rq.seed = seed
        rq.opt = _opts(a, b, cap, flags)
        _check(lib().ams_sort_request(self.handle, ctypes.byref(rq), _stream(stream)),
               "ams_sort_request")
        return keys_out

    def sync(self):
        _check(lib().ams_context_sync(self.handle), "ams_context_sync")

    def stats(self):
        s = Stats()
        _check(lib().ams_get_stats(self.handle, ctypes.byref(s)), "ams_get_stats")
        return s.as_dict()

    def scratch_bytes(self):
        return int(lib().ams_context_scratch_bytes(self.handle))

    def reserve(self, nbytes):
        """Grow the context's scratch to at least nbytes now (ams_context_reserve)."""
        _check(lib().ams_context_reserve(self.handle, int(nbytes)), "ams_context_reserve")

    def level_segments(self, level):
        """Segments sorted at distribution level `level` (1-based) by the last sort, with
        their a, S, L*, groups and pieces (ams_get_level_segments)."""
        n = ctypes.c_uint32()
        _check(lib().ams_get_level_segments(self.handle, level, ctypes.byref(n), None, 0),
               "ams_get_level_segments")
        arr = (SegmentInfo * max(1, n.value))()
        _check(lib().ams_get_level_segments(self.handle, level, ctypes.byref(n), arr, n.value),
               "ams_get_level_segments")
        return [{f: getattr(arr[i], f) for f, _ in SegmentInfo._fields_} for i in range(n.value)]

    def segment_tables(self, level, seg, nbucket_ids, npieces):
        """(bucket starts, piece of every id, piece starts) of one segment, as lists."""
        bs = (ctypes.c_uint32 * nbucket_ids)()
        po = (ctypes.c_uint16 * nbucket_ids)()
        ps = (ctypes.c_uint32 * max(1, npieces))()
        _check(lib().ams_get_segment_tables(self.handle, level, seg, bs, po, ps), "ams_get_segment_tables")
        return list(bs), list(po), list(ps)[:npieces]

    def close(self):
        if self.handle:
            _check(lib().ams_context_destroy(self.handle), "ams_context_destroy")
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _sizing_request(n, kt, levels, buckets, a=0, b=0, cap=0, pairs=False, nseg=1):
    """A request description for sizing only (no buffers: the size calls read n, the
    key type, the plan parameters and whether there are payloads or segments)."""
    bk = _buckets(buckets)
    rq = Request()
    rq.keys_in = rq.keys_out = 16
    rq.vals_in = rq.vals_out = 16 if pairs else None
    rq.d_offsets = 16 if nseg > 1 else None
    rq.nseg = nseg
    rq.n = n
    rq.kt = kt
    rq.levels = levels
    rq.buckets_per_level = ctypes.cast(bk, ctypes.POINTER(ctypes.c_uint32))
    rq.opt = _opts(a, b, cap, 0)
    return rq, bk


def request_scratch_bytes(n, kt, levels=2, buckets=(256, 256), a=0, b=0, cap=0, pairs=False, nseg=1) -> int:
    """Device scratch a sort of this shape needs in a context (ams_request_scratch_bytes)."""
    rq, _bk = _sizing_request(n, kt, levels, buckets, a, b, cap, pairs, nseg)
    return int(lib().ams_request_scratch_bytes(ctypes.byref(rq)))


def rlm_sort(keys_in, keys_out=None, vals_in=None, vals_out=None, run=8192, parts=(64, 64), seed=0,
             kt=None, ctx=None, stream=None):
    """RLM-sort (ams_rlm_sort, Section 5): same result as the sample sort calls."""
    keys_out = keys_in if keys_out is None else keys_out
    if vals_in is not None and vals_out is None:
        vals_out = vals_in
    pk = _buckets(parts) if len(parts) else None
    h = ctx.handle if ctx is not None else None
    _check(lib().ams_rlm_sort(h, _dev(keys_in), _dev(keys_out), _dev(vals_in) if vals_in is not None else None,
                              _dev(vals_out) if vals_out is not None else None, keys_in.numel(),
                              key_type(keys_in, kt), run, len(parts), pk, seed, _stream(stream)),
           "ams_rlm_sort")
    return keys_out if vals_in is None else (keys_out, vals_out)


def tune(n, kt, pairs=False, ctx=None, stream=None) -> dict:
    """The autotuner's plan for n keys of type kt (ams_tune): levels, buckets (r per
    level), b, a, cap (0 = defaults), and its score on synthetic keys.  The keys
    levels / buckets / b / a / cap can be passed to the sort calls as they are."""
    t = Tuned()
    h = ctx.handle if ctx is not None else None
    _check(lib().ams_tune(h, n, kt, 1 if pairs else 0, _stream(stream), ctypes.byref(t)), "ams_tune")
    return {"levels": t.levels, "buckets": list(t.buckets_per_level)[:t.levels], "b": t.overpartition_b,
            "a": t.oversample_a, "cap": t.basecase_cap, "candidates": t.candidates, "ms": t.ms}


class Server:
    """Serving loop (ams_server_*): submit sort requests on device tensors; they run
    on the server's worker streams with continuous batching.  The tensors must stay
    alive and untouched until the request is waited for."""

    def __init__(self, hbm_budget_bytes=0, streams=4, pack_max_keys=1 << 16):
        self.handle = ctypes.c_void_p()
        _check(lib().ams_server_create(hbm_budget_bytes, streams, pack_max_keys, ctypes.byref(self.handle)),
               "ams_server_create")
        self._keep = {}

    def reserve(self, n, kt, levels=2, buckets=(256, 256), a=0, b=0, cap=0, pairs=False):
        """Size every worker for requests up to this shape now (ams_server_reserve)."""
        rq, _bk = _sizing_request(n, kt, levels, buckets, a, b, cap, pairs)
        _check(lib().ams_server_reserve(self.handle, ctypes.byref(rq)), "ams_server_reserve")

    def submit(self, keys_in, keys_out=None, vals_in=None, vals_out=None, levels=2, buckets=(256, 256),
               seed=0, a=0, b=0, cap=0, kt=None):
        keys_out = keys_in if keys_out is None else keys_out
        if vals_in is not None and vals_out is None:
            vals_out = vals_in
        bk = _buckets(buckets)
        rq = Request()
        rq.keys_in = keys_in.data_ptr()
        rq.keys_out = keys_out.data_ptr()
        rq.vals_in = vals_in.data_ptr() if vals_in is not None else None
        rq.vals_out = vals_out.data_ptr() if vals_out is not None else None
        rq.d_offsets = None
        rq.nseg = 1
        rq.n = keys_in.numel()
        rq.kt = key_type(keys_in, kt)
        rq.levels = levels
        rq.buckets_per_level = ctypes.cast(bk, ctypes.POINTER(ctypes.c_uint32))
        rq.seed = seed
        rq.opt = _opts(a, b, cap, 0)
        t = ctypes.c_uint64()
        _check(lib().ams_server_submit(self.handle, ctypes.byref(rq), ctypes.byref(t)), "ams_server_submit")
        self._keep[t.value] = (keys_in, keys_out, vals_in, vals_out)
        return t.value

    def wait(self, ticket):
        """Waits for the request; returns (submit_ns, done_ns) host steady-clock times."""
        t0, t1 = ctypes.c_uint64(), ctypes.c_uint64()
        st = lib().ams_server_wait(self.handle, ticket, ctypes.byref(t0), ctypes.byref(t1))
        self._keep.pop(ticket, None)
        _check(st, "ams_server_wait")
        return t0.value, t1.value

    def done(self, ticket):
        return lib().ams_server_done(self.handle, ticket) == 1

    def counters(self):
        b, p = ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().ams_server_counters(self.handle, ctypes.byref(b), ctypes.byref(p)), "ams_server_counters")
        return {"batches": b.value, "packed_requests": p.value}

    def close(self):
        if self.handle:
            _check(lib().ams_server_destroy(self.handle), "ams_server_destroy")
            self.handle = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ building blocks
def step_sample(keys, count, seed, level, begin, kt=None, stream=None):
    torch = _torch()
    kt = key_type(keys, kt)
    out = torch.empty(count, dtype=torch.int64 if kt == U64 else torch.int32, device=keys.device)
    _check(lib().ams_step_sample(_dev(keys), keys.numel(), kt, count, seed, level, begin,
                                 _dev(out), _stream(stream)), "ams_step_sample")
    return out


def step_rank_sort(sample, kt, stream=None):
    out = _torch().empty_like(sample)
    _check(lib().ams_step_rank_sort(_dev(sample), sample.numel(), kt, _dev(out), _stream(stream)),
           "ams_step_rank_sort")
    return out


def step_splitters(sorted_sample, a, nbuckets, kt, stream=None):
    out = _torch().empty(nbuckets - 1, dtype=sorted_sample.dtype, device=sorted_sample.device)
    _check(lib().ams_step_splitters(_dev(sorted_sample), a, nbuckets, kt, _dev(out),
                                    _stream(stream)), "ams_step_splitters")
    return out


def step_classify(keys, splitters, nbuckets, kt=None, want_ids=True, stream=None):
    torch = _torch()
    kt = key_type(keys, kt)
    counts = torch.empty(2 * nbuckets - 1, dtype=torch.int32, device=keys.device)
    ids = torch.empty(keys.numel(), dtype=torch.int16, device=keys.device) if want_ids else None
    _check(lib().ams_step_classify(_dev(keys), keys.numel(), kt, _dev(splitters), nbuckets,
                                   _dev(counts), _dev(ids) if ids is not None else None,
                                   _stream(stream)), "ams_step_classify")
    return counts, ids


def step_bin_pack(counts, nbuckets, r, stream=None):
    torch = _torch()
    L = torch.empty(1, dtype=torch.int64, device=counts.device)
    ends = torch.empty(r, dtype=torch.int32, device=counts.device)
    ng = torch.empty(1, dtype=torch.int32, device=counts.device)
    _check(lib().ams_step_bin_pack(_dev(counts), nbuckets, r, _dev(L), _dev(ends), _dev(ng),
                                   _stream(stream)), "ams_step_bin_pack")
    return L, ends, ng


def step_partition(keys, splitters, nbuckets, vals=None, kt=None, stream=None):
    torch = _torch()
    out = torch.empty_like(keys)
    vout = torch.empty_like(vals) if vals is not None else None
    _check(lib().ams_step_partition(_dev(keys), _dev(out), _dev(vals) if vals is not None else None,
                                    _dev(vout) if vout is not None else None, keys.numel(),
                                    key_type(keys, kt), _dev(splitters), nbuckets,
                                    _stream(stream)), "ams_step_partition")
    return out if vals is None else (out, vout)


def step_partition_arrival(keys, splitters, nbuckets, kt=None, stream=None):
    """Keys-only delivery in arrival order inside every bucket (ams_step_partition_arrival)."""
    torch = _torch()
    out = torch.empty_like(keys)
    _check(lib().ams_step_partition_arrival(_dev(keys), _dev(out), keys.numel(), key_type(keys, kt),
                                            _dev(splitters), nbuckets, _stream(stream)),
           "ams_step_partition_arrival")
    return out


def step_base_case(keys, vals=None, kt=None, stream=None):
    _check(lib().ams_step_base_case(_dev(keys), _dev(vals) if vals is not None else None,
                                    keys.numel(), key_type(keys, kt), _stream(stream)),
           "ams_step_base_case")
    return keys if vals is None else (keys, vals)


# ------------------------------------------------------------------ allocation-free sort
NOALLOC_MAX_KEYS = 524288


def sort_small_noalloc(keys, vals=None, kt=None, stream=None):
    """In-place sort of at most NOALLOC_MAX_KEYS elements that allocates no device
    memory (for callers that cannot allow allocations at call time); its scratch is
    a fixed 8 MiB device array inside the library, shared by all calls on a device,
    so calls must not overlap on the GPU."""
    kt = key_type(keys, kt)
    if keys.element_size() != (8 if kt == U64 else 4):
        raise ValueError("key type does not match the key tensor's element size")
    if vals is not None and (vals.numel() != keys.numel() or vals.element_size() != 8):
        raise ValueError("payloads must be one 64-bit value per key")
    _check(lib().ams_sort_small_noalloc(_dev(keys), _dev(vals) if vals is not None else None,
                                        keys.numel(), kt, _stream(stream)),
           "ams_sort_small_noalloc")
    return keys if vals is None else (keys, vals)
