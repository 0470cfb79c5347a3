"""Seeded synthetic inputs for the sort (shared by the tests, the bench and the oracle).

This module holds no arithmetic of the sorting method.  Each generator takes
(n, seed) and returns keys (and, for pairs, payloads) built from a SplitMix64
stream; the same values come out of the numpy path (host) and the torch path
(device tensors, int64 arithmetic that wraps modulo 2**64), so the large
workloads can be generated directly in device memory.

Distributions (the workloads of the sample-sort evaluation, all synthetic):

* ``uniform``    -- i.i.d. uniform over the full key range.
* ``zipf``       -- Zipf(s=1.1) ranks over 2**20 values (inverse CDF); uint64 keys
                    scatter the rank through SplitMix64, uint32 keys are the rank.
* ``equal``      -- one value repeated n times.
* ``sorted`` / ``reverse`` -- uniform draws sorted ascending / descending.
* ``staggered``  -- blocks of 2**16 keys; block i draws uniformly from slot
                    2i+1 (first half of the blocks) or 2i-m (second half) of m equal
                    slots of the key range and is sorted inside.
* ``normal_f32`` -- float32 N(0,1) by Box-Muller with 5% exact zeros, half -0.0.
* ``dup1024``    -- uint64 keys drawn uniformly from 1024 distinct uniform values.
"""
from __future__ import annotations

import math

import numpy as np

_M64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15
_C1 = 0xBF58476D1CE4E5B9
_C2 = 0x94D049BB133111EB

DISTRIBUTIONS = ("uniform", "zipf", "equal", "sorted", "reverse", "staggered")
_TAGS = {"uniform": 1, "zipf": 2, "equal": 3, "sorted": 4, "reverse": 5, "staggered": 6,
         "normal_f32": 7, "dup1024": 8, "segments": 9, "requests": 10}


def _s64(x: int) -> int:
    """Python int in [0, 2**64) -> the int64 with the same bits."""
    x &= _M64
    return x - (1 << 64) if x >= (1 << 63) else x


def _mix_int(z: int) -> int:
    z &= _M64
    z = ((z ^ (z >> 30)) * _C1) & _M64
    z = ((z ^ (z >> 27)) * _C2) & _M64
    return z ^ (z >> 31)


def base_state(seed: int, tag: int) -> int:
    return _mix_int((seed & _M64) + tag * _GAMMA)


# ---------------------------------------------------------------- numpy stream
def _mix_np(z):
    with np.errstate(over="ignore"):
        z = z ^ (z >> np.uint64(30))
        z = z * np.uint64(_C1)
        z = z ^ (z >> np.uint64(27))
        z = z * np.uint64(_C2)
        return z ^ (z >> np.uint64(31))


def stream_np(state: int, start: int, count: int) -> np.ndarray:
    """Outputs start..start+count-1 of SplitMix64 from ``state`` (uint64 array)."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix_np(np.uint64(state) + k * np.uint64(_GAMMA))


# ---------------------------------------------------------------- torch stream
def _srl(z, k):
    return (z >> k) & ((1 << (64 - k)) - 1)


def _mix_t(z):
    z = z ^ _srl(z, 30)
    z = z * _s64(_C1)
    z = z ^ _srl(z, 27)
    z = z * _s64(_C2)
    return z ^ _srl(z, 31)


def stream_torch(state: int, start: int, count: int, device):
    import torch
    k = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    return _mix_t(k * _s64(_GAMMA) + _s64(state))


def _stream(xp, state, count, device):
    if xp == "np":
        return stream_np(state, 0, count)
    return stream_torch(state, 0, count, device)


def _zipf_cdf(nvals: int, s: float) -> np.ndarray:
    w = np.arange(1, nvals + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def generate(dist: str, n: int, seed: int, key_bits: int = 64, device=None):
    """Keys of one distribution.  ``key_bits`` is 32 or 64.  ``device=None`` returns a
    numpy array (uint32/uint64); otherwise an int32/int64 torch tensor on ``device``
    holding the same bits."""
    xp = "np" if device is None else "t"
    st = base_state(seed, _TAGS[dist])
    if xp == "t":
        import torch
    if dist in ("uniform", "sorted", "reverse"):
        x = _stream(xp, st, n, device)
        x = _to_bits(xp, x, key_bits)
        if dist != "uniform":
            x = _sort(xp, x, key_bits, descending=(dist == "reverse"))
        return x
    if dist == "equal":
        v = _mix_int(st + _GAMMA)
        v = v if key_bits == 64 else v >> 32
        if xp == "np":
            return np.full(n, v, dtype=np.uint64 if key_bits == 64 else np.uint32)
        return torch.full((n,), _s64(v) if key_bits == 64 else _s32(v),
                          dtype=torch.int64 if key_bits == 64 else torch.int32, device=device)
    if dist == "zipf":
        cdf = _zipf_cdf(1 << 20, 1.1)
        x = _stream(xp, st, n, device)
        if xp == "np":
            u = (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
            rank = np.searchsorted(cdf, u, side="right").astype(np.uint64) + np.uint64(1)
            if key_bits == 32:
                return rank.astype(np.uint32)
            return _mix_np(rank * np.uint64(_GAMMA) + np.uint64(st))
        u = _srl(x, 11).to(torch.float64) * (2.0 ** -53)
        rank = torch.searchsorted(torch.from_numpy(cdf).to(device), u, right=True) + 1
        if key_bits == 32:
            return rank.to(torch.int32)
        return _mix_t(rank * _s64(_GAMMA) + _s64(st))
    if dist == "staggered":
        blk = min(1 << 16, n) if n else 1
        m = max(1, -(-n // blk))
        x = _stream(xp, st, n, device)
        i = (np.arange(n, dtype=np.int64) // blk) if xp == "np" else \
            torch.arange(n, dtype=torch.int64, device=device) // blk
        if m == 1:
            slot = i * 0
        else:
            half = m // 2
            slot = (2 * i + 1) * (i < half) + (2 * i - m) * (i >= half) if xp == "np" else \
                torch.where(i < half, 2 * i + 1, 2 * i - m)
        span_bits = key_bits
        # value = slot * floor(2**bits / m) + (x mod floor(2**bits / m))
        width = (1 << span_bits) // m
        if xp == "np":
            xv = x if key_bits == 64 else (x >> np.uint64(32))
            if m == 1:
                val = xv
            else:
                val = slot.astype(np.uint64) * np.uint64(width) + xv % np.uint64(width)
            val = val.astype(np.uint64 if key_bits == 64 else np.uint32)
            out = val.copy()
            for b0 in range(0, n, blk):
                out[b0:b0 + blk] = np.sort(val[b0:b0 + blk])
            return out
        # torch: unsigned 64-bit modulo via the numpy path is avoided by requiring
        # m to be a power of two (true for the power-of-two sizes used here)
        if m & (m - 1):
            raise ValueError("staggered on device needs a power-of-two block count")
        lg = m.bit_length() - 1
        if key_bits == 64:
            low = x & _s64((1 << (64 - lg)) - 1) if lg else x
            val = (slot << (64 - lg)) | low if lg else low
        else:
            xv = _srl(x, 32)
            low = xv & ((1 << (32 - lg)) - 1)
            val = ((slot << (32 - lg)) | low) if lg else low
            val = (val - ((val >> 31) << 32)).to(torch.int32)
        out = torch.empty_like(val)
        nb = n // blk
        if nb:
            out[:nb * blk] = _sort("t", val[:nb * blk].view(nb, blk), key_bits, dim=1).reshape(-1)
        if n > nb * blk:
            out[nb * blk:] = _sort("t", val[nb * blk:], key_bits)
        return out
    raise ValueError(f"unknown distribution {dist}")


def _s32(v: int) -> int:
    v &= 0xFFFFFFFF
    return v - (1 << 32) if v >= (1 << 31) else v


def _to_bits(xp, x, key_bits):
    """Keep 64 bits, or the top 32 bits of each 64-bit draw."""
    if key_bits == 64:
        return x
    if xp == "np":
        return (x >> np.uint64(32)).astype(np.uint32)
    import torch
    hi = _srl(x, 32)
    return (hi - ((hi >> 31) << 32)).to(torch.int32)   # same bits as uint32


def _sort(xp, x, key_bits, descending=False, dim=-1):
    """Unsigned sort of keys held as numpy unsigned or torch signed tensors."""
    if xp == "np":
        s = np.sort(x, axis=dim)
        return np.flip(s, axis=dim).copy() if descending else s
    import torch
    flip = (1 << 63) if key_bits == 64 else (1 << 31)
    y = x ^ _s64(flip) if key_bits == 64 else x ^ _s32(flip)   # signed order == unsigned order
    y, _ = torch.sort(y, dim=dim, descending=descending, stable=True)
    return y ^ _s64(flip) if key_bits == 64 else y ^ _s32(flip)


def normal_f32(n: int, seed: int, zero_frac: float = 0.05) -> np.ndarray:
    """float32 N(0,1) via Box-Muller, with a fraction of exact zeros (half -0.0)."""
    st = base_state(seed, _TAGS["normal_f32"])
    x = stream_np(st, 0, 3 * n).reshape(n, 3)
    u1 = ((x[:, 0] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    u2 = (x[:, 1] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    z = (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)).astype(np.float32)
    u3 = (x[:, 2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    zero = u3 < zero_frac
    neg = (x[:, 2] & np.uint64(1)).astype(bool)
    z[zero & ~neg] = np.float32(0.0)
    z[zero & neg] = np.float32(-0.0)
    return z


def dup_keys_u64(n: int, seed: int, distinct: int = 1024) -> np.ndarray:
    """uint64 keys drawn uniformly from ``distinct`` (a power of two) uniform values."""
    st = base_state(seed, _TAGS["dup1024"])
    table = stream_np(_mix_int(st + 7), 0, distinct)
    x = stream_np(st, 0, n)
    lg = distinct.bit_length() - 1
    return table[(x >> np.uint64(64 - lg)).astype(np.int64)]


def segment_lengths(nseg: int, total: int, seed: int, max_log2: int = 20) -> np.ndarray:
    """Log-uniform segment lengths 2**(max_log2*U), rescaled to sum to about
    ``total`` (each at least 1)."""
    st = base_state(seed, _TAGS["segments"])
    u = (stream_np(st, 0, nseg) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    raw = np.power(2.0, max_log2 * u)
    ln = np.maximum(1, np.rint(raw * (total / raw.sum()))).astype(np.int64)
    return ln
