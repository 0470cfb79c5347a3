"""Parity at the evaluation's full sizes, in the launch configuration the benchmark
times (a context, out-of-place sort): 2^28 uint64 keys at two levels (r = 256 x 256,
b = 4) for the six input distributions, and 2^27 pairs (duplicate-heavy uint64 keys;
float32 keys with signed zeros) at three levels.

The oracle cannot sort these sizes in seconds, so the checks are properties that fix
the result uniquely, plus sampled positions the oracle computes one by one:
 * keys only: the output is non-decreasing and holds the input's multiset (count and
   an order-independent hash) -- the sorted permutation of a multiset is unique; the
   oracle's selection gives the values at sampled output positions;
 * pairs with payload = original index: (key, payload) strictly increasing and
   key_out[i] == key_in[payload_out[i]] -- only the definition's output satisfies
   both."""
import numpy as np
import pytest

import oracle as O
from paper_1410_6754_gb300 import inputs as I

from helpers import to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1410_6754_gb300 as ams  # noqa: E402

SIGN64 = -(1 << 63)


def _ord64(t):
    """int64 tensor of unsigned 64-bit keys -> int64 with the same order (signed)."""
    return t ^ SIGN64


def _multiset_hash(t):
    """Count and two order-independent 64-bit hashes (wrapping sums of SplitMix64
    finalised keys)."""
    return t.numel(), int(I._mix_t(t).sum().item()), int(I._mix_t(t + 1).sum().item())


@pytest.mark.parametrize("dist", I.DISTRIBUTIONS)
def test_two_level_2p28_u64(dist):
    n = 1 << 28
    src = I.generate(dist, n, 0, 64, device="cuda")
    dst = torch.empty_like(src)
    ctx = ams.Context()
    ctx.sort(src, dst, levels=2, buckets=[256, 256], b=4, seed=0, kt=1)
    ctx.sync()
    o = _ord64(dst)
    assert bool((o[1:] >= o[:-1]).all()), "output not sorted"
    assert _multiset_hash(src) == _multiset_hash(dst), "output is not a permutation of the input"
    # sampled positions against the oracle's selection on the same input
    ranks = np.unique(np.concatenate([[0, n - 1, n // 2], np.random.default_rng(1).integers(0, n, 13)]))
    host = src.cpu().numpy().view(np.uint64)
    want = O.select_ranks(O.KT_U64, host, ranks)
    got = dst[torch.from_numpy(ranks).cuda()].cpu().numpy().view(np.uint64)
    assert np.array_equal(got, want)
    del ctx


def _pairs_check(keys_np, kt, levels=3):
    n = len(keys_np)
    dk = to_dev(keys_np)
    vals = torch.arange(n, dtype=torch.int64, device="cuda")
    kin = dk.clone()
    ams.sort_pairs(dk, vals, levels=levels, buckets=[256, 256, 256], seed=0, kt=kt)
    ams.sync()
    if kt == O.KT_F32:
        b = dk.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
        t = torch.where(b >> 31 == 1, b ^ 0xFFFFFFFF, b | 0x80000000)  # order map, as int64
        same = torch.equal(dk.view(torch.int32), kin.view(torch.int32)[vals])
    else:
        t = _ord64(dk)
        same = torch.equal(dk, kin[vals])
    assert same, "a payload does not travel with its key"
    asc = (t[1:] > t[:-1]) | ((t[1:] == t[:-1]) & (vals[1:] > vals[:-1]))
    assert bool(asc.all()), "(key, index) not strictly increasing"
    seen = torch.zeros(n, dtype=torch.int32, device="cuda")
    seen[vals] = 1
    assert int(seen.sum().item()) == n, "payloads are not a permutation of the indices"


def test_pairs_2p27_duplicate_heavy():
    _pairs_check(I.dup_keys_u64(1 << 27, 2), O.KT_U64)


def test_pairs_2p27_f32_normal_with_signed_zeros():
    _pairs_check(I.normal_f32(1 << 27, 3), O.KT_F32)


def test_segmented_100k_u32():
    """Batched segmented sort at full size: 100,000 uint32 segments with log-uniform
    lengths rescaled to ~2^28 keys in total, uniform values, device offsets.  Every
    segment must come out sorted and hold its own input multiset; a sample of
    segments is compared with the oracle element by element."""
    lens = I.segment_lengths(100000, 1 << 28, 4, max_log2=20)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    n = int(off[-1])
    keys = I.generate("uniform", n, 4, 32, device="cuda")
    kin = keys.clone()
    doff = torch.from_numpy(off).cuda()
    ams.sort_segmented(keys, doff, levels=1, buckets=[16], kt=O.KT_U32)
    ams.sync()
    seg = torch.repeat_interleave(torch.arange(len(lens), device="cuda"), torch.from_numpy(lens).cuda())
    u = keys.to(torch.int64) & 0xFFFFFFFF
    ok = (u[1:] >= u[:-1]) | (seg[1:] != seg[:-1])
    assert bool(ok.all()), "a segment is not sorted"
    uin = kin.to(torch.int64) & 0xFFFFFFFF
    h_in = torch.zeros(len(lens), dtype=torch.int64, device="cuda").index_add_(0, seg, I._mix_t(uin))
    h_out = torch.zeros(len(lens), dtype=torch.int64, device="cuda").index_add_(0, seg, I._mix_t(u))
    assert torch.equal(h_in, h_out), "a segment does not hold its own keys"
    rng = np.random.default_rng(4)
    big = np.argsort(lens)[-3:]
    for s in np.concatenate([rng.integers(0, len(lens), 20), big]):
        lo, hi = int(off[s]), int(off[s + 1])
        want = O.sort_keys(O.KT_U32, kin[lo:hi].cpu().numpy().view(np.uint32))
        assert np.array_equal(keys[lo:hi].cpu().numpy().view(np.uint32), want)
