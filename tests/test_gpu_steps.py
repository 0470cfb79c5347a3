"""Per-kernel parity: every step of one distribution level, run through the C ABI on
the GPU, against the oracle's restatement of the same step (bit-exact)."""
import numpy as np
import pytest

import oracle as O
from paper_1410_6754_gb300 import inputs as I

from helpers import ordered_dtype, same_bits, to_dev, to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1410_6754_gb300 as ams  # noqa: E402

KTS = [(O.KT_U32, 32), (O.KT_U64, 64), (O.KT_F32, 32)]


def _keys(kt, bits, dist, n, seed):
    if kt == O.KT_F32:
        return I.normal_f32(n, seed)
    return I.generate(dist, n, seed, bits)


@pytest.mark.parametrize("kt,bits", KTS)
@pytest.mark.parametrize("n,count", [(1, 5), (1000, 2047), (1000, 2048), ((1 << 20) + 3, 5000),
                                     (77777, 14336)])
def test_sample(kt, bits, n, count):
    keys = _keys(kt, bits, "uniform", n, 3)
    for level, begin, seed in [(1, 0, 0), (2, 123456, 7), (3, 2**31, 2**63 + 5)]:
        got = ams.step_sample(to_dev(keys), count, seed, level, begin, kt=kt)
        torch.cuda.synchronize()
        exp = O.sample(O.ordered_keys(kt, keys), seed, level, begin, count)
        assert same_bits(to_np(got, ordered_dtype(kt)), exp.astype(ordered_dtype(kt)))


@pytest.mark.parametrize("kt,bits", [(O.KT_U32, 32), (O.KT_U64, 64)])
@pytest.mark.parametrize("S", [1, 2, 3, 100, 2047, 2048, 2049, 4096, 10240, 14336, 65536])
def test_rank_sort(kt, bits, S):
    dt = ordered_dtype(kt)
    rng = np.random.default_rng(S)
    cases = [I.generate("uniform", S, S, bits),
             rng.integers(0, 7, size=S).astype(dt),            # heavy ties
             np.full(S, 5, dtype=dt),                           # all equal
             np.sort(I.generate("uniform", S, 1, bits))[::-1].copy()]
    for s in cases:
        got = ams.step_rank_sort(to_dev(s), kt)
        torch.cuda.synchronize()
        _, exp = O.rank_sort(s.astype(np.uint64))
        assert same_bits(to_np(got, dt), exp.astype(dt))


@pytest.mark.parametrize("kt,bits", [(O.KT_U32, 32), (O.KT_U64, 64)])
@pytest.mark.parametrize("a,B", [(1, 2), (16, 256), (14, 1024), (10, 1024), (3, 2048), (2, 7)])
def test_splitters(kt, bits, a, B):
    dt = ordered_dtype(kt)
    srt = np.sort(I.generate("zipf", a * B, a + B, bits))
    got = ams.step_splitters(to_dev(srt), a, B, kt)
    torch.cuda.synchronize()
    assert same_bits(to_np(got, dt), O.splitters(srt.astype(np.uint64), a, B).astype(dt))


@pytest.mark.parametrize("kt,bits", KTS)
@pytest.mark.parametrize("B", [2, 3, 5, 256, 1000, 1024, 2048])
def test_classify(kt, bits, B):
    dt = ordered_dtype(kt)
    n = 300001
    keys = _keys(kt, bits, "zipf", n, B)
    t = O.ordered_keys(kt, keys)
    # splitters from the keys themselves (repeats included), plus the largest key
    rng = np.random.default_rng(B)
    spl = np.sort(t[rng.integers(0, n, size=B - 1)])
    if B > 3:
        spl[-1] = np.iinfo(dt).max
    keys2 = keys.copy()
    if kt != O.KT_F32:
        keys2[:5] = np.iinfo(dt).max
        t = O.ordered_keys(kt, keys2)
    counts, ids = ams.step_classify(to_dev(keys2), to_dev(spl.astype(dt)), B, kt=kt)
    torch.cuda.synchronize()
    exp_ids = O.classify(spl, B, t)
    assert np.array_equal(to_np(ids, np.uint16).astype(np.int64), exp_ids)
    assert np.array_equal(to_np(counts, np.uint32).astype(np.int64), O.bucket_counts(exp_ids, B))


@pytest.mark.parametrize("kt,bits", KTS)
@pytest.mark.parametrize("B", [2, 3, 17, 256, 1024, 2048])
def test_classify_uniform_short_spans(kt, bits, B):
    """Distinct, evenly spread splitters (the short-span path of the table classifier:
    at most three splitter values per cell), keys equal to splitters, keys below the
    first splitter, and keys equal to the largest key above every splitter."""
    dt = ordered_dtype(kt)
    n = 200003
    keys = _keys(kt, bits, "uniform", n, 1000 + B)
    t = O.ordered_keys(kt, keys)
    spl = np.unique(np.sort(t[np.random.default_rng(B).integers(0, n, size=B - 1)]))
    while len(spl) < B - 1:  # (distinct splitters)
        spl = np.unique(np.concatenate([spl, spl[-1:] + np.arange(1, B, dtype=np.uint64)]))[:B - 1]
    spl = spl.astype(np.uint64)
    if kt != O.KT_F32:
        keys = keys.copy()
        keys[:7] = np.iinfo(dt).max                       # above every splitter
        keys[7:14] = spl[np.arange(7) % len(spl)].astype(dt)  # equal to splitters
        keys[14:21] = 0
        t = O.ordered_keys(kt, keys)
    counts, ids = ams.step_classify(to_dev(keys), to_dev(spl.astype(dt)), B, kt=kt)
    torch.cuda.synchronize()
    exp_ids = O.classify(spl, B, t)
    assert np.array_equal(to_np(ids, np.uint16).astype(np.int64), exp_ids)
    assert np.array_equal(to_np(counts, np.uint32).astype(np.int64), O.bucket_counts(exp_ids, B))


def _golden_binpack():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "binpack_examples.txt")
    out = []
    for ln in open(path):
        ln = ln.strip()
        if not ln or ln.startswith("#"):
            continue
        r, w, L, ends = (p.strip() for p in ln.split(";"))
        out.append((int(r), [int(x) for x in w.split()], int(L), [int(x) for x in ends.split()]))
    return out


def _run_binpack(w, r):
    B = len(w)
    counts = np.zeros(2 * B - 1, dtype=np.uint32)
    counts[0::2] = w
    counts[1::2] = 3  # equality buckets weigh nothing
    L, ends, ng = ams.step_bin_pack(to_dev(counts), B, r)
    torch.cuda.synchronize()
    ng = int(ng.item())
    return int(L.item()), [int(x) for x in to_np(ends, np.uint32)[:ng]]


def test_bin_pack_golden():
    for r, w, L, ends in _golden_binpack():
        if len(w) < 2 or r > len(w):
            continue
        assert _run_binpack(w, r) == (L, ends)


@pytest.mark.parametrize("B", [2, 3, 16, 255, 1024, 2048])
def test_bin_pack_random(B):
    rng = np.random.default_rng(B)
    for trial in range(12):
        r = int(rng.integers(1, B + 1)) if trial % 3 else min(B, 256)
        kind = trial % 4
        if kind == 0:
            w = rng.integers(0, 1000, size=B)
        elif kind == 1:
            w = rng.poisson(262144, size=B)           # large, near-equal buckets
        elif kind == 2:
            w = rng.choice([0, 0, 1, 5, 100000], size=B)
        else:
            w = np.zeros(B, dtype=np.int64)
            w[rng.integers(0, B)] = 12345
        L, ends = O.bin_pack([int(x) for x in w], r)
        assert _run_binpack(w.astype(np.uint32), r) == (L, ends)


@pytest.mark.parametrize("kt,bits", KTS)
@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("n,B", [(5000, 2), (100003, 256), (1 << 20, 1024), (262147, 2048)])
def test_partition(kt, bits, pairs, n, B):
    dt = ordered_dtype(kt)
    keys = _keys(kt, bits, "zipf", n, n)
    t = O.ordered_keys(kt, keys)
    rng = np.random.default_rng(n)
    spl = np.sort(t[rng.integers(0, n, size=B - 1)])
    vals = np.arange(n, dtype=np.uint64) * np.uint64(3) + np.uint64(1)
    res = ams.step_partition(to_dev(keys), to_dev(spl.astype(dt)), B,
                             vals=to_dev(vals) if pairs else None, kt=kt)
    torch.cuda.synchronize()
    perm = O.stable_partition(O.classify(spl, B, t))
    out = res[0] if pairs else res
    # keys come back in order form
    assert same_bits(to_np(out, dt), t[perm].astype(dt))
    if pairs:
        assert np.array_equal(to_np(res[1], np.uint64), vals[perm])


@pytest.mark.parametrize("kt,bits", KTS)
@pytest.mark.parametrize("dist", ["uniform", "zipf", "sorted"])
@pytest.mark.parametrize("n,B", [(5000, 2), (100003, 256), (1 << 20, 1024), (262147, 2048)])
def test_partition_arrival(kt, bits, dist, n, B):
    """The keys-only delivery the sorts use: every bucket's range holds exactly the
    bucket's keys (the oracle's stable partition, compared as a multiset per bucket,
    since the order inside a bucket is arrival order)."""
    dt = ordered_dtype(kt)
    keys = _keys(kt, bits, dist, n, n + 7)
    t = O.ordered_keys(kt, keys)
    rng = np.random.default_rng(n + B)
    spl = np.sort(t[rng.integers(0, n, size=B - 1)])
    out = to_np(ams.step_partition_arrival(to_dev(keys), to_dev(spl.astype(dt)), B, kt=kt), dt)
    torch.cuda.synchronize()
    ids = O.classify(spl, B, t)
    expect = t[O.stable_partition(ids)].astype(dt)
    bucket_of_pos = np.repeat(np.arange(2 * B - 1), O.bucket_counts(ids, B))
    o1 = np.lexsort((out, bucket_of_pos))
    o2 = np.lexsort((expect, bucket_of_pos))
    assert same_bits(out[o1], expect[o2])


@pytest.mark.parametrize("kt,bits", KTS)
@pytest.mark.parametrize("pairs", [False, True])
def test_base_case(kt, bits, pairs):
    cap = ams.default_basecase_cap(kt, pairs)
    rng = np.random.default_rng(int(cap) + kt)
    for n in [1, 2, 3, 31, 100, 1000, 4095, 4096, cap - 1, cap]:
        for dist in ["uniform", "equal", "sorted", "few"]:
            if kt == O.KT_F32:
                keys = I.normal_f32(n, n)
                if dist == "few":
                    keys = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf], np.float32)[rng.integers(0, 6, n)]
                elif dist == "equal":
                    keys = np.full(n, -0.0, np.float32)
            elif dist == "few":
                keys = rng.integers(0, 3, size=n).astype(ordered_dtype(kt))
            else:
                keys = I.generate(dist, n, n, bits)
            vals = np.arange(n, dtype=np.uint64)
            dk = to_dev(keys)
            dv = to_dev(vals) if pairs else None
            ams.step_base_case(dk, dv, kt=kt)
            torch.cuda.synchronize()
            ek, ev = O.sort_pairs(kt, keys, vals)
            assert same_bits(to_np(dk, keys.dtype), ek), (n, dist)
            if pairs:
                assert np.array_equal(to_np(dv, np.uint64), ev), (n, dist)
