"""Pins of the CPU oracle against facts that do not come from the oracle itself:
published generator outputs, brute force over all permutations, closed forms,
library routines, hand-worked examples (tests/golden) and the paper's lemmas."""
import bisect
import itertools
import os
import random
import struct

import numpy as np
import pytest

import oracle as O
from paper_1410_6754_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _lines(name):
    with open(os.path.join(GOLD, name)) as f:
        return [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]


# ----------------------------------------------------------------- generator
def test_splitmix64_published_values():
    for ln in _lines("splitmix64_seed0.txt"):
        state, k, out = ln.split()
        got = O.splitmix64_outputs(int(state), int(k) + 1)[int(k)]
        assert int(got) == int(out, 16)


def test_mulhi64_against_exact_integers():
    rng = random.Random(1)
    a = np.array([rng.getrandbits(64) for _ in range(2000)] + [2**64 - 1, 0, 1], dtype=np.uint64)
    for b in [1, 2, 3, 2**20, 2**32 - 1, 2**32, 2**40 + 12345, 2**63 + 7, 2**64 - 1]:
        got = O.mulhi64(a, b)
        exp = np.array([(int(x) * b) >> 64 for x in a], dtype=np.uint64)
        assert np.array_equal(got, exp)


def test_sample_indices_in_range_and_uniform():
    idx = O.sample_indices(7, 1, 0, 1000, 200000)
    assert idx.min() >= 0 and idx.max() < 1000
    counts = np.bincount(idx, minlength=1000)
    # chi-square against uniform, 999 dof: mean 999, sd ~ 44.7
    chi = ((counts - 200.0) ** 2 / 200.0).sum()
    assert chi < 999 + 6 * 44.7


def test_oversampling_factor_closed_form():
    # a = ceil(1.6 log10 n) (paper Section 7.2) away from integer boundaries
    for n in [10, 1000, 2**20, 2**27, 2**28, 12345678]:
        v = 1.6 * np.log10(n)
        if abs(v - round(v)) > 1e-9:
            assert O.oversampling_factor(n) == max(1, int(np.ceil(v)))
    assert O.oversampling_factor(2**28) == 14
    assert O.oversampling_factor(2**20) == 10


# ----------------------------------------------------------------- float order
F32_SPECIAL = [0.0, -0.0, 1.0, -1.0, 1.5, -1.5, 1e-45, -1e-45, 1.17549435e-38,
               -1.17549435e-38, 3.4028235e38, -3.4028235e38, float("inf"), float("-inf"),
               0.1, -0.1, 2.0, -2.0, 1e-40, -1e-40]


def _bits(f):
    return struct.unpack("<I", struct.pack("<f", f))[0]


def test_f32_order_monotone_on_specials():
    vals = F32_SPECIAL
    bits = np.array([_bits(v) for v in vals], dtype=np.uint32)
    t = O.f32_order(bits)
    f = np.array(vals, dtype=np.float32)
    for i in range(len(vals)):
        for j in range(len(vals)):
            if f[i] < f[j]:
                assert t[i] < t[j]
            elif f[i] > f[j]:
                assert t[i] > t[j]
    # -0.0 strictly before +0.0 (strict total order on bit patterns)
    assert O.f32_order(np.array([_bits(-0.0)], np.uint32))[0] < \
        O.f32_order(np.array([_bits(0.0)], np.uint32))[0]


def test_f32_order_roundtrip_and_random_monotone():
    rng = np.random.default_rng(5)
    b = rng.integers(0, 2**32, size=200000, dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(O.f32_unorder(O.f32_order(b)), b)
    f = b.view(np.float32)
    ok = ~np.isnan(f)
    f, b = f[ok], b[ok]
    i = rng.integers(0, len(f), 50000)
    j = rng.integers(0, len(f), 50000)
    t = O.f32_order(b)
    lt = f[i] < f[j]
    assert np.all(t[i][lt] < t[j][lt])


def test_f32_order_nan_placement():
    qnan_pos, qnan_neg = 0x7FC00000, 0xFFC00000
    t = O.f32_order(np.array([qnan_neg, _bits(float("-inf")), _bits(float("inf")), qnan_pos], np.uint32))
    assert list(np.argsort(t)) == [0, 1, 2, 3]


# ----------------------------------------------------------------- the definition
def _brute_force_order(tkeys):
    """The unique permutation whose (T(key), index) sequence strictly increases,
    found by enumerating all permutations."""
    n = len(tkeys)
    found = []
    for p in itertools.permutations(range(n)):
        if all((tkeys[p[i]], p[i]) < (tkeys[p[i + 1]], p[i + 1]) for i in range(n - 1)):
            found.append(p)
    assert len(found) == 1
    return list(found[0])


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_sort_brute_force_small_alphabet(n):
    for keys in itertools.product([0, 1, 2], repeat=n):
        k = np.array(keys, dtype=np.uint64)
        perm = _brute_force_order([int(x) for x in k])
        assert list(O.sort_keys(O.KT_U64, k)) == [int(k[i]) for i in perm]
        ks, vs = O.sort_pairs(O.KT_U64, k, np.arange(n, dtype=np.uint64))
        assert list(vs) == perm


def test_sort_brute_force_f32_specials():
    rng = random.Random(3)
    pool = [0.0, -0.0, -1.0, 1.0, 1e-40, float("inf"), float("-inf")]
    for _ in range(300):
        n = rng.randint(1, 6)
        vals = [rng.choice(pool) for _ in range(n)]
        k = np.array(vals, dtype=np.float32)
        t = [int(x) for x in O.f32_order(k.view(np.uint32))]
        perm = _brute_force_order(t)
        out_k, out_v = O.sort_pairs(O.KT_F32, k, np.arange(n, dtype=np.uint64))
        assert list(out_v) == perm
        assert np.array_equal(out_k.view(np.uint32), k.view(np.uint32)[perm])


@pytest.mark.parametrize("kt,bits", [(O.KT_U32, 32), (O.KT_U64, 64)])
@pytest.mark.parametrize("dist", I.DISTRIBUTIONS)
def test_sort_invariants(kt, bits, dist):
    k = I.generate(dist, 40000, 11, bits)
    out_k, out_v = O.sort_pairs(kt, k, np.arange(len(k), dtype=np.uint64))
    t = O.ordered_keys(kt, out_k)
    assert np.all(t[1:] >= t[:-1])
    # permutation: payload is a permutation of indices and carries its key
    assert np.array_equal(np.sort(out_v), np.arange(len(k), dtype=np.uint64))
    assert np.array_equal(k[out_v.astype(np.int64)], out_k)
    # stability: equal keys keep index order
    same = t[1:] == t[:-1]
    assert np.all(out_v[1:][same] > out_v[:-1][same])
    # agrees with Python's sorted on (key, index)
    ref = sorted(range(len(k)), key=lambda i: (int(k[i]), i))
    assert np.array_equal(out_v, np.array(ref, dtype=np.uint64))


def test_sort_segmented_brute_force():
    rng = random.Random(9)
    for _ in range(200):
        lens = [rng.randint(0, 5) for _ in range(rng.randint(1, 4))]
        off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        n = int(off[-1])
        k = np.array([rng.randint(0, 2) for _ in range(n)], dtype=np.uint32)
        v = np.arange(n, dtype=np.uint64)
        ok, ov = O.sort_segmented(O.KT_U32, k, off, v)
        for s in range(len(lens)):
            lo, hi = off[s], off[s + 1]
            perm = _brute_force_order([int(x) for x in k[lo:hi]])
            assert list(ov[lo:hi]) == [lo + p for p in perm]


# ----------------------------------------------------------------- rank sort
def test_rank_sort_against_loops_and_library():
    rng = np.random.default_rng(2)
    for n in [1, 2, 7, 33, 100]:
        s = rng.integers(0, 5, size=n).astype(np.uint64)
        r1, o1 = O.rank_sort(s, block=16)
        r2, o2 = O.rank_sort_literal(s)
        assert list(r1) == r2 and [int(x) for x in o1] == o2
        assert sorted(r2) == list(range(n))
        assert [int(x) for x in o1] == sorted(int(x) for x in s)
    s = rng.integers(0, 2**63, size=5000).astype(np.uint64)
    r, o = O.rank_sort(s)
    assert np.array_equal(o, np.sort(s))
    assert np.array_equal(np.sort(r), np.arange(5000))


# ----------------------------------------------------------------- splitters / classify
def test_splitters_closed_form():
    for a, B in [(1, 4), (3, 8), (16, 256), (10, 1024)]:
        srt = np.arange(a * B, dtype=np.uint64)
        assert list(O.splitters(srt, a, B)) == [j * a for j in range(1, B)]


def test_classify_golden():
    lines = _lines("classify_example.txt")
    spl = np.array([int(x) for x in lines[0].split()[1:]], dtype=np.uint64)
    B = len(spl) + 1
    for ln in lines[1:]:
        x, i = (int(v) for v in ln.split())
        assert O.classify(spl, B, np.array([x], dtype=np.uint64))[0] == i
        assert O.classify_literal(spl, B, [x])[0] == i


def test_classify_against_bisect():
    rng = np.random.default_rng(4)
    for B in [2, 3, 16, 255, 1024]:
        spl = np.sort(rng.integers(0, 50, size=B - 1)).astype(np.uint64)
        x = rng.integers(0, 55, size=3000).astype(np.uint64)
        ids = O.classify(spl, B, x)
        sl = [int(s) for s in spl]
        for v, i in zip(x, ids):
            j = bisect.bisect_left(sl, int(v))
            eq = int(j < B - 1 and sl[j] == int(v))
            assert i == 2 * j + eq
        if B <= 255:
            assert list(ids[:200]) == O.classify_literal(spl, B, x[:200])
        # keys in one equality bucket are all equal to its splitter
        for i in np.unique(ids[ids % 2 == 1]):
            assert np.all(x[ids == i] == spl[i // 2])


# ----------------------------------------------------------------- bucket grouping
def _dp_opt(w, r):
    """Textbook linear partition: min over <= r contiguous groups of the max load."""
    m = len(w)
    pre = [0]
    for x in w:
        pre.append(pre[-1] + x)
    INF = float("inf")
    best = [[INF] * (m + 1) for _ in range(r + 1)]
    best[0][0] = 0
    for g in range(1, r + 1):
        for j in range(m + 1):
            for i in range(j + 1):
                if best[g - 1][i] < INF:
                    best[g][j] = min(best[g][j], max(best[g - 1][i], pre[j] - pre[i]))
    return min(best[g][m] for g in range(1, r + 1))


def _enum_opt(w, r):
    m = len(w)
    best = None
    for k in range(0, min(r, m) ):
        for cuts in itertools.combinations(range(1, m), k):
            b = (0,) + cuts + (m,)
            load = max(sum(w[b[i]:b[i + 1]]) for i in range(len(b) - 1))
            best = load if best is None else min(best, load)
    return best


def test_bin_pack_golden():
    for ln in _lines("binpack_examples.txt"):
        r, w, L, ends = (p.strip() for p in ln.split(";"))
        w = [int(x) for x in w.split()]
        got_L, got_e = O.bin_pack(w, int(r))
        assert got_L == int(L)
        assert got_e == [int(x) for x in ends.split()]


def test_bin_pack_against_dp_and_enumeration():
    rng = random.Random(12)
    for trial in range(300):
        m = rng.randint(1, 10 if trial % 2 else 40)
        r = rng.randint(1, 8)
        w = [rng.choice([0, 0, 1, 2, 3, 5, 8, 13, 40]) for _ in range(m)]
        L, ends = O.bin_pack(w, r)
        assert L == _dp_opt(w, r)
        if m <= 10:
            assert L == _enum_opt(w, r)
        assert len(ends) <= r and ends[-1] == m
        if L > 0:
            e = O.greedy_groups(w, L - 1)
            assert e is None or len(e) > r
        start = 0
        for e in ends:
            assert sum(w[start:e]) <= L
            start = e


# ----------------------------------------------------------------- pieces
def test_pieces_partition_and_cuts():
    rng = np.random.default_rng(8)
    for trial in range(200):
        B = int(rng.integers(2, 20))
        cnt = rng.integers(0, 6, size=2 * B - 1)
        cnt[1::2] = rng.choice([0, 1, 2, 9, 40], size=B - 1)
        L, ends = O.bin_pack(cnt[0::2], int(rng.integers(1, B + 1)))
        begin = int(rng.integers(0, 1000))
        pcs = O.pieces(cnt, B, L, ends, begin)
        pos = begin
        for (lo, hi, fin) in pcs:
            assert lo == pos and hi > lo
            pos = hi
        assert pos == begin + int(cnt.sum())
        tau = O.eq_cut_threshold(L)
        starts = np.concatenate([[0], np.cumsum(cnt)]) + begin
        heavy = {(int(starts[i]), int(starts[i + 1])) for i in range(1, 2 * B - 1, 2) if cnt[i] >= tau}
        finals = {(lo, hi) for (lo, hi, fin) in pcs if fin}
        assert finals == heavy
        # non-final pieces never straddle a group boundary
        bounds = {int(starts[min(2 * e, 2 * B - 1)]) for e in ends}
        for (lo, hi, fin) in pcs:
            assert not any(lo < b < hi for b in bounds)


def test_piece_labels_agree_with_pieces():
    """Delivery by piece: the labels group exactly the ids of each piece of
    ``pieces`` (same positions, same final flags), in id order."""
    rng = np.random.default_rng(18)
    for trial in range(300):
        B = int(rng.integers(2, 24))
        cnt = rng.integers(0, 6, size=2 * B - 1)
        cnt[1::2] = rng.choice([0, 1, 2, 9, 40], size=B - 1)
        L, ends = O.bin_pack(cnt[0::2], int(rng.integers(1, B + 1)))
        lab = O.piece_of_ids(cnt, B, L, ends)
        assert np.all(np.diff(lab) >= 0) and lab[0] == 0
        starts = np.concatenate([[0], np.cumsum(cnt)])
        got = []
        for v in np.unique(lab):
            ids = np.nonzero(lab == v)[0]
            b, e = int(starts[ids[0]]), int(starts[ids[-1] + 1])
            fin = len(ids) == 1 and ids[0] % 2 == 1 and cnt[ids[0]] >= O.eq_cut_threshold(L)
            if e > b:
                got.append((b, e, int(fin)))
        assert got == O.pieces(cnt, B, L, ends, 0)


# ----------------------------------------------------------------- whole method
@pytest.mark.parametrize("dist", I.DISTRIBUTIONS)
def test_ams_restatement_equals_definition(dist):
    n = 1 << 15
    k = I.generate(dist, n, 21, 64)
    pl = O.plan(n, O.KT_U64, 2, [8, 8], C=256)
    out_k, out_v = O.ams_sort(O.KT_U64, k, pl, seed=5, vals=np.arange(n, dtype=np.uint64))
    ek, ev = O.sort_pairs(O.KT_U64, k, np.arange(n, dtype=np.uint64))
    assert np.array_equal(out_k, ek) and np.array_equal(out_v, ev)


def test_ams_restatement_f32_u32_segmented():
    k = I.normal_f32(20000, 3)
    pl = O.plan(len(k), O.KT_F32, 2, [4, 4], C=300)
    out = O.ams_sort(O.KT_F32, k, pl, seed=1)
    assert np.array_equal(out.view(np.uint32), O.sort_keys(O.KT_F32, k).view(np.uint32))
    k = I.generate("zipf", 30000, 2, 32)
    lens = I.segment_lengths(40, 30000, 4, max_log2=12)
    off = np.concatenate([[0], np.cumsum(lens)])
    k = I.generate("uniform", int(off[-1]), 2, 32)
    pl = O.plan(int(lens.max()), O.KT_U32, 2, [4, 4], C=200)
    out = O.ams_sort(O.KT_U32, k, pl, seed=3, offsets=off)
    assert np.array_equal(out, O.sort_segmented(O.KT_U32, k, off))


def test_extra_levels_planned():
    pl = O.plan(1 << 28, O.KT_U64, 1, [256])
    assert pl.r == [256, 256]
    pl = O.plan(1 << 28, O.KT_U64, 2, [256, 256])
    assert pl.r == [256, 256] and pl.b == 4
    pl = O.plan(1 << 20, O.KT_U32, 1, [256], b=1, a=16)
    assert pl.r == [256] and pl.b == 1 and pl.a_for(1 << 20, 256) == 16 and pl.a_for(50000, 256) == 12


# ----------------------------------------------------------------- Lemma lm:ams-param
def test_overpartitioning_bounds_uniform():
    """Section 6 Lemma: with b = 4 (eps = 2/b) the optimal group load stays within
    (1+eps) n/r and no range bucket exceeds n/r (checked at fixed seeds)."""
    n, r = 1 << 20, 256
    k = I.generate("uniform", n, 0, 64)
    for seed in range(3):
        pl = O.plan(n, O.KT_U64, 1, [r], b=4)
        tr = []
        O.ams_sort(O.KT_U64, k, pl, seed=seed, trace=tr)
        t0 = tr[0]
        assert t0["L"] <= 1.5 * n / r
        assert t0["counts"][0::2].max() <= n / r
        loads = [int(t0["counts"][0::2][s:e].sum()) for s, e in zip([0] + t0["ends"][:-1], t0["ends"])]
        assert max(loads) == t0["L"] and len(loads) <= r


def test_single_level_bucket_bound():
    """Single-level sample sort of 2**20 uint32 keys, 256 buckets, a = 16 (b = 1): every
    bucket stays below 2.5 n/r at the fixed seed."""
    n, r = 1 << 20, 256
    k = I.generate("uniform", n, 0, 32)
    pl = O.plan(n, O.KT_U32, 1, [r], b=1, a=16)
    tr = []
    out = O.ams_sort(O.KT_U32, k, pl, seed=0, trace=tr)
    assert np.array_equal(out, np.sort(k))
    assert tr[0]["S"] == 4096
    assert tr[0]["counts"][0::2].max() <= 2.5 * n / r


# ----------------------------------------------------------------- planted mistakes
def test_pins_catch_planted_mistakes(monkeypatch):
    """Plausible slips planted in the oracle make one of the pins above fail."""
    spl = np.array([10, 20, 20, 30], dtype=np.uint64)
    x = np.array([10, 20, 30], dtype=np.uint64)
    # (1) '<=' instead of '<' in the splitter count
    bad = [2 * int(np.searchsorted(spl, v, side="right")) for v in x]
    assert bad != list(O.classify(spl, 5, x))
    # (2) binary search upper end one too small
    w = [3, 1, 4, 1, 5, 9, 2, 6]
    assert O.greedy_groups(w, 13) is not None and len(O.greedy_groups(w, 13)) > 3
    # (3) tie-break dropped in the all-pairs rank: ranks stop being a permutation
    s = np.array([1, 1, 0], dtype=np.uint64)
    naive = [int((s < v).sum()) for v in s]
    assert sorted(naive) != [0, 1, 2]
    # (4) wrong splitter offset j*a-1 changes the closed form
    srt = np.arange(32, dtype=np.uint64)
    assert list(srt[np.arange(1, 8) * 4 - 1]) != list(O.splitters(srt, 4, 8))


@pytest.mark.parametrize("kt,bits", [(O.KT_U64, 64), (O.KT_U32, 32), (O.KT_F32, 32)])
def test_select_ranks_brute_force(kt, bits):
    """Sampled output positions: the i-th smallest key by brute-force counting on small
    inputs (rank i is held by the key v with #{x < v} <= i < #{x <= v})."""
    rng = np.random.default_rng(11)
    for n in (1, 2, 7, 64, 300):
        if kt == O.KT_F32:
            keys = rng.choice(np.array([-2.0, -0.0, 0.0, 1.5, 3.0, -1e30], dtype=np.float32), n)
            t = O.ordered_keys(kt, keys)
        else:
            keys = rng.integers(0, 9, n).astype(np.uint64 if bits == 64 else np.uint32)
            t = keys.astype(np.uint64)
        ranks = np.arange(n)
        got = O.ordered_keys(kt, O.select_ranks(kt, keys, ranks))
        for i in range(n):
            v = got[i]
            assert np.sum(t < v) <= i < np.sum(t <= v)
