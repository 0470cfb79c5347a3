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


def test_sort_keys_f32_hand_order():
    """Float keys in float order with -0.0 before +0.0, written out by hand."""
    k = np.array([1.0, -0.0, float("-inf"), 0.0, -1.0, float("inf"), 1e-45, -1e-45, -1.0], dtype=np.float32)
    exp = np.array([float("-inf"), -1.0, -1.0, -1e-45, -0.0, 0.0, 1e-45, 1.0, float("inf")], dtype=np.float32)
    assert np.array_equal(O.sort_keys(O.KT_F32, k).view(np.uint32), exp.view(np.uint32))


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


# ----------------------------------------------------------------- sample stream
def test_sample_stream_golden():
    """Stream states and first draws written by tests/golden/make_sample_stream.py, which
    implements SplitMix64 in its stateful form with plain Python integers and imports
    nothing from this repository."""
    for ln in _lines("sample_stream.txt"):
        head, idx = ln.split(";")
        seed, level, begin, n_g, state = head.split()
        exp = [int(x) for x in idx.split()]
        assert O.stream_key(int(seed), int(level), int(begin)) == int(state, 16), ln
        got = O.sample_indices(int(seed), int(level), int(begin), int(n_g), len(exp))
        assert [int(x) for x in got] == exp, ln


def test_a_for_hand_values():
    """READING of the oversampling factor: ceil(1.6 log10 n_g) (or the fixed a), capped
    at max(1, n_g // (16 B)).  Values worked by hand."""
    pl = O.plan(1 << 20, O.KT_U64, 2, [256, 256])
    assert pl.a_for(1 << 20, 1024) == 10          # 1.6 * 6.02 = 9.63 -> 10; cap 64
    assert pl.a_for(100000, 1024) == 6            # 1.6 * 5 = 8; cap 100000 // 16384 = 6
    assert pl.a_for(20000, 1024) == 1             # cap 20000 // 16384 = 1
    assert pl.a_for(1000, 1024) == 1              # cap max(1, 0) = 1
    fixed = O.plan(1 << 20, O.KT_U32, 1, [256], b=1, a=16)
    assert fixed.a_for(1 << 20, 256) == 16        # cap 256
    assert fixed.a_for(50000, 256) == 12          # cap 50000 // 4096 = 12


# ----------------------------------------------------------------- pieces (reading)
def test_eq_cut_threshold_golden():
    for ln in _lines("eq_cut_threshold.txt"):
        L, t = (int(v) for v in ln.split())
        assert O.eq_cut_threshold(L) == t, ln


def _piece_cases():
    for ln in _lines("pieces_examples.txt"):
        B, cnt, r, L, ends, begin, pcs, lab = (p.strip() for p in ln.split(";"))
        yield (int(B), [int(x) for x in cnt.split()], int(r), int(L), [int(x) for x in ends.split()],
               int(begin), [tuple(int(v) for v in p.split(",")) for p in pcs.split()],
               [int(x) for x in lab.split()])


def test_pieces_golden():
    """Hand-worked pieces (tests/golden/pieces_examples.txt): the grouping, the final
    equality pieces (one at a group's end, one at a group's start, two in a row), the
    dropped empty runs and the per-id labels of the delivery order."""
    n = 0
    for B, cnt, r, L, ends, begin, pcs, lab in _piece_cases():
        gL, ge = O.bin_pack(cnt[0::2], r)
        assert (gL, ge) == (L, ends)
        assert O.pieces(np.array(cnt), B, L, ends, begin) == pcs
        assert list(O.piece_of_ids(np.array(cnt), B, L, ends)) == lab
        n += 1
    assert n == 5


# ----------------------------------------------------------------- RLM-sort (Section 5)
def _brute_split(seqs, k):
    """Split positions of rank k by listing every element as (key, sequence, position)
    and sorting the tuples (Python's sort; no numpy)."""
    els = sorted((int(v), i, j) for i, q in enumerate(seqs) for j, v in enumerate(q))
    cnt = [0] * len(seqs)
    for (_, i, _) in els[:k]:
        cnt[i] += 1
    return cnt


def test_multiseq_select_brute_force():
    """Section 4.1: the definition and the quickselect both equal the brute-force split
    for every rank of small sorted sequences with many ties (and empty sequences)."""
    rng = np.random.default_rng(31)
    for trial in range(250):
        p = int(rng.integers(1, 6))
        seqs = [np.sort(rng.integers(0, 4, int(rng.integers(0, 7)))).astype(np.uint64) for _ in range(p)]
        total = sum(len(q) for q in seqs)
        for k in range(total + 1):
            want = _brute_split(seqs, k)
            assert O.multiseq_select_definition(seqs, k) == want
            assert O.multiseq_select(seqs, k, seed=trial) == want


def test_multiseq_select_hand_example():
    # sequences (1 3 3 7), (3 5), (0 3): total order by (key, sequence, position):
    # 0(s2) 1(s0) 3(s0) 3(s0) 3(s1) 3(s2) 5(s1) 7(s0)
    seqs = [np.array([1, 3, 3, 7], np.uint64), np.array([3, 5], np.uint64), np.array([0, 3], np.uint64)]
    want = {0: [0, 0, 0], 1: [0, 0, 1], 2: [1, 0, 1], 4: [3, 0, 1], 5: [3, 1, 1], 6: [3, 1, 2],
            7: [3, 2, 2], 8: [4, 2, 2]}
    for k, cut in want.items():
        assert O.multiseq_select(seqs, k) == cut
        assert O.multiseq_select_definition(seqs, k) == cut


@pytest.mark.parametrize("dist", I.DISTRIBUTIONS)
def test_rlm_sort_equals_definition(dist):
    """Section 5: RLM-sort (runs sorted, parts by multisequence selection, pieces
    delivered, local merge) gives the definition's output, and every part of every
    level is perfectly balanced (sizes differ by at most one)."""
    n = 6000
    k = I.generate(dist, n, 13, 64)
    v = np.arange(n, dtype=np.uint64)
    tr = []
    ok, ov = O.rlm_sort(O.KT_U64, k, 257, [5, 4], vals=v, trace=tr)
    ek, ev = O.sort_pairs(O.KT_U64, k, v)
    assert np.array_equal(ok, ek) and np.array_equal(ov, ev)
    for t in tr:
        sizes = np.diff(t["ranks"])
        assert sizes.max() - sizes.min() <= 1
        assert sum(t["cuts"][-1]) == t["end"] - t["begin"]
    out = O.rlm_sort(O.KT_F32, I.normal_f32(3000, 2), 100, [7])
    assert np.array_equal(out.view(np.uint32), O.sort_keys(O.KT_F32, I.normal_f32(3000, 2)).view(np.uint32))


# ----------------------------------------------------------------- planted mistakes
import oracle.ams_oracle as _M  # noqa: E402


def _bad_classify_le(spl, nbuckets, x):            # '<=' instead of '<' in #{s < x}
    spl = np.asarray(spl, dtype=np.uint64)
    x = np.asarray(x, dtype=np.uint64)
    j = np.searchsorted(spl, x, side="right").astype(np.int64)
    jj = np.minimum(j, nbuckets - 2)
    eq = (j < nbuckets - 1) & (spl[jj] == x)
    return 2 * j + eq.astype(np.int64)


def _bad_splitters(sorted_sample, a, nbuckets):    # rank (i+1)a - 1 instead of (i+1)a
    idx = np.arange(1, nbuckets, dtype=np.int64) * a - 1
    return np.asarray(sorted_sample, dtype=np.uint64)[idx]


def _bad_rank_sort(s, block=512):                  # tie-break dropped
    s = np.asarray(s, dtype=np.uint64)
    rank = np.array([(s < v).sum() for v in s], dtype=np.int64)
    out = np.zeros_like(s)
    out[np.minimum(rank, len(s) - 1)] = s
    return rank, out


def _bad_bin_pack(w, r):                           # feasible only with fewer than r groups
    w = [int(x) for x in w]
    total = sum(w)
    lo = max((total + r - 1) // r, max(w) if w else 0)
    hi = max(lo, total)
    while lo < hi:
        mid = (lo + hi) // 2
        e = _M.greedy_groups(w, mid)
        if e is not None and len(e) < r:
            hi = mid
        else:
            lo = mid + 1
    return lo, _M.greedy_groups(w, lo)


def _bad_stream_key_level(seed, level, begin):    # level instead of level + 1
    s1 = _M.mix64((seed + level * _M._GAMMA) & _M._M64)
    return _M.mix64((s1 + (begin + 1) * _M._GAMMA) & _M._M64)


def _bad_stream_key_begin(seed, level, begin):    # begin instead of begin + 1
    s1 = _M.mix64((seed + (level + 1) * _M._GAMMA) & _M._M64)
    return _M.mix64((s1 + begin * _M._GAMMA) & _M._M64)


def _bad_mulhi64(a, b):                            # carry of the middle partial products dropped
    a = np.asarray(a, dtype=np.uint64)
    m32, s32 = np.uint64(0xFFFFFFFF), np.uint64(32)
    bh, bl = np.uint64(int(b) >> 32), np.uint64(int(b) & 0xFFFFFFFF)
    ah, al = a >> s32, a & m32
    with np.errstate(over="ignore"):
        return ah * bh + ((ah * bl) >> s32) + ((al * bh) >> s32)


def _bad_eq_cut(L):                                # L*/8 instead of L*/16
    return max(2, L >> 3)


def _bad_pieces(counts, nbuckets, L, ends, begin):  # empty runs kept
    counts = [int(c) for c in counts]
    nid = 2 * nbuckets - 1
    tau = _M.eq_cut_threshold(L)
    starts = [0] * (nid + 1)
    for i in range(nid):
        starts[i + 1] = starts[i] + counts[i]
    out, g0 = [], 0
    for e in ends:
        id_lo, id_hi = 2 * g0, min(2 * e, nid)
        run = starts[id_lo]
        for i in range(id_lo, id_hi):
            if (i & 1) and counts[i] >= tau:
                out.append((begin + run, begin + starts[i], 0))
                out.append((begin + starts[i], begin + starts[i + 1], 1))
                run = starts[i + 1]
        out.append((begin + run, begin + starts[id_hi], 0))
        g0 = e
    return [p for p in out if p[1] > p[0] or p[2] == 0]


def _bad_piece_of_ids(counts, nbuckets, L, ends):  # label run not restarted per group
    counts = [int(c) for c in counts]
    nid = 2 * nbuckets - 1
    tau = _M.eq_cut_threshold(L)
    label = np.zeros(nid, dtype=np.int64)
    run, g0 = 0, 0
    for e in ends:
        for i in range(2 * g0, min(2 * e, nid)):
            if (i & 1) and counts[i] >= tau:
                label[i] = i
                run = i + 1
            else:
                label[i] = run
        g0 = e
    return label


def _bad_sort_keys(kt, keys):                      # float map dropped (raw bit order)
    keys = np.asarray(keys)
    raw = keys.view(np.uint32) if keys.dtype == np.float32 else keys
    return keys[np.argsort(raw, kind="stable")]


def _bad_sort_pairs(kt, keys, vals):               # equal keys in reverse index order
    t = _M.ordered_keys(kt, keys)
    perm = len(t) - 1 - np.argsort(t[::-1], kind="stable")
    return np.asarray(keys)[perm], np.asarray(vals)[perm]


def _bad_f32_order(bits):                          # negative values not flipped
    return (np.asarray(bits, dtype=np.uint32) ^ np.uint32(0x80000000)).astype(np.uint32)


def _bad_oversampling(n_g):                        # floor instead of ceil
    return max(1, int(1.6 * np.log10(max(n_g, 1))))


def _bad_stable_partition(ids):                    # equal ids in reverse input order
    ids = np.asarray(ids, dtype=np.int64)
    return len(ids) - 1 - np.argsort(ids[::-1], kind="stable")


def _bad_count_before(q, key, i, pivot_seq, pivot_pos):  # sequence tie-break reversed
    if i < pivot_seq:
        return int(np.searchsorted(q, key, side="left"))
    if i > pivot_seq:
        return int(np.searchsorted(q, key, side="right"))
    return pivot_pos


def _bad_msel_definition(seqs, k):                 # ties not broken by sequence index
    keys = np.concatenate([np.asarray(q, dtype=np.uint64) for q in seqs])
    sid = np.concatenate([np.full(len(q), i, dtype=np.int64) for i, q in enumerate(seqs)])
    order = np.argsort(keys, kind="quicksort")
    return [int(np.sum(sid[order[:k]] == i)) for i in range(len(seqs))]


def _bad_a_for(self, n_g, nbuckets):               # sample-size cap dropped
    return self.a if self.a else _M.oversampling_factor(n_g)


PLANTED = [
    # (mistake, oracle attribute, replacement, pin that must fail, pin arguments)
    ("classify counts splitters <= x", "classify", _bad_classify_le, "test_classify_golden", {}),
    ("splitter rank shifted by one", "splitters", _bad_splitters, "test_splitters_closed_form", {}),
    ("rank tie-break dropped", "rank_sort", _bad_rank_sort, "test_rank_sort_against_loops_and_library", {}),
    ("bin-pack feasibility < r", "bin_pack", _bad_bin_pack, "test_bin_pack_golden", {}),
    ("stream level offset", "stream_key", _bad_stream_key_level, "test_sample_stream_golden", {}),
    ("stream begin offset", "stream_key", _bad_stream_key_begin, "test_sample_stream_golden", {}),
    ("multiply-high carry dropped", "mulhi64", _bad_mulhi64, "test_sample_stream_golden", {}),
    ("multiply-high carry dropped (exact)", "mulhi64", _bad_mulhi64, "test_mulhi64_against_exact_integers", {}),
    ("heavy-bucket threshold L/8", "eq_cut_threshold", _bad_eq_cut, "test_eq_cut_threshold_golden", {}),
    ("empty runs kept as pieces", "pieces", _bad_pieces, "test_pieces_golden", {}),
    ("piece labels not restarted per group", "piece_of_ids", _bad_piece_of_ids, "test_pieces_golden", {}),
    ("definition not stable", "sort_pairs", _bad_sort_pairs, "test_sort_brute_force_small_alphabet", {"n": 3}),
    ("keys sorted by raw float bits", "sort_keys", _bad_sort_keys, "test_sort_keys_f32_hand_order", {}),
    ("float map without the flip", "f32_order", _bad_f32_order, "test_f32_order_monotone_on_specials", {}),
    ("oversampling floor", "oversampling_factor", _bad_oversampling, "test_oversampling_factor_closed_form", {}),
    ("partition not stable", "stable_partition", _bad_stable_partition, "test_ams_restatement_equals_definition",
     {"dist": "zipf"}),
    ("a without its cap", "Plan.a_for", _bad_a_for, "test_a_for_hand_values", {}),
    ("multiselect tie-break reversed", "_count_before", _bad_count_before, "test_multiseq_select_hand_example", {}),
    ("multiselect ties unbroken", "multiseq_select_definition", _bad_msel_definition,
     "test_multiseq_select_brute_force", {}),
]


@pytest.mark.parametrize("what,attr,bad,pin,kw", PLANTED, ids=[p[0] for p in PLANTED])
def test_pins_catch_planted_mistakes(monkeypatch, what, attr, bad, pin, kw):
    """A plausible slip planted in the oracle (in its module and in the package's
    re-export) makes the named pin fail; the unpatched oracle passes the same pin."""
    pin_fn = globals()[pin]
    pin_fn(**kw)  # the real oracle passes
    if attr.startswith("Plan."):
        monkeypatch.setattr(_M.Plan, attr.split(".")[1], bad)
    else:
        monkeypatch.setattr(_M, attr, bad)
        if hasattr(O, attr):  # (private helpers are not re-exported)
            monkeypatch.setattr(O, attr, bad)
    with pytest.raises(AssertionError):
        pin_fn(**kw)


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
