"""Plain CPU oracle for AMS-sort (test infrastructure; see package docstring).

Every function states the passage of the paper it follows.  Section numbers refer
to Axtmann, Bingmann, Sanders, Schulz, "Practical Massively Parallel Sorting".
Readings of passages the paper leaves open are marked READING and are listed,
with the reason for each, in the repository's design notes.

Integer arithmetic on uint64 numpy arrays wraps modulo 2**64, which is what the
counter-based generator below is defined with.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "KT_U32", "KT_U64", "KT_F32",
    "mix64", "splitmix64_outputs", "mulhi64",
    "f32_order", "f32_unorder", "ordered_keys", "unordered_keys",
    "sort_keys", "sort_pairs", "sort_segmented", "select_ranks",
    "stream_key", "sample_indices", "oversampling_factor", "sample",
    "rank_sort", "rank_sort_literal", "splitters", "classify", "classify_literal",
    "bucket_counts", "greedy_groups", "bin_pack", "eq_cut_threshold", "pieces",
    "stable_partition", "piece_of_ids", "Plan", "plan", "ams_sort", "default_basecase_cap",
    "multiseq_select_definition", "multiseq_select", "rlm_sort",
]

KT_U32, KT_U64, KT_F32 = 0, 1, 2

_M64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15          # SplitMix64 increment (Steele, Lea, Flood 2014)
_MIX1 = 0xBF58476D1CE4E5B9           # SplitMix64 finaliser multipliers
_MIX2 = 0x94D049BB133111EB


# --------------------------------------------------------------------------------------
# Counter-based generator.  READING: Section 6 asks for a random sample of a*b*r
# elements without naming a generator; we draw with replacement from SplitMix64,
# implemented here from its published definition and independently in the CUDA code.
# --------------------------------------------------------------------------------------

def mix64(z):
    """SplitMix64 output function applied to a Python int or a uint64 array."""
    if isinstance(z, np.ndarray):
        z = z.astype(np.uint64, copy=True)
        with np.errstate(over="ignore"):
            z ^= z >> np.uint64(30)
            z *= np.uint64(_MIX1)
            z ^= z >> np.uint64(27)
            z *= np.uint64(_MIX2)
            z ^= z >> np.uint64(31)
        return z
    z &= _M64
    z = ((z ^ (z >> 30)) * _MIX1) & _M64
    z = ((z ^ (z >> 27)) * _MIX2) & _M64
    return z ^ (z >> 31)


def splitmix64_outputs(state: int, count: int) -> np.ndarray:
    """The first ``count`` outputs of SplitMix64 started at ``state``:
    output k (0-based) is mix64(state + (k+1) * gamma)."""
    k = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(state & _M64) + k * np.uint64(_GAMMA)
    return mix64(z)


def mulhi64(a: np.ndarray, b) -> np.ndarray:
    """High 64 bits of the 128-bit product a*b (a: uint64 array, b: int < 2**64),
    by schoolbook multiplication on 32-bit halves."""
    a = np.asarray(a, dtype=np.uint64)
    m32 = np.uint64(0xFFFFFFFF)
    s32 = np.uint64(32)
    bh, bl = np.uint64(int(b) >> 32), np.uint64(int(b) & 0xFFFFFFFF)
    ah, al = a >> s32, a & m32
    with np.errstate(over="ignore"):
        ll = al * bl
        hl = ah * bl
        lh = al * bh
        hh = ah * bh
        mid = (ll >> s32) + (hl & m32) + (lh & m32)
        return hh + (hl >> s32) + (lh >> s32) + (mid >> s32)


# --------------------------------------------------------------------------------------
# Key order.  The paper sorts 64-bit integers (Section 7).  READING for float32 keys:
# order by the bit pattern mapped so that unsigned order equals the float order, with
# -0.0 < +0.0 (a strict total order on bit patterns); the output keeps input bits.
# --------------------------------------------------------------------------------------

def f32_order(bits: np.ndarray) -> np.ndarray:
    """Order-preserving map of float32 bit patterns (uint32) to uint32: negative
    values have all bits flipped, non-negative values have the sign bit set."""
    bits = np.asarray(bits, dtype=np.uint32)
    neg = (bits >> np.uint32(31)).astype(bool)
    return np.where(neg, ~bits, bits | np.uint32(0x80000000)).astype(np.uint32)


def f32_unorder(u: np.ndarray) -> np.ndarray:
    """Inverse of ``f32_order``."""
    u = np.asarray(u, dtype=np.uint32)
    was_pos = (u >> np.uint32(31)).astype(bool)
    return np.where(was_pos, u & np.uint32(0x7FFFFFFF), ~u).astype(np.uint32)


def ordered_keys(kt: int, keys: np.ndarray) -> np.ndarray:
    """T(key) as uint64: identity for integer keys, ``f32_order`` for float32."""
    if kt == KT_U32:
        return np.asarray(keys, dtype=np.uint32).astype(np.uint64)
    if kt == KT_U64:
        return np.asarray(keys, dtype=np.uint64).copy()
    if kt == KT_F32:
        return f32_order(np.asarray(keys).view(np.uint32)).astype(np.uint64)
    raise ValueError(f"unknown key type {kt}")


def unordered_keys(kt: int, t: np.ndarray) -> np.ndarray:
    """Inverse of ``ordered_keys``: returns uint32 / uint64 / float32 arrays."""
    if kt == KT_U32:
        return t.astype(np.uint32)
    if kt == KT_U64:
        return t.astype(np.uint64)
    if kt == KT_F32:
        return f32_unorder(t.astype(np.uint32)).view(np.float32)
    raise ValueError(f"unknown key type {kt}")


# --------------------------------------------------------------------------------------
# The definition (Section 1 output requirement; Section 2 / Appendix D tie breaking):
# position i of the output holds the element whose (T(key), original index) is the
# i-th smallest.  This is a stable sort by T(key); numpy's stable argsort serves as
# the library step.
# --------------------------------------------------------------------------------------

def sort_keys(kt: int, keys: np.ndarray) -> np.ndarray:
    perm = np.argsort(ordered_keys(kt, keys), kind="stable")
    return np.asarray(keys)[perm]


def sort_pairs(kt: int, keys: np.ndarray, vals: np.ndarray):
    perm = np.argsort(ordered_keys(kt, keys), kind="stable")
    return np.asarray(keys)[perm], np.asarray(vals)[perm]


def sort_segmented(kt: int, keys: np.ndarray, offsets: np.ndarray, vals=None):
    """Apply the definition independently inside each [offsets[s], offsets[s+1])."""
    keys = np.asarray(keys)
    out_k = keys.copy()
    out_v = None if vals is None else np.asarray(vals).copy()
    offsets = np.asarray(offsets, dtype=np.int64)
    for s in range(len(offsets) - 1):
        lo, hi = int(offsets[s]), int(offsets[s + 1])
        if hi - lo < 2:
            continue
        perm = np.argsort(ordered_keys(kt, keys[lo:hi]), kind="stable") + lo
        out_k[lo:hi] = keys[perm]
        if out_v is not None:
            out_v[lo:hi] = np.asarray(vals)[perm]
    return out_k if out_v is None else (out_k, out_v)


def select_ranks(kt: int, keys: np.ndarray, ranks) -> np.ndarray:
    """Output positions ``ranks`` of the keys-only sort, one by one: the value at
    position i of the definition's output is the i-th smallest T(key) (keys alone
    carry no index to distinguish equal keys).  numpy's selection (introselect)
    serves as the library step, so a sampled position of a large sort is checked
    without sorting it."""
    ranks = np.asarray(ranks, dtype=np.int64)
    t = ordered_keys(kt, keys)
    part = np.partition(t, np.unique(ranks))
    return unordered_keys(kt, part[ranks])


# --------------------------------------------------------------------------------------
# Step 1 (Section 6): a random sample of size a*b*r from each segment.
# READING: with replacement; the j-th draw of the segment starting at position
# `begin` at recursion level `level` (1-based) is index floor(u_j * n_g / 2**64), with
# u_j the j-th SplitMix64 output from state stream_key(seed, level, begin).
# READING for a: the paper uses a = 1.6 log10 n (Section 7.2); we take the smallest
# integer a >= 1 with n_g <= 10**(a/1.6), i.e. a = ceil(1.6 log10 n_g), per segment.
# --------------------------------------------------------------------------------------

def stream_key(seed: int, level: int, begin: int) -> int:
    s1 = mix64((seed + (level + 1) * _GAMMA) & _M64)
    return mix64((s1 + (begin + 1) * _GAMMA) & _M64)


def sample_indices(seed: int, level: int, begin: int, n_g: int, count: int) -> np.ndarray:
    u = splitmix64_outputs(stream_key(seed, level, begin), count)
    return mulhi64(u, n_g).astype(np.int64)


def oversampling_factor(n_g: int) -> int:
    a = 1
    while float(n_g) > math.pow(10.0, a / 1.6):
        a += 1
    return a


def sample(seg_t: np.ndarray, seed: int, level: int, begin: int, count: int) -> np.ndarray:
    """Sample keys (already in T order, uint64) of one segment held in ``seg_t``."""
    idx = sample_indices(seed, level, begin, len(seg_t), count)
    return seg_t[idx]


# --------------------------------------------------------------------------------------
# Step 2 (Section 4.2): fast work-inefficient sorting.  The global rank of element i
# is the number of elements that precede it in the strict order (key, sample slot);
# summing the comparison results over all j gives exactly this.
# --------------------------------------------------------------------------------------

def rank_sort(s: np.ndarray, block: int = 512):
    """Returns (rank, sorted) with rank[i] = #{j: s[j] < s[i]} + #{j < i: s[j] == s[i]}
    and sorted[rank[i]] = s[i]; all-pairs comparisons in row blocks."""
    s = np.asarray(s, dtype=np.uint64)
    n = len(s)
    rank = np.empty(n, dtype=np.int64)
    j = np.arange(n)
    for lo in range(0, n, block):
        hi = min(n, lo + block)
        x = s[lo:hi, None]
        less = (s[None, :] < x).sum(axis=1)
        tie = ((s[None, :] == x) & (j[None, :] < np.arange(lo, hi)[:, None])).sum(axis=1)
        rank[lo:hi] = less + tie
    out = np.empty_like(s)
    out[rank] = s
    return rank, out


def rank_sort_literal(s):
    """The same definition as two explicit loops (for tiny inputs in the pins)."""
    s = [int(v) for v in s]
    n = len(s)
    rank = [0] * n
    for i in range(n):
        for j in range(n):
            if s[j] < s[i] or (s[j] == s[i] and j < i):
                rank[i] += 1
    out = [0] * n
    for i in range(n):
        out[rank[i]] = s[i]
    return rank, out


# --------------------------------------------------------------------------------------
# Step 3 (Section 6): br-1 splitters with equidistant rank in the sorted sample.
# READING: with S = a*B samples, splitter i (0-based, i < B-1) is sorted[(i+1)*a].
# --------------------------------------------------------------------------------------

def splitters(sorted_sample: np.ndarray, a: int, nbuckets: int) -> np.ndarray:
    idx = (np.arange(1, nbuckets, dtype=np.int64)) * a
    return np.asarray(sorted_sample, dtype=np.uint64)[idx]


# --------------------------------------------------------------------------------------
# Step 4 (Section 6, Section 2.2, Appendix D): partition into B range buckets plus an
# equality bucket per splitter.  With j = #{splitters < x}: id = 2j for the range
# bucket, 2j+1 when j < B-1 and x equals splitter j.  Key-only comparisons.
# A run of equal splitters sends x equal to them to the first copy's equality bucket.
# --------------------------------------------------------------------------------------

def classify(spl: np.ndarray, nbuckets: int, x: np.ndarray) -> np.ndarray:
    """Bucket ids; numpy's searchsorted (count of sorted splitters < x) is the library
    step for #{splitters < x}."""
    spl = np.asarray(spl, dtype=np.uint64)
    x = np.asarray(x, dtype=np.uint64)
    j = np.searchsorted(spl, x, side="left").astype(np.int64)
    jj = np.minimum(j, nbuckets - 2)
    eq = (j < nbuckets - 1) & (spl[jj] == x) if nbuckets > 1 else np.zeros(len(x), bool)
    return 2 * j + eq.astype(np.int64)


def classify_literal(spl, nbuckets, x):
    """Definition as explicit loops (tiny inputs in the pins)."""
    out = []
    for v in x:
        v = int(v)
        j = sum(1 for s in spl if int(s) < v)
        eq = 1 if (j < nbuckets - 1 and int(spl[j]) == v) else 0
        out.append(2 * j + eq)
    return out


def bucket_counts(ids: np.ndarray, nbuckets: int) -> np.ndarray:
    """Step 5 (Section 6, global bucket sizes): counts of each of the 2B-1 ids."""
    return np.bincount(np.asarray(ids, dtype=np.int64), minlength=2 * nbuckets - 1).astype(np.int64)


# --------------------------------------------------------------------------------------
# Step 6 (Section 6, bucket grouping; Lemma on the scanning algorithm; Appendix C):
# scan the bucket sizes, starting a new group when the load would exceed L; binary
# search for the smallest L that needs at most r groups.
# READING: equality buckets weigh 0 (they are final); weights are range-bucket sizes.
# --------------------------------------------------------------------------------------

def greedy_groups(w, L: int):
    """Group ends (exclusive bucket indices) of the scan with bound L, or None if some
    single bucket exceeds L."""
    ends = []
    load = 0
    for j, x in enumerate(w):
        x = int(x)
        if x > L:
            return None
        if load + x > L:
            ends.append(j)
            load = x
        else:
            load += x
    ends.append(len(w))
    return ends


def bin_pack(w, r: int):
    """(L*, ends): the smallest feasible L by binary search over the integers in
    [max(ceil(W/r), max w), W], and the scan's group ends at L*."""
    w = [int(x) for x in w]
    total = sum(w)
    lo = max((total + r - 1) // r, max(w) if w else 0)
    hi = max(lo, total)

    def feasible(L):
        e = greedy_groups(w, L)
        return e is not None and len(e) <= r

    while lo < hi:
        mid = (lo + hi) // 2
        if feasible(mid):
            hi = mid
        else:
            lo = mid + 1
    return lo, greedy_groups(w, lo)


def eq_cut_threshold(L: int) -> int:
    """READING: an equality bucket is cut out of its group as a final piece when it
    holds at least max(2, floor(L*/16)) elements; lighter ones stay in the group."""
    return max(2, L >> 4)


def pieces(counts, nbuckets: int, L: int, ends, begin: int):
    """Contiguous pieces of one segment after grouping.  Group k spans range buckets
    [s_k, e_k) and the ids [2 s_k, min(2 e_k, 2B-1)) (each group keeps the equality
    bucket after its last range bucket).  Heavy equality buckets (see
    ``eq_cut_threshold``) become final pieces; the rest of a group stays together.
    Returns a list of (begin, end, final) with empty pieces dropped."""
    counts = [int(c) for c in counts]
    nid = 2 * nbuckets - 1
    tau = eq_cut_threshold(L)
    starts = [0] * (nid + 1)
    for i in range(nid):
        starts[i + 1] = starts[i] + counts[i]
    out = []
    g0 = 0
    for e in ends:
        id_lo, id_hi = 2 * g0, min(2 * e, nid)
        run = starts[id_lo]
        for i in range(id_lo, id_hi):
            if (i & 1) and counts[i] >= tau:
                if starts[i] > run:
                    out.append((begin + run, begin + starts[i], 0))
                out.append((begin + starts[i], begin + starts[i + 1], 1))
                run = starts[i + 1]
        if starts[id_hi] > run:
            out.append((begin + run, begin + starts[id_hi], 0))
        g0 = e
    return out


def stable_partition(ids: np.ndarray) -> np.ndarray:
    """Step 7 (Section 6, data delivery): the order that moves every element to its
    bucket while keeping input order inside a bucket (stable; numpy's stable argsort
    of the ids is the library step)."""
    return np.argsort(np.asarray(ids, dtype=np.int64), kind="stable")


def piece_of_ids(counts, nbuckets: int, L: int, ends) -> np.ndarray:
    """READING of the delivery of Section 6 ("the data splitting defined by the bucket
    group is the input for data delivery"): elements are delivered to *pieces* -- a
    group's buckets between heavy equality buckets form one piece, each heavy
    equality bucket (see ``eq_cut_threshold``) is a piece of its own -- keeping input
    order inside a piece.  Returns, for every bucket id, the first id of its piece
    (a non-decreasing label, so a stable sort by it is the delivery order)."""
    counts = [int(c) for c in counts]
    nid = 2 * nbuckets - 1
    tau = eq_cut_threshold(L)
    label = np.zeros(nid, dtype=np.int64)
    g0 = 0
    for e in ends:
        id_lo, id_hi = 2 * g0, min(2 * e, nid)
        run = id_lo
        for i in range(id_lo, id_hi):
            if (i & 1) and counts[i] >= tau:
                label[i] = i
                run = i + 1
            else:
                label[i] = run
        g0 = e
    return label


# --------------------------------------------------------------------------------------
# Parameters of a run.  READINGS: `levels` is the largest number of distribution
# levels the caller asks for; if n / prod(r) still exceeds the base-case capacity C,
# further levels with the last r are added (at most 8 in total).  b defaults to 1 for
# one level and 4 otherwise; the number of range buckets per level is B = b*r.
# --------------------------------------------------------------------------------------

def default_basecase_cap(kt: int, pairs: bool) -> int:
    if pairs:
        return 8192
    return 16384 if kt in (KT_U32, KT_F32) else 8192


class Plan:
    def __init__(self, r, b, a, C, max_seg):
        self.r = list(r)               # groups per level
        self.b = b
        self.a = a                     # None: per-segment rule, else fixed
        self.C = C
        self.max_seg = max_seg

    @property
    def levels(self):
        return len(self.r)

    def nbuckets(self, level):         # 1-based level
        return self.b * self.r[level - 1]

    def a_for(self, n_g, nbuckets):
        """READING: a = the fixed value or ceil(1.6 log10 n_g), but never more than
        max(1, n_g // (16 B)), so a segment's sample stays within 1/16 of it."""
        a = self.a if self.a else oversampling_factor(n_g)
        return min(a, max(1, n_g // (16 * nbuckets)))


def plan(n_max: int, kt: int, levels: int, r, pairs=False, b=None, a=None, C=None) -> Plan:
    r = [int(x) for x in r][:levels]
    if levels < 1 or len(r) != levels or any(x < 2 for x in r):
        raise ValueError("levels >= 1 and one r >= 2 per level")
    if b is None or b == 0:
        b = 1 if levels == 1 else 4
    if C is None or C == 0:
        C = default_basecase_cap(kt, pairs)
    est = n_max
    for x in r:
        est = -(-est // x)
    while est > C and len(r) < 8:
        r.append(r[-1])
        est = -(-est // r[-1])
    return Plan(r, b, a, C, n_max)


# --------------------------------------------------------------------------------------
# The whole method (Section 6): per level, for every segment larger than C: sample,
# sort the sample, pick splitters, classify, count, group, deliver; recurse on the
# non-final pieces; sort the leaves sequentially (base case).
# --------------------------------------------------------------------------------------

def ams_sort(kt: int, keys: np.ndarray, pl: Plan, seed: int, vals=None, offsets=None,
             trace=None):
    """Returns sorted keys (and values).  If ``trace`` is a list, one dict per
    processed segment is appended with its intermediates."""
    keys = np.asarray(keys)
    n = len(keys)
    t = ordered_keys(kt, keys)
    src_idx = np.arange(n, dtype=np.int64)          # which input element sits here
    if offsets is None:
        segs = [(0, n)] if n else []
    else:
        offsets = [int(x) for x in offsets]
        segs = [(offsets[i], offsets[i + 1]) for i in range(len(offsets) - 1)
                if offsets[i + 1] > offsets[i]]
    leaves = []                                       # (begin, end, final)
    for level in range(1, pl.levels + 1):
        nxt = []
        B = pl.nbuckets(level)
        for (lo, hi) in segs:
            n_g = hi - lo
            if n_g <= pl.C:
                leaves.append((lo, hi, 0))
                continue
            a = pl.a_for(n_g, B)
            S = a * B
            seg = t[lo:hi]
            smp = sample(seg, seed, level, lo, S)
            _, srt = rank_sort(smp)
            spl = splitters(srt, a, B)
            ids = classify(spl, B, seg)
            cnt = bucket_counts(ids, B)
            L, ends = bin_pack(cnt[0::2], pl.r[level - 1])
            perm = stable_partition(piece_of_ids(cnt, B, L, ends)[ids])
            t[lo:hi] = seg[perm]
            src_idx[lo:hi] = src_idx[lo:hi][perm]
            pcs = pieces(cnt, B, L, ends, lo)
            if trace is not None:
                trace.append(dict(level=level, begin=lo, end=hi, a=a, S=S, sample=smp,
                                  sorted_sample=srt, splitters=spl, counts=cnt, L=L,
                                  ends=ends, pieces=pcs))
            for (pb, pe, fin) in pcs:
                if fin or (pe - pb) <= pl.C or level == pl.levels:
                    leaves.append((pb, pe, fin))
                else:
                    nxt.append((pb, pe))
        segs = nxt
    for (lo, hi) in segs:                             # only if no level ran
        leaves.append((lo, hi, 0))
    for (lo, hi, fin) in leaves:                      # base case: sequential sort
        if fin or hi - lo < 2:
            continue
        perm = np.argsort(t[lo:hi], kind="stable")
        t[lo:hi] = t[lo:hi][perm]
        src_idx[lo:hi] = src_idx[lo:hi][perm]
    out_k = unordered_keys(kt, t)
    if kt != KT_F32:
        out_k = out_k.astype(keys.dtype)
    if vals is None:
        return out_k
    return out_k, np.asarray(vals)[src_idx]


# --------------------------------------------------------------------------------------
# RLM-sort (Section 5, recurse-last multilevel multiway mergesort) and its building
# block, multisequence selection (Section 4.1).
#
# Sequences are sorted arrays of ordered keys (uint64); the total order among all
# their elements is (key, sequence index, position in the sequence), the tie breaking
# of Section 2 / Appendix D when the sequences hold consecutive input ranges in input
# order (then it is (key, original index)).
# --------------------------------------------------------------------------------------

def multiseq_select_definition(seqs, k: int):
    """The split positions (s_1, ..., s_p) of rank k: the first k elements of the total
    order are exactly the prefixes seqs[i][:s_i].  numpy's lexsort over (key, sequence,
    position) is the library step."""
    keys = np.concatenate([np.asarray(q, dtype=np.uint64) for q in seqs]) if seqs else np.zeros(0, np.uint64)
    sid = np.concatenate([np.full(len(q), i, dtype=np.int64) for i, q in enumerate(seqs)]) if seqs else \
        np.zeros(0, np.int64)
    order = np.lexsort((np.arange(len(keys)), keys))  # ties: concatenation order = (sequence, position)
    first = sid[order[:k]]
    return [int(np.sum(first == i)) for i in range(len(seqs))]


def _count_before(q, key, i, pivot_seq, pivot_pos):
    """Elements of sorted sequence q (index i) that precede the pivot element
    (key, pivot_seq, pivot_pos) in the total order."""
    if i < pivot_seq:
        return int(np.searchsorted(q, key, side="right"))
    if i > pivot_seq:
        return int(np.searchsorted(q, key, side="left"))
    return pivot_pos


def multiseq_select(seqs, k: int, seed: int = 0):
    """Section 4.1: quickselect on sorted sequences.  Windows [lo_i, hi_i) hold the split
    position of every sequence; a pivot drawn uniformly from the windows' elements
    (SplitMix64 stream from `seed`) is located in every sequence by binary search;
    if fewer than k elements precede it the pivot and everything before it are taken
    (lo moves up), otherwise the windows end at the pivot (hi moves down).  Returns the
    same positions as the definition (they are unique)."""
    seqs = [np.asarray(q, dtype=np.uint64) for q in seqs]
    p = len(seqs)
    lo = [0] * p
    hi = [len(q) for q in seqs]
    state = mix64((seed * _GAMMA + k) & _M64)
    while sum(lo) < k:
        sizes = [hi[i] - lo[i] for i in range(p)]
        total = sum(sizes)
        state = (state + _GAMMA) & _M64
        u = (mix64(state) * total) >> 64          # uniform index among the window elements
        ps = 0
        while u >= sizes[ps]:
            u -= sizes[ps]
            ps += 1
        pp = lo[ps] + u                             # pivot: element (seqs[ps][pp], ps, pp)
        key = seqs[ps][pp]
        before = [min(max(_count_before(seqs[i], key, i, ps, pp), lo[i]), hi[i]) for i in range(p)]
        a = sum(before)
        if a < k:                                   # pivot and all before it are in the first k
            lo = before
            lo[ps] = pp + 1
        else:                                       # the first k all precede the pivot
            hi = before
    return lo


def rlm_sort(kt: int, keys: np.ndarray, run: int, parts, vals=None, trace=None):
    """Section 5, RLM-sort ("recurse last") on one device, with a processing element's
    data played by a tile of `run` consecutive positions.  Level 0: every tile sorts
    its elements locally (stable: (key, original index)).  Level l = 1..len(parts):
    every current part is split into parts[l-1] parts of equal size (sizes
    floor(j m / r) apart) by multisequence selection over the part's tiles; part j
    receives from every tile the piece between its split positions, in tile order
    (data delivery); then every tile of the new part -- `run` consecutive positions
    from the part's start -- merges the pieces it holds locally (here a stable sort
    of the tile, the library step; the pieces are sorted, so this is their multiway
    merge), and those tiles are the sorted sequences the next level splits.  A part
    still larger than one tile after the last level is merged as a whole.  Returns
    the sorted keys (and values); `trace` gets, per level and part, its range, the
    split ranks and the split positions in each of its tiles."""
    keys = np.asarray(keys)
    n = len(keys)
    t = ordered_keys(kt, keys)
    idx = np.arange(n, dtype=np.int64)

    def merge_tiles(lo, hi):
        tiles = []
        for b in range(lo, hi, run):
            e = min(hi, b + run)
            perm = np.argsort(t[b:e], kind="stable")
            t[b:e] = t[b:e][perm]
            idx[b:e] = idx[b:e][perm]
            tiles.append((b, e))
        return tiles

    cur = [(0, n, merge_tiles(0, n))] if n else []
    for level, r in enumerate(parts, start=1):
        nxt = []
        for (lo, hi, sq) in cur:
            m = hi - lo
            ranks = [(j * m) // r for j in range(r + 1)]
            arrays = [t[b:e] for (b, e) in sq]
            cuts = [[0] * len(sq)] + [multiseq_select_definition(arrays, k) for k in ranks[1:-1]] + \
                   [[e - b for (b, e) in sq]]
            new_t = t[lo:hi].copy()
            new_i = idx[lo:hi].copy()
            pos = 0
            for j in range(r):
                for si, (b, e) in enumerate(sq):
                    pb, pe = b + cuts[j][si], b + cuts[j + 1][si]
                    new_t[pos:pos + pe - pb] = t[pb:pe]
                    new_i[pos:pos + pe - pb] = idx[pb:pe]
                    pos += pe - pb
            assert pos == m
            t[lo:hi] = new_t
            idx[lo:hi] = new_i
            if trace is not None:
                trace.append(dict(level=level, begin=lo, end=hi, ranks=ranks, cuts=cuts, tiles=list(sq)))
            for j in range(r):
                pb, pe = lo + ranks[j], lo + ranks[j + 1]
                nxt.append((pb, pe, merge_tiles(pb, pe)))
        cur = nxt
    for (lo, hi, sq) in cur:                          # a part of several tiles: merge it whole
        if len(sq) > 1:
            perm = np.argsort(t[lo:hi], kind="stable")
            t[lo:hi] = t[lo:hi][perm]
            idx[lo:hi] = idx[lo:hi][perm]
    out_k = unordered_keys(kt, t)
    if kt != KT_F32:
        out_k = out_k.astype(keys.dtype)
    if vals is None:
        return out_k
    return out_k, np.asarray(vals)[idx]
