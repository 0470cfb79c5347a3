"""The intermediates of whole two-level sorts -- per segment and level: the oversampling
factor a and sample size S, the global bucket sizes, the optimal group bound L*, the
number of groups and the delivery pieces with their final flags -- equal the oracle's
restatement of Section 6 (its ``trace``) bit for bit, for every input distribution.

Pair sorts deliver stably (input order inside a piece), as the restatement does, so
every level matches.  Keys-only sorts deliver in arrival order inside a piece (no
order is observable among equal keys, and the base case orders every leaf), so the
order inside a level-2 segment differs from the restatement's and so does the level-2
sample drawn from it: there, level 1 and the level-2 segments themselves (bounds, a,
S) are compared."""
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


def _gpu_pieces(seg, starts, piece_of, piece_starts):
    """Non-empty pieces (begin, end, final) of one GPU segment; final = every id of the
    piece is an equality bucket (odd id)."""
    n_p = seg["npieces"]
    ids_of = [[] for _ in range(n_p)]
    for i, p in enumerate(piece_of):
        ids_of[p].append(i)
    out = []
    for p in range(n_p):
        b = piece_starts[p]
        e = piece_starts[p + 1] if p + 1 < n_p else seg["end"] - seg["begin"]
        if e > b:
            fin = int(len(ids_of[p]) > 0 and all(i % 2 == 1 for i in ids_of[p]))
            out.append((seg["begin"] + b, seg["begin"] + e, fin))
    return out


@pytest.mark.parametrize("dist", I.DISTRIBUTIONS)
@pytest.mark.parametrize("kt,bits", [(O.KT_U64, 64), (O.KT_U32, 32)])
@pytest.mark.parametrize("pairs,cap", [(True, 0), (False, 0), (True, 4096), (False, 8192)])
def test_level_intermediates_match_oracle(dist, kt, bits, pairs, cap):
    # cap 4096 with pairs, 8192 with 32-bit keys: the base cases of half the capacity.
    # Both sides get the same C explicitly (the planner would pick the half capacity
    # for these leaf sizes on its own).
    if not pairs and cap and kt != O.KT_U32:
        pytest.skip("64-bit keys have one base-case capacity")
    n, r, seed = 1 << 20, ([16, 16] if not cap else [16, 32]), 3
    keys = I.generate(dist, n, 17, bits)
    vals = np.arange(n, dtype=np.uint64)
    C = cap or ams.default_basecase_cap(kt, pairs)
    pl = O.plan(n, kt, 2, r, pairs=pairs, C=C)
    trace = []
    ref = O.ams_sort(kt, keys, pl, seed=seed, trace=trace, vals=vals if pairs else None)
    ctx = ams.Context()
    src = to_dev(keys)
    dst = torch.empty_like(src)
    if pairs:
        vin = to_dev(vals)
        vout = torch.empty_like(vin)
        ctx.sort(src, dst, vin, vout, levels=2, buckets=r, seed=seed, kt=kt, cap=C)
    else:
        ctx.sort(src, dst, levels=2, buckets=r, seed=seed, kt=kt, cap=C)
    ctx.sync()
    if pairs:
        assert np.array_equal(dst.cpu().numpy().view(ref[0].dtype), ref[0])
        assert np.array_equal(vout.cpu().numpy().view(np.uint64), ref[1])
    else:
        assert np.array_equal(dst.cpu().numpy().view(ref.dtype), ref)
    for level in (1, 2):
        want = {t["begin"]: t for t in trace if t["level"] == level}
        got = ctx.level_segments(level) if level <= len(pl.r) else []
        assert sorted(s["begin"] for s in got) == sorted(want), (dist, level)
        for idx, seg in enumerate(got):
            t = want[seg["begin"]]
            assert seg["end"] == t["end"]
            assert (seg["a"], seg["S"]) == (t["a"], t["S"]), (dist, level, seg["begin"])
            if level > 1 and not pairs:
                continue  # (the keys-only segment's order differs: see above)
            assert (seg["L"], seg["ngroups"]) == (t["L"], len(t["ends"])), (dist, level, seg["begin"])
            starts, piece_of, piece_starts = ctx.segment_tables(level, idx, seg["nbucket_ids"], seg["npieces"])
            exp_starts = np.concatenate([[0], np.cumsum(t["counts"])[:-1]])
            assert np.array_equal(np.array(starts), exp_starts), (dist, level, seg["begin"])
            assert _gpu_pieces(seg, starts, piece_of, piece_starts) == t["pieces"], (dist, level, seg["begin"])
    ctx.close()
