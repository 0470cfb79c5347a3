"""End-to-end parity of whole sorts through the C ABI against the oracle's definition
(bit-exact): the synthetic workloads of the evaluation at sizes the oracle finishes
in seconds, edge cases, segmented and pair sorts, and the other entry points."""
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


def _sort_check(keys, kt, levels, buckets, seed=0, pairs=False, **kw):
    n = len(keys)
    dk = to_dev(keys)
    vals = np.arange(n, dtype=np.uint64)
    dv = to_dev(vals) if pairs else None
    if pairs:
        ams.sort_pairs(dk, dv, levels=levels, buckets=buckets, seed=seed, kt=kt, **kw)
    else:
        ams.sort_keys(dk, levels=levels, buckets=buckets, seed=seed, kt=kt, **kw)
    ams.sync()
    ek, ev = O.sort_pairs(kt, keys, vals)
    assert same_bits(to_np(dk, keys.dtype), ek)
    if pairs:
        assert np.array_equal(to_np(dv, np.uint64), ev)
    return ams.stats()


def test_single_level_2p20_u32():
    """Plain single-level sample sort: 2^20 uint32 uniform keys from seed 0, 256 buckets,
    oversampling 16 (4096 sample keys), b = 1."""
    keys = I.generate("uniform", 1 << 20, 0, 32)
    st = _sort_check(keys, O.KT_U32, 1, [256], seed=0, a=16, b=1)
    assert st["levels_planned"] == 1 and st["segments"][0] == 1
    assert st["kernel_elems"]["sample_sort"] == 4096


@pytest.mark.parametrize("dist", I.DISTRIBUTIONS)
def test_two_level_u64_distributions(dist):
    """Two-level sort of uint64 keys, k1 = k2 = 256, overpartitioning 4, at 2^22 keys."""
    keys = I.generate(dist, 1 << 22, 7, 64)
    st = _sort_check(keys, O.KT_U64, 2, [256, 256], seed=I.DISTRIBUTIONS.index(dist), b=4)
    assert st["levels_planned"] == 2


def test_pairs_duplicate_heavy_three_levels():
    keys = I.dup_keys_u64(1 << 22, 3)
    _sort_check(keys, O.KT_U64, 3, [256, 256, 256], seed=1, pairs=True)


def test_pairs_f32_normal_with_zeros():
    keys = I.normal_f32(1 << 22, 5)
    _sort_check(keys, O.KT_F32, 3, [256, 256, 256], seed=2, pairs=True)
    _sort_check(keys, O.KT_F32, 2, [64, 64], seed=3, pairs=False)


@pytest.mark.parametrize("kt,bits", [(O.KT_U32, 32), (O.KT_U64, 64)])
@pytest.mark.parametrize("n", [1, 2, 3, 17, 8191, 8192, 8193, 16384, 16385, (1 << 16) + 7, 1234567])
def test_sizes_and_ragged_tails(kt, bits, n):
    keys = I.generate("uniform", n, n, bits)
    _sort_check(keys, kt, 2, [16, 16], seed=n, pairs=(n % 2 == 1))


def test_extreme_keys():
    for bits, kt in [(32, O.KT_U32), (64, O.KT_U64)]:
        dt = ordered_dtype(kt)
        mx = np.iinfo(dt).max
        rng = np.random.default_rng(bits)
        keys = rng.choice(np.array([0, 1, mx - 1, mx], dtype=dt), size=300000)
        _sort_check(keys, kt, 2, [32, 32], pairs=True)
        _sort_check(np.full(200000, mx, dtype=dt), kt, 2, [32, 32], pairs=True)


def test_f32_special_values():
    rng = np.random.default_rng(11)
    pool = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, 1e-40, -1e-40, 3.4e38, -3.4e38],
                    dtype=np.float32)
    keys = pool[rng.integers(0, len(pool), size=500000)]
    nan_bits = np.array([0x7FC00000, 0xFFC00000, 0x7F800001], dtype=np.uint32).view(np.float32)
    keys[:3] = nan_bits
    _sort_check(keys, O.KT_F32, 2, [64, 64], pairs=True)


def test_seed_and_parameters_do_not_change_the_output():
    keys = I.generate("zipf", 1 << 21, 4, 64)
    exp = O.sort_keys(O.KT_U64, keys)
    for levels, buckets, b, a, seed in [(1, [256], 1, 0, 0), (2, [256, 256], 4, 0, 1),
                                        (2, [64, 512], 2, 3, 2), (3, [8, 8, 8], 16, 1, 3),
                                        (2, [1024, 2], 1, 0, 4)]:
        dk = to_dev(keys)
        ams.sort_keys(dk, levels=levels, buckets=buckets, seed=seed, a=a, b=b)
        ams.sync()
        assert same_bits(to_np(dk, np.uint64), exp), (levels, buckets, b, a, seed)


@pytest.mark.parametrize("kt,bits,dist", [(O.KT_U64, 64, "uniform"), (O.KT_U64, 64, "zipf"),
                                          (O.KT_U32, 32, "staggered"), (O.KT_F32, 32, None)])
def test_tree_classifier_same_output(kt, bits, dist):
    """The implicit-search-tree classifier (the paper's multisplitter) and the default
    cell-table classifier give the same sort."""
    keys = I.normal_f32(1 << 21, 8) if kt == O.KT_F32 else I.generate(dist, 1 << 21, 8, bits)
    _sort_check(keys, kt, 2, [256, 256], seed=4, pairs=True, flags=ams.FLAG_TREE_CLASSIFIER)
    _sort_check(keys, kt, 1, [1024], seed=5, flags=ams.FLAG_TREE_CLASSIFIER)


def test_fallback_for_groups_above_capacity():
    """With two buckets per level and a tiny base-case capacity, some groups stay above
    capacity after the last level and take the global-memory merge path."""
    keys = I.generate("uniform", 1 << 16, 9, 64)
    _sort_check(keys, O.KT_U64, 1, [2], cap=256, pairs=True)
    keys = I.generate("zipf", 1 << 17, 9, 32)
    _sort_check(keys, O.KT_U32, 1, [2], cap=300)


@pytest.mark.parametrize("kt,bits", [(O.KT_U32, 32), (O.KT_U64, 64), (O.KT_F32, 32)])
@pytest.mark.parametrize("pairs", [False, True])
def test_segmented(kt, bits, pairs):
    lens = I.segment_lengths(3000, 1 << 21, 4, max_log2=20)
    lens[5] = 0
    lens[17] = 0
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    n = int(off[-1])
    keys = I.normal_f32(n, 3) if kt == O.KT_F32 else I.generate("uniform", n, 3, bits)
    vals = np.arange(n, dtype=np.uint64)
    dk, dv, do = to_dev(keys), to_dev(vals), to_dev(off.view(np.uint64))
    res = ams.sort_segmented(dk, do, vals=dv if pairs else None, levels=2, buckets=[64, 64], kt=kt)
    ams.sync()
    if pairs:
        ek, ev = O.sort_segmented(kt, keys, off, vals)
        assert np.array_equal(to_np(dv, np.uint64), ev)
    else:
        ek = O.sort_segmented(kt, keys, off)
    assert same_bits(to_np(dk, keys.dtype), ek)
    assert res is not None


@pytest.mark.parametrize("kt,bits", [(O.KT_U32, 32), (O.KT_U64, 64), (O.KT_F32, 32)])
@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("dist", ["uniform", "zipf"])
def test_segmented_tiny_segments(kt, bits, pairs, dist):
    """Many segments of at most 2^12 keys: those of at most 256 keys go through the warp
    all-pairs rank sort, the others through the base case; every length from 0 to 300
    appears (ties by original index with payloads = index), out of place and in place."""
    rng = np.random.default_rng(kt * 7 + pairs + len(dist))
    lens = np.concatenate([np.arange(0, 301), rng.integers(0, 4097, 200), [1, 1, 2, 255, 256, 257]])
    rng.shuffle(lens)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    n = int(off[-1])
    if kt == O.KT_F32:
        keys = I.normal_f32(n, 5)
        if dist == "zipf":
            keys = np.array([0.0, -0.0, 1.0, -1.0, 2.5], np.float32)[rng.integers(0, 5, n)]
    else:
        keys = I.generate(dist, n, 5, bits)
    vals = np.arange(n, dtype=np.uint64)
    ek = O.sort_segmented(kt, keys, off, vals if pairs else None)
    do = to_dev(off.view(np.uint64))
    # in place
    dk, dv = to_dev(keys), to_dev(vals)
    ams.sort_segmented(dk, do, vals=dv if pairs else None, levels=2, buckets=[16, 16], kt=kt)
    ams.sync()
    if pairs:
        assert same_bits(to_np(dk, keys.dtype), ek[0])
        assert np.array_equal(to_np(dv, np.uint64), ek[1])
    else:
        assert same_bits(to_np(dk, keys.dtype), ek)
    # out of place, through a context
    ctx = ams.Context()
    kin, kout = to_dev(keys), torch.empty_like(to_dev(keys))
    vin, vout = (to_dev(vals), torch.empty_like(to_dev(vals))) if pairs else (None, None)
    ctx.sort(kin, kout, vin, vout, offsets=do, levels=2, buckets=[16, 16], kt=kt)
    ctx.sync()
    if pairs:
        assert same_bits(to_np(kout, keys.dtype), ek[0])
        assert np.array_equal(to_np(vout, np.uint64), ek[1])
    else:
        assert same_bits(to_np(kout, keys.dtype), ek)
    assert same_bits(to_np(kin, keys.dtype), keys)  # the input is left alone
    ctx.close()


@pytest.mark.parametrize("kt,bits", [(O.KT_U32, 32), (O.KT_U64, 64), (O.KT_F32, 32)])
@pytest.mark.parametrize("pairs", [False, True])
def test_small_arrays_through_the_warp_sort(kt, bits, pairs):
    for n in [2, 3, 31, 32, 33, 64, 100, 255, 256, 257]:
        keys = I.normal_f32(n, n) if kt == O.KT_F32 else I.generate("zipf", n, n, bits)
        _sort_check(keys, kt, 2, [64, 64], pairs=pairs)


def test_out_of_place_and_host_entry_points():
    keys = I.generate("staggered", 1 << 20, 2, 64)
    src = to_dev(keys)
    dst = torch.empty_like(src)
    ams.sort_keys_into(src, dst, levels=2, buckets=[64, 64])
    ams.sync()
    assert same_bits(to_np(dst, np.uint64), np.sort(keys))
    assert same_bits(to_np(src, np.uint64), keys)  # input untouched
    vals = np.arange(len(keys), dtype=np.uint64)
    vs, vd = to_dev(vals), torch.empty_like(to_dev(vals))
    ams.sort_pairs_into(src, dst, vs, vd, levels=2, buckets=[64, 64])
    ams.sync()
    ek, ev = O.sort_pairs(O.KT_U64, keys, vals)
    assert same_bits(to_np(dst, np.uint64), ek) and np.array_equal(to_np(vd, np.uint64), ev)
    h = keys.copy()
    hv = vals.copy()
    ams.sort_host(h, hv, levels=2, buckets=[256, 256])
    assert same_bits(h, ek) and np.array_equal(hv, ev)


@pytest.mark.parametrize("pairs", [False, True])
def test_host_async_two_contexts_two_streams(pairs):
    """ams_sort_host_async: six sorts of page-locked host arrays enqueued alternately on
    two contexts and two streams (each context on its own stream), all in flight at
    once; every array then holds its own sorted result (pairs: stable)."""
    ctxs = [ams.Context(), ams.Context()]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    n = (1 << 20) + 77
    keys = [I.generate(["uniform", "zipf", "sorted"][i % 3], n, 40 + i, 64) for i in range(6)]
    vals = np.arange(n, dtype=np.uint64)
    hk = [torch.from_numpy(k.view(np.int64).copy()).pin_memory() for k in keys]
    hv = [torch.from_numpy(vals.view(np.int64).copy()).pin_memory() for _ in keys] if pairs else [None] * 6
    for i in range(6):
        ams.sort_host_async(hk[i], hv[i], levels=2, buckets=[64, 64], seed=i, kt=O.KT_U64,
                            ctx=ctxs[i % 2], stream=streams[i % 2])
    for c in ctxs:
        c.sync()
    for i in range(6):
        ek, ev = O.sort_pairs(O.KT_U64, keys[i], vals)
        assert same_bits(hk[i].numpy().view(np.uint64), ek), i
        if pairs:
            assert np.array_equal(hv[i].numpy().view(np.uint64), ev), i
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("kt,bits,dist", [(O.KT_U64, 64, "uniform"), (O.KT_U32, 32, "uniform"),
                                          (O.KT_F32, 32, None), (O.KT_U64, 64, "zipf")])
@pytest.mark.parametrize("in_off,out_off", [(1, 3), (2, 1), (3, 2)])
def test_buffers_at_any_element_offset(kt, bits, dist, in_off, out_off):
    """Input and output views starting at element offsets (so not 16-byte aligned):
    the levels that write into the caller's buffer handle any 16-byte phase."""
    n = (1 << 21) + 13
    keys = I.normal_f32(n, 6) if kt == O.KT_F32 else I.generate(dist, n, 6, bits)
    big_in = to_dev(np.concatenate([np.zeros(in_off, keys.dtype), keys]))
    big_out = torch.zeros(n + out_off + 5, dtype=big_in.dtype, device="cuda")
    src = big_in[in_off:in_off + n]
    dst = big_out[out_off:out_off + n]
    ams.sort_keys_into(src, dst, levels=2, buckets=[64, 64], kt=kt)
    ams.sync()
    assert same_bits(to_np(dst, keys.dtype), O.sort_keys(kt, keys))
    rest = torch.cat([big_out[:out_off], big_out[out_off + n:]])
    assert int((rest != 0).sum().item()) == 0, "wrote outside the output view"


@pytest.mark.parametrize("kt,bits,dist,lg,pairs", [
    (O.KT_U32, 32, "zipf", 14, False), (O.KT_U32, 32, "zipf", 18, False), (O.KT_U32, 32, "zipf", 18, True),
    (O.KT_F32, 32, None, 18, False), (O.KT_F32, 32, None, 18, True), (O.KT_U64, 64, "zipf", 20, False)])
def test_skewed_leaves(kt, bits, dist, lg, pairs):
    """Leaves whose keys crowd into a few cells with several values (Zipf ranks, float
    bit patterns near zero) take the distribution-independent path of the base case."""
    n = 1 << lg
    keys = I.normal_f32(n, 5) if kt == O.KT_F32 else I.generate(dist, n, 5, bits)
    _sort_check(keys, kt, 2, [64, 64], pairs=pairs)


def test_contexts_budget_and_errors():
    keys = I.generate("uniform", 1 << 20, 1, 32)
    ctx = ams.Context()
    dk = to_dev(keys)
    ctx.sort(dk, levels=1, buckets=[256])
    ctx.sync()
    assert same_bits(to_np(dk, np.uint32), np.sort(keys))
    assert ctx.scratch_bytes() > 4 * len(keys)
    ctx.close()
    small = ams.Context(hbm_budget_bytes=1 << 16)
    with pytest.raises(ams.AmsError) as ei:
        small.sort(to_dev(keys), levels=1, buckets=[256])
    assert ei.value.status == ams.ERR_OOM
    small.close()
    with pytest.raises(ams.AmsError) as ei:
        ams.sort_keys(to_dev(keys), levels=0, buckets=[256])
    assert ei.value.status == ams.ERR_INVALID
    with pytest.raises(ams.AmsError) as ei:
        ams.sort_keys(to_dev(keys), levels=1, buckets=[1])
    assert ei.value.status == ams.ERR_INVALID
    with pytest.raises(ams.AmsError) as ei:
        ams.sort_keys(to_dev(keys), levels=1, buckets=[4096], b=1)
    assert ei.value.status == ams.ERR_UNSUPPORTED
    empty = torch.empty(0, dtype=torch.int64, device="cuda")
    ams.sort_keys(empty)
    ams.sync()


def test_phase_timers_and_stats():
    keys = I.generate("uniform", 1 << 22, 1, 64)
    dk = to_dev(keys)
    ams.stats()  # reading the statistics resets the launch and event tallies
    ams.sort_keys(dk, levels=2, buckets=[256, 256], flags=ams.FLAG_PHASE_TIMERS)
    st = ams.stats()
    assert st["device_status"] == 0
    assert st["kernel_calls"]["scatter"] == 2 and st["kernel_ms"]["scatter"] > 0
    assert st["kernel_elems"]["classify"] >= len(keys)
    assert st["kernel_launches"] == sum(st["kernel_calls"].values())
