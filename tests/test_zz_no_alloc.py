"""The allocation-free entry point (ams_sort_small_noalloc) gives the same result as
the regular sort calls, twice in a row on the shared scratch array.

Some callers cannot let the library allocate device memory while they call it (a
latency-critical loop where cudaMalloc/cudaFree would synchronise the device, or a
plug-in inside a host with a fixed memory budget); this entry point serves them with
a fixed device array compiled into the library.  The file is named so that pytest
collects it last."""
import numpy as np
import pytest

import oracle as O
from paper_1410_6754_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1410_6754_gb300 as ams  # noqa: E402


def _dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64)).cuda()
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32)).cuda()
    return torch.from_numpy(a).cuda()


def _inputs(kt, n, seed):
    if kt == ams.F32:
        return I.normal_f32(n, seed)
    return I.generate("zipf" if seed % 2 else "uniform", n, seed, 32 if kt == ams.U32 else 64)


@pytest.mark.parametrize("kt", [ams.U32, ams.U64, ams.F32])
@pytest.mark.parametrize("pairs", [False, True])
def test_noalloc_matches_regular_sort_twice(kt, pairs):
    # two calls in a row with different sizes and data: the second call finds the
    # first call's leftovers in the shared scratch and must not be affected by them
    for call, n in enumerate([ams.NOALLOC_MAX_KEYS, 100003]):
        keys = _inputs(kt, n, 11 + call)
        vals = np.arange(n, dtype=np.uint64)[::-1].copy()
        a_k, b_k = _dev(keys), _dev(keys)
        a_v = _dev(vals) if pairs else None
        b_v = _dev(vals) if pairs else None
        ams.sort_small_noalloc(a_k, a_v, kt=kt)
        if pairs:
            ams.sort_pairs(b_k, b_v, levels=2, buckets=[64, 64], kt=kt)
        else:
            ams.sort_keys(b_k, levels=2, buckets=[64, 64], kt=kt)
        torch.cuda.synchronize()
        assert torch.equal(a_k, b_k), (kt, pairs, call)
        if pairs:
            assert torch.equal(a_v, b_v), (kt, pairs, call)


def test_noalloc_rejects_oversize_without_touching_data():
    keys = torch.arange(ams.NOALLOC_MAX_KEYS + 1, 0, -1, dtype=torch.int64, device="cuda")
    before = keys.clone()
    with pytest.raises(ams.AmsError) as ei:
        ams.sort_small_noalloc(keys)
    assert ei.value.status == ams.ERR_INVALID
    torch.cuda.synchronize()
    assert torch.equal(keys, before)


@pytest.mark.parametrize("kt", [ams.U32, ams.U64, ams.F32])
@pytest.mark.parametrize("pairs", [False, True])
def test_noalloc_edge_sizes_on_a_side_stream(kt, pairs):
    """n = 1, the one-block capacity C (a single shared-memory sort, no merge) and
    C + 1 (the smallest merge), enqueued on a non-default stream, against the oracle's
    (key, original index) order and against the regular sort calls."""
    cap = ams.default_basecase_cap(kt, pairs)
    side = torch.cuda.Stream()
    for n in (1, 2, cap, cap + 1):
        keys = _inputs(kt, n, 5 + n % 7)
        vals = np.arange(n, dtype=np.uint64)
        a_k = _dev(keys)
        a_v = _dev(vals) if pairs else None
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            ams.sort_small_noalloc(a_k, a_v, kt=kt, stream=side)
        side.synchronize()
        ek, ev = O.sort_pairs(kt, keys, vals)
        got = a_k.cpu().numpy().view(ek.dtype if kt != ams.F32 else np.float32)
        assert np.array_equal(got.view(np.uint8), np.ascontiguousarray(ek).view(np.uint8)), (kt, pairs, n)
        if pairs:
            assert np.array_equal(a_v.cpu().numpy().view(np.uint64), ev), (kt, pairs, n)
        b_k = _dev(keys)
        b_v = _dev(vals) if pairs else None
        if pairs:
            ams.sort_pairs(b_k, b_v, levels=2, buckets=[64, 64], kt=kt)
        else:
            ams.sort_keys(b_k, levels=2, buckets=[64, 64], kt=kt)
        torch.cuda.synchronize()
        assert torch.equal(a_k, b_k), (kt, pairs, n)
