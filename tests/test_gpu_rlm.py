"""RLM-sort (Section 5) through the C ABI: the result equals the oracle's definition
(and the oracle's restatement of RLM-sort) bit for bit, for keys and pairs of every
key type, one to three levels, ragged tiles and parts, in place and out of place."""
import numpy as np
import pytest

import oracle as O
from paper_1410_6754_gb300 import inputs as I

from helpers import same_bits, to_dev, to_np

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1410_6754_gb300 as ams  # noqa: E402


def _keys(kt, bits, dist, n, seed):
    if kt == O.KT_F32:
        return I.normal_f32(n, seed)
    return I.generate(dist, n, seed, bits)


@pytest.mark.parametrize("kt,bits", [(O.KT_U32, 32), (O.KT_U64, 64), (O.KT_F32, 32)])
@pytest.mark.parametrize("pairs", [False, True])
@pytest.mark.parametrize("dist", I.DISTRIBUTIONS)
def test_rlm_two_levels(kt, bits, pairs, dist):
    n, run, parts = 300007, 2048, [16, 12]
    keys = _keys(kt, bits, dist, n, 7)
    vals = np.arange(n, dtype=np.uint64)
    kin = to_dev(keys)
    kout = torch.empty_like(kin)
    vin = to_dev(vals) if pairs else None
    vout = torch.empty_like(vin) if pairs else None
    ams.rlm_sort(kin, kout, vin, vout, run=run, parts=parts, seed=3, kt=kt)
    ams.sync()
    if pairs:
        ek, ev = O.sort_pairs(kt, keys, vals)
        assert np.array_equal(to_np(vout, np.uint64), ev)
    else:
        ek = O.sort_keys(kt, keys)
    assert same_bits(to_np(kout, keys.dtype), ek)
    assert same_bits(to_np(kin, keys.dtype), keys)  # input untouched


@pytest.mark.parametrize("n,run,parts", [(1, 64, []), (1000, 1024, []), (5000, 64, [100]),
                                         (100003, 512, [7, 5, 6]), (65536, 8192, [8]),
                                         ((1 << 20) + 17, 4096, [32, 9])])
def test_rlm_shapes_in_place(n, run, parts):
    keys = I.generate("zipf", n, n % 97, 64)
    vals = np.arange(n, dtype=np.uint64)
    dk, dv = to_dev(keys), to_dev(vals)
    ams.rlm_sort(dk, vals_in=dv, run=run, parts=parts, seed=1, kt=O.KT_U64)
    ams.sync()
    want = O.rlm_sort(O.KT_U64, keys, run, parts, vals=vals)
    assert np.array_equal(to_np(dk, np.uint64), want[0])
    assert np.array_equal(to_np(dv, np.uint64), want[1])


@pytest.mark.parametrize("kt,bits", [(O.KT_U32, 32), (O.KT_U64, 64), (O.KT_F32, 32)])
@pytest.mark.parametrize("pairs", [False, True])
def test_rlm_wide_first_level(kt, bits, pairs):
    """Few selections over many tiles (7 over 2049 tiles: the cluster selection), then
    many over about 257 tiles each (one block per selection)."""
    n, run, parts = (1 << 21) + 1234, 1024, [8, 300]
    keys = _keys(kt, bits, "uniform", n, 11)
    vals = np.arange(n, dtype=np.uint64)
    kin = to_dev(keys)
    kout = torch.empty_like(kin)
    vin = to_dev(vals) if pairs else None
    vout = torch.empty_like(vin) if pairs else None
    ams.rlm_sort(kin, kout, vin, vout, run=run, parts=parts, seed=5, kt=kt)
    ams.sync()
    if pairs:
        ek, ev = O.sort_pairs(kt, keys, vals)
        assert np.array_equal(to_np(vout, np.uint64), ev)
    else:
        ek = O.sort_keys(kt, keys)
    assert same_bits(to_np(kout, keys.dtype), ek)


def test_rlm_rejects_unfinished_parts():
    # the last level's parts must fit one tile
    k = torch.zeros(10000, dtype=torch.int64, device="cuda")
    with pytest.raises(ams.AmsError) as ei:
        ams.rlm_sort(k, run=1024, parts=[4], kt=O.KT_U64)
    assert ei.value.status == ams.ERR_UNSUPPORTED
