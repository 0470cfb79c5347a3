"""Sorts replayed from a CUDA graph per size class (AMS_FLAG_GRAPH): every size of a
class, fresh buffers on every call, every key type, in place and out of place -- the
result equals the oracle's definition; a class's second call replays its graph."""
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


@pytest.mark.parametrize("kt,bits", [(O.KT_U32, 32), (O.KT_U64, 64), (O.KT_F32, 32)])
def test_graph_replay_per_size_class(kt, bits):
    ctx = ams.Context()
    kw = dict(levels=2, buckets=[16, 16], seed=2, kt=kt, flags=ams.FLAG_GRAPH)
    sizes = [2, 1000, 1024, 1025, 40000, 65535, 65536, 65537, 70000, 131072, 300001]
    for rep in range(2):
        for i, n in enumerate(sizes):
            dist = ["uniform", "zipf", "sorted", "equal"][(i + rep) % 4]
            keys = I.normal_f32(n, n) if kt == O.KT_F32 else I.generate(dist, n, n + rep, bits)
            if kt != O.KT_F32 and n > 10:
                keys = keys.copy()
                keys[:3] = np.iinfo(keys.dtype).max  # keys equal to the pad value
            kin = to_dev(keys)
            if rep == 0:
                kout = torch.empty_like(kin)
                ctx.sort(kin, kout, **kw)
            else:
                kout = kin
                ctx.sort(kin, **kw)  # in place
            ctx.sync()
            assert same_bits(to_np(kout, keys.dtype), O.sort_keys(kt, keys)), (n, rep)
    st = ctx.stats()
    assert st["kernel_launches"] > 0
    ctx.close()


def test_graph_flag_ignored_for_pairs_and_segments():
    keys = I.generate("uniform", 5000, 3, 64)
    vals = np.arange(5000, dtype=np.uint64)
    dk, dv = to_dev(keys), to_dev(vals)
    ams.sort_pairs(dk, dv, levels=2, buckets=[8, 8], flags=ams.FLAG_GRAPH, kt=O.KT_U64)
    ams.sync()
    ek, ev = O.sort_pairs(O.KT_U64, keys, vals)
    assert np.array_equal(to_np(dk, np.uint64), ek) and np.array_equal(to_np(dv, np.uint64), ev)
