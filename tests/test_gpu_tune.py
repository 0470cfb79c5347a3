"""Autotuner (ams_tune): the plan it picks for a size class is a valid plan that
sorts correctly, and the second call for the class returns the cached plan."""
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


@pytest.mark.parametrize("kt,bits,pairs,lg", [(O.KT_U64, 64, False, 22), (O.KT_U32, 32, False, 20),
                                              (O.KT_U64, 64, True, 21), (O.KT_U32, 32, False, 12)])
def test_tuned_plan_sorts(kt, bits, pairs, lg):
    n = 1 << lg
    cfg = ams.tune(n, kt, pairs=pairs)
    assert 1 <= cfg["levels"] <= 3 and len(cfg["buckets"]) == cfg["levels"]
    assert all(2 <= r <= 2048 for r in cfg["buckets"]) and cfg["b"] in (1, 4, 16, 64)
    assert cfg["a"] in (0, 1) and cfg["cap"] in (0, ams.default_basecase_cap(kt, pairs) // 2)
    assert cfg["b"] * cfg["buckets"][0] <= 2048
    assert cfg["ms"] > 0 and cfg["candidates"] >= 1
    assert ams.tune(n - 1, kt, pairs=pairs) == cfg  # same size class: cached
    keys = I.generate("uniform", n - 3, 4, bits)
    dk = to_dev(keys)
    if pairs:
        vals = np.arange(len(keys), dtype=np.uint64)
        dv = to_dev(vals)
        ams.sort_pairs(dk, dv, levels=cfg["levels"], buckets=cfg["buckets"], b=cfg["b"], a=cfg["a"],
                       cap=cfg["cap"], kt=kt)
        ams.sync()
        ek, ev = O.sort_pairs(kt, keys, vals)
        assert np.array_equal(to_np(dv, np.uint64), ev)
    else:
        ams.sort_keys(dk, levels=cfg["levels"], buckets=cfg["buckets"], b=cfg["b"], a=cfg["a"], cap=cfg["cap"],
                      kt=kt)
        ams.sync()
        ek = O.sort_keys(kt, keys)
    assert same_bits(to_np(dk, keys.dtype), ek)
