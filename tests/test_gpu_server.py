"""Serving loop (ams_server_*): a stream of mixed requests -- uint32 / uint64 / float32
keys, uniform and Zipf values, sizes log-uniform in [2^10, 2^20], some pairs -- runs
with continuous batching (several worker streams, small keys-only requests packed
into shared segmented sorts).  Every result must equal the oracle's, and equal the
result the same request gets alone."""
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


def _requests(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(2 ** rng.uniform(10, 20))
        u = rng.random()
        kt = O.KT_U32 if u < 0.5 else (O.KT_U64 if u < 0.8 else O.KT_F32)
        if kt == O.KT_F32:
            keys = I.normal_f32(n, 100 + i)
        else:
            dist = "uniform" if rng.random() < 0.5 else "zipf"
            keys = I.generate(dist, n, 100 + i, 64 if kt == O.KT_U64 else 32)
        pairs = kt == O.KT_U64 and rng.random() < 0.2
        out.append((kt, keys, pairs))
    return out


def test_server_mixed_stream_matches_oracle_and_alone():
    reqs = _requests(300, 5)
    srv = ams.Server(hbm_budget_bytes=8 << 30, streams=4, pack_max_keys=1 << 16)
    tickets, bufs = [], []
    for kt, keys, pairs in reqs:
        kin = to_dev(keys)
        kout = torch.empty_like(kin)
        vin = torch.arange(len(keys), dtype=torch.int64, device="cuda") if pairs else None
        vout = torch.empty_like(vin) if pairs else None
        tickets.append(srv.submit(kin, kout, vin, vout, levels=2, buckets=[64, 64], kt=kt))
        bufs.append((kin, kout, vin, vout))
    lat = []
    for t in tickets:
        t0, t1 = srv.wait(t)
        assert t1 >= t0
        lat.append(t1 - t0)
    counters = srv.counters()
    srv.close()
    assert counters["packed_requests"] > 0, "no request was packed"
    for (kt, keys, pairs), (kin, kout, vin, vout) in zip(reqs, bufs):
        if pairs:
            ek, ev = O.sort_pairs(kt, keys, np.arange(len(keys), dtype=np.uint64))
            assert same_bits(to_np(kout, keys.dtype), ek)
            assert np.array_equal(to_np(vout, np.uint64), ev)
        else:
            assert same_bits(to_np(kout, keys.dtype), O.sort_keys(kt, keys))
    # the same requests alone (plain calls) give the same bits
    for (kt, keys, pairs), (kin, kout, vin, vout) in list(zip(reqs, bufs))[:40]:
        alone = torch.empty_like(kin)
        if pairs:
            va = torch.empty_like(vin)
            ams.sort_pairs_into(kin, alone, vin, va, levels=2, buckets=[64, 64], kt=kt)
            ams.sync()
            assert torch.equal(va, vout)
        else:
            ams.sort_keys_into(kin, alone, levels=2, buckets=[64, 64], kt=kt)
            ams.sync()
        assert torch.equal(alone, kout)


def test_server_budget_admits_one_large_request_alone():
    """A request larger than the whole budget still runs (alone); small ones queue
    behind it and complete."""
    srv = ams.Server(hbm_budget_bytes=1 << 20, streams=2, pack_max_keys=0)
    big = to_dev(I.generate("uniform", 1 << 20, 9, 64))
    small = [to_dev(I.generate("uniform", 3000 + i, 10 + i, 32)) for i in range(5)]
    ts = [srv.submit(big, levels=2, buckets=[64, 64], kt=O.KT_U64)]
    ts += [srv.submit(x, levels=1, buckets=[16], kt=O.KT_U32) for x in small]
    for t in ts:
        srv.wait(t)
    srv.close()
    o = big ^ (-(1 << 63))
    assert bool((o[1:] >= o[:-1]).all())
    for x in small:
        u = x.to(torch.int64) & 0xFFFFFFFF
        assert bool((u[1:] >= u[:-1]).all())
