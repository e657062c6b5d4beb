"""Batched rebuild of all the indexes of one table: each index must equal its
own unbatched rebuild and the oracle, bit for bit, whether the batch runs on
concurrent streams or as one replayed CUDA graph; the autotuner must pick a
legal digit width and serve it back from its cache."""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2009_11543_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2009_11543_gb300 import ck, pipeline  # noqa: E402

DEV = "cuda:0"
FANOUTS = [64, 64, 64, 64, 256, 256]


def table(n):
    cols = synth.table_columns(n, synth.BASE_SEED + 3)
    dev = [torch.from_numpy(c.view(np.int64) if c.dtype == np.uint64 else
                            (c.view(np.int32) if c.dtype == np.uint32 else c)).to(DEV) for c in cols]
    perms = [oracle.sort_rows(c) for c in cols]
    dmasks = [oracle.dmask(c, p) for c, p in zip(cols, perms)]
    return cols, dev, perms, dmasks


def check_part(r, col, perm, dmask, fanout):
    n = len(perm)
    assert np.array_equal(ck.u32(r.rid_sorted)[:n], perm)
    t = oracle.btree(col, perm, fanout)
    assert np.array_equal(r.tree["leaf_dbit"].cpu().numpy().view(np.uint16)[:n], t["leaf_dbit"])
    ni = int(r.shape.inner_entries)
    assert np.array_equal(r.tree["inner_dbit"].cpu().numpy().view(np.uint16)[:ni], t["dbit"])
    assert np.array_equal(ck.u32(r.tree["inner_high_rid"])[:ni], perm[t["high"]])
    assert list(ck.mask_to_host(r.refined)) == list(dmask)


def test_batched_streams_and_graph_match_oracle(tmp_path):
    n = 300_001
    cols, dev, perms, dmasks = table(n)
    cache = str(tmp_path / "tune.txt")
    b = pipeline.BatchedRebuild(dev, dmasks, FANOUTS, cache_path=cache, tune_reps=2)
    assert all(4 <= r.digit_bits <= 11 for r in b.parts)
    assert all(r.tile in ck.CK_SORT_TILES for r in b.parts)
    b.run()
    torch.cuda.synchronize()
    for r, c, p, m, f in zip(b.parts, cols, perms, dmasks, FANOUTS):
        check_part(r, c, p, m, f)
    # graph replay, twice, after clobbering the outputs
    for _ in range(2):
        for r in b.parts:
            r.rid_sorted.fill_(-1)
            r.tree["leaf_dbit"].fill_(0)
        b.launch()
        torch.cuda.synchronize()
        for r, c, p, m, f in zip(b.parts, cols, perms, dmasks, FANOUTS):
            check_part(r, c, p, m, f)
    b.close()
    assert ck.ck_device_status()[0] == ck.CK_OK
    # the autotuner's cache serves the same widths without timing anything
    b2 = pipeline.BatchedRebuild(dev, dmasks, FANOUTS, cache_path=cache)
    assert [r.digit_bits for r in b2.parts] == [r.digit_bits for r in b.parts]
    assert [r.tile for r in b2.parts] == [r.tile for r in b.parts]
    assert all(ms == 0.0 for ms in b2.tuned_ms)
    assert os.path.getsize(cache) > 0


def test_batched_equals_unbatched():
    n = 100_003
    cols, dev, perms, dmasks = table(n)
    b = pipeline.BatchedRebuild(dev, dmasks, FANOUTS, digit_bits=[4, 5, 6, 8, 9, 11],
                                tiles=[2048, 4096, 8192, 2048, 8192, 4096])
    b.run()
    torch.cuda.synchronize()
    for k, r in enumerate(b.parts):
        u = pipeline.Rebuild(dev[k], dmasks[k], fanout=FANOUTS[k], digit_bits=8)
        u.run()
        torch.cuda.synchronize()
        assert torch.equal(u.rid_sorted[:n], r.rid_sorted[:n])
        assert torch.equal(u.ck_sorted[:, :n], r.ck_sorted[:, :n])
        for name in ("leaf_dbit", "inner_dbit", "inner_high_ck"):
            assert torch.equal(u.tree[name], r.tree[name])


def test_overlapped_rebuild_matches_oracle():
    """A stream of five batches through pipeline.OverlappedRebuild (copies of
    neighbouring batches beside each rebuild): every batch's sorted row ids on
    the host equal the oracle's order of that batch."""
    n = 200_003
    batches = [synth.urls(n, synth.BASE_SEED + 60 + k) for k in range(5)]
    allk = np.concatenate(batches)
    vmask = oracle.variant_mask(allk, 0)          # a superset of every batch's D-bitmap
    hosts = [torch.from_numpy(b).pin_memory() for b in batches]
    outs = [torch.empty(n, dtype=torch.int32, pin_memory=True) for _ in batches]
    O = pipeline.OverlappedRebuild((n, 32), torch.uint8, vmask, DEV, fanout=64)
    O.begin()
    for h, o in zip(hosts, outs):
        O.submit(h, o)
    O.finish()
    torch.cuda.synchronize()
    for b, o in zip(batches, outs):
        assert np.array_equal(o.numpy().view(np.uint32), oracle.sort_rows(b))
    assert ck.ck_device_status()[0] == ck.CK_OK
