"""Full-size parity: the 64M x 32-byte URL workload in the launch configuration
the bench times (8-bit digits, fanout 64).

The oracle cannot sort 64M keys in seconds, so the permutation is checked by
properties that fix it uniquely -- it is a bijection, and consecutive rows are
in (key, row id) order -- and then every O(n) output is compared with the
oracle computed under that verified order: the D-bitmap (Theorem 1), every
leaf and inner entry of the tree, and a random sample of compressed keys."""
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

N = 64 * 2**20


def rows_ordered(keys: np.ndarray, perm: np.ndarray, chunk: int = 1 << 22) -> bool:
    """True if keys[perm] is non-decreasing, ties in increasing row id."""
    n, W = keys.shape
    assert W % 8 == 0
    prev = None
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        lo = s - 1 if s > 0 else 0
        p = perm[lo:e]
        kp = keys[p].view(">u8").reshape(len(p), W // 8)
        a, b = kp[:-1], kp[1:]
        lt = np.zeros(len(a), bool)
        eq = np.ones(len(a), bool)
        for c in range(W // 8):
            lt |= eq & (a[:, c] < b[:, c])
            eq &= a[:, c] == b[:, c]
        if not np.all(lt | (eq & (p[:-1] < p[1:]))):
            return False
        prev = p[-1]
    return prev is not None or n <= 1


def test_urls_64m_full_size():
    keys = synth.urls(N, synth.BASE_SEED + 2)
    kd = torch.from_numpy(keys).to("cuda:0")
    dmask = pipeline.first_build_dmask(kd)
    nbits = ck.popcount(dmask)
    assert 100 <= nbits <= 128, nbits            # packs into 128-bit compressed keys
    r = pipeline.Rebuild(kd, dmask, fanout=64, digit_bits=8)    # the bench configuration
    assert r.K == 4
    r.run()
    torch.cuda.synchronize()
    assert ck.ck_device_status()[0] == ck.CK_OK
    perm = ck.u32(r.rid_sorted)[:N]
    assert np.all(np.bincount(perm, minlength=N) == 1)          # a bijection
    assert rows_ordered(keys, perm)                             # in (key, row id) order
    D = oracle.dmask(keys, perm)                                # Theorem 1 under the verified order
    assert list(D) == list(dmask)
    assert list(ck.mask_to_host(r.refined)) == list(D)
    t = oracle.btree(keys, perm, 64)
    assert [int(r.shape.level_entries[i]) for i in range(r.shape.levels)] == t["levels"]
    assert np.array_equal(r.tree["leaf_dbit"].cpu().numpy().view(np.uint16)[:N], t["leaf_dbit"])
    assert np.array_equal(ck.u32(r.tree["leaf_rid"])[:N], perm)
    ni = int(r.shape.inner_entries)
    assert np.array_equal(ck.u32(r.tree["inner_high"])[:ni], t["high"].astype(np.uint32))
    assert np.array_equal(r.tree["inner_dbit"].cpu().numpy().view(np.uint16)[:ni], t["dbit"])
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(N, 200_000, replace=False))
    exp = oracle.compress(keys[idx], dmask, 4)
    assert np.array_equal(ck.u32(r.ck_in)[:, idx].T, exp)                 # extraction, input order
    assert np.array_equal(ck.u32(r.ck_sorted)[:, idx].T, oracle.compress(keys[perm[idx]], dmask, 4))
    hck = ck.u32(r.tree["inner_high_ck"])[:ni * 4].reshape(ni, 4)
    sel = np.sort(rng.choice(ni, min(ni, 50_000), replace=False))
    assert np.array_equal(hck[sel], oracle.compress(keys[perm[t["high"][sel]]], dmask, 4))


def check_full(keys, r, fanout):
    n = len(keys)
    kb = oracle.as_key_bytes(keys) if keys.ndim == 1 else keys
    perm = ck.u32(r.rid_sorted)[:n]
    assert np.all(np.bincount(perm, minlength=n) == 1)
    assert rows_ordered(kb if kb.shape[1] % 8 == 0 else np.pad(kb, ((0, 0), (0, 8 - kb.shape[1] % 8))), perm)
    D = oracle.dmask(kb, perm)
    assert list(D) == list(ck.mask_to_host(r.refined))
    t = oracle.btree(kb, perm, fanout)
    assert np.array_equal(r.tree["leaf_dbit"].cpu().numpy().view(np.uint16)[:n], t["leaf_dbit"])
    ni = int(r.shape.inner_entries)
    assert np.array_equal(r.tree["inner_dbit"].cpu().numpy().view(np.uint16)[:ni], t["dbit"])
    return perm


@pytest.mark.parametrize("name,n,fanout", [("zipf", 256 * 2**20, 64), ("dna", 200_000_000, 256)])
def test_learned_full_size(name, n, fanout):
    """The learned configurations at the bench's sizes: 256M Zipf(0.9) uint64
    keys and 200M DNA keys, learned partition in the bench's configuration."""
    keys = synth.zipf_tagged_u64(n, synth.BASE_SEED + 4, 0.9) if name == "zipf" else synth.dna(n, synth.BASE_SEED + 5)
    kd = torch.from_numpy(keys.view(np.int64) if keys.dtype == np.uint64 else keys).to("cuda:0")
    dmask = pipeline.first_build_dmask(kd)
    r = pipeline.Rebuild(kd, dmask, fanout=fanout, learned=True)
    r.run()
    torch.cuda.synchronize()
    assert ck.ck_device_status()[0] == ck.CK_OK
    assert r.learned_stats["fell_back"] == 0, r.learned_stats
    perm = check_full(keys, r, fanout)
    p = pipeline.Rebuild(kd, dmask, fanout=fanout)      # the plain path gives the same bits
    p.run()
    torch.cuda.synchronize()
    assert np.array_equal(ck.u32(p.rid_sorted)[:n], perm)
    assert torch.equal(p.ck_sorted, r.ck_sorted)


def test_batched_table_full_size():
    """16M rows x 6 indexes, batched graph with autotuned digit widths."""
    n = 16 * 2**20
    cols = synth.table_columns(n, synth.BASE_SEED + 3)
    dev = [torch.from_numpy(c.view(np.int64) if c.dtype == np.uint64 else
                            (c.view(np.int32) if c.dtype == np.uint32 else c)).to("cuda:0") for c in cols]
    dmasks = [pipeline.first_build_dmask(c) for c in dev]
    fan = [64, 64, 64, 64, 256, 256]
    b = pipeline.BatchedRebuild(dev, dmasks, fan, tune_reps=2)
    b.launch()
    torch.cuda.synchronize()
    for c, r, f in zip(cols, b.parts, fan):
        check_full(c, r, f)
    b.close()
