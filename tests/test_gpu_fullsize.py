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
