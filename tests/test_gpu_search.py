"""Partial-key leaves and search on the GPU (Sec. 4.2, Sec. 4.3 Search,
Sec. 5.3 bit sources).  Every leaf and inner partial key must equal the
oracle's (taken from the full keys), whichever way the bits are sourced: an
extraction mask extended for them (C a), the key rows (C b), or a tree built
from the row ids alone.  Every search result (lower-bound position and row id)
must equal the oracle's, for queries that are keys, keys one bit away, random
rows and the extremes."""
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


def structured(rng, n, W, nvary, dup_frac=0.1):
    base = rng.integers(0, 256, W, dtype=np.uint8)
    pos = rng.choice(8 * W, size=min(nvary, 8 * W), replace=False)
    keys = np.repeat(base[None, :], n, axis=0)
    bits = np.unpackbits(keys, axis=1)
    bits[:, pos] = rng.integers(0, 2, (n, len(pos)), dtype=np.uint8)
    keys = np.packbits(bits, axis=1)
    nd = int(n * dup_frac)
    if nd and n > 1:
        keys[rng.integers(0, n, nd)] = keys[rng.integers(0, n, nd)]
    return keys


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def u32(t, n):
    return t[:n].cpu().numpy().view(np.uint32)


def queries_for(rng, kb, m):
    """Index-key byte rows: keys, keys with one bit flipped, random rows, extremes."""
    n, W = kb.shape
    a = kb[rng.integers(0, n, m)]
    b = kb[rng.integers(0, n, m)].copy()
    flip = rng.integers(0, 8 * W, m)
    b[np.arange(m), flip // 8] ^= (0x80 >> (flip % 8)).astype(np.uint8)
    c = rng.integers(0, 256, (m // 4, W), dtype=np.uint8)
    ext = np.stack([np.zeros(W, np.uint8), np.full(W, 255, np.uint8), kb.min(axis=0), kb.max(axis=0)])
    return np.concatenate([a, b, c, ext])


def check_partial_keys(keys_np, r, leaf_pk, inner_pk, pk, f):
    n = keys_np.shape[0]
    perm = oracle.sort_rows(keys_np)
    t = oracle.btree(keys_np, perm, f)
    want_leaf, want_inner = oracle.partial_keys(keys_np, perm, t, pk)
    assert np.array_equal(u32(leaf_pk, n), want_leaf)
    ni = int(r.shape.inner_entries)
    assert ni == len(want_inner)
    if ni:
        assert np.array_equal(u32(inner_pk, ni), want_inner)


CASES = [  # W, n, nvary, f, pk
    (3, 20_011, 20, 16, 8),
    (8, 50_000, 40, 64, 16),
    (32, 30_007, 90, 14, 32),
    (35, 9_000, 50, 5, 4),
    (5, 3_000, 24, 2, 1),
]


@pytest.mark.parametrize("W,n,nvary,f,pk", CASES)
@pytest.mark.parametrize("source", ["extended_mask", "rows", "perm_only"])
def test_partial_keys_match_oracle(W, n, nvary, f, pk, source):
    rng = np.random.default_rng(W * 100 + pk)
    keys = structured(rng, n, W, nvary)
    kd = to_dev(keys)
    D, V = oracle.dmask(keys), oracle.variant_mask(keys, 7)
    ref = ck.reference_key(kd, 7)
    assert np.array_equal(ref, keys[7])
    mask = ck.ck_partial_key_mask(D, V, 8 * W, pk) if source == "extended_mask" else D
    r = pipeline.Rebuild(kd, mask, fanout=f, perm_only=source == "perm_only")
    r.run()
    if source == "extended_mask":   # every bit from the compressed keys or the reference key: no column
        leaf_pk, inner_pk = ck.ck_partial_keys(r.shape, r.tree, r.ck_sorted, r.K, mask, V, ref, pk,
                                               key_bytes=W)
    else:
        leaf_pk, inner_pk = r.partial_keys(V, ref, pk)
    torch.cuda.synchronize()
    check_partial_keys(keys, r, leaf_pk, inner_pk, pk, f)
    assert np.array_equal(ck.mask_to_host(r.refined), D)
    assert ck.ck_device_status()[0] == ck.CK_OK


def test_partial_keys_need_rows_without_extension():
    """With the plain D-bitmap some partial-key bits are variant and outside
    the compressed key: without a column they have no source, which the
    device status word records (CK_EINVAL); no column and no compressed keys
    is refused at once."""
    rng = np.random.default_rng(4)
    keys = structured(rng, 5000, 8, 30)
    kd = to_dev(keys)
    D, V = oracle.dmask(keys), oracle.variant_mask(keys, 0)
    assert not np.array_equal(ck.ck_partial_key_mask(D, V, 64, 8), D)
    r = pipeline.Rebuild(kd, D, fanout=16)
    r.run()
    assert ck.ck_device_status()[0] == ck.CK_OK
    ck.ck_partial_keys(r.shape, r.tree, r.ck_sorted, r.K, D, V, keys[0], 8, key_bytes=8)
    assert ck.ck_device_status()[0] == ck.CK_EINVAL
    ck.ck_clear_device_status()
    with pytest.raises(ck.CkError) as e:
        ck.ck_partial_keys(r.shape, r.tree, None, r.K, D, V, keys[0], 8, key_bytes=8)
    assert e.value.status == ck.CK_EINVAL


@pytest.mark.parametrize("W,n,nvary,f,pk", CASES)
@pytest.mark.parametrize("inner_partial", [True, False])
def test_search_matches_oracle(W, n, nvary, f, pk, inner_partial):
    rng = np.random.default_rng(W * 10 + f)
    keys = structured(rng, n, W, nvary)
    kd = to_dev(keys)
    D, V = oracle.dmask(keys), oracle.variant_mask(keys, 0)
    r = pipeline.Rebuild(kd, D, fanout=f)
    r.run()
    r.partial_keys(V, keys[0], pk)
    q = queries_for(rng, keys, 4000)
    pos, rid, derefs = r.search(to_dev(q), want_derefs=True, inner_partial=inner_partial)
    torch.cuda.synchronize()
    want_pos, want_rid = oracle.search(keys, oracle.sort_rows(keys), q)
    m = len(q)
    assert np.array_equal(u32(pos, m), want_pos)
    assert np.array_equal(u32(rid, m), want_rid)
    dr = u32(derefs, m)
    assert np.all(dr[want_rid != ck.CK_NO_ROW] >= 1)       # a match is confirmed on the full key
    assert dr.mean() < (int(r.shape.levels) + 2 if inner_partial else 3.0)   # ties of short partial keys
    assert ck.ck_device_status()[0] == ck.CK_OK


@pytest.mark.parametrize("kind,dtype", [(ck.CK_KIND_U64, np.uint64), (ck.CK_KIND_I32, np.int32),
                                        (ck.CK_KIND_F64, np.float64)])
def test_search_numeric_columns(kind, dtype):
    """Numeric columns (Sec. 4.1 key formats): partial keys from the mapped
    big-endian form, search with native query values."""
    rng = np.random.default_rng(21)
    n = 40_000
    if dtype == np.float64:
        vals = rng.standard_normal(n) * 1e3
        vals[:50] = np.array([0.0, -0.0, np.inf, -np.inf] * 12 + [1.5, -1.5])
    elif dtype == np.int32:
        vals = rng.integers(-2**31, 2**31, n).astype(np.int32)
    else:
        vals = rng.integers(0, 2**63, n, dtype=np.uint64)
    vals[rng.integers(0, n, 4000)] = vals[rng.integers(0, n, 4000)]
    vals = vals.astype(dtype)
    kb = oracle.as_key_bytes(vals)
    vd = to_dev(vals.view(np.int64 if vals.itemsize == 8 else np.int32))
    D, V = oracle.dmask(kb), oracle.variant_mask(kb, 3)
    ref = ck.reference_key(vd, 3, kind=kind)
    assert np.array_equal(ref, kb[3])
    r = pipeline.Rebuild(vd, D, fanout=32, kind=kind)
    r.run()
    leaf_pk, inner_pk = r.partial_keys(V, ref, 12)
    torch.cuda.synchronize()
    check_partial_keys(kb, r, leaf_pk, inner_pk, 12, 32)
    qv = np.concatenate([vals[rng.integers(0, n, 3000)], vals[rng.integers(0, n, 3000)] + 1]).astype(dtype)
    pos, rid, _ = r.search(to_dev(qv.view(np.int64 if qv.itemsize == 8 else np.int32)))
    torch.cuda.synchronize()
    want_pos, want_rid = oracle.search(kb, oracle.sort_rows(kb), oracle.as_key_bytes(qv))
    assert np.array_equal(u32(pos, len(qv)), want_pos)
    assert np.array_equal(u32(rid, len(qv)), want_rid)


@pytest.mark.parametrize("n", [1, 2, 3, 64, 65])
def test_search_small_and_equal_keys(n):
    """Single-leaf trees, a tree of n = 1, and all-equal keys (no offsets)."""
    rng = np.random.default_rng(n)
    W = 6
    for keys in (structured(rng, n, W, 10, dup_frac=0.0), np.repeat(structured(rng, 1, W, 10), n, axis=0)):
        kd = to_dev(keys)
        D, V = oracle.dmask(keys), oracle.variant_mask(keys, 0)
        r = pipeline.Rebuild(kd, D, fanout=8)
        r.run()
        leaf_pk, inner_pk = r.partial_keys(V, keys[0], 5)
        q = queries_for(rng, keys, 50)
        check_partial_keys(keys, r, leaf_pk, inner_pk, 5, 8)
        want_pos, want_rid = oracle.search(keys, oracle.sort_rows(keys), q)
        for inner_partial in (True, False):
            pos, rid, _ = r.search(to_dev(q), inner_partial=inner_partial)
            torch.cuda.synchronize()
            assert np.array_equal(u32(pos, len(q)), want_pos)
            assert np.array_equal(u32(rid, len(q)), want_rid)


def test_search_url_index_full_size():
    """The 64M-key URL column (32-byte keys, |D| = 121, fanout 64): 1M sampled
    queries land between their sorted neighbours (key[pos - 1] < q <=
    key[pos]), a query equal to a key returns that key's first row, and
    partial keys of sampled leaf entries equal the oracle's bits of the row."""
    n = 64 * 1024 * 1024
    keys = synth.urls(n, synth.BASE_SEED + 2)
    kd = to_dev(keys)
    dmask = pipeline.first_build_dmask(kd)
    vmask = ck.mask_to_host(ck.ck_variant_bits(kd, 0))
    r = pipeline.Rebuild(kd, dmask, fanout=64)
    r.run()
    leaf_pk, _ = r.partial_keys(vmask, keys[0], 16)
    rng = np.random.default_rng(5)
    m = 1 << 20
    q = np.concatenate([keys[rng.integers(0, n, m // 2)],                 # keys of the index
                        queries_for(rng, keys[rng.integers(0, n, 1 << 16)], m // 4)])
    qd = to_dev(q)
    pos, rid, derefs = r.search(qd, want_derefs=True)
    pos_f, rid_f, _ = r.search(qd, inner_partial=True)      # partial keys in the inner nodes too
    torch.cuda.synchronize()
    assert torch.equal(pos[:len(q)], pos_f[:len(q)]) and torch.equal(rid[:len(q)], rid_f[:len(q)])
    pos, rid = u32(pos, len(q)).astype(np.int64), u32(rid, len(q))
    perm = ck.u32(r.rid_sorted)[:n].astype(np.int64)
    sample = rng.integers(0, len(q), 20_000)
    for j in sample:
        qb = q[j].tobytes()
        p = pos[j]
        if p > 0:
            assert keys[perm[p - 1]].tobytes() < qb
        if p < n:
            assert qb <= keys[perm[p]].tobytes()
            assert rid[j] == (perm[p] if keys[perm[p]].tobytes() == qb else ck.CK_NO_ROW)
        else:
            assert rid[j] == ck.CK_NO_ROW
    assert np.all(rid[: m // 2] != ck.CK_NO_ROW)
    idx = rng.integers(0, n, 20_000)
    lp = u32(leaf_pk, n)
    ld = r.tree["leaf_dbit"][:n].cpu().numpy().view(np.uint16)
    rows = keys[perm[idx]]
    start = np.where(ld[idx] == oracle.NO_DBIT, 0, ld[idx].astype(np.int64) + 1)
    got_bits = lp[idx]
    for k in range(len(idx)):
        v = int.from_bytes(rows[k].tobytes(), "big") << 16
        assert int(got_bits[k]) == (v >> (256 - int(start[k]))) & 0xFFFF
    assert float(u32(derefs, len(q)).mean()) < 3.0
    assert ck.ck_device_status()[0] == ck.CK_OK
