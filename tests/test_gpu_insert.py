"""DS-metadata under batched inserts (Sec. 4.3, Insert): ck_insert_batch must
leave the D-bitmap and the variant bitmap exactly as the oracle's key-by-key
application of the paper's rule does, for byte and integer keys, duplicates,
inserts equal to indexed keys and new extremes; at a larger size the result
must equal the oracle's D-bitmap of the grown key set."""
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
from paper_2009_11543_gb300 import ck  # noqa: E402

DEV = "cuda:0"


def structured(rng, n, W, nvary):
    base = rng.integers(0, 256, W, dtype=np.uint8)
    pos = rng.choice(8 * W, size=nvary, replace=False)
    keys = np.repeat(base[None, :], n, axis=0)
    bits = np.unpackbits(keys, axis=1)
    bits[:, pos] = rng.integers(0, 2, (n, nvary), dtype=np.uint8)
    return np.packbits(bits, axis=1)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def mask_dev(m):
    return dev(np.asarray(m, np.uint64).view(np.int64))


def host_mask(t):
    return t.cpu().numpy().view(np.uint64)


def run_insert(old, new, ref, d_in, v_in, kind=None, old_dev=None, new_dev=None):
    """GPU update of (d_in, v_in) for `new` inserted into `old` (rows as in oracle)."""
    order = dev(oracle.sort_rows(old).view(np.int32))
    d, v = mask_dev(d_in), mask_dev(v_in)
    ck.ck_insert_batch(old_dev if old_dev is not None else dev(old), order,
                       new_dev if new_dev is not None else dev(new), ref, d, v, kind=kind)
    torch.cuda.synchronize()
    return host_mask(d), host_mask(v)


@pytest.mark.parametrize("W,n_old,m", [(1, 50, 20), (3, 4000, 700), (8, 20_000, 3000), (32, 12_000, 2500),
                                       (35, 3000, 1)])
def test_insert_matches_oracle_bytes(W, n_old, m):
    rng = np.random.default_rng(W * 1000 + m)
    allk = structured(rng, n_old + m, W, min(8 * W, 20))
    old, new = allk[:n_old].copy(), allk[n_old:].copy()
    if m > 3:
        new[: m // 4] = old[rng.integers(0, n_old, m // 4)]    # keys the index already holds
        new[m // 4] = 0                                         # a new minimum
        new[m // 4 + 1] = 255                                   # a new maximum
        new[m // 2: m // 2 + m // 8] = new[m // 2]              # a run of equal new keys
    ref = int(rng.integers(0, n_old))
    d0, v0 = oracle.dmask(old), oracle.variant_mask(old, ref)
    want_d, want_v = oracle.insert_batch(old, oracle.sort_rows(old), new, ref, d0, v0)
    got_d, got_v = run_insert(old, new, ref, d0, v0)
    assert np.array_equal(got_d, want_d) and np.array_equal(got_v, want_v)
    assert ck.ck_device_status()[0] == ck.CK_OK


@pytest.mark.parametrize("dtype", [np.uint32, np.uint64])
def test_insert_matches_oracle_integers(dtype):
    rng = np.random.default_rng(11)
    bits = 8 * np.dtype(dtype).itemsize
    vals = rng.integers(0, 1 << min(bits, 62), 30_000, dtype=np.uint64).astype(dtype)
    vals[rng.integers(0, 30_000, 3000)] = vals[0]
    old, new = vals[:25_000].copy(), vals[25_000:].copy()
    ref = 7
    ob, nb = oracle.as_key_bytes(old), oracle.as_key_bytes(new)
    d0, v0 = oracle.dmask(ob), oracle.variant_mask(ob, ref)
    want_d, want_v = oracle.insert_batch(ob, oracle.sort_rows(ob), nb, ref, d0, v0)
    view = np.int32 if dtype == np.uint32 else np.int64
    got_d, got_v = run_insert(ob, nb, ref, d0, v0, old_dev=dev(old.view(view)), new_dev=dev(new.view(view)))
    assert np.array_equal(got_d, want_d) and np.array_equal(got_v, want_v)


def test_insert_keeps_stale_bits_and_handles_equal_batches():
    """Bits a delete left behind stay set (Sec. 4.3); a batch of equal keys, a
    one-key batch and a batch of zero keys are handled."""
    rng = np.random.default_rng(5)
    old = structured(rng, 5000, 6, 12)
    ref = 0
    d0 = oracle.dmask(old)
    d0[0] |= np.uint64(1) << np.uint64(63)                      # a stale position 0
    v0 = oracle.variant_mask(old, ref)
    for new in (np.repeat(old[17:18], 40, axis=0), old[5:6].copy(), np.zeros((3, 6), np.uint8)):
        want_d, want_v = oracle.insert_batch(old, oracle.sort_rows(old), new, ref, d0, v0)
        got_d, got_v = run_insert(old, new, ref, d0, v0)
        assert np.array_equal(got_d, want_d) and np.array_equal(got_v, want_v)
        assert got_d[0] >> np.uint64(63) == 1


def test_insert_grown_url_index():
    """1M URL keys indexed, 100K more inserted: the maintained D-bitmap is the
    oracle's D-bitmap of all 1.1M keys and the variant bitmap theirs against
    the same reference key."""
    keys = synth.urls(1_100_000, synth.BASE_SEED + 2)
    old, new = keys[:1_000_000], keys[1_000_000:]
    ref = 0
    d0, v0 = oracle.dmask(old), oracle.variant_mask(old, ref)
    got_d, got_v = run_insert(old, new, ref, d0, v0)
    assert np.array_equal(got_d, oracle.dmask(keys))
    assert np.array_equal(got_v, oracle.variant_mask(keys, ref))


def test_insert_in_a_cuda_graph():
    """The call never waits for the GPU, so it can be captured: a replayed
    graph gives the bitmaps of the eager call."""
    rng = np.random.default_rng(21)
    allk = structured(rng, 60_000, 16, 40)
    old, new = allk[:50_000], allk[50_000:]
    ref = 3
    d0, v0 = oracle.dmask(old), oracle.variant_mask(old, ref)
    want_d, want_v = run_insert(old, new, ref, d0, v0)          # eager, also the library's first call here
    od, nd = dev(old), dev(new)
    order = dev(oracle.sort_rows(old).view(np.int32))
    d, v = mask_dev(d0), mask_dev(v0)
    ws = torch.empty(max(ck._lib().ck_insert_workspace_bytes(len(new), 16), 256), dtype=torch.uint8, device=DEV)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            ck.ck_insert_batch(od, order, nd, ref, d, v, ws=ws, stream=s)
    d.copy_(mask_dev(d0))
    v.copy_(mask_dev(v0))
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(host_mask(d), want_d) and np.array_equal(host_mask(v), want_v)
    assert ck.ck_device_status()[0] == ck.CK_OK


def test_insert_argument_errors():
    rng = np.random.default_rng(3)
    old = dev(structured(rng, 100, 8, 10))
    order = dev(np.arange(100, dtype=np.int32))
    d = torch.zeros(1, dtype=torch.int64, device=DEV)
    v = torch.zeros(1, dtype=torch.int64, device=DEV)
    with pytest.raises(ck.CkError) as e:                        # key width mismatch
        ck.ck_insert_batch(old, order, dev(structured(rng, 5, 4, 3)), 0, d, v)
    assert e.value.status == ck.CK_EINVAL
    with pytest.raises(ck.CkError) as e:                        # reference row out of range
        ck.ck_insert_batch(old, order, dev(structured(rng, 5, 8, 3)), 100, d, v)
    assert e.value.status == ck.CK_EINVAL
    small = torch.empty(256, dtype=torch.uint8, device=DEV)
    with pytest.raises(ck.CkError) as e:                        # workspace too small
        ck.ck_insert_batch(old, order, dev(structured(rng, 5000, 8, 30)), 0, d, v, ws=small)
    assert e.value.status == ck.CK_ENOMEM
    before = (d.clone(), v.clone())
    ck.ck_insert_batch(old, order, dev(np.zeros((0, 8), np.uint8)), 0, d, v)   # empty batch: no change
    assert torch.equal(d, before[0]) and torch.equal(v, before[1])
