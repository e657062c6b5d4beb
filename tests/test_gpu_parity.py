"""GPU parity: every libck output against the CPU oracle, bit for bit.

All calls go through the C ABI (the ctypes binding).  Sizes span several sort
tiles (8192 pairs) with a ragged tail; edge cases cover n = 0, 1, 2, all-equal
keys, |D| = 0, 1, 32, 33, 64, 65, every digit width, strided rows, and the
uint32 / uint64 / byte key kinds."""
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
TILE = ck.CK_SORT_TILE


# ---------------------------------------------------------------- helpers
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


def ck_rows(ck_dev, n):
    """word-major device ck [K, CK_LD(n)] -> row-major numpy [n, K] uint32"""
    return ck.ck_rows(ck_dev, n)


def ck_dev_of(ckr):
    """row-major [n, K] uint32 -> word-major device column with padded rows"""
    n, K = ckr.shape
    buf = np.zeros((K, max(ck.CK_LD(n), 64)), np.uint32)
    buf[:, :n] = ckr.T
    return to_dev(buf.view(np.int32))


def mask_of(positions, key_bits):
    m = np.zeros((key_bits + 63) // 64, np.uint64)
    for p in positions:
        m[p // 64] |= np.uint64(1 << (63 - p % 64))
    return m


def u64_keys_dev(v):
    return to_dev(v.view(np.int64))


# ------------------------------------------------------- variant / D-bits
@pytest.mark.parametrize("W", [1, 3, 4, 5, 8, 12, 16, 32, 35, 64])
def test_variant_and_dbits_bytes(W):
    rng = np.random.default_rng(100 + W)
    n = 3 * TILE + 77
    keys = structured(rng, n, W, min(8 * W, 20))
    kd = to_dev(keys)
    assert list(ck.mask_to_host(ck.ck_variant_bits(kd, 0))) == list(oracle.variant_mask(keys, 0))
    assert list(ck.mask_to_host(ck.ck_variant_bits(kd, 1234))) == list(oracle.variant_mask(keys, 1234))
    perm = oracle.sort_rows(keys)
    expect = oracle.dmask(keys, perm)
    got = ck.mask_to_host(ck.ck_distinction_bits(kd, to_dev(perm.view(np.int32))))
    assert list(got) == list(expect)
    got2 = ck.mask_to_host(ck.ck_distinction_bits(to_dev(keys[perm])))   # physically sorted
    assert list(got2) == list(expect)


@pytest.mark.parametrize("stride", [36, 40, 48, 64])
def test_dbits_extract_strided_rows(stride):
    """Rows padded to a stride: the kernel chooses 4/8/16-byte loads."""
    rng = np.random.default_rng(stride)
    n, W = 5000, 35
    keys = structured(rng, n, W, 40)
    padded = np.zeros((n, stride), np.uint8)
    padded[:, :W] = keys
    padded[:, W:] = 0xA5                     # garbage past the key must be ignored
    kd = to_dev(padded)[:, :W]
    perm = oracle.sort_rows(keys)
    got = ck.mask_to_host(ck.ck_distinction_bits(kd, to_dev(perm.view(np.int32))))
    assert list(got) == list(oracle.dmask(keys, perm))
    assert list(ck.mask_to_host(ck.ck_variant_bits(kd, 7))) == list(oracle.variant_mask(keys, 7))
    D = oracle.dmask(keys, perm)
    assert np.array_equal(ck_rows(ck.ck_extract(kd, D), n), oracle.compress(keys, D))


def test_extract_unaligned_column():
    """A column that starts off a 16-byte boundary is read without staging."""
    rng = np.random.default_rng(21)
    n, W = 3 * TILE + 3, 32
    keys = structured(rng, n, W, 90)
    buf = torch.zeros(n * W + 4, dtype=torch.uint8, device=DEV)
    buf[4:].copy_(to_dev(keys).view(-1))
    kd = buf[4:].view(n, W)
    D = oracle.dmask(keys)
    assert np.array_equal(ck_rows(ck.ck_extract(kd, D), n), oracle.compress(keys, D))


def test_integer_kinds():
    rng = np.random.default_rng(7)
    v64 = (rng.integers(0, 2**20, 40000, dtype=np.uint64) << np.uint64(37)) ^ np.uint64(0x5A5A)
    v32 = rng.integers(0, 2**31, 40000, dtype=np.uint64).astype(np.uint32)
    for v in (v64, v32):
        kd = to_dev(v.view(np.int64) if v.dtype == np.uint64 else v.view(np.int32))
        perm = oracle.sort_rows(v)
        D = oracle.dmask(v, perm)
        assert list(ck.mask_to_host(ck.ck_distinction_bits(kd, to_dev(perm.view(np.int32))))) == list(D)
        assert list(ck.mask_to_host(ck.ck_variant_bits(kd, 3))) == list(oracle.variant_mask(v, 3))
        assert np.array_equal(ck_rows(ck.ck_extract(kd, D), len(v)), oracle.compress(v, D))


@pytest.mark.parametrize("dtype", [np.int32, np.int64, np.float32, np.float64])
def test_signed_and_float_kinds(dtype):
    """Sec. 4.1 key formats read by the kernels: D-bitmap, variant bitmap,
    compressed keys, the sorted order and the tree of a signed or float column
    equal the oracle's on the encoded keys."""
    rng = np.random.default_rng(int(np.dtype(dtype).itemsize) + 40)
    n = 3 * TILE + 41
    if np.issubdtype(dtype, np.integer):
        v = rng.integers(-2**20, 2**20, n).astype(dtype)
    else:
        v = (rng.standard_normal(n) * 10.0 ** rng.integers(-5, 5, n)).astype(dtype)
        v[:4] = [-0.0, 0.0, -np.inf, np.inf]
    v[50:90] = v[3]
    kind = {np.int32: ck.CK_KIND_I32, np.int64: ck.CK_KIND_I64, np.float32: ck.CK_KIND_F32,
            np.float64: ck.CK_KIND_F64}[dtype]
    kd = to_dev(v)
    kb = oracle.as_key_bytes(v)
    perm = oracle.sort_rows(kb)
    D = oracle.dmask(kb, perm)
    assert list(ck.mask_to_host(ck.ck_distinction_bits(kd, to_dev(perm.view(np.int32)), kind=kind))) == list(D)
    assert list(ck.mask_to_host(ck.ck_variant_bits(kd, 5, kind=kind))) == list(oracle.variant_mask(kb, 5))
    assert np.array_equal(ck_rows(ck.ck_extract(kd, D, kind=kind), n), oracle.compress(kb, D))
    assert list(pipeline.first_build_dmask(kd, kind=kind)) == list(D)
    r = pipeline.Rebuild(kd, D, fanout=16, kind=kind)
    r.run()
    torch.cuda.synchronize()
    assert np.array_equal(ck.u32(r.rid_sorted)[:n], perm)
    t = oracle.btree(kb, perm, 16)
    assert np.array_equal(r.tree["leaf_dbit"].cpu().numpy().view(np.uint16)[:n], t["leaf_dbit"])


def test_dbits_small_and_degenerate():
    for keys in (np.zeros((0, 8), np.uint8), np.full((1, 8), 7, np.uint8), np.full((5000, 8), 9, np.uint8),
                 np.array([[0] * 8, [255] * 8], np.uint8)):
        kd = to_dev(keys) if len(keys) else torch.empty((0, 8), dtype=torch.uint8, device=DEV)
        got = ck.mask_to_host(ck.ck_distinction_bits(kd))
        assert list(got) == list(oracle.dmask(keys)) if len(keys) else list(got) == [0]
        got = ck.mask_to_host(ck.ck_variant_bits(kd, 0))
        assert list(got) == (list(oracle.variant_mask(keys)) if len(keys) else [0])


# ------------------------------------------------------------------ extract
def table3_mask():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table3_indbtab_dbitmap.txt")
    bits = "".join(l.strip().replace(" ", "") for l in open(path) if not l.startswith("#"))
    pos = [i for i, b in enumerate(bits) if b == "1"]
    return mask_of(pos, 280)


@pytest.mark.parametrize("ck_words", [2, 3, 5])
def test_extract_table3_mask(ck_words):
    rng = np.random.default_rng(ck_words)
    keys = rng.integers(0, 256, (3 * TILE + 5, 35), dtype=np.uint8)
    m = table3_mask()
    got = ck_rows(ck.ck_extract(to_dev(keys), m, ck_words), len(keys))
    assert np.array_equal(got, oracle.compress(keys, m, ck_words))


@pytest.mark.parametrize("W,npos", [(4, 1), (4, 32), (8, 33), (8, 64), (12, 65), (16, 96), (16, 128),
                                    (32, 117), (32, 256), (64, 300), (64, 512), (3, 24), (5, 17)])
def test_extract_masks(W, npos):
    rng = np.random.default_rng(W * 1000 + npos)
    keys = rng.integers(0, 256, (2 * TILE + 11, W), dtype=np.uint8)
    m = mask_of(sorted(rng.choice(8 * W, npos, replace=False)), 8 * W)
    got = ck_rows(ck.ck_extract(to_dev(keys), m), len(keys))
    assert np.array_equal(got, oracle.compress(keys, m))


def word_mask(words):
    """D-bitmap (uint64 words, big-endian bit order) from 32-bit mask words."""
    words = list(words) + [0] * (len(words) % 2)
    return np.array([(words[2 * i] << 32) | words[2 * i + 1] for i in range(len(words) // 2)], np.uint64)


WORD_FORM_MASKS = {
    # ASCII bytes (one run per byte), the URL column's words
    "ascii": [0, 0, 0x0000001F, 0x1F1F1F5F, 0x5F180000, 0x7F7F7F7F, 0x7F7F7F7F, 0x7F7F7F7F],
    # two runs per byte, the DNA column's words
    "dna": [0x16161616] * 4 + [0x16141400, 0, 0x16161616, 0x16161404],
    # one byte mask in all four bytes
    "bytes": [0x0E0E0E0E, 0x63636363, 0x81818181, 0x41414141, 0x3C3C3C3C, 0x16161616, 0x07070707, 0x18181818],
    # one- and two-run words: full, top, bottom, middle, split; then scattered bits
    "runs": [0xFFFFFFFF, 0xFFFFFFF8, 0x000000FF, 0x80000000, 0x00000001, 0x00FFFF00, 0xF000000F, 0x0003C000,
             0xCA94A8A1, 0x30BA202C, 0x55555555, 0],
}


@pytest.mark.parametrize("name", sorted(WORD_FORM_MASKS))
@pytest.mark.parametrize("extra_words", [0, 2])
def test_extract_word_forms(name, extra_words):
    """Every form of the per-word program (shift-and-mask runs, the network
    with some or all rounds) and every way a word's bits meet the output words
    (inside one, ending one exactly, straddling two), on a ragged row count;
    extra_words > 0 adds whole zero words at the top of the output.  The
    digit counts of the same pass match the oracle's compressed keys."""
    words = WORD_FORM_MASKS[name]
    m = word_mask(words)
    W = 4 * len(words)
    rng = np.random.default_rng(len(words) * 7 + extra_words)
    n = 3 * TILE + 301
    keys = rng.integers(0, 256, (n, W), dtype=np.uint8)
    nbits = oracle.popcount(m)
    K = ck.words_for(nbits) + extra_words
    want = oracle.compress(keys, m, K)
    assert np.array_equal(ck_rows(ck.ck_extract(to_dev(keys), m, K), n), want)
    ckd, hist = ck.ck_extract_hist(to_dev(keys), m, K, 8)
    assert np.array_equal(ck_rows(ckd, n), want)
    passes = (nbits + 7) // 8
    assert np.array_equal(hist[:passes].cpu().numpy().astype(np.int64), oracle_digit_hist(want, nbits, 8))


def test_extract_full_mask_is_the_key():
    rng = np.random.default_rng(3)
    keys = rng.integers(0, 256, (1000, 16), dtype=np.uint8)
    got = ck_rows(ck.ck_extract(to_dev(keys), pipeline.full_key_mask(128)), len(keys))
    ints = [int.from_bytes(bytes(r), "big") for r in keys]
    assert [sum(int(w) << (32 * k) for k, w in enumerate(row)) for row in got] == ints


def test_extract_empty_mask_zeroes():
    keys = np.arange(64, dtype=np.uint8).reshape(8, 8)
    got = ck_rows(ck.ck_extract(to_dev(keys), np.zeros(1, np.uint64), 2), len(keys))
    assert not got.any()


# ------------------------------------------------------------------ sort
def check_sort(ckr, rid_in=None, nbits=None, digit_bits=8, inplace=False, tile=0):
    """ckr: row-major [n, K] uint32 compressed keys (high bits above nbits zero)."""
    n, K = ckr.shape
    nbits = 32 * K if nbits is None else nbits
    ck_in = ck_dev_of(ckr)
    rid_dev = to_dev(rid_in.view(np.int32)) if rid_in is not None else None
    ws = torch.empty(max(ck.ck_sort_workspace_bytes(n, K, nbits, digit_bits, tile), 256), dtype=torch.uint8,
                     device=DEV)
    if inplace:
        ck_out = ck_in
        rid_out = rid_dev if rid_dev is not None else torch.empty(max(n, 1), dtype=torch.int32, device=DEV)
    else:
        ck_out = torch.empty_like(ck_in)
        rid_out = torch.empty(max(n, 1), dtype=torch.int32, device=DEV)
    ck.ck_sort(ck_in, rid_dev, ck_out, rid_out, n, K, nbits, ws, digit_bits=digit_bits, tile=tile)
    torch.cuda.synchronize()
    perm = oracle.sort_compressed(ckr)
    exp_rid = perm if rid_in is None else rid_in[perm]
    assert np.array_equal(ck.u32(rid_out)[:n], exp_rid)
    assert np.array_equal(ck_rows(ck_out, n), ckr[perm])
    assert ck.ck_device_status()[0] == ck.CK_OK


@pytest.mark.parametrize("digit_bits", [4, 5, 6, 7, 8, 9, 10, 11])
def test_sort_digit_widths(digit_bits):
    rng = np.random.default_rng(digit_bits)
    n = 4 * TILE + 123
    nbits = 45
    v = rng.integers(0, 2**45, n, dtype=np.uint64)
    v[rng.integers(0, n, 3000)] = v[rng.integers(0, n, 3000)]        # ties keep row order
    ckr = np.stack([(v & np.uint64(0xFFFFFFFF)).astype(np.uint32), (v >> np.uint64(32)).astype(np.uint32)], 1)
    check_sort(ckr, nbits=nbits, digit_bits=digit_bits)


@pytest.mark.parametrize("tile,digit_bits,nbits", [(2048, 8, 45), (8192, 8, 45), (2048, 4, 45), (8192, 11, 45),
                                                   (2048, 11, 96), (8192, 5, 96), (2048, 7, 1), (8192, 8, 128)])
def test_sort_tiles(tile, digit_bits, nbits):
    """The pass tiles the autotuner may pick (2048 and 8192 pairs besides the
    default): several tiles of each and a ragged last tile, ties by row id."""
    rng = np.random.default_rng(tile + digit_bits + nbits)
    n = 3 * 8192 + 77
    K = max(1, (nbits + 31) // 32)
    ckr = rng.integers(0, 2**32, (n, K), dtype=np.uint64).astype(np.uint32)
    top = nbits - 32 * (K - 1)
    if top < 32:
        ckr[:, K - 1] &= np.uint32((1 << top) - 1)
    ckr[rng.integers(0, n, 2000)] = ckr[rng.integers(0, n, 2000)]
    check_sort(ckr, nbits=nbits, digit_bits=digit_bits, tile=tile)


@pytest.mark.parametrize("nbits", [1, 7, 8, 24, 32, 33, 64, 65, 96, 120, 128])
def test_sort_key_widths(nbits):
    rng = np.random.default_rng(nbits)
    n = 3 * TILE + 999
    K = max(1, (nbits + 31) // 32)
    ckr = rng.integers(0, 2**32, (n, K), dtype=np.uint64).astype(np.uint32)
    top = nbits - 32 * (K - 1)
    if top < 32:
        ckr[:, K - 1] &= np.uint32((1 << top) - 1)
    ckr[rng.integers(0, n, 500)] = ckr[rng.integers(0, n, 500)]
    check_sort(ckr, nbits=nbits)


def test_sort_rid_in_and_inplace():
    rng = np.random.default_rng(5)
    n = 2 * TILE + 1
    ckr = rng.integers(0, 1 << 20, (n, 1), dtype=np.uint64).astype(np.uint32)
    rid = rng.permutation(n).astype(np.uint32)
    check_sort(ckr, rid_in=rid, nbits=20)
    check_sort(ckr, rid_in=rid, nbits=20, inplace=True)
    check_sort(ckr, nbits=20, inplace=True)
    low = ckr & np.uint32(0xFFFF)                                     # nbits = 16: no bits above
    check_sort(low, nbits=16, digit_bits=8, inplace=True)             # even pass count in place


@pytest.mark.parametrize("n", [0, 1, 2, 31, 32, 33, TILE - 1, TILE, TILE + 1])
def test_sort_small_sizes(n):
    rng = np.random.default_rng(n)
    ckr = rng.integers(0, 1 << 30, (n, 1), dtype=np.uint64).astype(np.uint32)
    if n == 0:
        ws = torch.empty(256, dtype=torch.uint8, device=DEV)
        e = torch.empty((1, 1), dtype=torch.int32, device=DEV)
        ck.ck_sort(e, None, e, torch.empty(1, dtype=torch.int32, device=DEV), 0, 1, 30, ws)
        return
    check_sort(ckr, nbits=30)


def test_sort_zero_bits_and_all_equal():
    n = TILE + 5
    check_sort(np.zeros((n, 1), np.uint32), nbits=0)
    check_sort(np.full((n, 2), 3, np.uint32), nbits=40)


def test_sort_timeout_is_reported_and_gpu_stays_usable():
    """Fault injection on the host: the first tile never publishes, so the
    bounded waits of the tiles after it run out; the call must report
    CK_ETIMEOUT for pass 0 and a waiting tile, and the next sort must be exact."""
    ck.ck_clear_device_status()
    rng = np.random.default_rng(9)
    n = 3 * TILE
    ckr = rng.integers(0, 1 << 24, (n, 1), dtype=np.uint64).astype(np.uint32)
    ck_in = ck_dev_of(ckr)
    ws = torch.empty(ck.ck_sort_workspace_bytes(n, 1, 24), dtype=torch.uint8, device=DEV)
    ck_out = torch.empty_like(ck_in)
    rid_out = torch.empty(n, dtype=torch.int32, device=DEV)
    ck.ck_sort(ck_in, None, ck_out, rid_out, n, 1, 24, ws, spin_limit=2000, inject=ck.CK_INJECT_STALL_FIRST_TILE)
    status, detail = ck.ck_device_status()
    assert status == ck.CK_ETIMEOUT
    assert detail & 0xFFFF == 0 and (detail >> 16) in (1, 2)   # pass 0, a tile waiting on tile 0
    ck.ck_clear_device_status()
    assert ck.ck_device_status()[0] == ck.CK_OK
    check_sort(ckr, nbits=24)


# --------------------------------------------------------------- B-tree
def check_tree(keys, fanout, fill=1.0, dmask=None, digit_bits=8, perm_only=False):
    kd = to_dev(keys) if keys.dtype == np.uint8 else u64_keys_dev(keys)
    perm = oracle.sort_rows(keys)
    D = oracle.dmask(keys, perm)
    m = D if dmask is None else dmask
    r = pipeline.Rebuild(kd, m, fanout=fanout, fill=fill, digit_bits=digit_bits, perm_only=perm_only)
    r.run()
    torch.cuda.synchronize()
    n = len(perm)
    assert np.array_equal(ck.u32(r.rid_sorted)[:n], perm)
    kb = oracle.as_key_bytes(keys)
    if not perm_only:
        assert np.array_equal(ck_rows(r.ck_sorted, n), oracle.compress(kb, m, r.K)[perm])
    f = oracle.entries_per_node(fanout, fill)
    t = oracle.btree(kb, perm, f)
    assert [int(r.shape.level_entries[i]) for i in range(r.shape.levels)] == t["levels"]
    assert np.array_equal(ck.u32(r.tree["leaf_rid"])[:n], perm)
    assert np.array_equal(r.tree["leaf_dbit"].cpu().numpy().view(np.uint16)[:n], t["leaf_dbit"])
    nodes0 = (n + f - 1) // f
    assert np.array_equal(ck.u32(r.tree["leaf_high"])[:nodes0],
                          np.minimum((np.arange(nodes0) + 1) * f, n) - 1)
    ni = int(r.shape.inner_entries)
    assert ni == len(t["child"])
    if ni:
        assert np.array_equal(ck.u32(r.tree["inner_child"])[:ni], t["child"])
        assert np.array_equal(ck.u32(r.tree["inner_high"])[:ni], t["high"].astype(np.uint32))
        assert np.array_equal(ck.u32(r.tree["inner_high_rid"])[:ni], perm[t["high"]])
        hck = ck.u32(r.tree["inner_high_ck"])[:ni * r.K].reshape(ni, r.K)
        assert np.array_equal(hck, oracle.compress(kb, m, r.K)[perm[t["high"]]])
        assert np.array_equal(r.tree["inner_dbit"].cpu().numpy().view(np.uint16)[:ni], t["dbit"])
    assert list(ck.mask_to_host(r.refined)) == list(D)      # Sec. 4.3 step 1 gives D exactly
    assert ck.ck_device_status()[0] == ck.CK_OK
    return r


@pytest.mark.parametrize("perm_only", [False, True])
@pytest.mark.parametrize("fanout,fill", [(64, 1.0), (14, 0.9), (9, 0.9), (256, 1.0), (2, 1.0)])
def test_btree_fanouts(fanout, fill, perm_only):
    rng = np.random.default_rng(fanout)
    keys = structured(rng, 3 * TILE + 300, 12, 50)
    check_tree(keys, fanout, fill, perm_only=perm_only)


@pytest.mark.parametrize("perm_only", [False, True])
def test_btree_from_superset_mask(perm_only):
    """Extraction with the variant bitmap (a superset of D): same permutation,
    same tree, and the refinement recovers D exactly."""
    rng = np.random.default_rng(11)
    keys = structured(rng, 2 * TILE + 9, 16, 60)
    check_tree(keys, 64, dmask=oracle.variant_mask(keys, 0), perm_only=perm_only)


@pytest.mark.parametrize("perm_only", [False, True])
@pytest.mark.parametrize("n", [1, 2, 63, 64, 65])
def test_btree_tiny(n, perm_only):
    rng = np.random.default_rng(n)
    keys = structured(rng, n, 8, 10, dup_frac=0.3)
    check_tree(keys, 8, perm_only=perm_only)


@pytest.mark.parametrize("perm_only", [False, True])
def test_btree_all_equal_keys(perm_only):
    keys = np.full((1000, 8), 42, np.uint8)
    check_tree(keys, 16, perm_only=perm_only)


@pytest.mark.parametrize("digit_bits", [4, 7, 8, 11])
@pytest.mark.parametrize("W,nvary", [(8, 24), (16, 70), (32, 117), (64, 200)])
def test_perm_only_sort_and_keys_tree(W, nvary, digit_bits):
    """The permutation-only sort (consumed key words dropped) and the tree
    built from the key column: identical to the oracle."""
    rng = np.random.default_rng(W * 100 + digit_bits)
    keys = structured(rng, 3 * TILE + 41, W, nvary)
    check_tree(keys, 64, digit_bits=digit_bits, perm_only=True)


# ------------------------------------------------------------ workloads
def test_pipeline_integer_column_1m():
    """1,000,000 uint64 keys with 24 seeded varying bits, fanout 64: the whole
    path (first build from the variant bitmap, then the rebuild) bit-exact."""
    keys, pos = synth.varying_bits_u64(1_000_000, synth.BASE_SEED + 1)
    kd = u64_keys_dev(keys)
    D_gpu = pipeline.first_build_dmask(kd)
    perm = oracle.sort_rows(keys)
    assert np.array_equal(np.argsort(keys, kind="stable").astype(np.uint32), perm)   # textbook sort agrees
    D = oracle.dmask(keys, perm)
    assert list(D_gpu) == list(D)
    r = check_tree(keys, 64)
    assert r.shape.levels == 4 and [int(r.shape.level_entries[i]) for i in range(4)] == [1_000_000, 15625, 245, 4]


def test_pipeline_urls_dna_titles():
    for keys in (synth.urls(150_000, synth.BASE_SEED + 2), synth.dna(150_000, synth.BASE_SEED + 5),
                 synth.titles(150_000, synth.BASE_SEED + 3, 32)):
        kd = to_dev(keys)
        D_gpu = pipeline.first_build_dmask(kd)
        perm = oracle.sort_rows(keys)
        assert list(D_gpu) == list(oracle.dmask(keys, perm))
        check_tree(keys, 64)
        check_tree(keys, 256, perm_only=True)


def test_full_key_baseline_same_permutation():
    keys = synth.urls(100_000, 77)
    r = pipeline.Rebuild(to_dev(keys), pipeline.full_key_mask(256))
    r.run()
    assert np.array_equal(ck.u32(r.rid_sorted), oracle.sort_rows(keys))


def oracle_digit_hist(ckr, nbits, rb):
    """Digit counts of the oracle's compressed keys ([n, K] words, least
    significant first): hist[q][v] = #keys with bits [q*rb, q*rb+rb) = v."""
    passes = (nbits + rb - 1) // rb
    vals = [sum(int(w) << (32 * k) for k, w in enumerate(row)) for row in ckr]
    h = np.zeros((passes, 1 << rb), np.int64)
    for v in vals:
        for q in range(passes):
            h[q, (v >> (q * rb)) & ((1 << rb) - 1)] += 1
    return h


@pytest.mark.parametrize("W,npos,rb", [(32, 117, 8), (8, 40, 4), (16, 100, 11), (5, 17, 8), (40, 200, 8),
                                       (12, 96, 7)])
def test_extract_hist_matches_oracle(W, npos, rb):
    """ck_extract_hist: the compressed keys as ck_extract's, and the digit
    counts those of the oracle's compressed keys -- counted in the extraction
    pass (up to 16 KB of counters) or by the sort's counting kernel after it
    (200 positions in 8-bit digits: 25 KB)."""
    rng = np.random.default_rng(W * 31 + rb)
    n = 2 * TILE + 777
    keys = structured(rng, n, W, npos, dup_frac=0.2)
    m = oracle.variant_mask(keys, 0)
    nbits = oracle.popcount(m)
    ckd, hist = ck.ck_extract_hist(to_dev(keys), m, ck.words_for(nbits), rb)
    want = oracle.compress(keys, m)
    assert np.array_equal(ck_rows(ckd, n), want)
    passes = (nbits + rb - 1) // rb
    got = hist[:passes].cpu().numpy().astype(np.int64)
    assert np.array_equal(got, oracle_digit_hist(want, nbits, rb))
    assert got.sum(axis=1).tolist() == [n] * passes


def test_sort_with_extracted_hist_equals_sort():
    """ck_sort given the extraction's digit counts gives the same pairs as
    ck_sort counting them itself, and the oracle's order."""
    rng = np.random.default_rng(17)
    n, W = 5 * TILE + 123, 32
    keys = structured(rng, n, W, 110)
    D = oracle.dmask(keys)
    nbits = oracle.popcount(D)
    K = ck.words_for(nbits)
    ckd, hist = ck.ck_extract_hist(to_dev(keys), D, K, 8)
    outs = []
    for h in (hist, None):
        ck_out = ck.ck_buffer(K, n, DEV)
        rid = torch.empty(n, dtype=torch.int32, device=DEV)
        ws = torch.empty(ck.ck_sort_workspace_bytes(n, K, nbits), dtype=torch.uint8, device=DEV)
        ck.ck_sort(ckd, None, ck_out, rid, n, K, nbits, ws, hist=h)
        outs.append((ck_rows(ck_out, n), ck.u32(rid)[:n]))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][1], oracle.sort_rows(keys))


def test_extract_hist_edge_cases():
    """Empty column (counts zeroed), all-equal keys (no digits: no counts
    needed), a digit width outside 4..11, and a one-row column."""
    W = 8
    empty = torch.empty((0, W), dtype=torch.uint8, device=DEV)
    m = mask_of([3, 17, 40], 8 * W)
    hist = torch.full((1, 256), 7, dtype=torch.int32, device=DEV)
    ck.ck_extract_hist(empty, m, 1, 8, out=torch.empty(64, dtype=torch.int32, device=DEV), hist=hist)
    assert int(hist.abs().sum()) == 0
    same = to_dev(np.repeat(np.arange(W, dtype=np.uint8)[None, :], 1000, axis=0))
    z = np.zeros(1, np.uint64)
    ckd, _ = ck.ck_extract_hist(same, z, 1, 8)
    assert int(ckd[:, :1000].abs().sum()) == 0
    with pytest.raises(ck.CkError) as e:
        ck.ck_extract_hist(same, m, 1, 12)
    assert e.value.status == ck.CK_EINVAL
    one = to_dev(np.full((1, W), 0xA5, np.uint8))
    ckd, h = ck.ck_extract_hist(one, m, 1, 4)
    v = int(oracle.compress(np.full((1, W), 0xA5, np.uint8), m)[0, 0])
    want = np.zeros((1, 16), np.int64)
    want[0, v & 15] = 1
    assert np.array_equal(h.cpu().numpy().astype(np.int64), want)


def test_ds_metadata_restart(tmp_path):
    """Checkpoint / resume as the paper has it (Sec. 4.2, 4.3): the first build's
    DS-metadata is saved; after a 'restart' the loaded D-bitmap drives the
    rebuild, which reproduces the oracle's order and refines to the same D."""
    keys = synth.urls(3 * TILE + 9, synth.BASE_SEED + 91)
    kd = to_dev(keys)
    m = pipeline.DSMetadata.from_keys(kd, ref_row=5)
    assert np.array_equal(m.dmask, oracle.dmask(keys))
    assert np.array_equal(m.vmask, oracle.variant_mask(keys, 5))
    assert np.array_equal(m.ref_key, keys[5])
    path = str(tmp_path / "ds.npz")
    m.save(path)
    loaded = pipeline.DSMetadata.load(path)
    r = pipeline.Rebuild(kd, loaded.dmask, fanout=64)
    r.run()
    torch.cuda.synchronize()
    assert np.array_equal(ck.u32(r.rid_sorted)[:len(keys)], oracle.sort_rows(keys))
    assert np.array_equal(ck.mask_to_host(r.refined), loaded.dmask)
