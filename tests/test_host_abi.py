"""Host-side checks that need no GPU: the C ABI library loads and exports every
function include/ck.h declares, the host planning code agrees with the
oracle and the closed forms, argument errors come back synchronously, and the
reported metric formulas reproduce Table 2 of the paper."""
import json
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ckmod():
    from paper_2009_11543_gb300 import build as b
    b.build()
    from paper_2009_11543_gb300 import ck
    return ck


def header_functions():
    src = open(os.path.join(ROOT, "include", "ck.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ck_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(ckmod):
    lib = ckmod._lib()
    names = header_functions()
    assert "ck_sort" in names and "ck_extract" in names
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(ckmod.EXPORTED) == names


def pext32(x, m):
    out, k = 0, 0
    for b in range(32):
        if (m >> b) & 1:
            out |= ((x >> b) & 1) << k
            k += 1
    return out


def test_compress_network_matches_pext(ckmod):
    rng = np.random.default_rng(0)
    masks = [0, 0xFFFFFFFF, 0x80000001, 0x0F0F0F0F, 0x00000001, 0x80000000] + \
            [int(x) for x in rng.integers(0, 2**32, 300, dtype=np.uint64)]
    for m in masks:
        for x in [0, 0xFFFFFFFF] + [int(v) for v in rng.integers(0, 2**32, 20, dtype=np.uint64)]:
            assert ckmod.ck_compress_word_host(x, m) == pext32(x, m)


def test_word_programs_match_pext(ckmod):
    """The per-word form the extraction kernel runs: one- and two-run masks
    (shift-and-mask terms, including a full word and runs touching bit 0 or
    bit 31), masks of three or more runs (the network with its zero rounds
    skipped; among them every byte mask repeated in all four bytes), and mask
    words of the URL, DNA, Zipf and integer workloads."""
    rng = np.random.default_rng(1)
    masks = [0xFFFFFFFF, 0x80000000, 0x00000001, 0x0000001F, 0xFFFFFFF8, 0x7F000000, 0xF000000F,
             0x00FF0F00, 0x7F7F7F7F, 0x1F1F1F5F, 0x5F180000, 0x16161616, 0x16141400, 0xCA94A8A1,
             0x30BA202C, 0x55555555, 0xAAAAAAAA,
             # one byte mask in all four bytes
             0x16161616, 0x0E0E0E0E, 0x63636363, 0x81818181, 0x7E7E7E7E, 0x3C3C3C3C, 0x41414141, 0x07070707,
             0xC0C0C0C0, 0x18181818, 0x01010101, 0x80808080]
    for b in range(1, 255):                    # every byte mask, in all four bytes
        masks.append(b * 0x01010101)
    for _ in range(200):                       # random one- and two-run masks
        a, b = sorted(int(v) for v in rng.integers(0, 33, 2))
        c, d = sorted(int(v) for v in rng.integers(0, 33, 2))
        run = lambda lo, hi: ((1 << hi) - 1) ^ ((1 << lo) - 1)
        masks += [run(a, b), run(a, b) | run(c, d)]
    masks += [int(x) for x in rng.integers(0, 2**32, 300, dtype=np.uint64)]
    for m in masks:
        for x in [0, 0xFFFFFFFF] + [int(v) for v in rng.integers(0, 2**32, 16, dtype=np.uint64)]:
            assert ckmod.ck_compress_word_program_host(x, m) == pext32(x, m), (hex(x), hex(m))


def test_btree_plan_matches_oracle(ckmod):
    for n in (0, 1, 2, 14, 15, 1000, 4097, 10**6, 200 * 10**6):
        for fanout, fill in ((64, 1.0), (256, 1.0), (14, 0.9), (9, 0.9), (10, 0.7)):
            s = ckmod.ck_btree_plan(n, fanout, fill)
            f = oracle.entries_per_node(fanout, fill)
            assert s.entries_per_node == f
            lv = oracle.btree_shape(n, f)
            assert s.levels == len(lv)
            assert [int(s.level_entries[i]) for i in range(s.levels)] == lv
            off = 0
            for l in range(1, s.levels):
                assert s.inner_offset[l] == off
                off += lv[l]
            assert s.inner_entries == off


def test_argument_errors_are_synchronous(ckmod):
    import ctypes
    lib = ckmod._lib()
    col = ckmod.ck_column(0, 10, 8, 8, ckmod.CK_KIND_BYTES)          # NULL keys with n > 0
    m = np.zeros(1, np.uint64)
    assert lib.ck_extract(ctypes.byref(col), m.ctypes.data, 1, None, None) == ckmod.CK_EINVAL
    col = ckmod.ck_column(4096, 10, 8, 4, ckmod.CK_KIND_BYTES)       # stride < key bytes
    assert lib.ck_variant_bits(ctypes.byref(col), 0, 4096, None) == ckmod.CK_EINVAL
    col = ckmod.ck_column(4096, 10, 600, 600, ckmod.CK_KIND_BYTES)   # key too wide
    assert lib.ck_distinction_bits(ctypes.byref(col), None, 4096, None) == ckmod.CK_EINVAL
    col = ckmod.ck_column(4096, 10, 8, 8, ckmod.CK_KIND_U32)         # U32 needs 4 bytes
    assert lib.ck_distinction_bits(ctypes.byref(col), None, 4096, None) == ckmod.CK_EINVAL
    col = ckmod.ck_column(4096, 10, 4, 4, ckmod.CK_KIND_BYTES)
    m = np.array([0xFFFFFFFFF0000000], np.uint64)                    # 36 set bits > 32 * 1 word
    assert lib.ck_extract(ctypes.byref(col), m.ctypes.data, 1, 4096, None) in (ckmod.CK_EINVAL,)
    m = np.array([0xFFFFFFFF00000000], np.uint64)
    col = ckmod.ck_column(4096, 10, 8, 8, ckmod.CK_KIND_BYTES)
    m2 = np.array([0xFFFFFFFF80000000], np.uint64)                   # 33 bits into 1 word
    assert lib.ck_extract(ctypes.byref(col), m2.ctypes.data, 1, 4096, None) == ckmod.CK_EOVERFLOW
    o = ckmod.ck_sort_opts(3, 0, 0, 0, None)                             # digit width out of range
    assert lib.ck_sort(4096, None, 8192, 12288, 100, 1, 20, ctypes.byref(o), None, 0, None) == ckmod.CK_EINVAL
    o = ckmod.ck_sort_opts(8, 0, 0, 0, None)
    assert lib.ck_sort(4096, None, 8192, 12288, 100, 1, 20, ctypes.byref(o), None, 0, None) == ckmod.CK_ENOMEM
    assert lib.ck_sort(4096, None, 8192, 12288, 100, 1, 40, ctypes.byref(o), None, 0, None) == ckmod.CK_EINVAL
    assert lib.ck_sort(4096, None, 8192, 12288, 1 << 30, 1, 20, None, None, 0, None) == ckmod.CK_EINVAL
    for tile in (1024, 3000, 16384):                                    # not a pass tile
        o = ckmod._opts(8, tile=tile)
        assert lib.ck_sort(4096, None, 8192, 12288, 100, 1, 20, ctypes.byref(o), None, 0, None) == ckmod.CK_EINVAL
        assert lib.ck_sort_workspace_bytes(100, 1, 20, ctypes.byref(o)) == 0
    o = ckmod._opts(8)
    o.reserved = 1
    assert lib.ck_sort(4096, None, 8192, 12288, 100, 1, 20, ctypes.byref(o), None, 0, None) == ckmod.CK_EINVAL
    s = ckmod.ck_btree_shape()
    assert lib.ck_btree_plan(100, 1, ctypes.c_float(1.0), ctypes.byref(s)) == ckmod.CK_EINVAL


@pytest.mark.parametrize("tile", [0, 2048, 4096, 8192])
def test_workspace_size_formula(ckmod, tile):
    """One look-back word per tile, digit and pass: the tile sets the count."""
    n, K, nbits = 10**6, 4, 120
    ws = ckmod.ck_sort_workspace_bytes(n, K, nbits, 8, tile)
    t = tile or ckmod.CK_SORT_TILE
    tiles = (n + t - 1) // t
    passes = 15
    ld = ckmod.CK_LD(n)
    assert ld % 64 == 0 and ld >= n
    body = 4 * K * ld + 4 * n + 4 * 256 * tiles * passes
    assert body <= ws < body + 4 * 256 * passes + 4 * passes + 5 * 256


def test_table2_metric_formulas():
    from paper_2009_11543_gb300 import metrics as mt
    with open(os.path.join(ROOT, "tests", "golden", "table2_dataset_stats.json")) as f:
        g = json.load(f)
    crs, skrs = [], []
    for i in range(6):
        cr = mt.compression_ratio(g["full_key_bits"][i], g["distinction_bits"][i])
        assert round(cr, 2) == g["compression_ratio"][i]
        fb = mt.full_sort_key_bytes(g["max_key_length_bytes"][i], g["record_id_bytes"])
        cb = mt.compressed_sort_key_bytes(g["distinction_bits"][i], g["record_id_variant_bits"][i])
        assert fb == g["full_sort_key_bytes"][i]
        assert cb == g["compressed_sort_key_bytes"][i]
        skr = mt.sort_key_ratio(fb, cb)
        assert round(skr, 2) == g["sort_key_ratio"][i]
        crs.append(cr)
        skrs.append(skr)
    assert round(sum(crs) / 6, 2) == g["average_compression_ratio"]
    assert round(sum(skrs) / 6, 2) == g["average_sort_key_ratio"]
    frac = sum(d / f for d, f in zip(g["distinction_bits"], g["full_key_bits"])) / 6
    assert round(100 * frac, 1) == g["average_distinction_fraction_percent"]


def test_perm_only_pass_bytes():
    """Permutation-only LSD sort of 121-bit keys in 4 words with 8-bit digits:
    word w is carried until its last digit is consumed."""
    from paper_2009_11543_gb300 import metrics as mt
    arrs = mt.perm_only_pass_arrays(4, 121, 8)
    assert len(arrs) == 16
    assert arrs[0] == (5, 5) and arrs[3] == (5, 4) and arrs[4] == (4, 4) and arrs[15] == (2, 1)
    assert sum(r + w for r, w in arrs) == 108            # vs 16 * 10 = 160 when every word is carried
    assert mt.perm_only_sort_bytes(10, 4, 121, 8) == 4 * 10 * 108
    assert mt.perm_only_pass_arrays(1, 20, 8) == [(2, 2), (2, 2), (2, 1)]


def test_header_constants_match_binding(ckmod):
    """The binding's copies of the header's size constants."""
    import re
    with open(os.path.join(ROOT, "include", "ck.h")) as f:
        hdr = f.read()
    for name in ("CK_SORT_TILE", "CK_MAX_LEVELS", "CK_MLP_HIDDEN", "CK_MAX_PARTIAL_KEY_BITS"):
        m = re.search(r"#define %s (\d+)u?" % name, hdr)
        assert m and int(m.group(1)) == getattr(ckmod, name), name
    m = re.search(r"#define CK_NO_ROW (0x[0-9A-Fa-f]+)u?", hdr)
    assert m and int(m.group(1), 16) == ckmod.CK_NO_ROW


@pytest.mark.parametrize("W,nvary,pk", [(1, 5, 1), (4, 14, 3), (9, 30, 16), (33, 60, 32), (64, 200, 7)])
def test_partial_key_mask_matches_oracle(ckmod, W, nvary, pk):
    """ck_partial_key_mask (host only, Sec. 5.3 C a) against the oracle's
    extension of the D-bitmap, on the D and variant bitmaps of random keys."""
    rng = np.random.default_rng(W * 7 + pk)
    base = rng.integers(0, 256, W, dtype=np.uint8)
    pos = rng.choice(8 * W, size=min(nvary, 8 * W), replace=False)
    keys = np.repeat(base[None, :], 300, axis=0)
    bits = np.unpackbits(keys, axis=1)
    bits[:, pos] = rng.integers(0, 2, (300, len(pos)), dtype=np.uint8)
    keys = np.packbits(bits, axis=1)
    D, V = oracle.dmask(keys), oracle.variant_mask(keys, 0)
    got = ckmod.ck_partial_key_mask(D, V, 8 * W, pk)
    assert np.array_equal(got, oracle.partial_key_mask(D, V, 8 * W, pk))


def test_partial_key_mask_argument_errors(ckmod):
    z = np.zeros(1, np.uint64)
    for key_bits, pk in ((0, 4), (8, 0), (8, 33)):
        with pytest.raises(ckmod.CkError) as e:
            ckmod.ck_partial_key_mask(z, z, key_bits, pk)
        assert e.value.status == ckmod.CK_EINVAL


def test_ds_metadata_round_trip(tmp_path, ckmod):
    """The persisted DS-metadata (Sec. 4.2) survives a save and a load
    unchanged, and mismatched sizes are refused."""
    from paper_2009_11543_gb300 import pipeline
    rng = np.random.default_rng(12)
    keys = rng.integers(0, 256, (500, 12), dtype=np.uint8)
    m = pipeline.DSMetadata(oracle.dmask(keys), oracle.variant_mask(keys, 4), keys[4], 96)
    path = str(tmp_path / "ds.npz")
    m.save(path)
    r = pipeline.DSMetadata.load(path)
    assert np.array_equal(r.dmask, m.dmask) and np.array_equal(r.vmask, m.vmask)
    assert np.array_equal(r.ref_key, keys[4]) and r.key_bits == 96
    with pytest.raises(ValueError):
        pipeline.DSMetadata(m.dmask, m.vmask, keys[4, :8], 96)


def test_argument_errors_of_later_entry_points(ckmod):
    """Digit counting, partial keys, search, inserts and key encoding refuse
    bad arguments synchronously, before any device work (the device pointers
    below are never touched)."""
    import ctypes
    lib = ckmod._lib()
    col = ckmod.ck_column(4096, 10, 8, 8, ckmod.CK_KIND_BYTES)
    m = np.array([0xFFFFF00000000000], np.uint64)                    # 20 positions
    for rb in (3, 12):
        assert lib.ck_extract_hist(ctypes.byref(col), m.ctypes.data, 1, 4096, rb, 8192, None) == ckmod.CK_EINVAL
    assert lib.ck_extract_hist(ctypes.byref(col), m.ctypes.data, 1, 4096, 8, None, None) == ckmod.CK_EINVAL
    t = ckmod.ck_btree()
    z = np.zeros(1, np.uint64)
    ref = np.zeros(8, np.uint8)
    for pk in (0, 33):
        assert lib.ck_partial_keys(ctypes.byref(t), 4096, 1, z.ctypes.data, z.ctypes.data, ref.ctypes.data,
                                   ctypes.byref(col), 8, pk, 8192, 8192, None) == ckmod.CK_EINVAL
        assert lib.ck_search(ctypes.byref(t), ctypes.byref(col), 4096, None, pk, ctypes.byref(col), 8192, None,
                             None, None) == ckmod.CK_EINVAL
    q32 = ckmod.ck_column(4096, 10, 4, 4, ckmod.CK_KIND_U32)            # queries of another kind
    assert lib.ck_search(ctypes.byref(t), ctypes.byref(col), 4096, None, 16, ctypes.byref(q32), 8192, None,
                         None, None) == ckmod.CK_EINVAL
    narrow = ckmod.ck_column(4096, 5, 4, 4, ckmod.CK_KIND_BYTES)        # batch of another width
    assert lib.ck_insert_batch(ctypes.byref(col), 8192, ctypes.byref(narrow), 0, 12288, 16384, None, 0,
                               None) == ckmod.CK_EINVAL
    parts = (ckmod.ck_key_part * 1)()
    assert lib.ck_encode_key(parts, 0, 10, 4096, 16, None) == ckmod.CK_EINVAL
    parts[0] = ckmod.ck_key_part(4096, None, ckmod.CK_KIND_DECIMAL, 10, 8)   # decimal of 10 bytes
    assert lib.ck_encode_key(parts, 1, 10, 8192, 16, None) == ckmod.CK_EINVAL


def test_learned_sort_argument_errors(ckmod):
    """The learned sort's binding marshals every argument (device stats and
    parameter buffers included) and the call refuses bad arguments
    synchronously, before any device work (the buffers below are host memory
    that is never touched)."""
    import torch
    ck_in = torch.zeros((1, 256), dtype=torch.int32)
    out = torch.zeros((1, 256), dtype=torch.int32)
    rid = torch.zeros(256, dtype=torch.int32)
    ws = torch.zeros(256, dtype=torch.uint8)
    stats = torch.zeros(ckmod.CK_LEARNED_STATS_BYTES // 4, dtype=torch.int32)
    params = torch.zeros(ckmod.CK_MLP_PARAMS, dtype=torch.float32)
    bad = [dict(ck_words=0), dict(ck_words=9), dict(nbits=33), dict(opts=ckmod.learned_opts(bucket_bits=16)),
           dict(opts=ckmod.learned_opts(flags=8)), dict(same=True)]
    for b in bad:
        kw = dict(ck_words=1, nbits=20, opts=None)
        kw.update({k: v for k, v in b.items() if k != "same"})
        src = out if b.get("same") else ck_in
        with pytest.raises(ckmod.CkError) as e:
            ckmod.ck_sort_learned(src, out, rid, 256, kw["ck_words"], kw["nbits"], ws, kw["opts"], stats=stats,
                                  params=params, stream=0)
        assert e.value.status == ckmod.CK_EINVAL, b
    assert ckmod.ck_learned_stats.from_buffer_copy(bytes(ckmod.CK_LEARNED_STATS_BYTES)).fell_back == 0
    assert ctypes_sizeof_stats(ckmod) == ckmod.CK_LEARNED_STATS_BYTES


def ctypes_sizeof_stats(ckmod):
    import ctypes
    return ctypes.sizeof(ckmod.ck_learned_stats)
