"""Pins for the CPU oracle: each test checks an oracle function against something
other than itself -- a fact the paper states for a worked example, a closed
form, a brute-force enumeration, or an independently written procedure -- so
that a dropped term, a wrong sign or index, or a transposed operand in the
oracle fails at least one of them.  CPU only."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers
def ints_to_rows(vals, nbits):
    """Big-integer keys of nbits bits -> [n, W] big-endian uint8 rows (zero-padded)."""
    W = (nbits + 7) // 8
    pad = 8 * W - nbits
    return np.array([list((v << pad).to_bytes(W, "big")) for v in vals], np.uint8).reshape(len(vals), W)


def positions_of(mask, key_bits):
    return [p for p in range(key_bits) if (int(mask[p // 64]) >> (63 - p % 64)) & 1]


def mask_of(positions, key_bits):
    m = np.zeros((key_bits + 63) // 64, np.uint64)
    for p in positions:
        m[p // 64] |= np.uint64(1 << (63 - p % 64))
    return m


def row_int(row):
    return int.from_bytes(bytes(row), "big")


def dbit_py(a: int, b: int, nbits: int) -> int:
    """Closed form on integers: nbits - bit_length(a xor b); -1 if equal."""
    x = a ^ b
    return -1 if x == 0 else nbits - x.bit_length()


def ck_ints(ck):
    return [sum(int(w) << (32 * k) for k, w in enumerate(row)) for row in ck]


def random_structured_keys(rng, n, W, nvary):
    """Keys sharing a random pattern except at nvary random positions."""
    base = rng.integers(0, 256, W, dtype=np.uint8)
    pos = rng.choice(8 * W, size=nvary, replace=False)
    keys = np.repeat(base[None, :], n, axis=0)
    bits = np.unpackbits(keys, axis=1)
    bits[:, pos] = rng.integers(0, 2, (n, nvary), dtype=np.uint8)
    return np.packbits(bits, axis=1)


# ------------------------------------------------ Sec. 3.1 worked example
def load_fig2():
    with open(os.path.join(GOLD, "fig2_worked_example.json")) as f:
        g = json.load(f)
    vals = [int(h, 16) for h in g["keys_sorted_hex"]]
    return g, vals


def test_fig2_stated_facts():
    g, vals = load_fig2()
    st, nb = g["stated"], g["key_bits"]
    rows = ints_to_rows(vals, nb)
    perm = oracle.sort_rows(rows)
    assert list(perm) == list(range(len(vals)))            # the carrier keys are sorted
    D = positions_of(oracle.dmask(rows), 8 * rows.shape[1])
    assert D == st["distinction_positions"]
    V = positions_of(oracle.variant_mask(rows), 8 * rows.shape[1])
    assert V == st["variant_positions"]
    inv = [p for p in range(nb) if p not in V]
    assert inv == st["invariant_positions"]
    adj = [oracle.dbit(bytes(rows[i - 1]), bytes(rows[i])) for i in range(1, len(vals))]
    assert adj[:4] == [st["D_1"], st["D_2"], st["D_3"], st["D_4"]]
    assert oracle.dbit(bytes(rows[1]), bytes(rows[3])) == st["dbit_key1_key3"]
    assert oracle.dbit(bytes(rows[0]), bytes(rows[2])) == st["dbit_key0_key2"]
    assert sorted(set(V) - set(D)) == st["variant_not_distinction"]
    # deletion example (Sec. 3.2): delete key3, then key0
    r3 = np.delete(rows, 3, axis=0)
    D3 = positions_of(oracle.dmask(r3), 16)
    assert (7 in D3) == st["after_deleting_key3"]["7_in_D"]
    assert (7 in positions_of(oracle.variant_mask(r3), 16)) == st["after_deleting_key3"]["7_variant"]
    r30 = np.delete(r3, 0, axis=0)
    assert positions_of(oracle.dmask(r30), 16) == D3
    assert (7 in positions_of(oracle.variant_mask(r30), 16)) == st["after_deleting_key3_and_key0"]["7_variant"]
    # partial key (Sec. 4.2): the pk = 4 bits following D_1 of key_1
    d1 = st["D_1"]
    pk = "".join(str((vals[1] >> (nb - 1 - p)) & 1) for p in range(d1 + 1, d1 + 5))
    assert pk == st["partial_key_of_key1_pk4"]


def test_remark1_not_minimal():
    with open(os.path.join(GOLD, "remark1_example.json")) as f:
        g = json.load(f)
    vals = [int(b, 2) for b in g["keys_sorted_bin"]]
    rows = ints_to_rows(vals, g["key_bits"])
    D = positions_of(oracle.dmask(rows), 8)
    assert D == g["stated"]["distinction_positions"]
    # brute force the smallest position subset whose slice orders the keys strictly
    best = None
    for size in range(1, 5):
        for sub in itertools.combinations(range(4), size):
            sl = [tuple((v >> (3 - p)) & 1 for p in sub) for v in vals]
            if all(sl[i] < sl[i + 1] for i in range(len(sl) - 1)):
                best = (size, list(sub))
                break
        if best:
            break
    assert best == (g["stated"]["minimum_size"], g["stated"]["minimal_slice"])
    assert len(D) > best[0]          # the method does not claim minimality


# --------------------------------------------------- Sec. 3.1 definitions
def test_dbit_closed_form_uint64():
    rng = np.random.default_rng(1)
    a = rng.integers(0, 2**63, 2000, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, 2000, dtype=np.uint64)
    b = a ^ (np.uint64(1) << rng.integers(0, 64, 2000, dtype=np.uint64))   # one flipped bit
    b[::3] = rng.integers(0, 2**63, len(b[::3]), dtype=np.uint64)
    b[5] = a[5]
    ab, bb = oracle.as_key_bytes(a), oracle.as_key_bytes(b)
    for i in range(len(a)):
        assert oracle.dbit(bytes(ab[i]), bytes(bb[i])) == dbit_py(int(a[i]), int(b[i]), 64)


def test_uint_keys_are_big_endian():
    v = np.array([0x0102030405060708], np.uint64)
    assert bytes(oracle.as_key_bytes(v)[0]) == bytes([1, 2, 3, 4, 5, 6, 7, 8])
    v32 = np.array([0xA1B2C3D4], np.uint32)
    assert bytes(oracle.as_key_bytes(v32)[0]) == bytes([0xA1, 0xB2, 0xC3, 0xD4])


def test_sort_rows_against_python_sorted():
    rng = np.random.default_rng(2)
    for W in (1, 3, 8, 13):
        keys = rng.integers(0, 4, (500, W), dtype=np.uint8)     # many duplicates
        perm = oracle.sort_rows(keys)
        ref = sorted(range(500), key=lambda i: (bytes(keys[i]), i))
        assert list(perm) == ref


def test_sort_u64_matches_numeric_stable_argsort():
    rng = np.random.default_rng(3)
    v = rng.integers(0, 1000, 3000, dtype=np.uint64) << np.uint64(40)
    assert list(oracle.sort_rows(v)) == list(np.argsort(v, kind="stable"))


def test_varchar_nul_rule():
    # Sec. 4.1 C: "AB" + NUL < "ABA" + NUL, and the D-bit falls in the NUL byte.
    rows = np.array([list(b"ABA\0"), list(b"AB\0\0")], np.uint8)
    assert list(oracle.sort_rows(rows)) == [1, 0]
    p = oracle.dbit(bytes(rows[1]), bytes(rows[0]))
    assert p // 8 == 2 and p == 16 + (8 - (ord("A")).bit_length())


# ----------------------------------------------------- Lemma 1, Theorem 1
def brute_dall(vals, nbits):
    s = set()
    for i in range(len(vals)):
        for j in range(i + 1, len(vals)):
            d = dbit_py(vals[i], vals[j], nbits)
            if d >= 0:
                s.add(d)
    return sorted(s)


def test_theorem1_exhaustive_tiny():
    """D_all == D_adj over every multiset of up to 5 keys of 4 bits."""
    nb = 4
    count = 0
    for size in range(1, 6):
        for combo in itertools.combinations_with_replacement(range(16), size):
            rows = ints_to_rows(list(combo), nb)
            D = positions_of(oracle.dmask(rows), 8)
            assert D == brute_dall(list(combo), nb)
            count += 1
    assert count > 6000


@pytest.mark.parametrize("seed", range(8))
def test_theorem1_random(seed):
    rng = np.random.default_rng(10 + seed)
    W = int(rng.integers(1, 6))
    keys = random_structured_keys(rng, int(rng.integers(2, 60)), W, int(rng.integers(1, 8 * W)))
    keys = keys[rng.permutation(len(keys))]
    vals = [row_int(r) for r in keys]
    D = positions_of(oracle.dmask(keys), 8 * W)
    assert D == brute_dall(vals, 8 * W)


def test_lemma1_min_over_adjacent():
    rng = np.random.default_rng(4)
    vals = sorted(set(int(x) for x in rng.integers(0, 2**20, 200)))
    nb = 24
    Dk = [None] + [dbit_py(vals[k - 1], vals[k], nb) for k in range(1, len(vals))]
    for _ in range(2000):
        i, j = sorted(rng.choice(len(vals), 2, replace=False))
        rows = ints_to_rows([vals[i], vals[j]], nb)
        assert oracle.dbit(bytes(rows[0]), bytes(rows[1])) == min(Dk[i + 1:j + 1])


# ------------------------------------------------------ variant bitmap
def test_variant_mask_brute_force():
    rng = np.random.default_rng(5)
    for W in (1, 4, 7):
        keys = random_structured_keys(rng, 40, W, 5)
        bits = np.unpackbits(keys, axis=1)
        expect = [p for p in range(8 * W) if len(set(bits[:, p])) > 1]
        for ref in (0, 17, 39):
            assert positions_of(oracle.variant_mask(keys, ref), 8 * W) == expect


# ------------------------------------------------------ Sec. 3.2 Compress
def test_compress_all_positions_is_identity():
    rng = np.random.default_rng(6)
    for W in (4, 8, 12, 5):
        keys = rng.integers(0, 256, (50, W), dtype=np.uint8)
        ck = oracle.compress(keys, mask_of(range(8 * W), 8 * W))
        assert ck_ints(ck) == [row_int(r) for r in keys]


def test_compress_single_position_and_order():
    rng = np.random.default_rng(7)
    keys = rng.integers(0, 256, (64, 6), dtype=np.uint8)
    for p in (0, 7, 8, 31, 47):
        ck = oracle.compress(keys, mask_of([p], 48))
        assert [int(r[0]) for r in ck] == [(row_int(k) >> (47 - p)) & 1 for k in keys]
    # first set position lands in the most significant bit
    ck = oracle.compress(keys, mask_of([3, 40], 48))
    for k, c in zip(keys, ck):
        v = row_int(k)
        assert int(c[0]) == (((v >> 44) & 1) << 1) | ((v >> 7) & 1)


def pext(x: int, m: int) -> int:
    """Parallel bit extract (BMI2 PEXT semantics) on Python integers."""
    out, k = 0, 0
    while m:
        low = m & -m
        if x & low:
            out |= 1 << k
        k += 1
        m ^= low
    return out


def paper_extract(key: bytes, mask_bytes: bytes) -> tuple[int, int]:
    """Sec. 5.1 procedure: 8-byte masks starting at the byte of the next 1,
    PEXT per mask, shift-and-OR concatenation.  Written independently of the
    oracle's bit-by-bit definition."""
    W = len(mask_bytes)
    out, nb, start, masks = 0, 0, 0, 0
    while True:
        while start < W and mask_bytes[start] == 0:
            start += 1
        if start >= W:
            break
        mseg = mask_bytes[start:start + 8].ljust(8, b"\0")
        kseg = key[start:start + 8].ljust(8, b"\0")
        m, x = int.from_bytes(mseg, "big"), int.from_bytes(kseg, "big")
        c = bin(m).count("1")
        out = (out << c) | pext(x, m)
        nb += c
        masks += 1
        start += 8
    return out, masks


def load_table3():
    with open(os.path.join(GOLD, "table3_indbtab_dbitmap.txt")) as f:
        bits = "".join(l.strip().replace(" ", "") for l in f if not l.startswith("#"))
    assert len(bits) == 35 * 8
    return bytes(int(bits[i:i + 8], 2) for i in range(0, len(bits), 8))


def test_table3_mask_facts_and_paper_extraction():
    mb = load_table3()
    m = np.zeros(5, np.uint64)
    big = int.from_bytes(mb, "big") << (320 - 280)
    for w in range(5):
        m[w] = np.uint64((big >> (64 * (4 - w))) & (2**64 - 1))
    pos = positions_of(m, 280)
    assert len(pos) == 56                                   # Table 2: 56 D-bits
    assert max(pos) // 8 + 1 == 22                          # last D-bit in byte 22
    assert (len(pos) + 7) // 8 == 7                         # fits in 7 bytes
    assert (pos[0], pos[-1]) == (23, 174)
    rng = np.random.default_rng(8)
    keys = rng.integers(0, 256, (300, 35), dtype=np.uint8)
    ck = oracle.compress(keys, m)
    assert ck.shape == (300, 2)
    masks = None
    for k, c in zip(keys, ck_ints(ck)):
        v, masks = paper_extract(bytes(k), mb)
        assert c == v
    assert masks == 3                                       # three 8-byte masks
    allones = oracle.compress(np.frombuffer(mb, np.uint8)[None, :], m)
    assert ck_ints(allones) == [2**56 - 1]


# ------------------------------------------------------ Theorem 2
@pytest.mark.parametrize("seed", range(6))
def test_theorem2_compressed_order_equals_full_order(seed):
    rng = np.random.default_rng(20 + seed)
    W = int(rng.integers(1, 9))
    keys = random_structured_keys(rng, 400, W, int(rng.integers(1, min(8 * W, 30))))
    keys[rng.integers(0, 400, 50)] = keys[rng.integers(0, 400, 50)]     # duplicates
    keys = keys[rng.permutation(400)]
    perm_full = oracle.sort_rows(keys)
    D = oracle.dmask(keys, perm_full)
    for mask in (D, oracle.variant_mask(keys),
                 D | mask_of(rng.choice(8 * W, 5), 8 * W)):
        ck = oracle.compress(keys, mask)
        assert list(oracle.sort_compressed(ck)) == list(perm_full)


@pytest.mark.parametrize("K", [1, 2, 3, 4, 8])
def test_parallel_sort_matches_sort_compressed(K):
    """The all-cores comparison sort (GCC parallel-mode stable sort) orders
    compressed keys as the single-thread oracle sort does, ties by row id:
    many equal values and values that differ only in the low word; 50,000
    rows so that the parallel sort splits the input across threads."""
    rng = np.random.default_rng(K)
    n = 50_000
    ck = rng.integers(0, 4, (n, K), dtype=np.uint64).astype(np.uint32)   # few distinct values
    ck[: n // 3, 0] = rng.integers(0, 2**32, n // 3, dtype=np.uint64).astype(np.uint32)
    for threads in (1, 0):
        perm, used = oracle.sort_compressed_parallel(ck, threads)
        assert used >= 1
        assert list(perm) == list(oracle.sort_compressed(ck))
    with pytest.raises(ValueError):
        oracle.sort_compressed_parallel(np.zeros((4, 9), np.uint32))


def test_theorem2_needs_every_dbit():
    """Dropping any position of D breaks the order for some row arrangement."""
    g, vals = load_fig2()
    rows = ints_to_rows(vals, 12)
    D = positions_of(oracle.dmask(rows), 16)
    for drop in D:
        m = mask_of([p for p in D if p != drop], 16)
        broken = False
        for order in itertools.permutations(range(len(vals))):
            r = rows[list(order)]
            if list(oracle.sort_compressed(oracle.compress(r, m))) != list(oracle.sort_rows(r)):
                broken = True
                break
        assert broken


# --------------------------------------- Sec. 4.3 rebuild step 1 / D-offset
@pytest.mark.parametrize("seed", range(5))
def test_refine_from_superset_equals_full_key_D(seed):
    rng = np.random.default_rng(40 + seed)
    W = int(rng.integers(2, 10))
    keys = random_structured_keys(rng, 300, W, int(rng.integers(2, min(40, 8 * W))))
    keys = keys[rng.permutation(300)]
    perm = oracle.sort_rows(keys)
    D = oracle.dmask(keys, perm)
    for sup in (oracle.variant_mask(keys), D | mask_of(rng.choice(8 * W, 7), 8 * W), D):
        ck = oracle.compress(keys, sup)
        p2 = oracle.sort_compressed(ck)
        assert list(oracle.refine(ck, p2, sup, 8 * W)) == list(D)


# ------------------------------------------------------ Sec. 5.3 bulk load
def test_btree_shape_closed_form():
    for n in (1, 2, 63, 64, 65, 4096, 4097, 1_000_000, 10**7 + 3):
        for f in (2, 3, 14, 64, 256):
            lv = oracle.btree_shape(n, f)
            m, expect = n, [n]
            while m > f:
                m = math.ceil(m / f)
                expect.append(m)
            assert lv == expect
            if n > f:
                assert len(lv) == math.ceil(math.log(math.ceil(n / f), f) - 1e-12) + 1
    assert oracle.btree_shape(0, 64) == []
    assert oracle.btree_shape(10**6, 64) == [10**6, 15625, 245, 4]


@pytest.mark.parametrize("n,f", [(1, 4), (5, 4), (1000, 8), (4097, 64), (3000, 3)])
def test_btree_entries(n, f):
    rng = np.random.default_rng(n + f)
    v = (rng.integers(0, 2**20, n, dtype=np.uint64) << np.uint64(30)) | np.uint64(7)
    perm = oracle.sort_rows(v)
    t = oracle.btree(v, perm, f)
    sv = [int(v[i]) for i in perm]
    # leaves: D-bit against the previous key, closed form on integers
    assert [int(x) for x in t["leaf_dbit"]] == [0xFFFF] + [
        (lambda d: 0xFFFF if d < 0 else d)(dbit_py(sv[i - 1], sv[i], 64)) for i in range(1, n)]
    off = 0
    for l, m in enumerate(t["levels"][1:], start=1):
        hi = t["high"][off:off + m]
        assert list(t["child"][off:off + m]) == list(range(m))
        assert [int(h) for h in hi] == [min((e + 1) * f ** l, n) - 1 for e in range(m)]
        for e in range(m):
            d = int(t["dbit"][off + e])
            if e == 0:
                assert d == 0xFFFF
            else:   # Lemma 1: min of the leaf D-bits over the covered range
                rng_d = [int(x) for x in t["leaf_dbit"][int(hi[e - 1]) + 1:int(hi[e]) + 1]]
                assert d == min(rng_d)
        off += m


# ------------------------------------------------------ generators sanity
def test_generator_shapes():
    keys, pos = synth.varying_bits_u64(20000, 7)
    assert len(set(pos)) == 24
    D = positions_of(oracle.dmask(keys), 64)
    assert set(D) <= set(pos) and len(D) >= 20
    u = synth.urls(2000, 3)
    assert all(bytes(r).startswith(b"http://www.") for r in u)
    d = synth.dna(2000, 4)
    assert set(np.unique(d)) <= set(b"ACGT")
    # 0x41,0x43,0x47,0x54: only bit positions 3, 5, 6 of each byte can distinguish
    Dd = positions_of(oracle.dmask(d), 256)
    assert set(p % 8 for p in Dd) <= {3, 5, 6}


# ------------------------------------------------------ learned CDF model
def test_mlp_oracle_finite_differences():
    """fp64 gradient of the oracle against central differences (h = 1e-6)."""
    rng = np.random.default_rng(77)
    p = rng.normal(0, 1, oracle.MLP_PARAMS)
    x = rng.random(300)
    t = np.sort(rng.random(300))
    _, g = oracle.mlp_loss_grad(p, x, t)
    h = 1e-6
    for k in range(oracle.MLP_PARAMS):
        a, b = p.copy(), p.copy()
        a[k] += h
        b[k] -= h
        fd = (oracle.mlp_loss_grad(a, x, t)[0] - oracle.mlp_loss_grad(b, x, t)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])


def test_mlp_oracle_closed_forms():
    """Special cases with a closed form: all hidden units off leaves only b2,
    and a single active unit is a straight line."""
    x = np.linspace(0.0, 1.0, 11)
    t = x.copy()
    p = np.zeros(oracle.MLP_PARAMS)
    p[3 * 16] = 0.25                                   # y = 0.25 everywhere
    loss, g = oracle.mlp_loss_grad(p, x, t)
    assert loss == pytest.approx(np.mean((0.25 - x) ** 2))
    assert g[48] == pytest.approx(2 * np.mean(0.25 - x))
    assert np.all(g[:48] == 0)
    p = np.zeros(oracle.MLP_PARAMS)
    p[0], p[16], p[32] = 1.0, 0.5, 2.0                 # y = 2 * (x + 0.5)
    assert oracle.mlp_forward(p, 0.3) == pytest.approx(1.6)
    loss, g = oracle.mlp_loss_grad(p, x, t)
    r = 2 * (x + 0.5) - t
    assert loss == pytest.approx(np.mean(r ** 2))
    assert g[32] == pytest.approx(np.mean(2 * r * (x + 0.5)))
    assert g[0] == pytest.approx(np.mean(2 * r * 2.0 * x))
    assert g[16] == pytest.approx(np.mean(2 * r * 2.0))


# ------------------------------------------- Sec. 4.3 DS-metadata under inserts
def test_insert_rule_on_fig2_keys():
    """Sec. 3.2 / 4.3 on the Fig. 2 carrier keys: with key3 deleted, position 7
    is no distinction bit; inserting key3 back by the paper's rule (set the
    larger of D-bit(A, K) and D-bit(K, B)) restores D = {1, 2, 5, 7}, and the
    variant bitmap is unchanged (key3 was already counted)."""
    g, vals = load_fig2()
    rows = ints_to_rows(vals, g["key_bits"])
    r3 = np.delete(rows, 3, axis=0)
    d3, v3 = oracle.dmask(r3), oracle.variant_mask(r3)
    assert 7 not in positions_of(d3, 16)
    d, v = oracle.insert_batch(r3, oracle.sort_rows(r3), rows[3:4], 0, d3, v3)
    assert positions_of(d, 16) == g["stated"]["distinction_positions"]
    assert positions_of(v, 16) == g["stated"]["variant_positions"]


@pytest.mark.parametrize("seed", range(6))
def test_inserts_keep_the_d_bitmap_exact(seed):
    """Sec. 4.3: with inserts only, the maintained D-bitmap is the D-bitmap of
    the grown key set recomputed from scratch (Theorem 1 on the union) and the
    variant bitmap is that of the union against the same reference key; the
    result does not depend on the order of the inserts."""
    rng = np.random.default_rng(700 + seed)
    W = int(rng.integers(1, 6))
    n_old, n_new = int(rng.integers(1, 300)), int(rng.integers(0, 200))
    allk = random_structured_keys(rng, n_old + n_new, W, int(rng.integers(1, 8 * W)))
    old, new = allk[:n_old].copy(), allk[n_old:].copy()
    if len(new) and seed % 2:   # some inserts equal to existing keys, some at the ends
        new[: len(new) // 3] = old[rng.integers(0, len(old), len(new) // 3)]
        new[-1] = 0
    ref = int(rng.integers(0, len(old)))
    d0, v0 = oracle.dmask(old), oracle.variant_mask(old, ref)
    d, v = oracle.insert_batch(old, oracle.sort_rows(old), new, ref, d0, v0)
    union = np.concatenate([old, new]) if len(new) else old
    assert np.array_equal(d, oracle.dmask(union))
    assert np.array_equal(v, oracle.variant_mask(union, ref))
    shuffled = new[rng.permutation(len(new))]
    d2, v2 = oracle.insert_batch(old, oracle.sort_rows(old), shuffled, ref, d0, v0)
    assert np.array_equal(d2, d) and np.array_equal(v2, v)


def test_deletes_leave_a_valid_d_bitmap():
    """Sec. 4.3 (Delete): deletes leave the D-bitmap as it is; the stale bitmap
    is a superset of the remaining keys' D, so sorting their compressed keys
    still gives the full-key order (Theorem 2 with any superset of D)."""
    rng = np.random.default_rng(71)
    keys = random_structured_keys(rng, 400, 4, 14)
    d = oracle.dmask(keys)
    keep = np.sort(rng.choice(400, 150, replace=False))
    rest = keys[keep]
    dr = oracle.dmask(rest)
    assert np.all((dr & ~d) == 0)
    K = (oracle.popcount(d) + 31) // 32
    assert np.array_equal(oracle.sort_compressed(oracle.compress(rest, d, K)), oracle.sort_rows(rest))


# ------------------------------------------------ Sec. 4.1 numeric key formats
@pytest.mark.parametrize("dtype", [np.int32, np.int64, np.float32, np.float64])
def test_numeric_key_format_orders_like_the_numbers(dtype):
    """Sec. 4.1 ([LKN] mapping): comparing the encoded keys byte by byte sorts
    the values as numpy sorts the numbers (stable, ties by position)."""
    rng = np.random.default_rng(int(np.dtype(dtype).itemsize) * 10 + (dtype in (np.float32, np.float64)))
    if np.issubdtype(dtype, np.integer):
        info = np.iinfo(dtype)
        v = rng.integers(info.min, info.max, 5000, dtype=dtype, endpoint=True)
        v[:6] = [info.min, info.min + 1, -1, 0, 1, info.max]
    else:
        v = (rng.standard_normal(5000) * 10.0 ** rng.integers(-40, 38, 5000)).astype(dtype)
        v[:5] = [-np.inf, np.inf, np.finfo(dtype).tiny, -np.finfo(dtype).max, np.finfo(dtype).smallest_subnormal]
        v[v == 0] = 1          # -0.0 and +0.0 are equal numbers but distinct keys: pinned below
    v[100:200] = v[7]          # equal values keep their row order
    kb = oracle.as_key_bytes(v)
    assert kb.shape == (5000, np.dtype(dtype).itemsize)
    assert np.array_equal(oracle.sort_rows(kb), np.argsort(v, kind="stable"))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_float_key_format_chain(dtype):
    """The float format is a total order: -inf < ... < -0.0 < +0.0 < ... < +inf."""
    f = np.finfo(dtype)
    chain = np.array([-np.inf, -f.max, -1.0, -f.tiny, -f.smallest_subnormal, -0.0, 0.0, f.smallest_subnormal,
                      f.tiny, 1.0, f.max, np.inf], dtype=dtype)
    kb = oracle.as_key_bytes(chain)
    rows = [bytes(r) for r in kb]
    assert all(a < b for a, b in zip(rows, rows[1:]))


def test_multi_column_key_orders_like_tuples():
    """Sec. 4.1: a key of several columns (int, varchar(8), decimal with NULLs,
    float) concatenates the columns' index keys; comparing the keys byte by
    byte is Python's lexicographic comparison of the tuples (a varchar as its
    string, a NULL decimal before every value), ties by row.  The paper's
    varchar example: AB followed by NUL sorts before ABA followed by NUL."""
    rng = np.random.default_rng(81)
    n = 3000
    part_id = rng.integers(-50, 50, n).astype(np.int32)
    words = [b"", b"A", b"AB", b"ABA", b"ABB", b"B", b"BA", b"ZZZZZZZ"]
    names = [words[i] for i in rng.integers(0, len(words), n)]
    name_rows = np.zeros((n, 8), np.uint8)
    for r, w in enumerate(names):
        name_rows[r, :len(w)] = np.frombuffer(w, np.uint8)
    dec = rng.integers(-10**6, 10**6, n).astype(np.int64)
    dec[rng.integers(0, n, 200)] = 0
    nulls = rng.random(n) < 0.1
    flt = rng.standard_normal(n).astype(np.float64)
    flt[rng.integers(0, n, 300)] = 1.5
    kb = oracle.encode_key([("numeric", part_id, 4, None), ("bytes", name_rows, 8, None),
                            ("decimal", dec, 4, nulls), ("numeric", flt, 8, None)])
    assert kb.shape == (n, 24)

    def tup(r):
        return (int(part_id[r]), names[r], (0,) if nulls[r] else (1, int(dec[r])), float(flt[r]), r)

    assert list(oracle.sort_rows(kb)) == sorted(range(n), key=tup)
    ab = oracle.encode_key([("bytes", np.array([[65, 66, 0, 0], [65, 66, 65, 0]], np.uint8), 4, None)])
    assert bytes(ab[0]) < bytes(ab[1])


# ------------------------------------- Sec. 6.3 Zipf(s, n, m) synthetic datasets
@pytest.mark.parametrize("s,n,m", [(2.5, 16, 0), (1.5, 24, 3), (1.5, 40, 5)])
def test_zipf_letters_generator(s, n, m):
    """The Zipf(s, n, m) definition: in every 8-byte word the first m bytes
    are one fixed character (the same in every key), the others lowercase
    letters with the Zipf(s) frequencies over 26 letters (rank 1 = 'a')."""
    keys = synth.zipf_letters(200_000, synth.BASE_SEED + 9, n, m, s)
    assert keys.shape == (200_000, n)
    fixed = [p for p in range(n) if p % 8 < m]
    free = [p for p in range(n) if p % 8 >= m]
    for p in fixed:
        assert np.all(keys[:, p] == keys[0, p])
    letters = keys[:, free]
    assert letters.min() >= ord("a") and letters.max() <= ord("z")
    w = np.arange(1, 27, dtype=np.float64) ** -s
    expect = w / w.sum() * letters.size
    got = np.bincount(letters.ravel() - ord("a"), minlength=26)
    assert np.all(np.abs(got - expect) <= 6 * np.sqrt(expect) + 1)


def test_table4_sort_key_sizes_follow_the_formula():
    """Table 4's full sort key sizes and sort key ratios follow the Sec. 6.2
    formulas (key + 8-byte record id, in 8-byte words; full / compressed)."""
    from paper_2009_11543_gb300 import metrics as mt
    with open(os.path.join(GOLD, "table4_synthetic_stats.json")) as f:
        g = json.load(f)
    assert len(g["rows"]) == 20
    for r in g["rows"]:
        assert mt.full_sort_key_bytes(r["n"]) == r["full_sort_key_bytes"]
        assert round(mt.sort_key_ratio(r["full_sort_key_bytes"], r["compressed_sort_key_bytes"]), 2) == \
            r["sort_key_ratio"]


def test_table4_zipf_1_5_40_4_distinction_bits():
    """Zipf(1.5, 40, 4) at the paper's 10M keys: only the 20 letter bytes vary,
    five bits each ('a' to 'z'), so |D| <= 100; the oracle's |D| with the
    record id's 29 variant bits gives Table 4's 24-byte compressed sort key,
    and the 40 + 8 bytes of a full sort key give its sort key ratio of 2.00."""
    from paper_2009_11543_gb300 import metrics as mt
    keys = synth.zipf_letters(10_000_000, synth.BASE_SEED + 43, 40, 4, 1.5)
    nd = oracle.popcount(oracle.dmask(keys))
    assert 90 <= nd <= 100
    ck_bytes = mt.compressed_sort_key_bytes(nd, 29)
    assert ck_bytes == 24
    assert mt.sort_key_ratio(mt.full_sort_key_bytes(40), ck_bytes) == 2.0


# ------------------------------------------------ partial keys and search
def test_partial_key_of_fig2_key1():
    """Sec. 4.2: with pk = 4 the partial key of key_1 (offset D_1 = 5) is 1010;
    key_3 (offset D_3 = 7) takes positions 8..11 and key_0, with no offset,
    its first four bits."""
    g, vals = load_fig2()
    nb = g["key_bits"]
    rows = ints_to_rows(vals, nb)
    perm = oracle.sort_rows(rows)
    leaf, _ = oracle.partial_keys(rows, perm, oracle.btree(rows, perm, 4), 4)
    assert format(int(leaf[1]), "04b") == g["stated"]["partial_key_of_key1_pk4"]
    assert int(leaf[3]) == (vals[3] >> (nb - 12)) & 0xF
    assert int(leaf[0]) == vals[0] >> (nb - 4)


@pytest.mark.parametrize("W,n,nvary,f,pk", [(2, 300, 9, 3, 32), (5, 800, 20, 4, 7), (9, 500, 40, 5, 16)])
def test_partial_keys_against_big_integers(W, n, nvary, f, pk):
    """Every leaf and inner partial key equals the key, read as one big
    integer, shifted so that the pk bits after the offset come out (positions
    past the key's end are zeros); duplicates and short keys included."""
    rng = np.random.default_rng(W * 31 + pk)
    keys = random_structured_keys(rng, n, W, nvary)
    keys[rng.integers(0, n, n // 5)] = keys[rng.integers(0, n, n // 5)]
    perm = oracle.sort_rows(keys)
    t = oracle.btree(keys, perm, f)
    leaf, inner = oracle.partial_keys(keys, perm, t, pk)
    kbits = 8 * W

    def expect(row, off):
        start = 0 if off == oracle.NO_DBIT else off + 1
        v = row_int(keys[row]) << pk                   # pk zero bits appended past the end
        return (v >> (kbits + pk - start - pk)) & ((1 << pk) - 1)

    for i in range(n):
        assert int(leaf[i]) == expect(perm[i], int(t["leaf_dbit"][i]))
    assert len(inner) == len(t["high"]) > 0
    for g_, (h, off) in enumerate(zip(t["high"], t["dbit"])):
        assert int(inner[g_]) == expect(perm[int(h)], int(off))


def test_partial_key_mask_covers_every_partial_key():
    """Sec. 5.3 C a): with the extended mask, each bit a partial key reads is
    in the compressed key or invariant; the mask lies between D and D plus the
    variant positions; it still orders the keys (Theorem 2) and the D-offset
    refinement of its compressed keys gives D back."""
    rng = np.random.default_rng(77)
    W, pk = 6, 5
    keys = random_structured_keys(rng, 2000, W, 22)
    keys[rng.integers(0, 2000, 300)] = keys[rng.integers(0, 2000, 300)]
    kbits = 8 * W
    perm = oracle.sort_rows(keys)
    D = oracle.dmask(keys, perm)
    V = oracle.variant_mask(keys, 3)
    E = oracle.partial_key_mask(D, V, kbits, pk)
    ps = set(positions_of(E, kbits))
    assert set(positions_of(D, kbits)) <= ps <= set(positions_of(D, kbits)) | set(positions_of(V, kbits))
    t = oracle.btree(keys, perm, 8)
    var = set(positions_of(V, kbits))
    for off in list(t["leaf_dbit"]) + list(t["dbit"]):
        start = 0 if off == oracle.NO_DBIT else int(off) + 1
        for p in range(start, min(start + pk, kbits)):
            assert p in ps or p not in var
    ck = oracle.compress(keys, E)
    cperm = oracle.sort_compressed(ck)
    assert np.array_equal(cperm, perm)
    assert np.array_equal(oracle.refine(ck, cperm, E, kbits), D)


def test_search_against_linear_scan():
    """The search result (lower bound and the matching row id) against a
    linear count of smaller keys, for queries equal to keys, one bit away from
    keys, below the minimum and above the maximum."""
    rng = np.random.default_rng(8)
    W = 3
    keys = random_structured_keys(rng, 400, W, 12)
    keys[rng.integers(0, 400, 60)] = keys[rng.integers(0, 400, 60)]
    perm = oracle.sort_rows(keys)
    q = np.concatenate([keys[rng.integers(0, 400, 100)], keys[rng.integers(0, 400, 100)],
                        np.zeros((1, W), np.uint8), np.full((1, W), 255, np.uint8)])
    flip = rng.integers(0, 8 * W, 100)
    for j in range(100):
        q[100 + j, flip[j] // 8] ^= np.uint8(0x80 >> (flip[j] % 8))
    pos, rid = oracle.search(keys, perm, q)
    ints = [row_int(r) for r in keys]
    for j in range(len(q)):
        v = row_int(q[j])
        assert pos[j] == sum(1 for x in ints if x < v)
        eq = [r for r in range(len(ints)) if ints[r] == v]
        assert rid[j] == (min(eq) if eq else 0xFFFFFFFF)          # ties keep row id order
