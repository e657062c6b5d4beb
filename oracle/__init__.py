"""Plain CPU oracle for the compressed key sort hot path (arXiv 2009.11543).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA path and never imports it.

Most of the arithmetic lives in ``ck_oracle.c`` (plain C, single thread),
which this module builds with gcc and calls on numpy arrays; the key formats,
partial keys, the partial-key mask and the search are written here in plain
numpy / Python.  Each function names the passage of the paper it follows:

* ``dbit``            -- Sec. 3.1, definition of the distinction bit position
* ``sort_rows``       -- Sec. 3.1, sorted (lexicographic) order; ties by row id
* ``dmask``           -- Theorem 1, D = {D_1..D_n} over adjacent sorted keys
* ``variant_mask``    -- Sec. 4.2 variant bitmap, computed as in Sec. 4.3
* ``compress``        -- Sec. 3.2, Compress(key), bit by bit
* ``sort_compressed`` -- Sec. 3.2, compressed key sort
* ``refine``          -- Sec. 4.3 rebuild step 1 with D-offset (Sec. 5.3)
* ``btree``           -- Sec. 4.2 / 5.3, bottom-up bulk load
* ``insert_batch``    -- Sec. 4.3 (Insert), the D-bitmap / variant bitmap rule
* ``encode_key``      -- Sec. 4.1 index key formats (numpy)
* ``partial_keys``    -- Sec. 4.2 partial keys (pk bits after the offset), numpy
* ``partial_key_mask``-- Sec. 5.3 option C a), the extraction mask extended by
                         the variant positions partial keys need, numpy
* ``search``          -- lower bound of each query in the sorted keys (Python
                         bisect): the result a search of Sec. 4.3 reaches
* ``mlp_loss_grad``   -- the learned CDF model (not in the paper), fp64 forward
                         and backward by the chain rule

Layout conventions are stated in the header of ``ck_oracle.c``: bitmaps are
uint64 words most-significant-first (position p = bit 63 - p%64 of word p/64),
compressed keys are row-major ``[n, K]`` uint32 words, least significant first.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ck_oracle.c")
_LIB = os.path.join(_HERE, "libck_oracle.so")
_PAR_SRC = os.path.join(_HERE, "ck_oracle_par.cpp")
_PAR_LIB = os.path.join(_HERE, "libck_oracle_par.so")
NO_DBIT = 0xFFFF
MAX_LEVELS = 64

_lib = None
_par_lib = None


def build(force: bool = False) -> str:
    """Compile ck_oracle.c with gcc into oracle/libck_oracle.so, and the
    all-cores comparison sort (ck_oracle_par.cpp, g++ with OpenMP) into
    oracle/libck_oracle_par.so."""
    for src, lib, cmd in ((_SRC, _LIB, ["gcc", "-O2", "-std=c11"]),
                          (_PAR_SRC, _PAR_LIB, ["g++", "-O2", "-std=c++17", "-fopenmp"])):
        if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
            tmp = lib + ".tmp%d" % os.getpid()
            subprocess.check_call(cmd + ["-shared", "-fPIC", "-o", tmp, src])
            os.replace(tmp, lib)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        U64, U32, I64 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64
        lib.cko_uint_to_bytes.argtypes = [P, U64, U32, P]
        lib.cko_encode_numeric.argtypes = [P, U64, U32, P]
        lib.cko_dbit.argtypes = [P, P, U32]
        lib.cko_dbit.restype = I64
        lib.cko_sort_rows.argtypes = [P, U64, U32, U32, P]
        lib.cko_dmask.argtypes = [P, U64, U32, U32, P, P]
        lib.cko_variant_mask.argtypes = [P, U64, U32, U32, P, P]
        lib.cko_compress.argtypes = [P, U64, U32, U32, P, U32, P]
        lib.cko_compress.restype = I64
        lib.cko_sort_compressed.argtypes = [P, U64, U32, P]
        lib.cko_refine.argtypes = [P, P, U64, U32, P, U32, P]
        lib.cko_btree_shape.argtypes = [U64, U32, P, U32]
        lib.cko_btree_shape.restype = U32
        lib.cko_btree_leaf_dbits.argtypes = [P, U64, U32, U32, P, P]
        lib.cko_btree_inner.argtypes = [P, U64, U32, U32, P, U32, U32, P, P, P, P]
        lib.cko_insert_batch.argtypes = [P, U64, U32, P, P, U64, P, P, P]
        lib.cko_mlp_forward.argtypes = [P, ctypes.c_double]
        lib.cko_mlp_forward.restype = ctypes.c_double
        lib.cko_mlp_loss_grad.argtypes = [P, P, P, U64, P]
        lib.cko_mlp_loss_grad.restype = ctypes.c_double
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


_NUMERIC_KIND = {np.dtype(np.uint32): 1, np.dtype(np.uint64): 2, np.dtype(np.int32): 3, np.dtype(np.int64): 4,
                 np.dtype(np.float32): 5, np.dtype(np.float64): 6}


def as_key_bytes(keys: np.ndarray) -> np.ndarray:
    """Sec. 4.1: numeric columns (unsigned, signed, float) become their
    binary-comparable big-endian index keys; a 2-D uint8 array of rows is used
    as given.  Returns a C-contiguous [n, W] uint8."""
    keys = np.asarray(keys)
    if keys.dtype == np.uint8 and keys.ndim == 2:
        return np.ascontiguousarray(keys)
    if keys.dtype in _NUMERIC_KIND and keys.ndim == 1:
        k = np.ascontiguousarray(keys)
        w = k.dtype.itemsize
        out = np.empty((k.shape[0], w), np.uint8)
        _load().cko_encode_numeric(_ptr(k), k.shape[0], _NUMERIC_KIND[k.dtype], _ptr(out))
        return out
    raise TypeError("keys must be [n, W] uint8 rows or a 1-D numeric column")


def encode_key(parts) -> np.ndarray:
    """Sec. 4.1 (Index Key Format): the index key of a row of several columns
    is the concatenation of the columns' index keys.  parts: a list of
    (kind, values, width, nulls) with kind "bytes" (a [n, width] uint8 array:
    fixed-size strings, or varchars zero-padded with their terminating NUL,
    used as they are), "numeric" (a 1-D numpy integer or float column, its
    Sec. 4.1 format) or "decimal" (int64 values scaled by 10^s, optional bool
    nulls; Sec. 4.1 A: header byte with bit 1 = not null and bit 0 = sign,
    then the magnitude in width - 1 big-endian bytes; the sign bit toggled and,
    for a negative value, every magnitude bit).  Returns [n, total width] uint8."""
    cols = []
    for kind, values, width, nulls in parts:
        if kind == "bytes":
            b = np.ascontiguousarray(values, np.uint8)
            assert b.shape[1] == width
            cols.append(b)
        elif kind == "numeric":
            cols.append(as_key_bytes(np.asarray(values)))
        elif kind == "decimal":
            v = np.asarray(values, np.int64)
            n = v.shape[0]
            null = np.zeros(n, bool) if nulls is None else np.asarray(nulls, bool)
            out = np.zeros((n, width), np.uint8)
            for r in range(n):
                x = 0 if null[r] else int(v[r])
                neg = x < 0
                header = (0 if null[r] else 2) | (1 if neg else 0)
                mag = -x if neg else x
                mb = width - 1
                assert mag < 256 ** mb
                if neg:
                    mag = (256 ** mb - 1) - mag          # every magnitude bit toggled
                out[r, 0] = header ^ 1                   # the sign bit toggled
                out[r, 1:] = np.frombuffer(mag.to_bytes(mb, "big"), np.uint8)
            cols.append(out)
        else:
            raise ValueError(kind)
    return np.ascontiguousarray(np.concatenate(cols, axis=1))


def mask_words(key_bits: int) -> int:
    return (key_bits + 63) // 64


def dbit(a: bytes, b: bytes) -> int:
    """Sec. 3.1: most significant differing bit position; -1 if equal."""
    assert len(a) == len(b)
    aa = np.frombuffer(bytes(a), np.uint8).copy()
    bb = np.frombuffer(bytes(b), np.uint8).copy()
    return int(_load().cko_dbit(_ptr(aa), _ptr(bb), len(a)))


def sort_rows(keys) -> np.ndarray:
    """Sorted order of the rows (lexicographic on the key bytes, ties by row id)."""
    kb = as_key_bytes(keys)
    n, W = kb.shape
    perm = np.empty(n, np.uint32)
    _load().cko_sort_rows(_ptr(kb), n, W, W, _ptr(perm))
    return perm


def dmask(keys, perm=None) -> np.ndarray:
    """Theorem 1: the D-bitmap of the keys from adjacent pairs in sorted order."""
    kb = as_key_bytes(keys)
    n, W = kb.shape
    if perm is None:
        perm = sort_rows(kb)
    perm = np.ascontiguousarray(perm, np.uint32)
    out = np.zeros(mask_words(8 * W), np.uint64)
    _load().cko_dmask(_ptr(kb), n, W, W, _ptr(perm), _ptr(out))
    return out


def variant_mask(keys, ref_row: int = 0) -> np.ndarray:
    """Sec. 4.2/4.3: OR over all keys of (key xor reference key)."""
    kb = as_key_bytes(keys)
    n, W = kb.shape
    out = np.zeros(mask_words(8 * W), np.uint64)
    if n == 0:
        return out
    ref = np.ascontiguousarray(kb[ref_row])
    _load().cko_variant_mask(_ptr(kb), n, W, W, _ptr(ref), _ptr(out))
    return out


def insert_batch(keys, perm, batch, ref_row: int, dmask_in: np.ndarray, vmask_in: np.ndarray):
    """Sec. 4.3 (Insert): the D-bitmap and variant bitmap after inserting the
    rows of `batch`, one by one in the given order, into the sorted keys
    (order `perm`); the reference key is row ref_row of `keys`."""
    kb = as_key_bytes(keys)
    bb = as_key_bytes(batch)
    n, W = kb.shape
    assert bb.shape[1] == W or bb.shape[0] == 0
    d = np.array(dmask_in, np.uint64, copy=True)
    v = np.array(vmask_in, np.uint64, copy=True)
    ref = np.ascontiguousarray(kb[ref_row])
    p = np.ascontiguousarray(perm, np.uint32)
    _load().cko_insert_batch(_ptr(kb), n, W, _ptr(p), _ptr(np.ascontiguousarray(bb)), bb.shape[0], _ptr(ref),
                             _ptr(d), _ptr(v))
    return d, v


def popcount(mask: np.ndarray) -> int:
    return int(sum(bin(int(w)).count("1") for w in np.asarray(mask, np.uint64)))


def compress(keys, mask: np.ndarray, K: int | None = None) -> np.ndarray:
    """Sec. 3.2: Compress(key) for every row -> [n, K] uint32, least significant word first."""
    kb = as_key_bytes(keys)
    n, W = kb.shape
    m = np.ascontiguousarray(mask, np.uint64)
    assert m.shape[0] == mask_words(8 * W)
    nbits = popcount(m)
    if K is None:
        K = max(1, (nbits + 31) // 32)
    out = np.zeros((n, K), np.uint32)
    r = _load().cko_compress(_ptr(kb), n, W, W, _ptr(m), K, _ptr(out))
    if r < 0:
        raise ValueError("mask has more set positions than %d words hold" % K)
    return out


def sort_compressed(ck: np.ndarray) -> np.ndarray:
    """Sec. 3.2: sort the rows by their compressed value (ties by row id)."""
    ck = np.ascontiguousarray(ck, np.uint32)
    n, K = ck.shape
    perm = np.empty(n, np.uint32)
    _load().cko_sort_compressed(_ptr(ck), n, K, _ptr(perm))
    return perm


def sort_compressed_parallel(ck: np.ndarray, threads: int = 0) -> tuple[np.ndarray, int]:
    """Sec. 3.2's sort of the rows by compressed value (ties by row id) with
    GCC's parallel-mode stable sort on `threads` host threads (0: every
    core), the multi-core CPU sort of the paper's evaluation (Sec. 6).
    Returns (perm, threads used)."""
    global _par_lib
    if _par_lib is None:
        build()
        lib = ctypes.CDLL(_PAR_LIB)
        lib.cko_par_sort_compressed.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                                ctypes.c_void_p, ctypes.c_int]
        lib.cko_par_sort_compressed.restype = ctypes.c_int
        _par_lib = lib
    ck = np.ascontiguousarray(ck, np.uint32)
    n, K = ck.shape
    perm = np.empty(n, np.uint32)
    t = _par_lib.cko_par_sort_compressed(_ptr(ck), n, K, _ptr(perm), int(threads))
    if t < 0:
        raise ValueError("compressed keys of %d words are not supported (1..8)" % K)
    return perm, t


def refine(ck: np.ndarray, perm: np.ndarray, old_mask: np.ndarray, key_bits: int) -> np.ndarray:
    """Sec. 4.3 step 1 + D-offset (Sec. 5.3): new D-bitmap from sorted compressed keys."""
    ck = np.ascontiguousarray(ck, np.uint32)
    n, K = ck.shape
    perm = np.ascontiguousarray(perm, np.uint32)
    om = np.ascontiguousarray(old_mask, np.uint64)
    out = np.zeros(mask_words(key_bits), np.uint64)
    _load().cko_refine(_ptr(ck), _ptr(perm), n, K, _ptr(om), key_bits, _ptr(out))
    return out


def btree_shape(n: int, f: int) -> list[int]:
    """Entries per level (level 0 = leaves) of the canonical bulk-loaded tree."""
    le = np.zeros(MAX_LEVELS, np.uint64)
    levels = _load().cko_btree_shape(n, f, _ptr(le), MAX_LEVELS)
    return [int(x) for x in le[:levels]]


def entries_per_node(fanout: int, fill: float) -> int:
    """Sec. 5.3: nodes are filled up to max fanout x fill factor."""
    return max(1, int(fanout * fill))


def btree(keys, perm: np.ndarray, f: int) -> dict:
    """Sec. 4.2 / 5.3 bottom-up bulk load over the sorted permutation.

    Returns ``levels`` (entries per level), ``leaf_dbit`` [n] and, for the inner
    levels concatenated (level 1 first), ``child``, ``high`` (sorted index of the
    highest key) and ``dbit`` (vs the previous entry's highest key)."""
    kb = as_key_bytes(keys)
    n, W = kb.shape
    perm = np.ascontiguousarray(perm, np.uint32)
    shape = btree_shape(n, f)
    le = np.array(shape + [0], np.uint64)
    lib = _load()
    leaf = np.empty(n, np.uint16)
    lib.cko_btree_leaf_dbits(_ptr(kb), n, W, W, _ptr(perm), _ptr(leaf))
    ninner = int(sum(shape[1:]))
    child = np.empty(max(ninner, 1), np.uint32)
    high = np.empty(max(ninner, 1), np.uint64)
    idbit = np.empty(max(ninner, 1), np.uint16)
    lib.cko_btree_inner(_ptr(kb), n, W, W, _ptr(perm), f, len(shape), _ptr(le),
                        _ptr(child), _ptr(high), _ptr(idbit))
    return {"levels": shape, "leaf_dbit": leaf, "child": child[:ninner],
            "high": high[:ninner], "dbit": idbit[:ninner]}


# ------------------------------------------------------------ learned model
MLP_HIDDEN = 16
MLP_PARAMS = 3 * MLP_HIDDEN + 1


def mlp_forward(params, x: float) -> float:
    """fp64 forward of the 1-16-1 ReLU CDF model (parameters [w1, b1, w2, b2])."""
    p = np.ascontiguousarray(params, np.float64)
    return float(_load().cko_mlp_forward(_ptr(p), float(x)))


def mlp_loss_grad(params, x, t):
    """fp64 mean squared error of the model on (x, t) and its gradient."""
    p = np.ascontiguousarray(params, np.float64)
    xs = np.ascontiguousarray(x, np.float64)
    ts = np.ascontiguousarray(t, np.float64)
    g = np.zeros(MLP_PARAMS, np.float64)
    loss = _load().cko_mlp_loss_grad(_ptr(p), _ptr(xs), _ptr(ts), len(xs), _ptr(g))
    return float(loss), g


# ------------------------------------------------------------- partial keys
def _bits_after(kb: np.ndarray, rows: np.ndarray, start: np.ndarray, pk: int) -> np.ndarray:
    """Bits [start, start + pk) of each key kb[rows] as a pk-bit integer (the
    first bit most significant); positions past the key read 0."""
    n, W = kb.shape
    padded = np.zeros((n, W + 5), np.uint8)
    padded[:, :W] = kb
    b = (start >> 3).astype(np.int64)
    window = np.zeros(len(rows), np.uint64)      # 40 bits from byte b on
    for j in range(5):
        window = (window << np.uint64(8)) | padded[rows, b + j].astype(np.uint64)
    shift = (40 - (start & 7) - pk).astype(np.uint64)
    return ((window >> shift) & np.uint64((1 << pk) - 1)).astype(np.uint32)


def partial_keys(keys, perm: np.ndarray, tree: dict, pk: int):
    """Sec. 4.2 (after [BMR]): the partial key of an entry is the pk bits of
    its key that follow its distinction bit position, the offset.  Leaf entry
    i holds sorted key i with offset D-bit(key_{i-1}, key_i); an inner entry
    holds its highest key with the offset against the previous entry's highest
    key.  An entry without an offset (the first of its level, or a key equal
    to the previous one) takes the key's first pk bits.  Returns (leaf [n],
    inner [inner entries]) as uint32, 1 <= pk <= 32."""
    assert 1 <= pk <= 32
    kb = as_key_bytes(keys)
    perm = np.asarray(perm, np.int64)

    def of(sorted_idx, offsets):
        o = np.asarray(offsets, np.int64)
        start = np.where(o == NO_DBIT, 0, o + 1)
        return _bits_after(kb, perm[np.asarray(sorted_idx, np.int64)], start, pk)

    n = kb.shape[0]
    leaf = of(np.arange(n), tree["leaf_dbit"]) if n else np.zeros(0, np.uint32)
    inner = of(tree["high"], tree["dbit"]) if len(tree["high"]) else np.zeros(0, np.uint32)
    return leaf, inner


def partial_key_mask(dmask: np.ndarray, vmask: np.ndarray, key_bits: int, pk: int) -> np.ndarray:
    """Sec. 5.3 C a): every position a partial key can read is either in the
    compressed key or invariant once the D-bitmap is extended by the variant
    positions among the pk positions after each D position, and among the
    first pk positions (entries without an offset)."""
    D = [p for p in range(key_bits) if (int(dmask[p // 64]) >> (63 - p % 64)) & 1]
    want = set(D)
    for start in [0] + [d + 1 for d in D]:
        for p in range(start, min(start + pk, key_bits)):
            if (int(vmask[p // 64]) >> (63 - p % 64)) & 1:
                want.add(p)
    out = np.zeros(mask_words(key_bits), np.uint64)
    for p in want:
        out[p // 64] |= np.uint64(1 << (63 - p % 64))
    return out


def search(keys, perm: np.ndarray, queries):
    """For each query: the first sorted position whose key is >= the query
    (n if none), and the row id there if that key equals the query, else
    0xFFFFFFFF.  Keys and queries compare as index-key bytes (Sec. 4.1)."""
    import bisect
    kb, qb = as_key_bytes(keys), as_key_bytes(queries)
    perm = np.asarray(perm, np.int64)
    srt = [kb[r].tobytes() for r in perm]
    pos = np.empty(qb.shape[0], np.uint32)
    rid = np.full(qb.shape[0], 0xFFFFFFFF, np.uint32)
    for j in range(qb.shape[0]):
        q = qb[j].tobytes()
        i = bisect.bisect_left(srt, q)
        pos[j] = i
        if i < len(srt) and srt[i] == q:
            rid[j] = perm[i]
    return pos, rid
