"""Thin Python binding of libck (include/ck.h), argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: device buffers are torch CUDA tensors (uint32 data
is carried in int32 tensors and uint64 bitmaps in int64 tensors, bit for bit),
host bitmaps are numpy uint64 arrays.  There is no CPU fallback: if libck.so
is missing the import fails with an error that says how to build it.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libck.so")

CK_OK, CK_EINVAL, CK_ENOMEM, CK_ECUDA, CK_EOVERFLOW, CK_ETIMEOUT, CK_EVERIFY = range(7)
CK_KIND_BYTES, CK_KIND_U32, CK_KIND_U64, CK_KIND_I32, CK_KIND_I64, CK_KIND_F32, CK_KIND_F64 = 0, 1, 2, 3, 4, 5, 6
CK_KIND_DECIMAL = 7
CK_MAX_KEY_PARTS = 16
CK_MAX_ROWS = (1 << 30) - 1
CK_MAX_KEY_BYTES = 512
CK_NO_DBIT = 0xFFFF
CK_MAX_LEVELS = 32
CK_SORT_TILE = 4096
CK_SORT_TILES = (2048, 4096, 8192)
CK_INJECT_STALL_FIRST_TILE = 1
CK_SORT_PERM_ONLY = 1
CK_MAX_PARTIAL_KEY_BITS = 32
CK_NO_ROW = 0xFFFFFFFF

EXPORTED = ["ck_variant_bits", "ck_distinction_bits", "ck_extract", "ck_sort_workspace_bytes", "ck_sort",
            "ck_btree_plan", "ck_build_index", "ck_device_status", "ck_clear_device_status",
            "ck_status_string", "ck_launch_count", "ck_compress_word_host", "ck_compress_word_program_host",
            "ck_sort_static", "ck_build_index_keys",
            "ck_sort_learned_workspace_bytes", "ck_sort_learned", "ck_mlp_workspace_bytes", "ck_mlp_loss_grad",
            "ck_build_batched", "ck_graph_capture_batched", "ck_graph_launch", "ck_graph_destroy",
            "ck_autotune_sort", "ck_model_separators", "ck_insert_workspace_bytes", "ck_insert_batch", "ck_encode_key",
            "ck_partial_key_mask", "ck_partial_keys", "ck_search", "ck_extract_hist"]
CK_SORT_STATIC_SCRATCH_BYTES = 32 << 20
CK_LEARNED_STATS_BYTES = 64


class CkError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__("%s failed: %s" % (what, _lib().ck_status_string(status).decode()))
        self.status = status


class ck_column(ctypes.Structure):
    _fields_ = [("keys", ctypes.c_void_p), ("n", ctypes.c_uint64), ("key_bytes", ctypes.c_uint32),
                ("row_stride", ctypes.c_uint32), ("kind", ctypes.c_uint32)]


class ck_sort_opts(ctypes.Structure):
    _fields_ = [("digit_bits", ctypes.c_uint32), ("spin_limit", ctypes.c_uint32), ("inject", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("pass_events", ctypes.c_void_p), ("hist", ctypes.c_void_p),
                ("tile", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class ck_learned_opts(ctypes.Structure):
    _fields_ = [("bucket_bits", ctypes.c_uint32), ("sample_div", ctypes.c_uint32), ("epochs", ctypes.c_uint32),
                ("lr", ctypes.c_float), ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("phase_events", ctypes.c_void_p)]


class ck_learned_stats(ctypes.Structure):
    _fields_ = [("train_loss", ctypes.c_float), ("mean_search_steps", ctypes.c_float),
                ("max_search_steps", ctypes.c_uint32), ("buckets", ctypes.c_uint32),
                ("sample_size", ctypes.c_uint32), ("max_bucket", ctypes.c_uint32),
                ("sorted_segments", ctypes.c_uint32), ("constant_buckets", ctypes.c_uint32),
                ("oversize_buckets", ctypes.c_uint32), ("fell_back", ctypes.c_uint32),
                ("model_buckets", ctypes.c_uint32), ("model_boundaries", ctypes.c_uint32),
                ("model_boundary_frac", ctypes.c_float), ("heavy_keys", ctypes.c_uint32),
                ("capacity", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


class ck_btree_shape(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_uint32), ("entries_per_node", ctypes.c_uint32), ("n", ctypes.c_uint64),
                ("level_entries", ctypes.c_uint64 * CK_MAX_LEVELS), ("level_nodes", ctypes.c_uint64 * CK_MAX_LEVELS),
                ("inner_offset", ctypes.c_uint64 * CK_MAX_LEVELS), ("inner_entries", ctypes.c_uint64)]


class ck_btree(ctypes.Structure):
    _fields_ = [("shape", ck_btree_shape), ("leaf_rid", ctypes.c_void_p), ("leaf_dbit", ctypes.c_void_p),
                ("leaf_high", ctypes.c_void_p), ("inner_child", ctypes.c_void_p), ("inner_high", ctypes.c_void_p),
                ("inner_high_rid", ctypes.c_void_p), ("inner_high_ck", ctypes.c_void_p),
                ("inner_dbit", ctypes.c_void_p)]


class ck_index_job(ctypes.Structure):
    _fields_ = [("col", ck_column), ("dmask", ctypes.c_void_p), ("ck_words", ctypes.c_uint32),
                ("digit_bits", ctypes.c_uint32), ("tile", ctypes.c_uint32), ("fanout", ctypes.c_uint32),
                ("fill", ctypes.c_float),
                ("ck", ctypes.c_void_p), ("ck_sorted", ctypes.c_void_p), ("rid_sorted", ctypes.c_void_p),
                ("tree", ctypes.POINTER(ck_btree)), ("refined_mask", ctypes.c_void_p), ("ws", ctypes.c_void_p),
                ("ws_bytes", ctypes.c_size_t)]


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libck.so is not built (%s); run __graft_entry__.build() or "
                               "python -m paper_2009_11543_gb300.build" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        P, U64, U32, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        CP = ctypes.POINTER(ck_column)
        lib.ck_variant_bits.argtypes = [CP, U64, P, P]
        lib.ck_distinction_bits.argtypes = [CP, P, P, P]
        lib.ck_extract.argtypes = [CP, P, U32, P, P]
        lib.ck_extract_hist.argtypes = [CP, P, U32, P, U32, P, P]
        lib.ck_sort_workspace_bytes.argtypes = [U64, U32, U32, ctypes.POINTER(ck_sort_opts)]
        lib.ck_sort_workspace_bytes.restype = ctypes.c_size_t
        lib.ck_sort.argtypes = [P, P, P, P, U64, U32, U32, ctypes.POINTER(ck_sort_opts), P, ctypes.c_size_t, P]
        lib.ck_sort_static.argtypes = [P, P, P, P, U64, U32, U32, ctypes.POINTER(ck_sort_opts), P]
        lib.ck_btree_plan.argtypes = [U64, U32, ctypes.c_float, ctypes.POINTER(ck_btree_shape)]
        lib.ck_build_index.argtypes = [P, P, U64, U32, P, U32, U32, ctypes.c_float, ctypes.POINTER(ck_btree), P, P]
        lib.ck_build_index_keys.argtypes = [CP, P, P, U32, U32, ctypes.c_float, ctypes.POINTER(ck_btree), P, P]
        LO = ctypes.POINTER(ck_learned_opts)
        lib.ck_sort_learned_workspace_bytes.argtypes = [U64, U32, U32, LO]
        lib.ck_sort_learned_workspace_bytes.restype = ctypes.c_size_t
        lib.ck_sort_learned.argtypes = [P, P, P, U64, U32, U32, LO, P, P, P, ctypes.c_size_t, P]
        lib.ck_mlp_workspace_bytes.restype = ctypes.c_size_t
        lib.ck_mlp_loss_grad.argtypes = [P, P, P, U64, P, P, P, ctypes.c_size_t, P]
        JP = ctypes.POINTER(ck_index_job)
        lib.ck_build_batched.argtypes = [JP, U32, P]
        lib.ck_graph_capture_batched.argtypes = [JP, U32, ctypes.POINTER(ctypes.c_void_p)]
        lib.ck_graph_launch.argtypes = [P, P]
        lib.ck_graph_destroy.argtypes = [P]
        lib.ck_autotune_sort.argtypes = [P, P, P, U64, U32, U32, P, ctypes.c_size_t, U32, ctypes.c_char_p,
                                         ctypes.POINTER(U32), ctypes.POINTER(U32), ctypes.POINTER(ctypes.c_float), P]
        lib.ck_model_separators.argtypes = [P, ctypes.POINTER(ck_btree), U32, U32, P, P, P]
        lib.ck_encode_key.argtypes = [ctypes.POINTER(ck_key_part), U32, U64, P, U32, P]
        lib.ck_insert_workspace_bytes.argtypes = [U64, U32]
        lib.ck_insert_workspace_bytes.restype = ctypes.c_size_t
        lib.ck_insert_batch.argtypes = [CP, P, CP, U64, P, P, P, ctypes.c_size_t, P]
        lib.ck_partial_key_mask.argtypes = [P, P, U32, U32, P]
        lib.ck_partial_keys.argtypes = [ctypes.POINTER(ck_btree), P, U32, P, P, P, CP, U32, U32, P, P, P]
        lib.ck_search.argtypes = [ctypes.POINTER(ck_btree), CP, P, P, U32, CP, P, P, P, P]
        lib.ck_device_status.argtypes = [ctypes.POINTER(U64)]
        lib.ck_status_string.argtypes = [I]
        lib.ck_status_string.restype = ctypes.c_char_p
        lib.ck_launch_count.restype = U64
        lib.ck_compress_word_host.argtypes = [U32, U32]
        lib.ck_compress_word_host.restype = U32
        lib.ck_compress_word_program_host.argtypes = [U32, U32]
        lib.ck_compress_word_program_host.restype = U32
        for name in EXPORTED:
            if name not in ("ck_sort_workspace_bytes", "ck_status_string", "ck_launch_count",
                            "ck_compress_word_host", "ck_compress_word_program_host",
                            "ck_sort_learned_workspace_bytes", "ck_mlp_workspace_bytes"):
                getattr(lib, name).restype = I
        _LIB = lib
    return _LIB


def lib_path() -> str:
    return LIB_PATH


def _check(status: int, what: str) -> None:
    if status != CK_OK:
        raise CkError(status, what)


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return ctypes.c_void_p(t.ctypes.data)
    return ctypes.c_void_p(t.data_ptr())


class ck_key_part(ctypes.Structure):
    _fields_ = [("values", ctypes.c_void_p), ("nulls", ctypes.c_void_p), ("kind", ctypes.c_uint32),
                ("width", ctypes.c_uint32), ("stride", ctypes.c_uint32)]


def ck_encode_key(parts, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Index keys of several columns (ck_encode_key).  parts: a list of
    (tensor, kind, width) or (tensor, kind, width, nulls) on the device;
    byte parts are [n, width] uint8, numeric and decimal parts 1-D."""
    arr = (ck_key_part * len(parts))()
    n = None
    total = 0
    for i, part in enumerate(parts):
        t, kind, width = part[0], part[1], part[2]
        nulls = part[3] if len(part) > 3 else None
        rows = t.shape[0]
        n = rows if n is None else n
        if rows != n:
            raise ValueError("parts differ in row count")
        stride = t.stride(0) * t.element_size() if rows > 0 else max(width, t.element_size())
        arr[i] = ck_key_part(t.data_ptr(), nulls.data_ptr() if nulls is not None else None, kind, width, stride)
        total += width
    if out is None:
        out = torch.empty((n, total), dtype=torch.uint8, device=parts[0][0].device)
    _check(_lib().ck_encode_key(arr, len(parts), n, _ptr(out), out.stride(0) if n else total, _stream(stream)),
           "ck_encode_key")
    return out


def column(keys: torch.Tensor, kind: int | None = None) -> ck_column:
    """ck_column over a CUDA tensor: [n, W] uint8 rows (bytes), or a 1-D
    4-byte (uint32) / 8-byte (uint64) integer column."""
    if keys.dim() == 2:
        if keys.element_size() != 1:
            raise ValueError("2-D key columns must be uint8 rows")
        n, W = keys.shape
        stride = keys.stride(0) if n > 0 else W  # an empty column's strides carry no layout
        k = CK_KIND_BYTES if kind is None else kind
        if n > 0 and keys.stride(1) != 1:
            raise ValueError("key rows must be contiguous")
    elif keys.dim() == 1:
        n = keys.shape[0]
        W = keys.element_size()
        stride = W * keys.stride(0)
        if kind is not None:
            k = kind
        elif keys.dtype in (torch.float32, torch.float64):
            k = CK_KIND_F32 if W == 4 else CK_KIND_F64
        else:
            k = {4: CK_KIND_U32, 8: CK_KIND_U64}[W]   # integer tensors hold unsigned keys unless kind says so
    else:
        raise ValueError("keys must be 1-D or 2-D")
    return ck_column(keys.data_ptr(), n, W, stride, k)


def mask_words(key_bits: int) -> int:
    return (key_bits + 63) // 64


def CK_LD(n: int) -> int:
    """Leading dimension of word-major compressed key columns (include/ck.h)."""
    return (n + 63) & ~63


def ck_buffer(ck_words: int, n: int, device) -> torch.Tensor:
    """Device storage for a word-major compressed key column: [ck_words, CK_LD(n)]."""
    return torch.empty((ck_words, max(CK_LD(n), 64)), dtype=torch.int32, device=device)


def ck_variant_bits(keys: torch.Tensor, ref_row: int = 0, out: torch.Tensor | None = None, kind=None, stream=None):
    col = column(keys, kind)
    if out is None:
        out = torch.empty(mask_words(8 * col.key_bytes), dtype=torch.int64, device=keys.device)
    _check(_lib().ck_variant_bits(ctypes.byref(col), ref_row, _ptr(out), _stream(stream)), "ck_variant_bits")
    return out


def ck_distinction_bits(keys: torch.Tensor, order: torch.Tensor | None = None, out: torch.Tensor | None = None,
                        kind=None, stream=None):
    col = column(keys, kind)
    if out is None:
        out = torch.empty(mask_words(8 * col.key_bytes), dtype=torch.int64, device=keys.device)
    _check(_lib().ck_distinction_bits(ctypes.byref(col), _ptr(order), _ptr(out), _stream(stream)),
           "ck_distinction_bits")
    return out


def ck_insert_batch(keys: torch.Tensor, order: torch.Tensor, batch: torch.Tensor, ref_row: int,
                    dmask: torch.Tensor, vmask: torch.Tensor, kind=None, ws: torch.Tensor | None = None, stream=None):
    """Updates dmask and vmask (device, in place) for the rows of `batch`
    inserted into the index over `keys` whose sorted order is `order`."""
    col, bcol = column(keys, kind), column(batch, kind)
    need = _lib().ck_insert_workspace_bytes(bcol.n, bcol.key_bytes)
    if ws is None:
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device=keys.device)
    _check(_lib().ck_insert_batch(ctypes.byref(col), _ptr(order), ctypes.byref(bcol), ref_row, _ptr(dmask),
                                  _ptr(vmask), _ptr(ws), ws.numel(), _stream(stream)), "ck_insert_batch")
    return dmask, vmask


def popcount(mask: np.ndarray) -> int:
    return int(sum(bin(int(w)).count("1") for w in np.asarray(mask, np.uint64)))


def words_for(nbits: int) -> int:
    return max(1, (nbits + 31) // 32)


def ck_extract(keys: torch.Tensor, dmask: np.ndarray, ck_words: int | None = None, out: torch.Tensor | None = None,
               kind=None, stream=None):
    col = column(keys, kind)
    m = np.ascontiguousarray(np.asarray(dmask, np.uint64))
    if ck_words is None:
        ck_words = words_for(popcount(m))
    if out is None:
        out = ck_buffer(ck_words, col.n, keys.device)
    _check(_lib().ck_extract(ctypes.byref(col), _ptr(m), ck_words, _ptr(out), _stream(stream)), "ck_extract")
    return out


def ck_extract_hist(keys: torch.Tensor, dmask: np.ndarray, ck_words: int, digit_bits: int = 8,
                    out: torch.Tensor | None = None, hist: torch.Tensor | None = None, kind=None, stream=None):
    """Compressed keys and, in the same pass, their radix digit counts;
    returns (ck, hist) with hist [passes, 2^digit_bits] int32 (uint32 counts)."""
    col = column(keys, kind)
    m = np.ascontiguousarray(np.asarray(dmask, np.uint64))
    passes = (popcount(m) + digit_bits - 1) // digit_bits
    if out is None:
        out = ck_buffer(ck_words, col.n, keys.device)
    if hist is None:
        hist = torch.empty((max(passes, 1), 1 << digit_bits), dtype=torch.int32, device=keys.device)
    _check(_lib().ck_extract_hist(ctypes.byref(col), _ptr(m), ck_words, _ptr(out), digit_bits, _ptr(hist),
                                  _stream(stream)), "ck_extract_hist")
    return out, hist


def _opts(digit_bits=0, spin_limit=0, inject=0, pass_events=None, flags=0, hist=None, tile=0):
    return ck_sort_opts(digit_bits, spin_limit, inject, flags, pass_events,
                        hist.data_ptr() if hist is not None else None, tile, 0)


def event_handles(events) -> ctypes.Array:
    """cudaEvent_t array for the pass_events hook, from torch.cuda.Event objects."""
    arr = (ctypes.c_void_p * len(events))()
    for i, e in enumerate(events):
        arr[i] = e.cuda_event
    return arr


def ck_sort_workspace_bytes(n: int, ck_words: int, nbits: int, digit_bits: int = 0, tile: int = 0) -> int:
    o = _opts(digit_bits, tile=tile)
    return int(_lib().ck_sort_workspace_bytes(n, ck_words, nbits, ctypes.byref(o)))


def ck_sort(ck_in: torch.Tensor, rid_in: torch.Tensor | None, ck_out: torch.Tensor, rid_out: torch.Tensor, n: int,
            ck_words: int, nbits: int, ws: torch.Tensor, digit_bits: int = 0, spin_limit: int = 0, inject: int = 0,
            pass_events=None, perm_only: bool = False, hist: torch.Tensor | None = None, tile: int = 0,
            stream=None) -> None:
    o = _opts(digit_bits, spin_limit, inject,
              ctypes.cast(pass_events, ctypes.c_void_p) if pass_events is not None else None,
              CK_SORT_PERM_ONLY if perm_only else 0, hist, tile)
    _check(_lib().ck_sort(_ptr(ck_in), _ptr(rid_in), _ptr(ck_out), _ptr(rid_out), n, ck_words, nbits,
                          ctypes.byref(o), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)), "ck_sort")


def ck_sort_static(ck_in: torch.Tensor, rid_in: torch.Tensor | None, ck_out: torch.Tensor, rid_out: torch.Tensor,
                   n: int, ck_words: int, nbits: int, digit_bits: int = 0, perm_only: bool = False,
                   stream=None) -> None:
    """ck_sort without a caller workspace: the library's fixed scratch array is
    used instead (for callers that cannot allocate device memory; see ck.h)."""
    o = _opts(digit_bits, flags=CK_SORT_PERM_ONLY if perm_only else 0)
    _check(_lib().ck_sort_static(_ptr(ck_in), _ptr(rid_in), _ptr(ck_out), _ptr(rid_out), n, ck_words, nbits,
                                 ctypes.byref(o), _stream(stream)), "ck_sort_static")


def ck_btree_plan(n: int, fanout: int, fill: float = 1.0) -> ck_btree_shape:
    s = ck_btree_shape()
    _check(_lib().ck_btree_plan(n, fanout, fill, ctypes.byref(s)), "ck_btree_plan")
    return s


def alloc_btree(shape: ck_btree_shape, ck_words: int, device) -> dict:
    """Device arrays for a tree of the given shape (torch allocations)."""
    n = int(shape.n)
    ni = int(shape.inner_entries)
    nodes0 = int(shape.level_nodes[0]) if shape.levels else 0

    def e(sz, dt):
        return torch.empty(max(sz, 1), dtype=dt, device=device)
    return {"leaf_rid": e(n, torch.int32), "leaf_dbit": e(n, torch.int16), "leaf_high": e(nodes0, torch.int32),
            "inner_child": e(ni, torch.int32), "inner_high": e(ni, torch.int32), "inner_high_rid": e(ni, torch.int32),
            "inner_high_ck": e(ni * ck_words, torch.int32), "inner_dbit": e(ni, torch.int16)}


def ck_build_index(sorted_ck: torch.Tensor, sorted_rid: torch.Tensor, n: int, ck_words: int, dmask: np.ndarray,
                   key_bits: int, fanout: int, fill: float = 1.0, arrays: dict | None = None,
                   refined_out: torch.Tensor | None = None, stream=None):
    """Returns (shape, arrays); arrays are allocated when not given."""
    shape = ck_btree_plan(n, fanout, fill)
    if arrays is None:
        arrays = alloc_btree(shape, ck_words, sorted_rid.device if sorted_rid is not None else "cuda")
    t = ck_btree()
    for name, tensor in arrays.items():
        setattr(t, name, tensor.data_ptr())
    m = np.ascontiguousarray(np.asarray(dmask, np.uint64))
    _check(_lib().ck_build_index(_ptr(sorted_ck), _ptr(sorted_rid), n, ck_words, _ptr(m), key_bits, fanout, fill,
                                 ctypes.byref(t), _ptr(refined_out), _stream(stream)), "ck_build_index")
    return t.shape, arrays


def ck_build_index_keys(keys: torch.Tensor, sorted_rid: torch.Tensor, dmask: np.ndarray, ck_words: int, fanout: int,
                        fill: float = 1.0, arrays: dict | None = None, refined_out: torch.Tensor | None = None,
                        kind=None, stream=None):
    """Returns (shape, arrays); arrays are allocated when not given."""
    col = column(keys, kind)
    shape = ck_btree_plan(col.n, fanout, fill)
    if arrays is None:
        arrays = alloc_btree(shape, ck_words, keys.device)
    t = ck_btree()
    for name, tensor in arrays.items():
        setattr(t, name, tensor.data_ptr())
    m = np.ascontiguousarray(np.asarray(dmask, np.uint64))
    _check(_lib().ck_build_index_keys(ctypes.byref(col), _ptr(sorted_rid), _ptr(m), ck_words, fanout, fill,
                                      ctypes.byref(t), _ptr(refined_out), _stream(stream)), "ck_build_index_keys")
    return t.shape, arrays


CK_MLP_HIDDEN = 16
CK_MLP_PARAMS = 3 * CK_MLP_HIDDEN + 1
CK_LEARNED_NO_MODEL = 1
CK_LEARNED_INJECT_VERIFY_FAIL = 2
CK_LEARNED_INJECT_RID_SWAP = 4


CK_LEARNED_PHASES = 5


def learned_opts(bucket_bits=0, sample_div=0, epochs=0, lr=0.0, flags=0, phase_events=None) -> ck_learned_opts:
    """phase_events: None, or a ctypes array of CK_LEARNED_PHASES + 1 event handles (event_handles())."""
    return ck_learned_opts(bucket_bits, sample_div, epochs, lr, flags, 0,
                           ctypes.cast(phase_events, ctypes.c_void_p) if phase_events is not None else None)


def ck_sort_learned_workspace_bytes(n: int, ck_words: int, nbits: int, opts: ck_learned_opts | None = None) -> int:
    return int(_lib().ck_sort_learned_workspace_bytes(n, ck_words, nbits,
                                                      ctypes.byref(opts) if opts is not None else None))


def learned_stats_buffer(device) -> torch.Tensor:
    """Device buffer for one ck_learned_stats (read it with learned_stats())."""
    return torch.zeros(CK_LEARNED_STATS_BYTES // 4, dtype=torch.int32, device=device)


def learned_stats(buf: torch.Tensor) -> dict:
    """The ck_learned_stats a learned sort wrote into buf (synchronises with the copy)."""
    raw = buf.cpu().numpy().tobytes()
    return ck_learned_stats.from_buffer_copy(raw).as_dict()


def ck_sort_learned(ck_in: torch.Tensor, ck_out: torch.Tensor, rid_out: torch.Tensor, n: int, ck_words: int,
                    nbits: int, ws: torch.Tensor, opts: ck_learned_opts | None = None, stats: torch.Tensor | None = None,
                    params: torch.Tensor | None = None, stream=None) -> None:
    """Queues the learned sort (asynchronous; nothing is read back).  stats: a
    learned_stats_buffer() or None; params: a device float32 tensor of
    CK_MLP_PARAMS or None.  A fallback to the plain sort shows as CK_EVERIFY in
    ck_device_status()."""
    st = _lib().ck_sort_learned(_ptr(ck_in), _ptr(ck_out), _ptr(rid_out), n, ck_words, nbits,
                                ctypes.byref(opts) if opts is not None else None,
                                _ptr(stats) if stats is not None else None,
                                _ptr(params) if params is not None else None,
                                _ptr(ws), ws.numel() * ws.element_size(), _stream(stream))
    if st != CK_OK:
        raise CkError(st, "ck_sort_learned")


def ck_mlp_workspace_bytes() -> int:
    return int(_lib().ck_mlp_workspace_bytes())


def ck_mlp_loss_grad(params: torch.Tensor, x: torch.Tensor, t: torch.Tensor | None, ws: torch.Tensor,
                     stream=None):
    """Device fwd + bwd of the CDF model: returns (loss, grad) device tensors."""
    grad = torch.empty(CK_MLP_PARAMS, dtype=torch.float32, device=params.device)
    loss = torch.empty(1, dtype=torch.float32, device=params.device)
    _check(_lib().ck_mlp_loss_grad(_ptr(params), _ptr(x), _ptr(t), x.numel(), _ptr(grad), _ptr(loss), _ptr(ws),
                                   ws.numel() * ws.element_size(), _stream(stream)), "ck_mlp_loss_grad")
    return loss, grad


def ck_build_batched(jobs, stream=None) -> None:
    """jobs: a ctypes array of ck_index_job (see pipeline.BatchedRebuild)."""
    _check(_lib().ck_build_batched(jobs, len(jobs), _stream(stream)), "ck_build_batched")


def ck_graph_capture_batched(jobs):
    h = ctypes.c_void_p()
    _check(_lib().ck_graph_capture_batched(jobs, len(jobs), ctypes.byref(h)), "ck_graph_capture_batched")
    return h


def ck_graph_launch(graph, stream=None) -> None:
    _check(_lib().ck_graph_launch(graph, _stream(stream)), "ck_graph_launch")


def ck_graph_destroy(graph) -> None:
    _check(_lib().ck_graph_destroy(graph), "ck_graph_destroy")


def ck_autotune_sort(ck_in: torch.Tensor, ck_out: torch.Tensor, rid_out: torch.Tensor, n: int, ck_words: int,
                     nbits: int, ws: torch.Tensor, reps: int = 3, cache_path: str | None = None,
                     tune_tile: bool = True, stream=None):
    """Returns (best digit width, best tile, its median ms; 0.0 when read from
    the cache).  tune_tile=False keeps the default tile."""
    d = ctypes.c_uint32(0)
    t = ctypes.c_uint32(CK_SORT_TILE)
    ms = ctypes.c_float(0.0)
    _check(_lib().ck_autotune_sort(_ptr(ck_in), _ptr(ck_out), _ptr(rid_out), n, ck_words, nbits, _ptr(ws),
                                   ws.numel() * ws.element_size(), reps,
                                   cache_path.encode() if cache_path else None, ctypes.byref(d),
                                   ctypes.byref(t) if tune_tile else None, ctypes.byref(ms),
                                   _stream(stream)), "ck_autotune_sort")
    return int(d.value), int(t.value), float(ms.value)


def ck_model_separators(params: torch.Tensor, shape: ck_btree_shape, arrays: dict, ck_words: int, nbits: int,
                        stream=None):
    """Returns (proposals, hits) device tensors (see ck.h)."""
    t = ck_btree()
    t.shape = shape
    for name, tensor in arrays.items():
        setattr(t, name, tensor.data_ptr())
    ni = int(shape.inner_entries)
    prop = torch.empty(max(ni, 1), dtype=torch.int32, device=params.device)
    hits = torch.zeros(1, dtype=torch.int32, device=params.device)
    _check(_lib().ck_model_separators(_ptr(params), ctypes.byref(t), ck_words, nbits, _ptr(prop), _ptr(hits),
                                      _stream(stream)), "ck_model_separators")
    return prop, hits


def _tree(shape: ck_btree_shape, arrays: dict) -> ck_btree:
    t = ck_btree()
    t.shape = shape
    for name, tensor in arrays.items():
        setattr(t, name, tensor.data_ptr())
    return t


def ck_partial_key_mask(dmask: np.ndarray, vmask: np.ndarray, key_bits: int, pk: int) -> np.ndarray:
    """The extraction mask with the bits partial keys need (host only)."""
    d = np.ascontiguousarray(np.asarray(dmask, np.uint64))
    v = np.ascontiguousarray(np.asarray(vmask, np.uint64))
    out = np.zeros(mask_words(key_bits), np.uint64)
    _check(_lib().ck_partial_key_mask(_ptr(d), _ptr(v), key_bits, pk, _ptr(out)), "ck_partial_key_mask")
    return out


def reference_key(keys: torch.Tensor, ref_row: int, kind=None) -> np.ndarray:
    """Row ref_row of a key column in index-key byte order (through ck_encode_key)."""
    col = column(keys, kind)
    row = keys[ref_row:ref_row + 1]
    width = int(col.key_bytes)
    enc = ck_encode_key([(row, int(col.kind), width)])
    return enc.cpu().numpy().reshape(-1)[:width].copy()


def ck_partial_keys(shape: ck_btree_shape, arrays: dict, sorted_ck: torch.Tensor | None, ck_words: int,
                    emask: np.ndarray, vmask: np.ndarray, ref_key: np.ndarray, pk: int,
                    keys: torch.Tensor | None = None, key_bytes: int | None = None, kind=None,
                    leaf_pk: torch.Tensor | None = None, inner_pk: torch.Tensor | None = None, stream=None):
    """Partial keys of every leaf and inner entry; returns (leaf_pk, inner_pk)
    device int32 tensors (uint32 values)."""
    t = _tree(shape, arrays)
    col = column(keys, kind) if keys is not None else None
    W = int(col.key_bytes) if col is not None else int(key_bytes)
    dev = arrays["leaf_rid"].device
    n, ni = int(shape.n), int(shape.inner_entries)
    if leaf_pk is None:
        leaf_pk = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    if inner_pk is None:
        inner_pk = torch.empty(max(ni, 1), dtype=torch.int32, device=dev)
    e = np.ascontiguousarray(np.asarray(emask, np.uint64))
    v = np.ascontiguousarray(np.asarray(vmask, np.uint64))
    r = np.ascontiguousarray(np.asarray(ref_key, np.uint8))
    _check(_lib().ck_partial_keys(ctypes.byref(t), _ptr(sorted_ck), ck_words, _ptr(e), _ptr(v), _ptr(r),
                                  ctypes.byref(col) if col is not None else None, W, pk, _ptr(leaf_pk),
                                  _ptr(inner_pk), _stream(stream)), "ck_partial_keys")
    return leaf_pk, inner_pk


def ck_search(shape: ck_btree_shape, arrays: dict, keys: torch.Tensor, leaf_pk: torch.Tensor, pk: int,
              queries: torch.Tensor, kind=None, pos: torch.Tensor | None = None, rid: torch.Tensor | None = None,
              derefs: torch.Tensor | None = None, want_rid: bool = True, want_derefs: bool = False,
              inner_pk: torch.Tensor | None = None, stream=None):
    """Lower-bound search of every query row; returns (pos, rid, derefs)
    device int32 tensors (rid / derefs None unless wanted or given).  With
    inner_pk the inner nodes are scanned by partial keys too."""
    t = _tree(shape, arrays)
    col, qcol = column(keys, kind), column(queries, kind)
    q = int(qcol.n)
    dev = queries.device
    if pos is None:
        pos = torch.empty(max(q, 1), dtype=torch.int32, device=dev)
    if rid is None and want_rid:
        rid = torch.empty(max(q, 1), dtype=torch.int32, device=dev)
    if derefs is None and want_derefs:
        derefs = torch.empty(max(q, 1), dtype=torch.int32, device=dev)
    _check(_lib().ck_search(ctypes.byref(t), ctypes.byref(col), _ptr(leaf_pk), _ptr(inner_pk), pk,
                            ctypes.byref(qcol), _ptr(pos), _ptr(rid), _ptr(derefs), _stream(stream)), "ck_search")
    return pos, rid, derefs


def ck_device_status() -> tuple[int, int]:
    d = ctypes.c_uint64(0)
    s = _lib().ck_device_status(ctypes.byref(d))
    return int(s), int(d.value)


def ck_clear_device_status() -> None:
    _check(_lib().ck_clear_device_status(), "ck_clear_device_status")


def ck_status_string(status: int) -> str:
    return _lib().ck_status_string(status).decode()


def ck_launch_count() -> int:
    return int(_lib().ck_launch_count())


def ck_compress_word_host(x: int, mask: int) -> int:
    return int(_lib().ck_compress_word_host(x & 0xFFFFFFFF, mask & 0xFFFFFFFF))


def ck_compress_word_program_host(x: int, mask: int) -> int:
    return int(_lib().ck_compress_word_program_host(x & 0xFFFFFFFF, mask & 0xFFFFFFFF))


def mask_to_host(mask: torch.Tensor) -> np.ndarray:
    """Device bitmap (int64 storage) -> numpy uint64 words."""
    return mask.cpu().numpy().view(np.uint64)


def u32(t: torch.Tensor) -> np.ndarray:
    """Device uint32 data (int32 storage) -> numpy uint32."""
    return t.cpu().numpy().view(np.uint32)


def ck_rows(ck_dev: torch.Tensor, n: int) -> np.ndarray:
    """Word-major device column [K, CK_LD(n)] -> row-major numpy [n, K] uint32."""
    return np.ascontiguousarray(u32(ck_dev)[:, :n].T)
