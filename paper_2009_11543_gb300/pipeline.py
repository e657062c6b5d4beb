"""Index reconstruction on the GPU (Sec. 5 of the paper): the four C-ABI calls
in order, with device buffers allocated once through torch.

``Rebuild`` is the rebuild with stored DS-metadata (the D-bitmap kept from the
previous build, Sec. 4.2): extract -> sort -> bulk load, the bulk load also
recomputing the D-bitmap (Sec. 4.3, step 1).  ``first_build_dmask`` derives
the D-bitmap when there is none yet: the variant bitmap is a superset of D
(every distinction position is variant), so extracting with it, sorting and
refining gives the exact D (Sec. 4.3 reads the first D from full keys; the
refined set is the same by Theorem 2 and the D-offset mapping of Sec. 5.3).

Python only marshals arguments; every step runs in libck's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ck


class DSMetadata:
    """The state an index keeps across restarts (Sec. 4.2): the D-bitmap, the
    variant bitmap and the reference key value.  The index itself is never
    persisted; after a restart it is rebuilt from the table with the stored
    D-bitmap (Sec. 4.3).  save() / load() use one numpy .npz file."""

    def __init__(self, dmask: np.ndarray, vmask: np.ndarray, ref_key: np.ndarray, key_bits: int):
        words = ck.mask_words(key_bits)
        self.dmask = np.ascontiguousarray(np.asarray(dmask, np.uint64))
        self.vmask = np.ascontiguousarray(np.asarray(vmask, np.uint64))
        self.ref_key = np.ascontiguousarray(np.asarray(ref_key, np.uint8))
        self.key_bits = int(key_bits)
        if self.dmask.shape != (words,) or self.vmask.shape != (words,) or self.ref_key.size * 8 != key_bits:
            raise ValueError("DS-metadata sizes do not match a key of %d bits" % key_bits)

    @classmethod
    def from_keys(cls, keys: torch.Tensor, ref_row: int = 0, kind: int | None = None) -> "DSMetadata":
        """First build: the exact D-bitmap, the variant bitmap and the reference key of a column."""
        col = ck.column(keys, kind)
        return cls(first_build_dmask(keys, kind=kind), ck.mask_to_host(ck.ck_variant_bits(keys, ref_row, kind=kind)),
                   ck.reference_key(keys, ref_row, kind=kind), 8 * int(col.key_bytes))

    def save(self, path: str) -> None:
        np.savez(path, dmask=self.dmask, vmask=self.vmask, ref_key=self.ref_key,
                 key_bits=np.array([self.key_bits], np.int64))

    @classmethod
    def load(cls, path: str) -> "DSMetadata":
        with np.load(path) as z:
            return cls(z["dmask"], z["vmask"], z["ref_key"], int(z["key_bits"][0]))


class Rebuild:
    """Buffers and launches for one key column and one D-bitmap.

    keys:   CUDA tensor, [n, W] uint8 rows or a 1-D uint32 / uint64 column.
    dmask:  host numpy uint64 bitmap over the key positions (the D-bitmap).
    """

    def __init__(self, keys: torch.Tensor, dmask: np.ndarray, fanout: int = 64, fill: float = 1.0,
                 digit_bits: int = 8, ck_words: int | None = None, kind: int | None = None, perm_only: bool = False,
                 learned: bool = False, learned_opts=None, tile: int = 0):
        self.keys = keys
        self.kind = kind
        self.col = ck.column(keys, kind)
        self.n = int(self.col.n)
        self.key_bits = 8 * int(self.col.key_bytes)
        self.dmask = np.ascontiguousarray(np.asarray(dmask, np.uint64))
        self.nbits = ck.popcount(self.dmask)
        self.K = ck_words or ck.words_for(self.nbits)
        self.fanout, self.fill, self.digit_bits, self.tile = fanout, fill, digit_bits, tile
        # perm_only: the sort returns only the permutation (and stops carrying
        # consumed key words); the tree is then built from the key column
        self.perm_only = perm_only
        # learned: the sort is the learned-partition sort (same output bits)
        self.learned = learned
        self.learned_opts = learned_opts
        self.hist = None                  # digit counts from the last extract (plain sort)
        dev = keys.device
        n = max(self.n, 1)
        self.ck_in = ck.ck_buffer(self.K, n, dev)
        self.ck_sorted = ck.ck_buffer(self.K, n, dev)
        self.rid_sorted = torch.empty(n, dtype=torch.int32, device=dev)
        wsb = ck.ck_sort_workspace_bytes(self.n, self.K, self.nbits, digit_bits, tile)
        if learned:
            wsb = max(wsb, ck.ck_sort_learned_workspace_bytes(self.n, self.K, self.nbits, learned_opts))
            self.stats_buf = ck.learned_stats_buffer(dev)
            self.params_buf = torch.zeros(ck.CK_MLP_PARAMS, dtype=torch.float32, device=dev)
        self.ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device=dev)
        self.shape = ck.ck_btree_plan(self.n, fanout, fill)
        self.tree = ck.alloc_btree(self.shape, self.K, dev)
        self.tree["leaf_rid"] = self.rid_sorted      # the sort writes the leaves' row ids in place
        self.refined = torch.empty(ck.mask_words(self.key_bits), dtype=torch.int64, device=dev)

    def extract(self, stream=None):
        if self.learned:
            ck.ck_extract(self.keys, self.dmask, self.K, out=self.ck_in, kind=self.kind, stream=stream)
            return
        # the plain sort's digit counts come out of the extraction pass
        passes = (self.nbits + self.digit_bits - 1) // self.digit_bits
        if getattr(self, "hist", None) is None or self.hist.shape != (max(passes, 1), 1 << self.digit_bits):
            self.hist = torch.empty((max(passes, 1), 1 << self.digit_bits), dtype=torch.int32,
                                    device=self.keys.device)
        ck.ck_extract_hist(self.keys, self.dmask, self.K, self.digit_bits, out=self.ck_in, hist=self.hist,
                           kind=self.kind, stream=stream)

    def sort(self, stream=None, pass_events=None):
        """pass_events: ctypes event handles recorded around every radix pass
        (plain sort) or at the CK_LEARNED_PHASES phase boundaries (learned sort)."""
        if self.learned:
            o = self.learned_opts
            if pass_events is not None:
                base = o or ck.learned_opts()
                o = ck.learned_opts(base.bucket_bits, base.sample_div, base.epochs, base.lr, base.flags,
                                    phase_events=pass_events)
            ck.ck_sort_learned(self.ck_in, self.ck_sorted, self.rid_sorted, self.n, self.K, self.nbits, self.ws,
                               o, stats=self.stats_buf, params=self.params_buf, stream=stream)
            return
        ck.ck_sort(self.ck_in, None, self.ck_sorted, self.rid_sorted, self.n, self.K, self.nbits, self.ws,
                   digit_bits=self.digit_bits, pass_events=pass_events, perm_only=self.perm_only, hist=self.hist,
                   tile=self.tile, stream=stream)

    def build(self, stream=None):
        if self.perm_only:
            ck.ck_build_index_keys(self.keys, self.rid_sorted, self.dmask, self.K, self.fanout, self.fill,
                                   arrays=self.tree, refined_out=self.refined, kind=self.kind, stream=stream)
        else:
            ck.ck_build_index(self.ck_sorted, self.rid_sorted, self.n, self.K, self.dmask, self.key_bits,
                              self.fanout, self.fill, arrays=self.tree, refined_out=self.refined, stream=stream)

    @property
    def learned_stats(self) -> dict:
        """Statistics of the last learned sort (reads them back: synchronises)."""
        return ck.learned_stats(self.stats_buf) if self.learned else None

    @property
    def learned_params(self):
        """The model the last learned sort trained, as numpy float32 (synchronises)."""
        no_model = self.learned_opts is not None and (self.learned_opts.flags & ck.CK_LEARNED_NO_MODEL)
        return None if not self.learned or no_model else self.params_buf.cpu().numpy()

    def separators(self, stream=None):
        """Model-proposed inner separators of the built tree (learned mode):
        returns (proposals, hit count); the tree itself is not changed."""
        if not self.learned:
            raise RuntimeError("no trained model: not a learned rebuild")
        prop, hits = ck.ck_model_separators(self.params_buf, self.shape, self.tree, self.K, self.nbits,
                                            stream=stream)
        return prop, hits

    def partial_keys(self, vmask: np.ndarray, ref_key: np.ndarray, pk: int, stream=None):
        """Partial keys of the built tree (Sec. 4.2): bits at positions of the
        extraction mask from the compressed keys, invariant ones from ref_key,
        any other from the key rows (Sec. 5.3 C b).  Kept for search()."""
        sorted_ck = None if self.perm_only else self.ck_sorted
        self.pk = pk
        self.leaf_pk, self.inner_pk = ck.ck_partial_keys(
            self.shape, self.tree, sorted_ck, self.K, self.dmask, vmask, ref_key, pk, keys=self.keys, kind=self.kind,
            leaf_pk=getattr(self, "leaf_pk", None), inner_pk=getattr(self, "inner_pk", None), stream=stream)
        return self.leaf_pk, self.inner_pk

    def search(self, queries: torch.Tensor, pos=None, rid=None, derefs=None, want_derefs: bool = False,
               inner_partial: bool = False, stream=None):
        """Lower-bound search of the query rows in the built tree (Sec. 4.3):
        full keys in the inner nodes, partial keys in the leaves;
        inner_partial=True scans the inner nodes by partial keys as well
        (same result; slower on wide nodes, where the binary search over full
        keys takes fewer dependent steps)."""
        return ck.ck_search(self.shape, self.tree, self.keys, self.leaf_pk, self.pk, queries, kind=self.kind,
                            pos=pos, rid=rid, derefs=derefs, want_derefs=want_derefs,
                            inner_pk=self.inner_pk if inner_partial and self.shape.inner_entries else None,
                            stream=stream)

    def run(self, stream=None):
        """One full rebuild: extract, sort, bulk load (+ refined D-bitmap)."""
        self.extract(stream)
        self.sort(stream)
        self.build(stream)

    def launches_per_run(self) -> int:
        passes = (self.nbits + self.digit_bits - 1) // self.digit_bits
        if passes == 0:
            return 1 + 1 + (2 if self.shape.inner_entries else 1)
        bins = 1 << self.digit_bits
        chunk = 65536 // (4 * bins)
        up = (passes + chunk - 1) // chunk
        btree = 1 + (1 if self.shape.inner_entries else 0)
        return 1 + up + 1 + passes + btree


def full_key_mask(key_bits: int) -> np.ndarray:
    """Bitmap with every key position set: Compress is then the key itself,
    and the same kernels sort the full keys (the full-key baseline)."""
    m = np.zeros(ck.mask_words(key_bits), np.uint64)
    for p in range(key_bits):
        m[p // 64] |= np.uint64(1 << (63 - p % 64))
    return m


def first_build_dmask(keys: torch.Tensor, kind: int | None = None, digit_bits: int = 8) -> np.ndarray:
    """D-bitmap of a column with no stored DS-metadata: variant bitmap ->
    extract -> sort -> refine (all on the GPU)."""
    variant = ck.mask_to_host(ck.ck_variant_bits(keys, 0, kind=kind))
    r = Rebuild(keys, variant, digit_bits=digit_bits, kind=kind)
    r.run()
    return ck.mask_to_host(r.refined)


class OverlappedRebuild:
    """Rebuilds of a stream of key batches of one shape and D-bitmap, with the
    copies hidden behind the kernels: while batch i is rebuilt on the compute
    stream, batch i + 1 travels host -> device on one copy stream and the
    sorted row ids of batch i - 1 travel device -> host on another.  Two
    Rebuild slots alternate; events order every reuse of a slot (its keys are
    overwritten only after its previous rebuild, its row ids only after they
    reached the host).  Extra keyword arguments go to Rebuild."""

    def __init__(self, shape, dtype, dmask: np.ndarray, device, **rebuild_kw):
        self.slots = [Rebuild(torch.empty(shape, dtype=dtype, device=device), dmask, **rebuild_kw) for _ in range(2)]
        self.h2d = torch.cuda.Stream(device)
        self.d2h = torch.cuda.Stream(device)
        self.copied = [torch.cuda.Event() for _ in range(2)]   # slot's keys are on the device
        self.built = [torch.cuda.Event() for _ in range(2)]    # slot's rebuild finished
        self.fetched = [torch.cuda.Event() for _ in range(2)]  # slot's row ids reached the host
        cur = torch.cuda.current_stream(device)
        for e in self.copied + self.built + self.fetched:
            e.record(cur)
        self.i = 0

    def begin(self, stream=None):
        """Orders the copy streams after the work queued so far on `stream`."""
        comp = stream or torch.cuda.current_stream()
        self.h2d.wait_stream(comp)
        self.d2h.wait_stream(comp)

    def submit(self, host_keys: torch.Tensor, host_rid: torch.Tensor, stream=None) -> Rebuild:
        """Queues one batch (pinned host keys in, sorted row ids out to pinned
        host_rid); asynchronous.  Returns the slot that rebuilds it."""
        s = self.i % 2
        r = self.slots[s]
        comp = stream or torch.cuda.current_stream()
        self.h2d.wait_event(self.built[s])
        with torch.cuda.stream(self.h2d):
            r.keys.copy_(host_keys, non_blocking=True)
            self.copied[s].record(self.h2d)
        comp.wait_event(self.copied[s])
        comp.wait_event(self.fetched[s])
        r.run(comp)
        self.built[s].record(comp)
        self.d2h.wait_event(self.built[s])
        with torch.cuda.stream(self.d2h):
            host_rid.copy_(r.rid_sorted[:r.n], non_blocking=True)
            self.fetched[s].record(self.d2h)
        self.i += 1
        return r

    def finish(self, stream=None):
        """Makes `stream` wait for every queued copy."""
        comp = stream or torch.cuda.current_stream()
        comp.wait_stream(self.h2d)
        comp.wait_stream(self.d2h)


class BatchedRebuild:
    """All the indexes of one table rebuilt together (one Rebuild per column,
    concurrently through ck_build_batched, optionally as one CUDA graph).

    columns: list of CUDA key columns (same row count); dmasks: their stored
    D-bitmaps; digit_bits: per column, or None to run the autotuner on each
    column's own keys (ck_autotune_sort over digit width and pass tile, cached
    in cache_path); tiles: per column when digit_bits is given (default tile
    otherwise)."""

    def __init__(self, columns, dmasks, fanouts, fill: float = 1.0, digit_bits=None, cache_path: str | None = None,
                 tune_reps: int = 3, tiles=None, tune_tile: bool = True):
        import ctypes
        self.parts = [Rebuild(c, m, fanout=f, fill=fill, digit_bits=8) for c, m, f in zip(columns, dmasks, fanouts)]
        self.tuned_ms = []
        for k, r in enumerate(self.parts):
            if digit_bits is not None:
                r.digit_bits = int(digit_bits[k])
                r.tile = int(tiles[k]) if tiles is not None else 0
            else:
                r.extract()
                wsb = max(ck.ck_sort_workspace_bytes(r.n, r.K, r.nbits, d, t)
                          for d in range(4, 12) for t in ck.CK_SORT_TILES)
                if wsb > r.ws.numel():
                    r.ws = torch.empty(wsb, dtype=torch.uint8, device=r.keys.device)
                r.digit_bits, r.tile, ms = ck.ck_autotune_sort(r.ck_in, r.ck_sorted, r.rid_sorted, r.n, r.K, r.nbits,
                                                               r.ws, tune_reps, cache_path, tune_tile=tune_tile)
                self.tuned_ms.append(ms)
            # the sort's workspace, then room for the digit counts taken while extracting
            need = (ck.ck_sort_workspace_bytes(r.n, r.K, r.nbits, r.digit_bits, r.tile) + 255) // 256 * 256
            need += 4 * ((r.nbits + r.digit_bits - 1) // r.digit_bits << r.digit_bits)
            if need > r.ws.numel():
                r.ws = torch.empty(need, dtype=torch.uint8, device=r.keys.device)
        self._trees = []
        self.jobs = (ck.ck_index_job * len(self.parts))()
        for k, r in enumerate(self.parts):
            t = ck.ck_btree()
            for name, tensor in r.tree.items():
                setattr(t, name, tensor.data_ptr())
            self._trees.append(t)
            j = self.jobs[k]
            j.col = r.col
            j.dmask = r.dmask.ctypes.data
            j.ck_words, j.digit_bits, j.tile, j.fanout, j.fill = r.K, r.digit_bits, r.tile, r.fanout, r.fill
            j.ck, j.ck_sorted, j.rid_sorted = r.ck_in.data_ptr(), r.ck_sorted.data_ptr(), r.rid_sorted.data_ptr()
            j.tree = ctypes.pointer(t)
            j.refined_mask = r.refined.data_ptr()
            j.ws, j.ws_bytes = r.ws.data_ptr(), r.ws.numel()
        self.graph = None

    def run(self, stream=None):
        """One batched rebuild, the jobs on concurrent internal streams."""
        ck.ck_build_batched(self.jobs, stream)

    def capture(self):
        """Captures one batched rebuild as a CUDA graph (replayed by launch())."""
        if self.graph is None:
            self.graph = ck.ck_graph_capture_batched(self.jobs)
        return self.graph

    def launch(self, stream=None):
        ck.ck_graph_launch(self.capture(), stream)

    def run_sequential(self, stream=None):
        """The same rebuilds one after another on one stream (the unbatched path)."""
        for r in self.parts:
            r.run(stream)

    def close(self):
        if self.graph is not None:
            ck.ck_graph_destroy(self.graph)
            self.graph = None
