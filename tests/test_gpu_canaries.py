"""Guard bands around every output: each call writes its outputs into the
middle of a larger buffer whose ends (and, for row outputs with a stride,
the gaps between rows) hold a sentinel; afterwards the sentinels must be
intact.  Sizes are ragged (several sort tiles plus a tail) so that the last
tile, the last node and the last word of every array are exercised."""
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
G = 4096            # guard words on each side
SENT = 0x5A5AA5A5  # sentinel word (a positive int32)


class Guarded:
    """A 1-D int32 device buffer with G sentinel words on both sides."""

    def __init__(self, words: int):
        self.words = words
        self.flat = torch.full((words + 2 * G,), SENT, dtype=torch.int32, device=DEV)
        self.mid = self.flat[G:G + words]

    def intact(self) -> bool:
        torch.cuda.synchronize()
        return bool((self.flat[:G] == SENT).all()) and bool((self.flat[G + self.words:] == SENT).all())


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


N = 3 * ck.CK_SORT_TILE + 123


def test_pipeline_outputs_stay_in_bounds():
    keys = synth.urls(N, synth.BASE_SEED + 77)
    kd = to_dev(keys)
    D = oracle.dmask(keys)
    nbits = oracle.popcount(D)
    K = ck.words_for(nbits)
    ld = ck.CK_LD(N)
    # extraction with the sort's digit counts
    ckg, hg = Guarded(K * ld), Guarded(((nbits + 7) // 8) * 256)
    ck.ck_extract_hist(kd, D, K, 8, out=ckg.mid.view(K, ld), hist=hg.mid.view(-1, 256))
    assert ckg.intact() and hg.intact()
    # sort (workspace guarded too)
    outg, ridg = Guarded(K * ld), Guarded(N)
    wsb = ck.ck_sort_workspace_bytes(N, K, nbits)
    wsg = Guarded((wsb + 255) // 4 + 64)
    ws = wsg.mid.view(torch.uint8)
    off = (-ws.data_ptr()) % 256          # the workspace must start 256-byte aligned
    ck.ck_sort(ckg.mid.view(K, ld), None, outg.mid.view(K, ld), ridg.mid, N, K, nbits, ws[off:off + wsb],
               hist=hg.mid.view(-1, 256))
    assert outg.intact() and ridg.intact() and wsg.intact()
    assert np.array_equal(ck.u32(ridg.mid)[:N], oracle.sort_rows(keys))
    # bulk load
    shape = ck.ck_btree_plan(N, 64)
    plain = ck.alloc_btree(shape, K, DEV)
    guards = {name: Guarded(t.numel() * t.element_size() // 4 + 1) for name, t in plain.items()}
    arrays = {name: g.mid.view(torch.uint8)[:plain[name].numel() * plain[name].element_size()].view(plain[name].dtype)
              for name, g in guards.items()}
    refg = Guarded(2 * ck.mask_words(8 * keys.shape[1]))
    ck.ck_build_index(outg.mid.view(K, ld), ridg.mid, N, K, D, 8 * keys.shape[1], 64, arrays=arrays,
                      refined_out=refg.mid.view(torch.int64))
    assert all(g.intact() for g in guards.values()) and refg.intact()
    assert np.array_equal(ck.mask_to_host(refg.mid.view(torch.int64)), D)
    # partial keys and search
    V = oracle.variant_mask(keys, 0)
    lpk, ipk = Guarded(N), Guarded(max(int(shape.inner_entries), 1))
    ck.ck_partial_keys(shape, arrays, outg.mid.view(K, ld), K, D, V, keys[0], 16, keys=kd, leaf_pk=lpk.mid,
                       inner_pk=ipk.mid)
    assert lpk.intact() and ipk.intact()
    q = np.concatenate([keys[::7], np.full((5, keys.shape[1]), 255, np.uint8)])
    pos, rid, der = Guarded(len(q)), Guarded(len(q)), Guarded(len(q))
    for inner in (None, ipk.mid):
        ck.ck_search(shape, arrays, kd, lpk.mid, 16, to_dev(q), pos=pos.mid, rid=rid.mid, derefs=der.mid,
                     inner_pk=inner)
        assert pos.intact() and rid.intact() and der.intact()
    assert ck.ck_device_status()[0] == ck.CK_OK


def test_insert_and_encode_stay_in_bounds():
    rng = np.random.default_rng(3)
    keys = synth.urls(N, synth.BASE_SEED + 78)
    kd = to_dev(keys)
    perm = oracle.sort_rows(keys)
    W = keys.shape[1]
    mw = ck.mask_words(8 * W)
    dg, vg = Guarded(2 * mw), Guarded(2 * mw)
    dg.mid.view(torch.int64).copy_(to_dev(oracle.dmask(keys).view(np.int64)))
    vg.mid.view(torch.int64).copy_(to_dev(oracle.variant_mask(keys, 0).view(np.int64)))
    new = synth.urls(5000, synth.BASE_SEED + 79)
    ck.ck_insert_batch(kd, to_dev(perm.view(np.int32)), to_dev(new), 0, dg.mid.view(torch.int64),
                       vg.mid.view(torch.int64))
    assert dg.intact() and vg.intact()
    # two columns into rows of a wider stride: the gaps between rows stay untouched
    n = 10_001
    a = rng.integers(-2**31, 2**31, n).astype(np.int32)
    b = rng.integers(0, 256, (n, 5), dtype=np.uint8)
    stride = 16                                   # 4 + 5 key bytes, 7 bytes of gap per row
    og = Guarded((n * stride + 3) // 4)
    out = og.mid.view(torch.uint8)[:n * stride].view(n, stride)
    ck.ck_encode_key([(to_dev(a), ck.CK_KIND_I32, 4), (to_dev(b), ck.CK_KIND_BYTES, 5)], out=out[:, :9])
    assert og.intact()
    torch.cuda.synchronize()
    gaps = out[:, 9:].cpu().numpy()
    assert np.all(gaps == np.frombuffer(np.array([SENT], np.int32).tobytes(), np.uint8)[(np.arange(9, 16) % 4)])
    assert ck.ck_device_status()[0] == ck.CK_OK
