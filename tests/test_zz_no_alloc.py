"""ck_sort_static: the sort for callers that cannot allocate device memory.

A host that owns all device memory through its own memory manager (a database
engine restoring its indexes after a restart, say) may forbid its components
to call cudaMalloc, and cudaMalloc / cudaFree can synchronise the device.
ck_sort_static takes the sort's scratch from a fixed array inside libck
instead of a caller workspace.  These checks call it through the C ABI twice in
a row, on different inputs, and require the same bits as ck_sort with a
workspace; the second call must not see anything left over from the first.
This file is collected last so that a run stopping at its first failure has
already run every other test; it also passes on its own in a fresh process,
where its first call performs the per-device set-up."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2009_11543_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2009_11543_gb300 import ck  # noqa: E402

DEV = "cuda:0"


def keys_on_device(rng, n, nbits):
    K = (nbits + 31) // 32
    rows = rng.integers(0, 2**32, (n, K), dtype=np.uint64).astype(np.uint32)
    top = nbits - 32 * (K - 1)
    if top < 32:
        rows[:, K - 1] &= np.uint32((1 << top) - 1)
    rows[rng.integers(0, n, n // 10)] = rows[rng.integers(0, n, n // 10)]   # equal keys keep row order
    buf = np.zeros((K, ck.CK_LD(n)), np.uint32)
    buf[:, :n] = rows.T
    return torch.from_numpy(buf.view(np.int32)).to(DEV), K


def sort_with_workspace(ck_in, n, K, nbits):
    ws = torch.empty(ck.ck_sort_workspace_bytes(n, K, nbits), dtype=torch.uint8, device=DEV)
    ck_out = torch.empty_like(ck_in)
    rid_out = torch.empty(n, dtype=torch.int32, device=DEV)
    ck.ck_sort(ck_in, None, ck_out, rid_out, n, K, nbits, ws)
    return ck_out, rid_out


def sort_static(ck_in, n, K, nbits):
    ck_out = torch.empty_like(ck_in)
    rid_out = torch.empty(n, dtype=torch.int32, device=DEV)
    ck.ck_sort_static(ck_in, None, ck_out, rid_out, n, K, nbits)
    return ck_out, rid_out


def test_static_scratch_matches_workspace_sort_twice():
    rng = np.random.default_rng(2024)
    for n, nbits in ((300_001, 121), (123_457, 45)):       # two calls in a row, different inputs
        ck_in, K = keys_on_device(rng, n, nbits)
        assert ck.ck_sort_workspace_bytes(n, K, nbits) <= ck.CK_SORT_STATIC_SCRATCH_BYTES
        ref_ck, ref_rid = sort_with_workspace(ck_in, n, K, nbits)
        got_ck, got_rid = sort_static(ck_in, n, K, nbits)
        torch.cuda.synchronize()
        assert torch.equal(got_rid, ref_rid)
        assert torch.equal(got_ck[:, :n], ref_ck[:, :n])
        assert ck.ck_device_status()[0] == ck.CK_OK


def test_static_scratch_rejects_oversized_sorts():
    n, K, nbits = 4_000_000, 4, 128
    assert ck.ck_sort_workspace_bytes(n, K, nbits) > ck.CK_SORT_STATIC_SCRATCH_BYTES
    dummy = torch.empty(16, dtype=torch.int32, device=DEV)   # never touched: rejected on the host
    with pytest.raises(ck.CkError) as e:
        ck.ck_sort_static(dummy, None, dummy, dummy, n, K, nbits)
    assert e.value.status == ck.CK_ENOMEM
