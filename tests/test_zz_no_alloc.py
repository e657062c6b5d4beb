"""ck_sort_static: the sort for callers that cannot allocate device memory.

A host that owns all device memory through its own memory manager (a database
engine restoring its indexes after a restart, say) may forbid its components
to call cudaMalloc, and cudaMalloc / cudaFree can synchronise the device.
ck_sort_static takes the sort's scratch from a fixed array inside libck
instead of a caller workspace.  These checks call it through the C ABI four
times in a row, on different inputs, digit widths and outputs, and require the
same bits as ck_sort with a workspace; no call may see anything left over from
the one before, and after the first call none allocates device memory.
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


def sort_with_workspace(ck_in, n, K, nbits, digit_bits=8, perm_only=False):
    ws = torch.empty(ck.ck_sort_workspace_bytes(n, K, nbits, digit_bits), dtype=torch.uint8, device=DEV)
    ck_out = torch.empty_like(ck_in)
    rid_out = torch.empty(n, dtype=torch.int32, device=DEV)
    ck.ck_sort(ck_in, None, ck_out, rid_out, n, K, nbits, ws, digit_bits=digit_bits, perm_only=perm_only)
    return ck_out, rid_out


# (n, nbits, digit bits, permutation only): the second call is smaller than
# the first, the third larger than the second with another digit width (so
# look-back words and histograms of a different layout are left over), the
# fourth returns only the permutation
CALLS = ((300_001, 121, 8, False), (123_457, 45, 8, False), (600_001, 90, 6, False), (250_007, 77, 11, True))


def test_static_scratch_matches_workspace_sort_in_a_row():
    """Four calls in a row on different inputs give the bits of ck_sort with a
    workspace; across every call after the first (which may load the array on
    the device) the free device memory does not change: nothing is allocated."""
    rng = np.random.default_rng(2024)
    cases = []
    for n, nbits, d, perm in CALLS:                   # inputs, references and outputs, allocated up front
        ck_in, K = keys_on_device(rng, n, nbits)
        assert ck.ck_sort_workspace_bytes(n, K, nbits, d) <= ck.CK_SORT_STATIC_SCRATCH_BYTES
        ref_ck, ref_rid = sort_with_workspace(ck_in, n, K, nbits, d, perm)
        cases.append((n, nbits, d, perm, K, ck_in, ref_ck, ref_rid, torch.empty_like(ck_in),
                      torch.empty(n, dtype=torch.int32, device=DEV)))
    torch.cuda.synchronize()
    for i, (n, nbits, d, perm, K, ck_in, ref_ck, ref_rid, got_ck, got_rid) in enumerate(cases):
        # free device memory right before and right after the call (torch's
        # own small allocations, e.g. for the comparisons below, fall outside)
        free_before = torch.cuda.mem_get_info()[0]
        ck.ck_sort_static(ck_in, None, got_ck, got_rid, n, K, nbits, digit_bits=d, perm_only=perm)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        if i > 0:
            assert free_after == free_before, (i, free_before, free_after)
        assert torch.equal(got_rid, ref_rid)
        if not perm:
            assert torch.equal(got_ck[:, :n], ref_ck[:, :n])
        assert ck.ck_device_status()[0] == ck.CK_OK


def test_static_scratch_limit_and_rejection():
    """The documented limit: 1,396,736 pairs of 128-bit keys fit the array,
    one more does not, and an oversized sort is rejected with CK_ENOMEM before
    anything is launched."""
    assert ck.ck_sort_workspace_bytes(1_396_736, 4, 128, 8) <= ck.CK_SORT_STATIC_SCRATCH_BYTES
    assert ck.ck_sort_workspace_bytes(1_396_737, 4, 128, 8) > ck.CK_SORT_STATIC_SCRATCH_BYTES
    n, K, nbits = 4_000_000, 4, 128
    dummy = torch.empty(16, dtype=torch.int32, device=DEV)   # never touched: rejected on the host
    with pytest.raises(ck.CkError) as e:
        ck.ck_sort_static(dummy, None, dummy, dummy, n, K, nbits)
    assert e.value.status == ck.CK_ENOMEM
