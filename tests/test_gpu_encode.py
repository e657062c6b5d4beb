"""Index keys from several columns (Sec. 4.1): ck_encode_key writes the
oracle's bytes exactly, and the rebuild of an index on the encoded keys sorts
the rows as the tuples of column values sort."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2009_11543_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2009_11543_gb300 import ck, pipeline  # noqa: E402

DEV = "cuda:0"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def table(n, seed):
    rng = np.random.default_rng(seed)
    a = rng.integers(-2**31, 2**31 - 1, n, endpoint=True).astype(np.int32)
    a[: n // 2] = a[0]
    s = rng.integers(0, 256, (n, 11), dtype=np.uint8)
    s[:, 5:] = 0
    s[rng.random(n) < 0.5, 2:] = 0
    d = rng.integers(-2**40, 2**40, n).astype(np.int64)
    d[rng.random(n) < 0.3] = 17
    nulls = (rng.random(n) < 0.05).astype(np.uint8)
    f = rng.standard_normal(n).astype(np.float32)
    f[:3] = np.array([-np.inf, np.inf, -0.0], np.float32)[:n]
    u = rng.integers(0, 2**62, n, dtype=np.uint64)
    return a, s, d, nulls, f, u


@pytest.mark.parametrize("n", [1, 777, 50_003])
def test_encode_matches_oracle_and_sorts_like_tuples(n):
    a, s, d, nulls, f, u = table(n, n)
    want = oracle.encode_key([("numeric", a, 4, None), ("bytes", s, 11, None), ("decimal", d, 7, nulls.astype(bool)),
                              ("numeric", f, 4, None), ("numeric", u, 8, None)])
    got = ck.ck_encode_key([(dev(a), ck.CK_KIND_I32, 4), (dev(s), ck.CK_KIND_BYTES, 11),
                            (dev(d), ck.CK_KIND_DECIMAL, 7, dev(nulls)), (dev(f), ck.CK_KIND_F32, 4),
                            (dev(u.view(np.int64)), ck.CK_KIND_U64, 8)])
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), want)
    assert ck.ck_device_status()[0] == ck.CK_OK
    # an index on the encoded keys: rebuilt on the GPU, ordered as the oracle orders the keys
    D = pipeline.first_build_dmask(got)
    r = pipeline.Rebuild(got, D, fanout=32)
    r.run()
    torch.cuda.synchronize()
    assert np.array_equal(ck.u32(r.rid_sorted)[:n], oracle.sort_rows(want))


def test_encode_decimal_overflow_and_errors():
    d = dev(np.array([5, -70000, 3], np.int64))
    ck.ck_clear_device_status()
    ck.ck_encode_key([(d, ck.CK_KIND_DECIMAL, 3)])           # |-70000| needs 3 magnitude bytes, 2 given
    assert ck.ck_device_status()[0] == ck.CK_EOVERFLOW
    ck.ck_clear_device_status()
    with pytest.raises(ck.CkError) as e:
        ck.ck_encode_key([(d, ck.CK_KIND_DECIMAL, 10)])       # width past 9
    assert e.value.status == ck.CK_EINVAL
    with pytest.raises(ck.CkError) as e:
        ck.ck_encode_key([(d, ck.CK_KIND_F32, 8)])            # a 4-byte kind with width 8
    assert e.value.status == ck.CK_EINVAL
