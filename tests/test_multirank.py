"""The N > 1 path of bench.py on the CPU: replicas only (each rank rebuilds its
own copy; no data-path collective), so what multi-rank code there is -- the
maximum of the ranks' timings and rank 0 alone reporting -- runs here as two
gloo ranks on 127.0.0.1."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 3.5], world)
        np.save(os.path.join(out_dir, "max_%d.npy" % rank), got)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks(tmp_path):
    """Every rank ends with the element-wise maximum of the ranks' timings."""
    port = free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        assert np.load(tmp_path / ("max_%d.npy" % r)).tolist() == [2.0, 10.0, 3.5]


def test_max_over_ranks_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([4.0, 2.0], 1).tolist() == [4.0, 2.0]


def test_reference_arm_under_torchrun_prints_one_line():
    """`bench.py --impl reference` launched with two ranks: rank 0 times the
    oracle on a bounded sample and prints one JSON line; rank 1 does no work
    and exits 0."""
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--workload", "int1m", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"


def test_bench_roofline_inputs():
    """The bench's roofline inputs: the measured HBM peak from the committed
    peaks file, and each kernel's ncu traffic record scaled by n only while
    the kernel's source file still has the hash it was captured with."""
    sys.path.insert(0, ROOT)
    import bench
    peak, src = bench.peaks()
    have = os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json"))
    assert src == ("measured" if have else "fallback") and peak > 1000
    with open(bench.TRAFFIC_FILE) as f:
        recs = json.load(f)
    assert recs
    for kernel, rec in recs.items():
        t = bench.ncu_traffic(kernel, 2 * rec["n"], rec["ck_words"])
        if rec["kernel_src_sha"] == bench.file_sha(os.path.join(ROOT, rec["kernel_src"])):  # counters of this kernel
            assert t == 2 * rec["dram_bytes_per_launch"]
        else:                                                                        # changed since: no figure
            assert t is None
        assert bench.ncu_traffic(kernel, rec["n"], rec["ck_words"] + 1) is None
    assert bench.ncu_traffic("no_such_kernel", 1000, 1) is None
