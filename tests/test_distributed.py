"""Multi-rank logic of bench.py on CPU with the gloo backend (world size 2):
the max-over-ranks timing, whole-job aggregation, and the reference arm's
rank rule (only rank 0 runs and prints)."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    local_ms = [3.0, 5.0][rank]          # rank 1 is the slower one
    dist.barrier()
    m = bench.max_over_ranks(local_ms, dist, "cpu")
    gbs = bench.aggregate_gbs(432 * 1000, ws, m)
    with open(os.path.join(out, "r%d.json" % rank), "w") as f:
        json.dump({"max": m, "gbs": gbs}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_aggregate(tmp_path):
    ws = 2
    mp.spawn(_worker, args=(ws, free_port(), str(tmp_path)), nprocs=ws, join=True)
    res = [json.load(open(tmp_path / ("r%d.json" % r))) for r in range(ws)]
    for r in res:
        assert r["max"] == 5.0
        assert r["gbs"] == pytest.approx(432 * 1000 * 2 / 5e-3 / 1e9)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, None, "cpu") == 2.5
    assert bench.aggregate_gbs(1e9, 1, 1000.0) == pytest.approx(1.0)


def test_reference_arm_nonzero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_e2e_host_memory_guard():
    """Each rank pins its own end-to-end host buffers (~23 GB at 48^4); the
    bench reports the shortage instead of failing when the node cannot hold
    every rank's buffers."""
    sys.path.insert(0, ROOT)
    import bench
    per_rank = bench.e2e_host_bytes((48, 48, 48, 48))
    assert 20e9 < per_rank < 26e9
    assert bench.e2e_host_shortage((48, 48, 48, 48), 1, 209e9) is None
    assert bench.e2e_host_shortage((48, 48, 48, 48), 8, None) is None
    msg = bench.e2e_host_shortage((48, 48, 48, 48), 8, 150e9)
    assert msg.startswith("host memory: 8 ranks")
