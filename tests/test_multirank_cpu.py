"""The N > 1 host logic of bench.py on CPU with gloo, world size 2: the process-group
set-up, the barrier and the max-over-ranks reduction of the timing, and the reference arm,
whose rank 0 alone runs the oracle and prints one JSON line.  The path shards as independent
replicas (one problem per rank, seed = rank), so no data-path collective is involved."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "FMMPC_BENCH_BACKEND": "gloo"})
    sys.path.insert(0, ROOT)
    import bench
    w, r, _, pg = bench.dist_setup()
    assert (w, r) == (world, rank) and pg is not None
    bench.barrier(pg)
    v = bench.max_over_ranks(1.5 + rank, pg, "cpu")
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as fh:
        fh.write(repr(v))
    pg.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        assert float(open(tmp_path / f"rank{r}.txt").read()) == 2.5


def test_reference_arm_prints_one_line_from_rank_zero(tmp_path):
    pytest.importorskip("torch")
    env = dict(os.environ, FMMPC_BENCH_BACKEND="gloo", PYTHONPATH=ROOT)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "2",
           "--warmup", "1", "--side", "64", "--p", "8"]
    res = subprocess.run(cmd, cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["value"] > 0
    assert rec["e2e"]["h2d_bytes_per_step"] == 0
