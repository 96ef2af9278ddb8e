"""The N > 1 path of bench.py on CPU (gloo, world size 2).

The path shards by instance (each rank solves its own seeded instance, weak
scaling, no data exchange); the only collective is the max over ranks of the
step time, from which the whole-job throughput is computed.  Checked here
without a GPU: the max-over-ranks reduction over gloo, the per-rank seeds,
the job value, and the reference arm under torchrun (rank 0 alone prints one
JSON line, the other rank exits 0).
"""
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


def _rank_main(rank, ws, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(ws),
                       "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t = bench.max_over_ranks(1.0 + 1.5 * rank)
    res = {"rank": rank, "t": t, "seed": bench.rank_seed(7, rank),
           "env": bench.dist_env(),
           "value": bench.job_value(ws, 1000, t)}
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump(res, f)


def test_max_over_ranks_and_job_value_over_gloo(tmp_path):
    import torch.multiprocessing as mp
    ws, port = 2, _free_port()
    mp.spawn(_rank_main, args=(ws, port, str(tmp_path)), nprocs=ws,
             join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(ws)]
    for r, d in enumerate(res):
        assert d["t"] == 2.5                 # the slower rank's time, on both
        assert d["env"] == [ws, r, r]
        assert d["value"] == pytest.approx(2 * 1000 / 2.5e-3)
    assert res[0]["seed"] != res[1]["seed"]  # independent instances


def test_max_over_ranks_is_identity_without_a_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.job_value(1, 100, 2.0) == pytest.approx(5e4)


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
           "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
           "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--small", "--gpus", "2", "--steps", "1",
           "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    p = subprocess.run(cmd, capture_output=True, text=True, timeout=600,
                       cwd=ROOT, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
