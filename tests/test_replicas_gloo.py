"""The multi-process path (one process per GPU, independent solves) on the CPU with gloo.

RLOBPCG's solves do not exchange data, so the only collectives are the barrier around the timed
region and the max over ranks of the elapsed time; these tests run them with world_size 2 on
the CPU, and run the benchmark's reference arm under torchrun with two ranks (rank 0 alone
works and prints one line; rank 1 exits cleanly).
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    from paper_2602_16797_gb300 import replicas
    r, w, lr = replicas.world_from_env()
    replicas.init(w, "gloo")
    replicas.barrier(w)
    # rank r "took" (r + 1) * 1.5 ms: the job time is the slowest rank's
    t = replicas.max_over_ranks((r + 1) * 1.5, w)
    rate = replicas.job_rate(10, w, t * 1e-3)
    replicas.finish(w)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"rank": r, "world": w, "local_rank": lr, "t": t, "rate": rate}, f)


def test_max_over_ranks_and_job_rate_gloo(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert [x["rank"] for x in res] == [0, 1] and all(x["world"] == 2 for x in res)
    assert all(x["t"] == 3.0 for x in res)                 # max of 1.5 and 3.0
    assert all(abs(x["rate"] - 2 * 10 / 3e-3) < 1e-6 for x in res)


def test_single_process_is_a_no_op():
    from paper_2602_16797_gb300 import replicas
    replicas.init(1, "gloo")
    replicas.barrier(1)
    assert replicas.max_over_ranks(2.5, 1) == 2.5
    assert replicas.job_rate(4, 1, 2.0) == 2.0
    replicas.finish(1)


def test_reference_arm_under_torchrun_two_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 1 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
