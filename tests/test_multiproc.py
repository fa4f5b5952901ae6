"""The multi-process host path of bench.py on CPU (gloo, world size 2).

The bench's own bookkeeping between ranks: the barrier around the timed
region, the maximum of the per-rank times, and one JSON line printed by rank 0
(the data exchange of the sharded fit is tested in test_sharded_cpu.py and, on
a GPU, in test_gpu_sharded.py).  These tests run that logic as two gloo ranks
on 127.0.0.1, without a GPU.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench

    w, r, _ = bench.dist_init()
    assert (w, r) == (world, rank)
    bench.barrier(w)
    m = bench.allmax(w, 1.5 + rank)  # rank-dependent "times"
    bench.barrier(w)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as fh:
        fh.write(repr(m))
    dist.destroy_process_group()


@pytest.mark.skipif(torch.cuda.is_available(), reason="with CUDA the bench's ranks use NCCL, one GPU each")
def test_allmax_and_barrier_over_two_gloo_ranks(tmp_path):
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    vals = [float((tmp_path / f"rank{r}.txt").read_text()) for r in range(2)]
    assert vals == [2.5, 2.5]  # every rank sees the slowest rank's time


def test_single_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.allmax(1, 3.25) == 3.25
    bench.barrier(1)  # no-op


@pytest.mark.skipif(torch.cuda.is_available(), reason="the CPU launch of the reference arm")
def test_reference_arm_two_ranks_prints_one_line_from_rank_0():
    env = dict(os.environ)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-rows", "500"]
    res = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, res.stdout
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["steps"] == 1
    assert rec["value"] > 0 and rec["cpu_baseline"]["kind"] == "oracle"
    assert rec["e2e"]["h2d_bytes_per_step"] == 0
