"""The multi-process path of bench.py (replicas, one rank per GPU) on the CPU:
two gloo ranks set up through bench.dist_setup, meet at bench.barrier and agree
on the slowest rank's time through bench.max_over_ranks; the reference arm
returns at once on ranks other than 0."""
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, types
sys.path.insert(0, sys.argv[1])
import bench
world, rank, local = bench.dist_setup()
assert world == 2 and rank == local
bench.barrier(world)
t = bench.max_over_ranks(10.0 + 5.0 * rank, world)
bench.barrier(world)
args = types.SimpleNamespace(gpus=2, steps=1, warmup=1)
bench.run_reference(args, world, rank) if rank != 0 else None
print("rank", rank, "max", t, flush=True)
import torch.distributed as dist
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_agree_on_max():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), SHT_BENCH_GLOO="1")
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True))
    outs = []
    for p in procs:
        out, _ = p.communicate(timeout=120)
        outs.append(out)
        assert p.returncode == 0, out
    for rank, out in enumerate(outs):
        assert f"rank {rank} max 15.0" in out, out
