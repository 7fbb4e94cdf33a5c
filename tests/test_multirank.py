"""The multi-rank (replica) logic of bench.py on CPU: two gloo ranks, as torchrun launches
them.  Trajectories are independent, so ranks share nothing but the timing barrier and the
max-over-ranks reduction; each rank advances its own block of trajectory ids."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["FM_ROOT"])
import torch.distributed as dist
dist.init_process_group("gloo", init_method="env://")
import bench
world, rank, local = bench.setup_distributed(None)
bench.barrier(world)
t = bench.max_over_ranks(1.5 + rank, world)
print(json.dumps({"rank": rank, "world": world, "local": local, "t": t,
                  "traj0": bench.replica_traj_id(rank, 4)}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_time_and_trajectory_blocks():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r), WORLD_SIZE="2",
                   LOCAL_RANK=str(r), FM_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    outs.sort(key=lambda d: d["rank"])
    assert [d["world"] for d in outs] == [2, 2]
    assert [d["t"] for d in outs] == [2.5, 2.5]          # the slowest rank's time, on every rank
    assert [d["traj0"] for d in outs] == [0, 4]          # disjoint trajectory blocks
    assert [d["local"] for d in outs] == [0, 1]
