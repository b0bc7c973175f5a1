"""The multi-rank host logic of weak scaling (ranks.py), on two gloo processes on CPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

from paper_2501_17267_gb300 import ranks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_WORKER = r"""
import json, os, sys
sys.path.insert(0, os.getcwd())
import torch
import torch.distributed as dist
from paper_2501_17267_gb300 import ranks
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
mine = ranks.rank_units(rank, 16)
everyone = [torch.zeros(16, dtype=torch.int64) for _ in range(world)]
dist.all_gather(everyone, torch.tensor(mine, dtype=torch.int64))
ms = 100.0 + 7.0 * rank          # this rank's step time
mx = ranks.max_over_ranks(ms, device="cpu")
print(json.dumps(dict(rank=rank, units=[e.tolist() for e in everyone], max_ms=mx,
                      rate=ranks.job_rate(1e9, world, 3, mx))))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_rank_units_are_disjoint_and_cover_the_job():
    got = [ranks.rank_units(r, 16) for r in range(4)]
    assert sorted(sum(got, [])) == list(range(64))
    assert ranks.job_rate(1e9, 4, 3, 500.0) == pytest.approx(1e9 * 4 * 3 / 0.5)
    assert ranks.max_over_ranks(12.5) == 12.5  # no process group: the value itself


def test_two_gloo_ranks_shard_and_take_the_slowest_time():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", _WORKER], cwd=ROOT, env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=240)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["max_ms"] == 107.0  # both ranks see the slowest rank's time
        assert o["rate"] == pytest.approx(1e9 * 2 * 3 / 0.107)
        assert sorted(sum(o["units"], [])) == list(range(32))  # disjoint, complete
