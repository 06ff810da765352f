"""Host logic of multi-GPU runs, on CPU: rank bookkeeping, the max-over-ranks
timing with world_size-2 `gloo` process groups, the whole-job throughput, the
ensemble-member split, and the reference arm's non-lead ranks doing no work."""
import json
import os
import socket
import subprocess
import sys

import pytest

from paper_1805_02144_gb300.ranks import Ranks, from_env, job_rate, max_over_ranks, member_shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_from_env_defaults_and_torchrun_values():
    assert from_env({}) == Ranks(1, 0, 0)
    r = from_env({"WORLD_SIZE": "4", "RANK": "3", "LOCAL_RANK": "3"})
    assert (r.world, r.rank, r.local, r.lead) == (4, 3, 3, False)
    assert from_env({"WORLD_SIZE": "2", "RANK": "0"}).lead
    for bad in ({"WORLD_SIZE": "2", "RANK": "2"}, {"WORLD_SIZE": "0"}, {"RANK": "-1"}):
        with pytest.raises(ValueError):
            from_env(bad)


def test_job_rate_counts_every_rank_over_the_slowest_time():
    assert job_rate(1, 20, 200.0) == pytest.approx(100.0)
    assert job_rate(8, 20, 250.0) == pytest.approx(640.0)
    assert max_over_ranks(3.5) == 3.5          # no process group: the value itself
    with pytest.raises(ValueError):
        job_rate(2, 10, 0.0)


@pytest.mark.parametrize("n,world", [(64, 1), (64, 2), (64, 3), (64, 8), (5, 8), (0, 2)])
def test_member_shard_partitions_the_members(n, world):
    shards = [member_shard(n, world, r) for r in range(world)]
    assert [i for s in shards for i in s] == list(range(n))      # in order, each once
    sizes = [len(s) for s in shards]
    assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        member_shard(n, world, world)


_CHILD = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import torch.distributed as dist
from paper_1805_02144_gb300.ranks import from_env, job_rate, max_over_ranks
rk = from_env()
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:{port}", world_size=rk.world, rank=rk.rank)
dist.barrier()
t_ms = 100.0 + 50.0 * rk.rank                 # rank r "took" 100 + 50 r ms
t = max_over_ranks(t_ms, dist, "cpu")
dist.barrier()
out = {{"rank": rk.rank, "lead": rk.lead, "t": t, "rate": job_rate(rk.world, 10, t)}}
dist.destroy_process_group()
print(json.dumps(out))
"""


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_agree_on_the_slowest_time():
    port = _free_port()
    code = _CHILD.format(root=ROOT, port=port)
    procs = []
    for r in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(r), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e[-2000:]
        outs.append(json.loads(o.strip().splitlines()[-1]))
    outs.sort(key=lambda d: d["rank"])
    assert [d["lead"] for d in outs] == [True, False]
    for d in outs:
        assert d["t"] == 150.0                       # max over ranks, seen by both
        assert d["rate"] == pytest.approx(2 * 10 / 0.150)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench

    class Args:
        steps, warmup, gpus = 1, 1, 2

    def boom(*a, **k):
        raise AssertionError("a non-lead rank must not run the oracle")

    monkeypatch.setattr(bench, "run_oracle_subprocess", boom)
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    bench.reference_arm(Args())
    assert capsys.readouterr().out == ""
