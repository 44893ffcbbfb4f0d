"""Host logic of the multi-rank benchmark on CPU: two gloo ranks.

The render path does not shard (views are independent), so several GPUs run
replicas; what needs checking is the host side: every rank renders its own
poses, the timed window is the slowest rank's, the job value counts every
rank's frames, and the reference arm runs on rank 0 only.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import json
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    value, ms = bench.job_throughput(local_ms, 20.0, world)
    bench.barrier(world)
    poses = [[bench.pose_batch(list(range(bench.N_POSES)), step, rank)] for step in range(bench.N_POSES)]
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"value": value, "ms": ms, "poses": poses}, f)
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks(tmp_path):
    import json
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r = [json.load(open(tmp_path / f"r{k}.json")) for k in range(2)]
    for k in range(2):
        assert r[k]["ms"] == 150.0  # max over ranks
        assert r[k]["value"] == pytest.approx(40.0 / 0.150)  # all ranks' frames / slowest time
    # within a step the two ranks render different poses
    for step in range(len(r[0]["poses"])):
        assert not set(r[0]["poses"][step][0]) & set(r[1]["poses"][step][0])


def test_reference_arm_other_ranks_do_nothing(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "run_oracle_subprocess", lambda **kw: called.append(kw))

    class A:
        gpus, steps, warmup = 2, 3, 3
    bench.reference_arm(A())
    assert called == [] and capsys.readouterr().out == ""
