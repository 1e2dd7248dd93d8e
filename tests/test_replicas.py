"""The N > 1 path of bench.py on the CPU: two gloo ranks of the replica bookkeeping.

One real-time iteration does not shard, so a run on N GPUs steps N independent replicas and
combines only the timing: a barrier, the max over ranks of the milliseconds per step, and
the whole-job rate N x 1000 / that max.  The reference arm's non-leader ranks do no work.
"""
import json
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import sys
    sys.path.insert(0, ROOT)
    from paper_2602_17601_b300.replicas import Replicas
    reps = Replicas("gloo", device="cpu")
    ms = 10.0 + 5.0 * rank                   # rank 1 is the slow one
    reps.barrier()
    m = reps.max_over_ranks(ms)
    res = {"rank": reps.rank, "world": reps.world, "leader": reps.leader, "max_ms": m,
           "steps_per_s": reps.steps_per_s(m)}
    reps.barrier()
    reps.close()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)


def test_two_gloo_ranks_combine_timing(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, d in enumerate(res):
        assert d["rank"] == r and d["world"] == world and d["leader"] == (r == 0)
        assert d["max_ms"] == 15.0                       # every rank sees the slowest rank's time
        assert d["steps_per_s"] == pytest.approx(world * 1000.0 / 15.0)


def test_single_process_needs_no_process_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_2602_17601_b300.replicas import Replicas
    reps = Replicas("gloo")
    assert reps.world == 1 and reps.leader
    assert reps.max_over_ranks(3.5) == 3.5
    assert reps.steps_per_s(4.0) == 250.0
    reps.barrier()
    reps.close()


def test_reference_arm_non_leader_rank_does_no_work(monkeypatch, capsys):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(bench, "workload", lambda name: pytest.fail("a non-leader rank built a workload"))
    bench.run_reference(bench.parse(["--impl", "reference", "--gpus", "2"]))
    assert capsys.readouterr().out == ""
