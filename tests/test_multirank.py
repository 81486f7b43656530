"""The multi-rank logic of the benchmark on CPU (gloo, world size 2): the
path shards by views (every rank renders its own frame, no data-path
collective); the timing is the largest over the ranks and the value counts
the rays of all ranks; the reference arm runs on rank 0 only."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2311_02542_gb300 import synth as S
    r, w, _ = bench.dist_env()
    ms = bench.max_over_ranks(1.5 + rank)
    sc = S.make_scene("room", with_params=False)
    c2w, _, _ = S.camera_room(sc.occ, sc.cfg, 2 + r, 64, 64)  # each rank's own view
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, ms, c2w[0].tolist()))


def test_two_ranks_time_is_the_slowest_and_views_differ():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[2] == 2.5 for o in out)  # max over ranks, seen by both
    assert out[0][3] != out[1][3]


def test_whole_job_value_and_single_rank():
    import bench
    assert bench.whole_job_mrays(2048 * 2048, 2, 2.5) == pytest.approx(2 * 4194304 / 2.5e-3 / 1e6)
    assert bench.max_over_ranks(3.25) == 3.25  # no process group: the value itself


def test_reference_arm_is_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    class A:
        gpus, steps, warmup, variant = 2, 1, 0, "room"
    assert bench.reference_arm(A()) == 0
    assert capsys.readouterr().out == ""
