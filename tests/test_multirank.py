"""Host side of the multi-GPU benchmark path, on CPU with gloo (two ranks): each rank runs an
independent replica (the lattices share nothing), the whole-job time is the slowest rank's,
and the whole-job rate counts every rank's lattice updates.  Only rank 0 runs and prints the
oracle reference arm."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        seconds = bench.max_over_ranks(1.5 + rank)  # rank 1 is the slow one
        rate = bench.whole_job_mlups(1000, 2000, ws, seconds)
        q.put((rank, bench._dist(), seconds, rate))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_all_updates():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, dist_env, seconds, rate in out:
        assert dist_env == (2, rank, rank)
        assert seconds == pytest.approx(2.5)                # max over ranks
        assert rate == pytest.approx(1000 * 2000 * 2 / 2.5 / 1e6)


def test_single_process_has_no_group():
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.whole_job_mlups(10, 100, 1, 2.0) == pytest.approx(5e-4)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup = 1, 3
    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""
