"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): each rank
draws its own seeded chains (no data-path collective), the step time is the
max over ranks and the value counts every rank's draws."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 * (rank + 1)
    step = bench.max_over_ranks(ms, world)
    P = bench.make_workload(rank, small=True)
    out[rank] = (step, bench.job_value(world, step), float(P.omega[0, 0]), float(P.tau[0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=240)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 20.0                 # max over ranks
    assert res[0][1] == pytest.approx(2 * 16 / 0.020)    # whole-job draws/s
    assert res[0][2] != res[1][2] and res[0][3] != res[1][3]   # distinct chains per rank


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    class A:
        steps, warmup, small, gpus = 1, 1, True, 2
    bench.run_reference(A)
    assert capsys.readouterr().out == ""
