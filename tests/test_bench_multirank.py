"""The N > 1 host logic of bench.py on CPU: two gloo ranks report different
step times; both see the slowest one, and the value counts both ranks' work;
the configuration rank 0 tuned reaches the other rank."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    assert bench.dist_env() == (rank, world, rank)
    t_ms = 2.0 if rank == 0 else 3.0          # rank 1 is the slow one
    dist.barrier()
    t_max, value = bench.aggregate_over_ranks(t_ms, 6e9)
    tuned = bench.from_rank0(((16, 16, 4, 2, 1, 1), 5576, {"brute": {"evals": 5576}}) if rank == 0 else None)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t_max, value, tuned))


def test_two_gloo_ranks_take_the_slowest_step():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted((q.get(timeout=5) for _ in range(2)), key=lambda r: r[0])
    for rank, t_max, value, tuned in res:
        assert t_max == 3.0
        assert value == pytest.approx(2 * 6e9 / 3e-3 / 1e9)
        assert tuned == ((16, 16, 4, 2, 1, 1), 5576, {"brute": {"evals": 5576}})


def _rank_fail(rank, world, port, q):
    import sys
    import time
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import datetime
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(minutes=10))
    import bench

    def tune():
        raise ValueError("no configuration compiled")
    t0 = time.time()
    try:
        bench.run_on_rank0(tune)
        outcome = "returned"
    except bench.Rank0Failed as e:
        outcome = "Rank0Failed: " + str(e)
    except ValueError as e:
        outcome = "ValueError: " + str(e)
    q.put((rank, outcome, time.time() - t0))
    dist.destroy_process_group()


def test_rank0_failure_reaches_the_other_rank_at_once():
    """Rank 0's tuning raises: rank 0 re-raises its own error, rank 1 raises
    Rank0Failed with rank 0's message within seconds, not at the process
    group's timeout (10 minutes here)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_fail, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = dict((r, (o, t)) for r, o, t in (q.get(timeout=5) for _ in range(2)))
    assert res[0][0] == "ValueError: no configuration compiled"
    assert res[1][0].startswith("Rank0Failed") and "no configuration compiled" in res[1][0]
    assert res[1][1] < 60.0


def test_single_process_needs_no_collective():
    import bench
    t, v = bench.aggregate_over_ranks(2.0, 4e9)
    assert t == 2.0 and v == pytest.approx(4e9 / 2e-3 / 1e9)
    assert bench.from_rank0({"a": 1}) == {"a": 1}
    assert bench.run_on_rank0(lambda: 5) == 5
