"""The multi-rank path of the benchmark on CPU (gloo, two processes): each
rank draws its own share of a family of independent systems and the job's
time is the maximum over ranks; no data-path collective is involved."""
import multiprocessing
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    try:
        import bench
        from paper_0911_4348_gb300 import workloads as W
        dist, r, w, _ = bench._dist("gloo")
        t = bench.max_over_ranks(dist, 1.5 + 2.0 * r, device="cpu")
        mine = [(s.name, tuple(s.Z), tuple(s.R), s.n_elem, s.order, s.u)
                for s in W.batch_systems(6, config_id=bench.rank_config(4, r))]
        allsys = [None] * w
        dist.all_gather_object(allsys, mine)
        dist.barrier()
        dist.destroy_process_group()
        q.put((r, w, t, allsys))
    except Exception as e:  # report, never hang the parent
        q.put((rank, -1, repr(e), None))


def test_two_ranks_max_time_and_distinct_systems():
    port = _free_port()
    ctx = multiprocessing.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    results.sort()
    for r, w, t, allsys in results:
        assert w == 2, t
        assert t == pytest.approx(3.5)  # max of 1.5 and 3.5
        assert allsys[0] != allsys[1]   # each rank draws its own systems
    assert results[0][3] == results[1][3]
