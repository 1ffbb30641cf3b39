"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas) with
different step times; the job's time is the maximum over ranks and its value
counts the units of both ranks.  Each rank seeds its own workload."""
import math
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import sys
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms = 2.0 + rank          # rank 1 is the slow one
    e2e = 3.0 + 2 * rank
    res = bench.aggregate_over_ranks(ms, e2e, 1e6, ws, torch.device("cpu"))
    w = bench.make_workload(N=4, m=50, seed=bench.SEED + rank)
    dist.barrier()
    dist.destroy_process_group()
    out[rank] = (res, float(w["y"][0, 0]))


def test_two_gloo_ranks_take_the_max_and_count_all_units():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    (r0, y0), (r1, y1) = out[0], out[1]
    assert r0 == r1                                  # every rank sees the same aggregate
    ms, e2e, value, e2e_val = r0
    assert ms == 3.0 and e2e == 5.0                  # the maximum over ranks
    assert math.isclose(value, 2 * 1e6 / 3e-3 / 1e9)
    assert math.isclose(e2e_val, 2 * 1e6 / 5e-3 / 1e9)
    assert y0 != y1                                  # replicas run different seeded inputs


def test_single_rank_needs_no_collective():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    ms, e2e, value, e2e_val = bench.aggregate_over_ranks(4.0, float("nan"), 2e6, 1, None)
    assert ms == 4.0 and value == pytest.approx(2e6 / 4e-3 / 1e9) and e2e_val is None
