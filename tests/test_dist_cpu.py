"""Multi-rank path of the benchmark on CPU (gloo, world size 2): ranks take
disjoint blocks of the same seeded candidate population (weak scaling, no
data-path collective), and the whole-job throughput uses the slowest rank's
time and the units summed over ranks."""
import os
import socket
import types

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    args = types.SimpleNamespace(workload="c4", candidates=3)
    wl = bench.load_workload(args, rank)
    seeds = [c.pulse.p for c in wl.candidates]
    value, ms, units = bench.aggregate(100.0 + 50.0 * rank, 1000.0 * (rank + 1), dist)
    q.put((rank, seeds, value, ms, units))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_aggregation():
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
    (r0, s0, v0, ms0, u0), (r1, s1, v1, ms1, u1) = out
    assert not set(s0) & set(s1)                 # disjoint candidate blocks
    assert ms0 == ms1 == 150.0                   # slowest rank
    assert u0 == u1 == 3000.0                    # all ranks' units
    assert v0 == pytest.approx(3000.0 / 0.150)


def test_rank_blocks_continue_the_population():
    import bench
    import lr_inputs as li
    args = types.SimpleNamespace(workload="c4", candidates=4)
    full = li.c4(n_candidates=8)
    got = bench.load_workload(args, 0).candidates + bench.load_workload(args, 1).candidates
    assert [c.pulse.p for c in got] == [c.pulse.p for c in full.candidates]
