"""Host logic of the multi-GPU bench path on CPU with two gloo ranks: the step
time is the slowest rank's, and each rank of the batched form draws its own
problems (weak scaling, no data-path collective)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import argparse

    import bench
    t = bench.max_over_ranks(10.0 + 5.0 * rank, ws, device="cpu")
    args = argparse.Namespace(workload="batched2d", batch=6, tol_inner=1e-10, form="mixed", form_default=True,
                              n=1024, gammas=[100.0], rank=rank)
    wk = bench.Workload(args)
    sides = [p["n"][0] for p in wk.problems]
    first = float(wk.problems[0]["g"][0])
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t, sides, first))


@pytest.mark.timeout(300)
def test_two_gloo_ranks_max_time_and_own_batches():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    (r0, t0, s0, g0), (r1, t1, s1, g1) = res
    assert t0 == t1 == 15.0                 # both ranks report the slowest rank's time
    assert len(s0) == len(s1) == 6
    assert all(s % 32 == 0 and 64 <= s <= 512 for s in s0 + s1)
    assert (s0, g0) != (s1, g1)             # distinct problems per rank


def test_single_rank_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.batch_seed_offset(0) == 6 and bench.batch_seed_offset(1) != bench.batch_seed_offset(0)
