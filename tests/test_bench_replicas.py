"""Replica helpers of bench.py on two gloo ranks (CPU): rendezvous, barrier,
max-over-ranks timing, and the rule that only rank 0 runs the reference arm."""
import os
import socket
import sys

import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(ws),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    got_ws, got_rank, local = bench.dist_init()
    try:
        bench.barrier(got_ws)
        # each rank reports a different time; every rank must see the maximum
        m = bench.max_over_ranks(got_ws, 1.5 + rank, torch.device("cpu"))

        class A:
            workload = "taylor_green_2d"
            steps = 1
            warmup = 0
            gpus = ws
        printed = []
        real_print = print
        import builtins
        builtins.print = lambda *a, **k: printed.append(a)
        try:
            if rank != 0:
                bench.run_reference(A, got_ws, got_rank)
        finally:
            builtins.print = real_print
        out.put((rank, got_ws, got_rank, local, m, len(printed)))
        bench.barrier(got_ws)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_barrier_and_max():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got_ws, got_rank, local, m, nprinted in res:
        assert (got_ws, got_rank, local) == (ws, rank, rank)
        assert m == 2.5
        assert nprinted == 0   # non-zero ranks exit the reference arm without work or output
