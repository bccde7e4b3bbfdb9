"""Workers for the multi-process (gloo, CPU) tests: each runs in a spawned
process with a torch.distributed group of the given size and returns a
picklable result."""
import os

import torch
import torch.distributed as dist


def run_group(fn, world: int = 2, timeout: float = 120.0):
    """Run fn(rank, world) in `world` spawned processes joined by a gloo group on
    127.0.0.1; returns the results in rank order."""
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, fn, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(world):
            rank, res = q.get(timeout=timeout)
            out[rank] = res
    finally:
        for p in procs:
            p.join(timeout=10)
            if p.is_alive():
                p.kill()
    return [out[r] for r in range(world)]


def _worker(rank, world, port, fn, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = fn(rank, world)
    except Exception as e:  # reported to the parent, which fails the test
        res = ("error", repr(e))
    finally:
        dist.destroy_process_group()
    q.put((rank, res))


# ---- the functions under test, one per case --------------------------------------
def gather_case(rank, world):
    from paper_2606_06329_gb300 import shard
    n = 11
    b, e = shard.row_range(rank, world, n)
    local = torch.stack([torch.arange(b, e, dtype=torch.float32), -torch.arange(b, e, dtype=torch.float32)], 1)
    return shard.gather_rows(local, n).tolist()


def timing_case(rank, world):
    import bench
    return bench.aggregate_timing(100.0 + 50.0 * rank, 1000, 3, dist)


class _FakeCtx:
    """Stands in for api.Context: kappa of row i is 0.5 i + 1."""

    def mecuco_curvature_range(self, X, k, b, e, **kw):
        return 0.5 * torch.arange(b, e, dtype=torch.float32) + 1.0


def sharded_case(rank, world):
    from paper_2606_06329_gb300 import shard
    X = torch.zeros((9, 4))
    return shard.curvature_sharded(_FakeCtx(), X, 3).tolist()
