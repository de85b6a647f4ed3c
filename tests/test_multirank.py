"""The multi-rank benchmark path on CPU: two gloo ranks, each with its own
seeded shard (no data exchange), the whole-job figures reduced as the bench
does on GPUs (max time, summed instances).  Each rank's device solve is
stood in for by the oracle."""
import os
import socket
import time

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_2404_18034_gb300 import inputs
    p = inputs.load_params()
    B = 2 + rank  # uneven shards
    x0 = inputs.dispersion(p, B, bench.shard_seed(inputs.config_seed(2), rank), "bj")
    dist.barrier()
    t = time.perf_counter()
    r = oracle.solve_batch(p, x0, np.full(B, 10, np.int32), nthreads=1)
    ms = 1e3 * (time.perf_counter() - t)
    conv = int(np.sum(r["status"] == 0))
    agg = bench.reduce_over_ranks(ms, conv, B, dist, "cpu")
    q.put((rank, ms, conv, B, agg, x0[0].tolist()))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=300) for _ in range(2))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    (r0, ms0, c0, b0, agg0, x00), (r1, ms1, c1, b1, agg1, x01) = res
    assert agg0 == agg1
    assert agg0[0] == pytest.approx(max(ms0, ms1))
    assert agg0[1] == c0 + c1 and agg0[2] == b0 + b1
    assert not np.allclose(x00, x01)  # independent shards
