"""Host logic of bench.py: whole-job aggregation over ranks (gloo, 2 ranks)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    secs = [2.0, 3.0][rank]
    t = bench.reduce_max(secs, world)
    units = 1000 * (rank + 1)
    dist.barrier()
    q.put((rank, t, bench.aggregate([1000, 2000], [2.0, 3.0])))
    dist.destroy_process_group()


def test_replica_aggregation_uses_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(t == 3.0 for _, t, _ in out)
    assert out[0][2] == pytest.approx(3000 / 3.0)


def test_clock_rejection_rules():
    import bench
    assert bench.clocks_rejected({"reasons": ["hw_slowdown"], "sm_mhz": 1900, "sm_max_mhz": 2070})
    assert not bench.clocks_rejected({"reasons": ["sw_power_cap"], "sm_mhz": 1500, "sm_max_mhz": 2070})
    assert bench.clocks_rejected({"reasons": [], "sm_mhz": 600, "sm_max_mhz": 2070})
