"""The multi-rank path on CPU: two gloo ranks as independent replicas.

Each rank draws its own instance (distinct seeds), and the whole-job
throughput is the units of all ranks over the slowest rank's time, computed
with the same helper bench.py uses under torchrun.
"""
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    from paper_1705_09366_gb300 import replicas, synth

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        w = synth.small(seed_offset=replicas.instance_offset(rank))
        units = float(w.n) * (rank + 1)        # rank r "processes" (r + 1) n units
        secs = 0.5 + rank                      # in 0.5 + r seconds
        dist.barrier()
        value, tmax, total = replicas.job_throughput(dist, units, secs, device="cpu")
        q.put((rank, value, tmax, total, float(w.points[:, 0].sum())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_as_replicas():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    n = 2000.0
    for rank, value, tmax, total, _ in res:
        assert tmax == pytest.approx(1.5)
        assert total == pytest.approx(3 * n)
        assert value == pytest.approx(3 * n / 1.5)
    # the two replicas computed different instances
    assert res[0][4] != res[1][4]


def test_single_process_path():
    from paper_1705_09366_gb300 import replicas

    assert replicas.job_throughput(None, 10.0, 2.0) == (5.0, 2.0, 10.0)
