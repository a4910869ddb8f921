"""The multi-GPU bench path on CPU: two gloo ranks take disjoint position blocks that together cover
the scan once per pass, and the step time is the maximum over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, B, Ntot, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = bench.rank_batches(rank, world, B, Ntot, n=Ntot // (B * world))
    flat = torch.tensor([p for b in mine for p in b], dtype=torch.int64)
    gathered = [torch.empty_like(flat) for _ in range(world)]
    dist.all_gather(gathered, flat)
    t = bench.max_over_ranks(10.0 + rank, dist, "cpu")
    if rank == 0:
        q.put((sorted(int(x) for g in gathered for x in g), [len(g) for g in gathered], t))
    dist.destroy_process_group()


@pytest.mark.parametrize("world,B,Ntot", [(2, 512, 4096), (2, 64, 256), (4, 16, 256)])
def test_ranks_cover_the_scan_once_and_time_is_the_max(world, B, Ntot):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, B, Ntot, q)) for r in range(world)]
    for p in procs:
        p.start()
    allpos, sizes, t = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert allpos == list(range(Ntot))  # disjoint blocks covering every position exactly once
    assert sizes == [Ntot // world] * world
    assert t == 10.0 + world - 1
