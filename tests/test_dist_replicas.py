"""CPU test of the N > 1 benchmark path with world_size 2 over gloo: ranks
run independent replicas (different seeds), the timed region is the slowest
rank's, and the whole-job value counts every rank's site updates."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, lr, w = bench.dist_env()
        ms_local = 100.0 + 50.0 * rank  # rank 1 is the slow one
        ms = bench.max_over_ranks(torch, dist, ms_local, "cpu")
        out[rank] = (r, w, bench.replica_seed(r), ms, bench.whole_job_mlups(1000, w, 10, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_over_gloo():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    assert sorted(out.keys()) == [0, 1]
    seeds = {out[r][2] for r in out.keys()}
    assert len(seeds) == world  # independent replicas
    for r in out.keys():
        rank, w, _, ms, value = out[r]
        assert (rank, w) == (r, world)
        assert ms == 150.0  # max over ranks
        assert value == pytest.approx(1000 * 2 * 10 / 0.150 / 1e6)


def test_single_rank_defaults(monkeypatch):
    import bench
    for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 0, 1)
    assert bench.max_over_ranks(torch, None, 12.5, "cpu") == 12.5
