"""The multi-GPU bookkeeping on CPU: two `gloo` ranks in separate processes
(the GPU runs use one process per GPU the same way).  Each rank derives its
replica problem, times its own work, and the job throughput counts both ranks'
work at the slower rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2010_00520_gb300.replicas import (job_throughput, max_over_ranks, ranks_from_env,  # noqa: E402
                                             replica_seed)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r = ranks_from_env()
        seconds = 0.5 + r.rank                     # rank 1 is the slower one
        worst = max_over_ranks(seconds, dist)
        dist.barrier()
        out[r.rank] = (r.world, r.rank, replica_seed(1002, r.rank), worst,
                       job_throughput(1000.0, r.world, worst))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_timing_and_throughput():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    seeds = {res[r][2] for r in res}
    assert len(seeds) == 2 and res[0][2] == 1002          # distinct problems, rank 0 keeps the seed
    for r in res:
        assert res[r][0] == world and res[r][1] == r
        assert res[r][3] == 1.5                           # both ranks see the slowest time
        assert res[r][4] == pytest.approx(2 * 1000.0 / 1.5)


def test_ranks_from_env_alone_and_invalid():
    r = ranks_from_env({})
    assert (r.world, r.rank, r.local, r.leader) == (1, 0, 0, True)
    with pytest.raises(ValueError):
        ranks_from_env({"WORLD_SIZE": "2", "RANK": "2"})
    assert max_over_ranks(3.0) == 3.0


def test_direction_blocks_partition_the_grid():
    from paper_2010_00520_gb300.replicas import direction_block
    for n_dir, world in ((162, 1), (162, 2), (162, 4), (162, 8), (98, 8), (8, 8), (435, 3)):
        blocks = [direction_block(n_dir, world, r) for r in range(world)]
        assert blocks[0][0] == 0 and sum(c for _, c in blocks) == n_dir
        for (f0, c0), (f1, _) in zip(blocks, blocks[1:]):
            assert f1 == f0 + c0                       # contiguous, in rank order
        assert max(c for _, c in blocks) - min(c for _, c in blocks) <= 1
    with pytest.raises(ValueError):
        direction_block(3, 4, 0)


def _shard_worker(rank, world, port, out, fmt=3, dec=1):
    """Each rank compresses its block of directions (host FP64 set-up) with a
    shard plan; rank 0 gathers the restored operators.  3D formats decompose
    each direction on its own; 4D formats decompose the whole grid's T_4D and
    keep the block's rows of the direction factor."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import numpy as np
        import paper_2010_00520_gb300 as F
        from paper_2010_00520_gb300.replicas import direction_block
        K, L = (6, 5, 7), 3
        n_dir = 2 * (L + 1) ** 2
        first, count = direction_block(n_dir, world, rank)
        h = F.fmmfft_plan_create(*K, 0.5, 2 * np.pi, L, fmt, dec, 1e-4)
        try:
            F.fmmfft_plan_set(h, F.FMMFFT_KEY_DIR_FIRST, first)
            F.fmmfft_plan_set(h, F.FMMFFT_KEY_DIR_COUNT, count)
            assert F.fmmfft_plan_stats(h)["n_dir"] == count
            ranks, restored = F.fmmfft_compress_host(h)
        finally:
            F.fmmfft_plan_destroy(h)
        parts = [None] * world
        dist.all_gather_object(parts, (first, ranks, restored))
        if rank == 0:
            out["parts"] = parts
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("fmt,dec", [(3, 1), (4, 1), (4, 3), (4, 2)])
def test_direction_shards_on_gloo_ranks_equal_the_whole_plan(fmt, dec):
    """The shards' restored operators, concatenated in rank order, equal the
    whole plan's bit for bit (Sec. II.C: directions are restored
    independently; for the 4D formats from one global decomposition, so the
    result does not depend on the number of ranks)."""
    import numpy as np
    import paper_2010_00520_gb300 as F
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_worker, args=(world, _free_port(), out, fmt, dec), nprocs=world, join=True)
        parts = out["parts"]
    K, L = (6, 5, 7), 3
    h = F.fmmfft_plan_create(*K, 0.5, 2 * np.pi, L, fmt, dec, 1e-4)
    try:
        ranks, restored = F.fmmfft_compress_host(h)
    finally:
        F.fmmfft_plan_destroy(h)
    parts = sorted(parts, key=lambda t: t[0])
    if fmt == 3:
        assert np.array_equal(np.concatenate([p[1] for p in parts]), ranks)
    else:
        for p in parts:
            assert np.array_equal(p[1], ranks)           # the global ranks on every shard
    assert np.array_equal(np.concatenate([p[2] for p in parts]), restored)
