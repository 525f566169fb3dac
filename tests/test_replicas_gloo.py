"""Multi-process host logic of multi-GPU runs, on CPU with the gloo backend.

A multi-GPU job shards the signals across ranks (no data-path collective);
the host-side pieces -- the shard assignment, the barrier-bracketed timing,
the maximum of per-rank step times and the whole-job throughput -- are
checked here with world_size 2 on 127.0.0.1.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1507_02525_gb300 import inputs, replicas  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_covers_every_signal_once():
    lengths = [int(v) for v in inputs.ragged_lengths(1024, 8, 18, seed=3)]
    for world in (1, 2, 3, 4, 8):
        parts = [replicas.shard(lengths, r, world) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(lengths)))
        # contiguous blocks, in rank order
        for p in parts:
            assert p == list(range(p[0], p[-1] + 1)) if p else True
        # balance: no rank holds more than its share plus one longest signal
        total = sum(lengths)
        for p in parts:
            assert sum(lengths[i] for i in p) <= total / world + max(lengths)


def test_shard_uniform_batch_and_degenerate():
    assert replicas.shard([1 << 16] * 256, 1, 4) == list(range(64, 128))
    # fewer signals than ranks: some ranks get nothing, none gets a signal twice
    parts = [replicas.shard([1 << 24], r, 4) for r in range(4)]
    assert sorted(i for p in parts for i in p) == [0]
    with pytest.raises(ValueError):
        replicas.shard([8, 8], 2, 2)


def test_job_throughput():
    assert replicas.job_throughput(2 * (1 << 24), 2.0) == pytest.approx(2 * (1 << 24) / 2e-3)
    with pytest.raises(ValueError):
        replicas.job_throughput(1.0, 0.0)


def _worker(rank, world, port, lengths, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        info = replicas.rank_info()
        mine = replicas.shard(lengths, info.rank, info.world)
        samples = sum(lengths[i] for i in mine)
        replicas.barrier()
        # rank-dependent "step time": the job is as slow as its slowest rank
        ms = 1.0 + info.rank
        ms_max = replicas.max_over_ranks(ms)
        total = replicas.sum_over_ranks(samples)
        replicas.barrier()
        q.put((info.rank, info.world, mine, ms_max, total, replicas.job_throughput(total, ms_max)))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_timing_and_shards():
    lengths = [int(v) for v in inputs.ragged_lengths(64, 8, 18, seed=3)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, lengths, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert sorted(res[0][2] + res[1][2]) == list(range(len(lengths)))
    for r in res:
        assert r[3] == 2.0                      # max of 1.0 and 2.0
        assert r[4] == float(sum(lengths))      # every sample counted once
        assert r[5] == pytest.approx(sum(lengths) / 2e-3)
