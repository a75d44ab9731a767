"""Multi-process host logic on CPU (gloo, world size 2): sharding a stream by
output spectra with a T-1 halo reproduces the unsharded transform, and the
timing reduction takes the maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_1511_03599_gb300 import dist as pdist
from paper_1511_03599_gb300 import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shards_partition_exactly():
    for S in (1, 7, 100, 1 << 20):
        for world in (1, 2, 3, 8):
            if world > S:
                continue
            covered = []
            for r in range(world):
                s0, s1, r0, r1 = pdist.shard_spectra(S, 8, r, world)
                assert r0 == s0 and r1 == s1 + 7
                covered.extend(range(s0, s1))
            assert covered == list(range(S))
    with pytest.raises(ValueError):
        pdist.shard_spectra(10, 8, 2, 2)


def _worker(rank, world, port, C, T, S, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    h = synth.design_taps(C, T)
    x = synth.stream(C, S + T - 1, "ci16", 2000.0, 99)        # every rank sees the same stream
    s0, s1, r0, r1 = pdist.shard_spectra(S, T, rank, world)
    y = oracle.pfb(x[r0 * C:r1 * C], h, C, T)                 # the rank's shard, halo included
    parts = [None] * world
    dist.all_gather_object(parts, (s0, s1, y))
    t = pdist.max_over_ranks(1.0 + rank)
    pdist.barrier()
    if rank == 0:
        full = np.zeros((S, C), dtype=np.complex128)
        for a, b, yy in parts:
            full[a:b] = yy
        np.save(os.path.join(out_dir, "sharded.npy"), full)
        with open(os.path.join(out_dir, "tmax.txt"), "w") as f:
            f.write(str(t))
    dist.destroy_process_group()


def test_sharded_transform_equals_whole_gloo(tmp_path):
    C, T, S, world = 32, 8, 61, 2
    mp.spawn(_worker, args=(world, _free_port(), C, T, S, str(tmp_path)), nprocs=world, join=True)
    sharded = np.load(tmp_path / "sharded.npy")
    whole = oracle.pfb(synth.stream(C, S + T - 1, "ci16", 2000.0, 99), synth.design_taps(C, T), C, T)
    assert np.max(np.abs(sharded - whole)) <= 1e-9 * np.max(np.abs(whole))
    assert float((tmp_path / "tmax.txt").read_text()) == 2.0


def test_max_over_ranks_without_group():
    assert pdist.max_over_ranks(3.5) == 3.5
    assert pdist.env_rank_world()[2] >= 1
