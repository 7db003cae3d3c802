"""Multi-process (gloo, world size 2) test of the image-sharded path on CPU.

Each rank compresses its shard of a mixed-size batch (the CPU oracle stands in
for the per-rank GPU compute, which needs no collective) and the per-image
PSNRs are gathered on the host.  The gathered result must equal the
single-process result, item for item."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_1606_05562_gb300 import shard, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _batch():
    imgs = synth.mixed_batch(7, lo=16, hi=96, seed=5)
    rs = [1, 6, 16, 36, 64, 100, 256][: len(imgs)]
    return imgs, rs


def _worker(rank, world, port, outdir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    imgs, rs = _batch()
    shards = shard.balanced_shards([im.size for im in imgs], world)
    mine = shards[rank]
    vals = [O.compress_zonal_exact(imgs[i], rs[i])["psnr"] for i in mine]
    gathered = [None] * world
    dist.all_gather_object(gathered, (mine, vals))
    if rank == 0:
        idx = [g[0] for g in gathered]
        res = shard.merge_results(idx, [g[1] for g in gathered], len(imgs))
        np.save(os.path.join(outdir, "psnr.npy"), np.array(res))
    dist.destroy_process_group()


def test_two_rank_gloo_matches_single_process(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    got = np.load(tmp_path / "psnr.npy")
    imgs, rs = _batch()
    ref = np.array([O.compress_zonal_exact(im, r)["psnr"] for im, r in zip(imgs, rs)])
    assert np.array_equal(got, ref)


def _bench_worker(rank, world, port, outdir):
    # the multi-GPU bench's image assignment, run by gloo ranks on CPU
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = bench.rank_images(world, rank, n_per_rank=4, side=32)
    imgs = synth.image_batch_512(4 * world, 32, first_seed=100, indices=mine)
    sums = [int(im.astype(np.int64).sum()) for im in imgs]
    gathered = [None] * world
    dist.all_gather_object(gathered, (list(mine), sums))
    if rank == 0:
        np.save(os.path.join(outdir, "assign.npy"), np.array([g[0] for g in gathered]))
        np.save(os.path.join(outdir, "sums.npy"), np.array([g[1] for g in gathered]))
    dist.destroy_process_group()


def test_bench_sharding_two_ranks(tmp_path):
    port = _free_port()
    mp.start_processes(_bench_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    assign = np.load(tmp_path / "assign.npy")
    sums = np.load(tmp_path / "sums.npy")
    # every image of the whole job exactly once, the same count per rank
    assert sorted(assign.ravel().tolist()) == list(range(8))
    assert [len(a) for a in assign] == [4, 4]
    # each rank drew exactly the images the single-process batch holds there
    full = synth.image_batch_512(8, 32, first_seed=100)
    for r in range(2):
        for i, s in zip(assign[r], sums[r]):
            assert int(full[i].astype(np.int64).sum()) == s


def test_shard_helpers():
    assert [list(shard.contiguous_shard(10, 3, r)) for r in range(3)] == [[0, 1, 2, 3], [4, 5, 6], [7, 8, 9]]
    sizes = [100, 90, 80, 10, 10, 5]
    s = shard.balanced_shards(sizes, 2)
    assert sorted(s[0] + s[1]) == list(range(6))
    loads = [sum(sizes[i] for i in x) for x in s]
    assert max(loads) - min(loads) <= max(sizes)
    with pytest.raises(ValueError):
        shard.merge_results([[0, 1], [1]], [[1, 2], [3]], 2)
    with pytest.raises(ValueError):
        shard.merge_results([[0]], [[1]], 2)
