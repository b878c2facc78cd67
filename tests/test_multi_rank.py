"""The N>1 path on CPU: two gloo ranks shard the field points (no exchange on
the data path), each evaluates its share, and the slowest rank's time sets
the job rate.  The evaluation is the oracle's, so this runs without a GPU;
what is tested is the sharding and the reduction that bench.py uses."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from paper_1606_03743_gb300 import shard


@pytest.mark.parametrize("n", [0, 1, 7, 4096, 4097])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_point_range_partitions(n, world):
    ranges = [shard.point_range(n, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 == b0
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1


def test_point_range_rejects_bad_rank():
    with pytest.raises(ValueError):
        shard.point_range(10, 2, 2)
    with pytest.raises(ValueError):
        shard.point_range(10, 0, 0)


def test_rank_seeds_give_distinct_batches():
    a = synth.coax_points(seed=shard.rank_seed(2, 0), n=64)
    b = synth.coax_points(seed=shard.rank_seed(2, 1), n=64)
    assert not np.array_equal(a, b)


def test_job_rate():
    assert shard.job_rate(2e9, 1000.0) == pytest.approx(2e9)
    with pytest.raises(ValueError):
        shard.job_rate(1.0, 0.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mesh = synth.plate_mesh(seed=1, n=4)
        pts = synth.plate_points(seed=1, n=301)
        lo, hi = shard.point_range(len(pts), rank, world)
        phi, E = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, pts[lo:hi], nthreads=1)
        parts = [None] * world
        dist.all_gather_object(parts, (lo, hi, phi, E))  # test-only gather; bench.py gathers nothing
        slow = shard.slowest_rank_ms(10.0 + rank, dist)
        if rank == 0:
            np.savez(os.path.join(out_dir, "gathered.npz"),
                     lo=np.array([p[0] for p in parts]), hi=np.array([p[1] for p in parts]),
                     phi=np.concatenate([p[2] for p in parts]), E=np.concatenate([p[3] for p in parts]),
                     slow=np.array([slow]))
        else:
            np.save(os.path.join(out_dir, f"slow{rank}.npy"), np.array([slow]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_one(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    oracle.build()
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    g = np.load(tmp_path / "gathered.npz")
    mesh = synth.plate_mesh(seed=1, n=4)
    pts = synth.plate_points(seed=1, n=301)
    phi, E = oracle.eval_field(mesh.types, mesh.verts, mesh.sigma, pts, nthreads=1)
    assert list(g["lo"]) == [0, 151] and list(g["hi"]) == [151, 301]
    # per-point sums do not depend on the sharding: bit-identical
    np.testing.assert_array_equal(g["phi"], phi)
    np.testing.assert_array_equal(g["E"], E)
    # every rank sees the slowest rank's time
    assert g["slow"][0] == 11.0
    assert np.load(tmp_path / "slow1.npy")[0] == 11.0
