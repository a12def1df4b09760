"""Multi-process host logic on CPU ranks (gloo, world size 2).

Covers the helpers the benchmark uses under torchrun (max over ranks, the
job-wide rate) and the frame partition that a frame-sharded step would use:
the adjoint of Eq. 2 summed over ranks' frame ranges with one all-reduce must
equal the adjoint over all frames, and each rank's pose gradients are the
rows of the all-frame pose gradient for its frames.  The arithmetic here is
the FP64 oracle's; only the partition and the collectives are under test.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2604_09643_b300 import replicas, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _small_scan():
    geom = synth.make_geom((10, 9, 8), 0.2, 9, 5, 160)
    rng = np.random.default_rng(41)
    p0 = rng.uniform(0.0, 1.0, size=(10, 9, 8)).astype(np.float32)
    elem = synth.planar_array(3, 3, 0.7)
    poses = synth.sweep_poses(5, 0.3, synth.top_face_z(geom) + 1.5, np.random.default_rng(42))
    g = np.random.default_rng(43).standard_normal((5, 9, 160))
    return geom, p0, elem, poses, g


def _rank_main(rank, world, port, out_dir):
    import oracle

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = {}
        res["max"] = replicas.max_over_ranks(1.5 + rank)
        res["rate"] = replicas.job_throughput(10, replicas.max_over_ranks(2.0 + rank), world)

        geom, p0, elem, poses, g = _small_scan()
        b, e = replicas.frame_ranges(geom["n_frames"], world)[rank]
        gl = dict(geom, n_frames=e - b)
        xw = oracle.element_positions(gl, elem, poses[b:e])
        vol = torch.from_numpy(oracle.adjoint(gl, g[b:e], xw))
        dist.all_reduce(vol, op=dist.ReduceOp.SUM)
        grad6, _ = oracle.pose_grad(gl, p0, g[b:e], xw)
        np.save(os.path.join(out_dir, f"vol{rank}.npy"), vol.numpy())
        np.save(os.path.join(out_dir, f"grad6_{rank}.npy"), grad6)
        np.save(os.path.join(out_dir, f"res{rank}.npy"), np.array([res["max"], res["rate"]]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_frame_ranges_partition():
    for F in (0, 1, 5, 64, 400):
        for world in (1, 2, 3, 8):
            r = replicas.frame_ranges(F, world)
            assert len(r) == world and r[0][0] == 0 and r[-1][1] == F
            assert all(r[i][1] == r[i + 1][0] for i in range(world - 1))
            sizes = [e - b for b, e in r]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.frame_ranges(4, 0)


def test_single_process_helpers():
    assert replicas.max_over_ranks(3.25) == 3.25
    assert replicas.job_throughput(20, 2.0, 4) == 40.0
    with pytest.raises(ValueError):
        replicas.job_throughput(1, 0.0, 1)


def test_two_gloo_ranks_shard_frames(tmp_path):
    import oracle

    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    for r in range(world):
        mx, rate = np.load(tmp_path / f"res{r}.npy")
        assert mx == 2.5
        assert rate == pytest.approx(world * 10 / 3.0)

    geom, p0, elem, poses, g = _small_scan()
    xw = oracle.element_positions(geom, elem, poses)
    vol_all = oracle.adjoint(geom, g, xw)
    grad6_all, _ = oracle.pose_grad(geom, p0, g, xw)
    assert np.abs(vol_all).max() > 0
    for r in range(world):
        vol = np.load(tmp_path / f"vol{r}.npy")
        np.testing.assert_allclose(vol, vol_all, rtol=1e-12, atol=1e-12 * np.abs(vol_all).max())
    shards = np.concatenate([np.load(tmp_path / f"grad6_{r}.npy") for r in range(world)])
    np.testing.assert_allclose(shards, grad6_all, rtol=0, atol=0)
