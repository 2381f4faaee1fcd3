"""Host logic of the ray-sharded data-parallel step (Sec. 3.5: rays are independent units), on CPU: two gloo ranks
each back-propagate their shard of one batch (dp.shard_bounds; hash ids of the whole batch; loss normalised by
the whole batch) through the FP64 oracle, all-reduce (sum) the gradients, and must get the single-rank gradient
of the whole batch.  A shard split that dropped or repeated a ray, restarted the hash ids, or normalised by the
shard would fail."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2305_13220_b300.dp import shard_bounds

N_SAMPLES = 24


def _problem():
    import oracle
    import synth
    sc = synth.scene_tiny_room(0)
    keys = synth.band_blocks(sc, 0.04, 3)
    g = synth.fill_grid(sc, keys, 0.04, 3)
    O = oracle.Grid(0.04, 0.02).set(keys, g["sdf"], g["rgb"])
    rays = synth.view_rays(synth.random_poses(sc, 1, seed=3)[0], 10, 7, synth.intrinsics(10, 7)).numpy()
    rng = np.random.default_rng(0)
    t_rgb = rng.uniform(0, 1, (len(rays), 3))
    t_depth = rng.uniform(0.5, 2.0, len(rays))
    return O, rays, t_rgb, t_depth


def _shard_grad(O, rays, t_rgb, t_depth, a, b, n):
    """Oracle gradient of rays [a, b) of the batch, the loss a mean over all n rays of the batch."""
    import oracle
    out = O.render(rays[a:b], N_SAMPLES, seed=5, ray_id0=a)
    _, s = oracle.loss(out["rgb"], out["depth"], t_rgb[a:b], t_depth[a:b], 0.1)
    k = (b - a) / n  # oracle.loss means over its own rays: rescale to the batch's n
    g = O.backward(rays[a:b], N_SAMPLES, s["rgb"] * k, s["depth"] * k, seed=5, ray_id0=a)
    return np.concatenate([g["sdf"][..., None], g["rgb"]], -1)


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    O, rays, t_rgb, t_depth = _problem()
    a, b = shard_bounds(len(rays), rank, world)
    g = torch.from_numpy(_shard_grad(O, rays, t_rgb, t_depth, a, b, len(rays)))
    dist.all_reduce(g, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(out, g.numpy())
    dist.destroy_process_group()


def test_shard_bounds_cover_the_batch_once():
    for n in (0, 1, 5, 70, 1 << 18):
        for w in (1, 2, 3, 8):
            b = [shard_bounds(n, r, w) for r in range(w)]
            assert b[0][0] == 0 and b[-1][1] == n and all(b[i][1] == b[i + 1][0] for i in range(w - 1))
            assert max(y - x for x, y in b) - min(y - x for x, y in b) <= 1


def test_two_gloo_ranks_sum_to_the_whole_batch(tmp_path):
    out = str(tmp_path / "g.npy")
    port = 29500 + os.getpid() % 1000
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    O, rays, t_rgb, t_depth = _problem()
    want = _shard_grad(O, rays, t_rgb, t_depth, 0, len(rays), len(rays))
    assert np.abs(want).max() > 0
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-12 * np.abs(want).max())
