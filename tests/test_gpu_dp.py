"""The ray-sharded data-parallel step on one GPU, ranks emulated by replicas (no kernel waits on another): two
grids holding the same voxels each run dp.shard_train on their shard of one batch, their gradient channels are
summed (what the all-reduce does across GPUs), both take the optimiser step; the summed gradient must equal the
whole batch's gradient from one grid, and both replicas must end bit-identical to each other and equal to the
unsharded step where the gradient is not at FP32 noise level (Adam's first step is sign-like there)."""
import numpy as np
import pytest
import torch

import synth
from paper_2305_13220_b300 import dp
from tests.gpu_util import assert_grad_close, make_pair

pytestmark = pytest.mark.gpu


def test_sharded_step_equals_unsharded_step():
    import paper_2305_13220_b300 as sdg
    A = sdg._abi
    sc = synth.scene_tiny_room(0)
    keys = synth.band_blocks(sc, 0.04, 3)
    grids = [make_pair(sc, keys, 0.04, 3, 0.02)[0] for _ in range(3)]  # rank 0, rank 1, unsharded
    rays = synth.view_rays(synth.random_poses(sc, 1, seed=9)[0], 64, 48, synth.intrinsics(64, 48)).cuda()
    n = rays.shape[0]
    g = torch.Generator(device="cuda").manual_seed(2)
    t_rgb = torch.rand((n, 3), generator=g, device="cuda")
    t_depth = 2.0 * torch.rand(n, generator=g, device="cuda")
    for G in grids:
        G.zero_grad()
        G.step = 0
    shards = [dp.shard_train(grids[r], rays, t_rgb, t_depth, r, 2, n_samples=64, seed=4) for r in range(2)]
    assert shards == [(0, n // 2), (n // 2, n)]
    sdg.train_step_rays(grids[2], rays, t_rgb, t_depth, n_samples=64, seed=4)
    torch.cuda.synchronize()
    # the all-reduce, emulated: sum the two ranks' gradient channels into both
    for t0, t1 in zip(dp.grad_tensors(grids[0]), dp.grad_tensors(grids[1])):
        s = t0 + t1
        t0.copy_(s)
        t1.copy_(s)
    whole = dp.grad_tensors(grids[2])[0].double().cpu().numpy()
    summed = dp.grad_tensors(grids[0])[0].double().cpu().numpy()
    assert_grad_close(summed[..., 0], whole[..., 0], what="sdf")
    assert_grad_close(summed[..., 1:], whole[..., 1:], what="rgb")
    for G in grids:
        G.adam_step(lr=1e-3)
    torch.cuda.synchronize()
    th = [G.channel(A.GROUP_GEO)[:G.num_blocks].double().cpu().numpy() for G in grids]
    assert np.array_equal(th[0], th[1])
    big = np.abs(whole) > 1e-3 * np.abs(whole).max()
    assert big.sum() > 1000
    np.testing.assert_allclose(th[0][big], th[2][big], rtol=0, atol=1e-6)
