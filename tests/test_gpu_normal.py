"""The fused training pass with the normal loss (Eq. 14, grad f of Eq. 17 at every sample) against the oracle:
loss terms and voxel gradients, in both storage layouts; with lambda_normal = 0 it reduces to the plain pass."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import assert_grad_close, check_placement, gpu_samples, grad_arrays, tiny_room

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sdg():
    import paper_2305_13220_b300 as m
    return m


def _dev(x):
    return torch.as_tensor(x, dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("rgb_dtype", ["f32", "bf16"])
def test_normal_loss_matches_oracle(sdg, rgb_dtype):
    sc, G, O, _, _ = tiny_room(rgb_dtype=rgb_dtype)
    P = synth.random_poses(sc, 1, seed=12)
    rays = synth.view_rays(P[0], 64, 48, synth.intrinsics(64, 48))
    # every ray: the oracle runs on the GPU's own samples (placement checked against the oracle's first)
    tr = sdg.trace(G, rays.cuda(), 64, stratified=False)
    check_placement(O, rays, tr, 64, stratified=False)
    gv = gpu_samples(tr)
    ref = O.render(rays, 64, stratified=False, given=gv)
    n = rays.shape[0]
    rng = np.random.default_rng(1)
    t_rgb = ref["rgb"] + rng.choice([-0.05, 0.05], size=(n, 3))
    t_depth = ref["depth"] + rng.choice([-0.1, 0.1], size=n)
    t_normal = ref["normal"] + rng.choice([-0.05, 0.05], size=(n, 3))
    L1, seeds = oracle.loss(ref["rgb"], ref["depth"], t_rgb, t_depth, 0.1)
    Ln, gN = oracle.loss_normal(ref["normal"], t_normal, 0.05)
    want = O.backward(rays, 64, seeds["rgb"], seeds["depth"], stratified=False, g_normal=gN, given=gv)
    assert np.abs(gN).max() > 0 and np.abs(ref["normal"]).max() > 0.5
    G.zero_grad()
    loss = torch.empty(n, device="cuda")
    sdg.train_step_rays_normal(G, rays.cuda(), _dev(t_rgb), _dev(t_depth), _dev(t_normal), n_samples=64,
                               stratified=False, lambda_normal=0.05, loss=loss)
    torch.cuda.synchronize()
    assert loss.sum().item() == pytest.approx(L1 + Ln, rel=1e-4)
    got = grad_arrays(G, G.num_blocks)
    assert_grad_close(got["sdf"], want["sdf"], what="sdf")
    assert_grad_close(got["rgb"], want["rgb"], what="rgb")
    # lambda_normal = 0: the plain fused pass
    G.zero_grad()
    sdg.train_step_rays_normal(G, rays.cuda(), _dev(t_rgb), _dev(t_depth), _dev(t_normal), n_samples=64,
                               stratified=False, lambda_normal=0.0)
    zero = grad_arrays(G, G.num_blocks)
    G.zero_grad()
    sdg.train_step_rays(G, rays.cuda(), _dev(t_rgb), _dev(t_depth), n_samples=64, stratified=False)
    plain = grad_arrays(G, G.num_blocks)
    assert_grad_close(zero["sdf"], plain["sdf"], rel=1e-5, floor=1e-5, what="sdf (lambda_n = 0)")


def test_normal_pass_rejects_what_it_does_not_support(sdg):
    sc, G, O, _, _ = tiny_room(n_sem=4)
    r = torch.zeros((4, 8), device="cuda")
    r[:, 6] = 1.0
    r[:, 7] = 1.0
    t3, t1 = torch.zeros((4, 3), device="cuda"), torch.zeros(4, device="cuda")
    with pytest.raises(sdg.SdgError):
        sdg.train_step_rays_normal(G, r, t3, t1, t3, n_samples=16)
