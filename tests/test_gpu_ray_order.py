"""Processing order of a training batch (sdg_train_step_rays, ray_order): a ray's samples, loss term and gradient
contributions do not depend on the order in which the batch is processed.  Surface order against the given order:
per-ray loss terms bit-identical (the loss buffer starts as NaN, so every ray was processed), summed loss identical
(deterministic reduction of the same terms), gradients equal up to the order of FP32 accumulation."""
import numpy as np
import pytest
import torch

import synth
from tests.gpu_util import assert_grad_close, grad_arrays, tiny_room

pytestmark = pytest.mark.gpu


def _run(sdg, G, rays, t_rgb, t_depth, order, n_samples=64):
    n = rays.shape[0]
    loss = torch.full((n,), float("nan"), device="cuda")
    s = torch.zeros(1, device="cuda")
    G.zero_grad()
    sdg.train_step_rays(G, rays, t_rgb, t_depth, n_samples=n_samples, seed=5, loss=loss, loss_sum=s,
                        ray_order=order)
    torch.cuda.synchronize()
    return loss.cpu().numpy(), s.item(), grad_arrays(G, max(G.num_blocks, 1))


def _compare(sdg, G, rays, t_rgb, t_depth, order="surface"):
    l0, s0, g0 = _run(sdg, G, rays, t_rgb, t_depth, "given")
    l1, s1, g1 = _run(sdg, G, rays, t_rgb, t_depth, order)
    finite = np.isfinite(t_depth.cpu().numpy())
    assert not np.isnan(l1[finite]).any()
    np.testing.assert_array_equal(l1, l0)
    assert s1 == s0 or (np.isnan(s1) and np.isnan(s0))
    for k in g0:
        if np.abs(g0[k]).max() == 0:  # no ray reached an allocated voxel
            assert np.abs(g1[k]).max() == 0, k
        else:
            assert_grad_close(g1[k], g0[k], what=k)
    return l1


@pytest.fixture(scope="module")
def sdg():
    import paper_2305_13220_b300 as m
    return m


@pytest.mark.parametrize("n", [1, 777, 8192, 65536])
def test_surface_order_matches_given_order(sdg, n):
    sc, G, O, _, _ = tiny_room()
    poses = synth.random_poses(sc, 6, seed=2)
    K = synth.intrinsics(64, 48)
    b = synth.training_batch(sc, poses, 64, 48, K, n, seed=3, device="cuda")
    _compare(sdg, G, b["rays"], b["rgb"], b["depth"])
    if n == 65536:  # the automatic choice at this size is the surface order
        _compare(sdg, G, b["rays"], b["rgb"], b["depth"], order="auto")


def test_rays_without_a_usable_target_depth(sdg):
    """NaN, infinite, zero and negative target depths take the last bucket; the rays still run once each."""
    sc, G, O, _, _ = tiny_room()
    poses = synth.random_poses(sc, 3, seed=4)
    K = synth.intrinsics(32, 24)
    b = synth.training_batch(sc, poses, 32, 24, K, 2048, seed=6, device="cuda")
    d = b["depth"].clone()
    d[::7] = float("nan")
    d[1::11] = float("inf")
    d[2::13] = 0.0
    d[3::17] = -1.0
    l1 = _compare(sdg, G, b["rays"], b["rgb"], d)
    dn = d.cpu().numpy()
    assert np.isnan(l1[np.isnan(dn)]).all()  # |depth - NaN| is NaN: the term is reported as is
    assert np.isinf(l1[np.isinf(dn)]).all()


def test_empty_grid_runs_in_given_order(sdg):
    G = sdg.Grid(0.04, 16, beta=0.02)
    rays = synth.pack_rays(torch.zeros(300, 3, dtype=torch.float64),
                           torch.nn.functional.normalize(torch.randn(300, 3, dtype=torch.float64), dim=-1),
                           0.0, 10.0).cuda()
    t_rgb = torch.rand(300, 3, device="cuda")
    t_depth = torch.rand(300, device="cuda") * 3
    _compare(sdg, G, rays, t_rgb, t_depth)


@pytest.mark.parametrize("span", [256, 5000])
def test_wide_grids_coarsen_the_buckets(sdg, span):
    """A block AABB 256 blocks wide needs 18 Morton bits (buckets merge 8 codes); 5000 wide also needs coarser
    cells to fit 10 bits per axis.  The order changes, the results do not."""
    keys = np.array([[0, 0, 0], [span - 1, 0, 0], [0, 40, 0], [0, 0, 40], [span // 2, 20, 20]], np.int32)
    G = sdg.Grid(0.04, 64, beta=0.02)
    G.activate_keys(torch.as_tensor(keys, device="cuda"))
    geo = G.channel(sdg._abi.GROUP_GEO)
    torch.manual_seed(0)
    geo[:5] = torch.rand_like(geo[:5]) - 0.5
    rays = synth.random_rays_through(keys, 0.04, 4096, seed=1).cuda()
    t_rgb = torch.rand(4096, 3, device="cuda")
    t_depth = torch.rand(4096, device="cuda") * span * 0.32
    _compare(sdg, G, rays, t_rgb, t_depth)


def test_unknown_order_is_rejected(sdg):
    sc, G, O, _, _ = tiny_room()
    A = sdg._abi
    import ctypes as C
    rays = torch.zeros(4, 8, device="cuda")
    rays[:, 6] = 1.0
    rays[:, 7] = 1.0
    t = torch.zeros(4, 3, device="cuda")
    td = torch.zeros(4, device="cuda")
    o = sdg.render_opts(16)
    lo = A.LossOpts(lambda_depth=0.1, lambda_sem=0.1, ray_order=7)
    rc = A.lib().sdg_train_step_rays(G.handle, rays.data_ptr(), 4, t.data_ptr(), td.data_ptr(), None, C.byref(o),
                                     C.byref(lo), None, None)
    assert rc == A.ERR_ARG
    assert b"ray_order" in A.lib().sdg_last_error()
    with pytest.raises(ValueError):
        sdg.train_step_rays(G, rays, t, td, ray_order="sorted")
