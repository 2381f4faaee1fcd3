"""Prepared training batches (sdg_train_prepare): a batch's ordering and traversal enqueued ahead on the grid's
auxiliary stream, beside the previous step's optimiser.  A pipeline of prepared steps over several batches (two
slots, each prepared after the previous step's training pass and before its optimiser step) must leave the
grid as the same steps unprepared do: per-ray loss terms bit-identical, gradients equal up to the order of FP32
accumulation.  Misuse is refused."""
import pytest
import torch

import synth
from tests.gpu_util import assert_grad_close, grad_arrays, make_pair

pytestmark = pytest.mark.gpu


def _batches(sc, k, W=96, H=72):
    out = []
    g = torch.Generator(device="cuda").manual_seed(7)
    for i in range(k):
        T = synth.random_poses(sc, 1, seed=20 + i)[0]
        rays = synth.view_rays(T, W, H, synth.intrinsics(W, H)).cuda()
        n = rays.shape[0]
        out.append((rays, torch.rand((n, 3), generator=g, device="cuda"), 2.0 * torch.rand(n, generator=g,
                                                                                          device="cuda")))
    return out


@pytest.mark.parametrize("order", ["given", "surface"])
def test_prepared_pipeline_equals_unprepared_steps(order):
    """Four batches through two slots, each prepared right after the previous batch's training pass; the same
    batches unprepared on a twin grid.  No optimiser step changes the voxels in between, so per-ray loss terms
    must be bit-identical and gradients equal up to the order of FP32 accumulation."""
    import paper_2305_13220_b300 as sdg
    sc = synth.scene_tiny_room(0)
    keys = synth.band_blocks(sc, 0.04, 3)
    Gp, _, _, _ = make_pair(sc, keys, 0.04, 3, 0.02)
    Gu, _, _, _ = make_pair(sc, keys, 0.04, 3, 0.02)
    batches = _batches(sc, 4)
    slot = 0
    sdg.train_prepare(Gp, batches[0][0], batches[0][2], slot, ray_order=order)
    for i, (rays, t_rgb, t_depth) in enumerate(batches):
        n = rays.shape[0]
        res = {}
        for G, tag in ((Gp, "p"), (Gu, "u")):
            G.zero_grad()
            loss = torch.full((n,), float("nan"), device="cuda")
            sdg.train_step_rays(G, rays, t_rgb, t_depth, n_samples=64, seed=i, loss=loss, ray_order=order,
                                prepared=slot if tag == "p" else None)
            if tag == "p" and i + 1 < len(batches):
                sdg.train_prepare(G, batches[i + 1][0], batches[i + 1][2], 1 - slot, ray_order=order)
            torch.cuda.synchronize()
            res[tag] = (loss, grad_arrays(G, G.num_blocks))
        slot = 1 - slot
        assert not torch.isnan(res["p"][0]).any()
        assert torch.equal(res["p"][0], res["u"][0])
        for k in ("sdf", "rgb"):
            assert_grad_close(res["p"][1][k], res["u"][1][k], what=k)


def test_prepared_slot_misuse_is_refused():
    import paper_2305_13220_b300 as sdg
    sc = synth.scene_tiny_room(0)
    keys = synth.band_blocks(sc, 0.04, 3)
    G, _, _, _ = make_pair(sc, keys, 0.04, 3, 0.02)
    (r0, c0, d0), (r1, c1, d1) = _batches(sc, 2, 16, 8)
    with pytest.raises(sdg.SdgError):  # nothing prepared
        sdg.train_step_rays(G, r0, c0, d0, n_samples=16, prepared=0)
    sdg.train_prepare(G, r0, d0, 0)
    with pytest.raises(sdg.SdgError):  # prepared for other rays
        sdg.train_step_rays(G, r1, c1, d1, n_samples=16, prepared=0)
    with pytest.raises(sdg.SdgError):
        sdg.train_prepare(G, r0, d0, 2)
    sdg.train_step_rays(G, r0, c0, d0, n_samples=16, prepared=0)
    with pytest.raises(sdg.SdgError):  # a prepared batch is used once
        sdg.train_step_rays(G, r0, c0, d0, n_samples=16, prepared=0)
    torch.cuda.synchronize()
