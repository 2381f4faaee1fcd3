"""Rays crossing more allocated block cells than the records kernel takes (32): with up to 64 they are rendered from
their records two per lane (the mid list), with more walked in-warp (the overflow list).  A slab of 40 blocks sends
every ray to the mid list, one of 80 to the overflow list; there a pass whose list is longer than the strided
overflow kernel takes in one turn renders its first entries with one warp each (sized from the list length the
grid's previous pass left), the rest with the strided kernel.  The outputs equal the trace's bit for bit (the
trace takes the strided kernels), and the oracle over the trace's samples."""
import numpy as np
import pytest
import torch

import synth
from tests.gpu_util import (assert_grad_close, assert_trace_equals_render, check_placement, gpu_samples,
                            grad_arrays, make_pair)

pytestmark = pytest.mark.gpu

N = 64


@pytest.fixture(scope="module", params=[40, 80], ids=["mid-list", "overflow-list"])
def slab(request):
    import paper_2305_13220_b300 as sdg
    # L x 3 x 3 allocated blocks (0.04 m voxels, 0.32 m blocks) viewed down x from one end through a narrow field
    # of view: every ray crosses about L + 1 cells
    L = request.param
    sc = synth.scene_room(0, size=(0.32 * L + 1.0, 2.0, 2.0), n_objects=0)
    keys = np.array([(x, y, z) for x in range(L) for y in range(3) for z in range(3)], np.int32)
    G, O, _, _ = make_pair(sc, keys, 0.04, 3, 0.02, "f32")
    T = np.array([[0.0, 0.0, 1.0, 0.1], [1.0, 0.0, 0.0, 0.48], [0.0, 1.0, 0.0, 0.48]])
    W = H = 80  # 6,400 rays, more than the strided kernel's 4,736 warps
    rays = synth.view_rays(T, W, H, synth.intrinsics(W, H, fov_deg=1.5))
    return sdg, G, O, rays


def test_long_overflow_list_forward(slab):
    sdg, G, O, rays = slab
    r = rays.cuda()
    sdg.render(G, r[:100].contiguous(), N, seed=2)  # a short list: the next pass takes the strided kernel
    first = sdg.render(G, r, N, seed=2)   # leaves the list length as the next pass's hint
    second = sdg.render(G, r, N, seed=2)  # its overflow list goes to the one-warp-per-entry kernel
    tr = sdg.trace(G, r, N, seed=2)
    torch.cuda.synchronize()
    assert int((tr["n_cells"] < 0).sum()) == rays.shape[0]
    assert_trace_equals_render(tr, first)
    assert_trace_equals_render(tr, second)
    rn = rays.numpy()
    for i in np.arange(0, rays.shape[0], 263):  # the oracle on a spread of 25 rays
        t1 = {k: v[int(i):int(i) + 1] for k, v in tr.items()}
        check_placement(O, rn[i:i + 1], t1, N, seed=2, ray_id0=int(i))
        ref = O.render(rn[i:i + 1], N, seed=2, ray_id0=int(i), given=gpu_samples(t1))
        for k in ("rgb", "depth", "opac"):
            assert np.abs(second[k][int(i):int(i) + 1].double().cpu().numpy() - ref[k]).max() <= 1e-4, (i, k)


def test_long_overflow_list_training(slab):
    """Two fused training passes over the same rays: the first renders the overflow list with the strided kernel,
    the second (with the hint) one warp per entry; per-ray losses are equal bit for bit and the gradients within
    the order of the FP32 atomic sums."""
    sdg, G, O, rays = slab
    r = rays.cuda()
    out = sdg.render(G, r, N, seed=4)
    t_rgb = (out["rgb"] + 0.05).contiguous()
    t_depth = (out["depth"] - 0.1).contiguous()
    n = rays.shape[0]
    sdg.render(G, r[:100].contiguous(), N, seed=4)  # a short list: the first pass takes the strided kernel
    losses, grads = [], []
    for _ in range(2):
        G.zero_grad()
        loss = torch.empty(n, device="cuda")
        sdg.train_step_rays(G, r, t_rgb, t_depth, n_samples=N, seed=4, loss=loss, ray_order="given")
        torch.cuda.synchronize()
        losses.append(loss.cpu())
        grads.append(grad_arrays(G, G.num_blocks))
    assert torch.equal(losses[0], losses[1])
    for k in ("sdf", "rgb"):
        assert_grad_close(grads[1][k], grads[0][k], rel=1e-5, floor=1e-5, what=k)
