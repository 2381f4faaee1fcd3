"""Parity at the room workload's full size, in the launch configuration bench.py times.

The room-scale grid (6x6x3 m, 1 cm voxels, 4-voxel band) is activated on the GPU from all 50 synthetic 640x480
depth maps and compared bit-exactly with the oracle's key set; then the fused training pass runs on a full
2^18-ray batch with 128 samples per ray (surface-ordered, as timed), and sampled rays' losses and rendered
colour / depth / opacity, a subset's gradients (through the surface-ordered path and in the given order) and
sampled Adam updates are checked against the oracle one by one.  No ray is skipped: the oracle runs on the GPU's
own samples (sdg_debug_trace), whose placement is first checked against the oracle's FP64 traversal."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import assert_grad_close, check_placement, gpu_samples

pytestmark = pytest.mark.gpu

VS, BAND, W, H, N = 0.01, 4, 640, 480, 128


@pytest.fixture(scope="module")
def room():
    import paper_2305_13220_b300 as sdg
    sc = synth.scene_room(0)
    poses = synth.random_poses(sc, 50, seed=0)
    K = synth.intrinsics(W, H)
    depths = [synth.depth_map(sc, T, W, H, K, device="cuda") for T in poses]
    G = sdg.Grid(VS, 80_000, beta=0.5 * VS)
    for T, d in zip(poses, depths):
        G.activate_depth(d, K, T, BAND)
    gk = G.keys().cpu().numpy()
    vals = synth.fill_grid(sc, gk, VS, BAND, device="cuda")
    A = sdg._abi
    nb = len(gk)
    geo = G.channel(A.GROUP_GEO)
    geo[:nb, :, 0] = vals["sdf"].to(torch.float32)
    geo[:nb, :, 1:4] = vals["rgb"].to(torch.float32)
    del vals
    stored = geo[:nb].double().cpu().numpy()
    O = oracle.Grid(VS, 0.5 * VS).set(gk, stored[..., 0], stored[..., 1:4])
    return sdg, sc, poses, K, [d.cpu() for d in depths], G, O, gk


def test_full_activation_is_bit_exact(room):
    sdg, sc, poses, K, depths, G, O, gk = room
    # oracle: per batch (one depth map each), new keys in ascending (z, y, x) order
    ks = oracle.KeySet()
    order = []
    seen = set()
    for T, d in zip(poses, depths):
        ks.add_depth(d, K, T, VS, BAND)
        for k in map(tuple, ks.keys().tolist()):
            if k not in seen:
                seen.add(k)
                order.append(k)
    np.testing.assert_array_equal(np.array(order, np.int32), gk)
    assert len(gk) > 40_000


def test_full_batch_sampled_rays_match_oracle(room):
    """The timed launch: 2^18 rays in surface order.  256 sampled rays' loss terms from that launch, and their
    rendered colour / depth / opacity from a full-batch forward, against the oracle over the GPU's samples."""
    sdg, sc, poses, K, depths, G, O, gk = room
    b = synth.training_batch(sc, poses, W, H, K, 1 << 18, seed=7, device="cuda", order="pixel")
    n = b["rays"].shape[0]
    loss = torch.empty(n, device="cuda")
    G.zero_grad()
    sdg.train_step_rays(G, b["rays"], b["rgb"], b["depth"], n_samples=N, seed=3, loss=loss)
    tr = sdg.trace(G, b["rays"], N, seed=3)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(n, 256, replace=False))
    sel = torch.as_tensor(idx, device="cuda")
    rays = b["rays"].cpu().numpy()
    t_rgb = b["rgb"].double().cpu().numpy()
    t_d = b["depth"].double().cpu().numpy()
    got = loss.double().cpu().numpy()
    sub = {k: v[sel] for k, v in tr.items()}
    assert (sub["n_cells"] >= 0).float().mean() > 0.9  # most rays placed from the traversal pass's records
    for j, i in enumerate(idx):
        one = {k: v[j:j + 1] for k, v in sub.items()}
        check_placement(O, rays[i:i + 1], one, N, seed=3, ray_id0=int(i))
        ref = O.render(rays[i:i + 1], N, seed=3, ray_id0=int(i), given=gpu_samples(one))
        for k in ("rgb", "depth", "opac"):
            assert np.abs(one[k].double().cpu().numpy() - ref[k]).max() <= 1e-4, (i, k)
        # per-ray loss term: (sum |C - C^| / 3 + 0.1 |D - D^|) / n, |dL_i| <= (|dC| + 0.1 |dD|) / n
        e = np.abs(ref["rgb"][0] - t_rgb[i]).sum() / 3 + 0.1 * abs(ref["depth"][0] - t_d[i])
        assert abs(got[i] * n - e) <= 2e-4, (i, got[i] * n, e)


def test_overflow_rays_match_oracle(room):
    """Rays crossing more allocated cells than a traversal record holds (32) are rendered by the in-warp kernel
    after the records kernel: in the timed launch (surface order), their loss terms and rendered outputs against
    the oracle over the GPU's samples."""
    sdg, sc, poses, K, depths, G, O, gk = room
    b = synth.training_batch(sc, poses, W, H, K, 1 << 18, seed=7, device="cuda", order="pixel")
    n = b["rays"].shape[0]
    loss = torch.empty(n, device="cuda")
    G.zero_grad()
    sdg.train_step_rays(G, b["rays"], b["rgb"], b["depth"], n_samples=N, seed=3, loss=loss)
    tr = sdg.trace(G, b["rays"], N, seed=3)
    torch.cuda.synchronize()
    ov = np.flatnonzero(tr["n_cells"].cpu().numpy() < 0)
    assert 50 < len(ov) < n // 100, len(ov)
    sel = ov[np.random.default_rng(3).choice(len(ov), 48, replace=False)]
    rays = b["rays"].cpu().numpy()
    t_rgb, t_d = b["rgb"].double().cpu().numpy(), b["depth"].double().cpu().numpy()
    got = loss.double().cpu().numpy()
    for i in np.sort(sel):
        one = {k: v[int(i):int(i) + 1] for k, v in tr.items()}
        check_placement(O, rays[i:i + 1], one, N, seed=3, ray_id0=int(i))
        ref = O.render(rays[i:i + 1], N, seed=3, ray_id0=int(i), given=gpu_samples(one))
        assert ref["S"][0] > 0
        for k in ("rgb", "depth", "opac"):
            assert np.abs(one[k].double().cpu().numpy() - ref[k]).max() <= 1e-4, (i, k)
        e = np.abs(ref["rgb"][0] - t_rgb[i]).sum() / 3 + 0.1 * abs(ref["depth"][0] - t_d[i])
        assert abs(got[i] * n - e) <= 2e-4, (i, got[i] * n, e)


@pytest.mark.parametrize("order", ["surface", "given"])
def test_subset_gradients_match_oracle(room, order):
    """Gradients of a 2048-ray subset of the full batch, through the surface-ordered path the timed launch takes
    (ray_order = surface) and in the given order, against the oracle over the GPU's samples."""
    sdg, sc, poses, K, depths, G, O, gk = room
    b = synth.training_batch(sc, poses, W, H, K, 1 << 18, seed=8, device="cuda", order="pixel")
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(1 << 18, 2048, replace=False))
    rays = b["rays"].cpu().numpy()[idx]
    rd = torch.as_tensor(rays, device="cuda")
    tr = sdg.trace(G, rd, N, stratified=False)
    check_placement(O, rays, tr, N, stratified=False)
    gv = gpu_samples(tr)
    ref = O.render(rays, N, stratified=False, given=gv)
    n = len(rays)
    t_rgb = ref["rgb"] + rng.choice([-0.05, 0.05], size=(n, 3))
    t_depth = ref["depth"] + rng.choice([-0.1, 0.1], size=n)
    _, seeds = oracle.loss(ref["rgb"], ref["depth"], t_rgb, t_depth, 0.1)
    want = O.backward(rays, N, seeds["rgb"], seeds["depth"], stratified=False, given=gv)
    G.zero_grad()
    sdg.train_step_rays(G, rd, torch.as_tensor(t_rgb, dtype=torch.float32, device="cuda"),
                        torch.as_tensor(t_depth, dtype=torch.float32, device="cuda"), n_samples=N, stratified=False,
                        ray_order=order)
    torch.cuda.synchronize()
    A = sdg._abi
    got = G.channel(A.GROUP_GEO, A.KIND_GRAD)[:len(gk)].double().cpu().numpy()
    touched = np.unique(np.nonzero(np.abs(want["sdf"]) + np.abs(want["rgb"]).sum(-1))[0])
    assert len(touched) > 100
    assert_grad_close(got[touched, :, 0], want["sdf"][touched], what="sdf")
    assert_grad_close(got[touched, :, 1:4], want["rgb"][touched], what="rgb")
    untouched = np.setdiff1d(np.arange(len(gk)), touched)
    assert np.abs(got[untouched]).max() == 0


def test_full_size_adam_sampled_voxels(room):
    sdg, sc, poses, K, depths, G, O, gk = room
    A = sdg._abi
    nb = len(gk)
    geo, grad = G.channel(A.GROUP_GEO), G.channel(A.GROUP_GEO, A.KIND_GRAD)
    m, v = G.channel(A.GROUP_GEO, A.KIND_ADAM_M), G.channel(A.GROUP_GEO, A.KIND_ADAM_V)
    torch.manual_seed(0)
    grad[:nb] = torch.randn_like(grad[:nb]) * 1e-3
    m[:nb] = 0
    v[:nb] = 0
    G.step = 0
    sel = torch.as_tensor(np.random.default_rng(2).choice(nb * 512, 4096, replace=False), device="cuda")
    flat = lambda t: t[:nb].reshape(-1, 4)
    th0, g0 = flat(geo)[sel].double().cpu().numpy().reshape(-1), flat(grad)[sel].double().cpu().numpy().reshape(-1)
    G.adam_step(lr=1e-3)
    torch.cuda.synchronize()
    th, gg, mo, vo = th0.copy(), g0.copy(), np.zeros_like(th0), np.zeros_like(th0)
    oracle.adam(th, gg, mo, vo, lr=1e-3, step=1)
    np.testing.assert_allclose(flat(geo)[sel].double().cpu().numpy().reshape(-1), th, rtol=0, atol=2e-7)
    assert torch.all(grad[:nb] == 0)
