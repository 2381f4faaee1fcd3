"""GPU parity of the rendering path (Sec. 3.5.1, Eq. 12-15; trilinear Eq. 17) against the FP64 oracle.

Tolerances (FP32 on the GPU vs FP64): rendered colour / depth / opacity max-abs 1e-4; gradients relative 1e-3
elementwise with a floor of 1e-5 of the channel's largest entry (FP32 atomics sum in arbitrary order).

Every ray is compared.  The GPU exports where it placed each sample (sdg_debug_trace); check_placement asserts
that this placement is the oracle's own up to FP32 rounding (a sample on a joint between allocated stretches may
sit at either end of the joint, a cell at either side of a face within rounding), and the oracle, fed those
samples, computes everything after the placement for every ray: forward outputs and the whole batch's gradients.
Rays the oracle's own placement reproduces are also compared with the plain oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import (assert_forward_all_rays, assert_grad_close, assert_trace_equals_render,
                            check_placement, gpu_samples, grad_arrays, tiny_room)

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def sdg():
    import paper_2305_13220_b300 as m
    return m


@pytest.fixture(scope="module")
def room():
    return tiny_room()


def _view(sc, W=64, H=48, seed=0):
    T = synth.random_poses(sc, 1, seed=seed)[0]
    return synth.view_rays(T, W, H, synth.intrinsics(W, H))


def _cmp_forward(out, ref, nd, ns=0):
    """Rays the oracle's own placement reproduces (not flagged degenerate) against the plain oracle."""
    for k in ("rgb", "depth", "opac") + (("sem",) if ns else ()):
        got = out[k].double().cpu().numpy()
        d = np.abs(got - ref[k])[nd]
        lim = TOL * 10 if k == "sem" else TOL   # logits reach ~5 in magnitude
        assert d.size == 0 or d.max() <= lim, (k, d.max())


def _all_rays(sdg, G, O, rays, N, seed=0, stratified=True, bg=(0, 0, 0), ns=0, ray_id0=0):
    """Forward of every ray against the oracle fed the GPU's samples, after checking the placement; returns the
    trace and the oracle's plain render (for the non-degenerate comparison)."""
    out = sdg.render(G, rays.cuda(), N, seed=seed, stratified=stratified, bg=bg, ray_id0=ray_id0)
    tr = sdg.trace(G, rays.cuda(), N, seed=seed, stratified=stratified, bg=bg, ray_id0=ray_id0)
    assert_trace_equals_render(tr, out)
    n_joint, n_tie = check_placement(O, rays, tr, N, seed=seed, ray_id0=ray_id0, stratified=stratified)
    given = O.render(rays, N, seed=seed, stratified=stratified, bg=bg, ray_id0=ray_id0, given=gpu_samples(tr))
    assert np.array_equal(given["n_valid"], tr["valid"].sum(1).double().cpu().numpy())  # same validity decisions
    assert_forward_all_rays(out, given, TOL, ns)
    ref = O.render(rays, N, seed=seed, stratified=stratified, bg=bg, ray_id0=ray_id0)
    _cmp_forward(out, ref, ~ref["degenerate"], ns)
    print(f"rays {len(rays)}: oracle-degenerate {ref['degenerate'].mean():.4f}, joint samples in {n_joint}, "
          f"cell ties in {n_tie}")
    return tr, ref


@pytest.mark.parametrize("stratified,bg", [(True, (0, 0, 0)), (False, (0.2, 0.5, 0.9)), (True, (1, 1, 1))])
def test_forward_matches_oracle(sdg, room, stratified, bg):
    sc, G, O, _, _ = room
    rays = _view(sc)
    tr, ref = _all_rays(sdg, G, O, rays, 64, seed=5, stratified=stratified, bg=bg)
    assert ref["opac"].max() > 0.99 and ref["n_valid"].mean() > 30


@pytest.mark.parametrize("N", [1, 17, 48, 100, 128, 192, 256])
def test_forward_sample_counts(sdg, room, N):
    sc, G, O, _, _ = room
    rays = _view(sc, 24, 16, seed=1)
    _all_rays(sdg, G, O, rays, N, seed=9)


def test_in_warp_traversal_matches_oracle(sdg, room):
    """The in-warp traversal (serving loop, allocation-free pass): every ray against the oracle fed its samples."""
    sc, G, O, _, _ = room
    rays = _view(sc, 48, 32, seed=3)
    tr = sdg.trace(G, rays.cuda(), 128, seed=2, walk="in_warp")
    assert (tr["n_cells"] == -1).all()
    check_placement(O, rays, tr, 128, seed=2)
    given = O.render(rays, 128, seed=2, given=gpu_samples(tr))
    assert_forward_all_rays(tr, given, TOL)


def test_rays_missing_the_grid_and_empty_batches(sdg, room):
    sc, G, O, _, _ = room
    r = np.array([[10, 10, 10, 0, 1, 0, 0, 100], [-5, 1, 1, 0.0, 1, 0, 0, 0.01],  # misses; too short to reach
                  [1, 1, 1, 5.0, 1, 0, 0, 4.0]], np.float32)                           # tnear > tfar
    out = sdg.render(G, torch.as_tensor(r, device="cuda"), 64, bg=(0.3, 0.2, 0.1))
    np.testing.assert_allclose(out["rgb"].cpu().numpy(), np.tile([0.3, 0.2, 0.1], (3, 1)), atol=1e-7)
    assert torch.all(out["depth"] == 0) and torch.all(out["opac"] == 0)
    out0 = sdg.render(G, torch.zeros((0, 8), device="cuda"), 64)
    assert out0["rgb"].shape == (0, 3)
    E = sdg.Grid(0.04, 16)
    oute = sdg.render(E, torch.as_tensor(r, device="cuda"), 64)
    assert torch.all(oute["opac"] == 0)


@pytest.mark.parametrize("mode", ["recompute", "store"])
@pytest.mark.parametrize("stratified", [True, False])
@pytest.mark.parametrize("N", [64, 192])  # 192: 6 samples per lane, where the forward reuses a cell's corners
def test_backward_matches_oracle(sdg, room, mode, stratified, N):
    """The whole batch's gradients against the oracle's backward over the GPU's samples (no ray left out)."""
    sc, G, O, _, _ = room
    rays = _view(sc, seed=2)
    bg = (0.3, 0.1, 0.7)
    n = len(rays)
    gen = torch.Generator().manual_seed(0)
    gc, gd, go = (torch.randn(s, generator=gen) for s in ((n, 3), (n,), (n,)))
    tr = sdg.trace(G, rays.cuda(), N, seed=3, stratified=stratified, bg=bg)
    check_placement(O, rays, tr, N, seed=3, stratified=stratified)
    G.zero_grad()
    o = sdg.render(G, rays.cuda(), N, seed=3, stratified=stratified, bg=bg, want_ctx=True, mode=mode)
    sdg.backward(o["ctx"], gc.cuda(), gd.cuda(), go.cuda())
    o["ctx"].release()
    torch.cuda.synchronize()
    got = grad_arrays(G, G.num_blocks)
    want = O.backward(rays.numpy(), N, gc.double().numpy(), gd.double().numpy(), go.double().numpy(), seed=3,
                      stratified=stratified, bg=bg, given=gpu_samples(tr))
    assert_grad_close(got["sdf"], want["sdf"], what="sdf")
    assert_grad_close(got["rgb"], want["rgb"], what="rgb")


@pytest.mark.parametrize("N", [128, 256])
def test_store_and_recompute_agree(sdg, room, N):
    """At 256 samples (8 per lane) both forwards reuse a cell's corners and the recompute backward does not."""
    sc, G, O, _, _ = room
    rays = _view(sc, seed=4).cuda()
    n = rays.shape[0]
    g = torch.randn((n, 3), device="cuda"), torch.randn(n, device="cuda"), torch.randn(n, device="cuda")
    res = {}
    for mode in ("recompute", "store"):
        G.zero_grad()
        o = sdg.render(G, rays, N, seed=1, want_ctx=True, mode=mode)
        sdg.backward(o["ctx"], *g)
        res[mode] = grad_arrays(G, G.num_blocks)
        res[mode + "_out"] = o["rgb"].clone()
    assert torch.allclose(res["recompute_out"], res["store_out"], rtol=0, atol=1e-6)
    for k in ("sdf", "rgb"):
        # the two modes compute the same per-sample values; only the FP32 atomic summation order differs
        assert_grad_close(res["store"][k], res["recompute"][k], rel=1e-5, floor=1e-5, what=k)


def test_autograd_function_accumulates_same_gradients(sdg, room):
    sc, G, O, _, _ = room
    A = sdg._abi
    rays = _view(sc, 32, 24, seed=5).cuda()
    n = rays.shape[0]
    w = torch.randn((n, 3), device="cuda"), torch.randn(n, device="cuda"), torch.randn(n, device="cuda")
    G.zero_grad()
    o = sdg.render(G, rays, 64, seed=2, want_ctx=True)
    sdg.backward(o["ctx"], *w)
    explicit = G.channel(A.GROUP_GEO, A.KIND_GRAD)[:G.num_blocks].clone()
    G.zero_grad()
    R = sdg.DifferentiableRenderer(G)
    rgb, depth, opac = R(rays, 64, seed=2)
    loss = (rgb * w[0]).sum() + (depth * w[1]).sum() + (opac * w[2]).sum()
    loss.backward()
    torch.cuda.synchronize()
    viaauto = G.channel(A.GROUP_GEO, A.KIND_GRAD)[:G.num_blocks]
    assert torch.allclose(viaauto, explicit, rtol=1e-5, atol=1e-6 * explicit.abs().max().item())
    assert explicit.abs().max() > 0


def test_fused_train_step_matches_oracle(sdg, room):
    """Fused forward + L1 losses + backward over every ray of a view, against the oracle over the GPU's samples."""
    sc, G, O, _, _ = room
    rays = _view(sc, seed=6)
    tr = sdg.trace(G, rays.cuda(), 64, stratified=False)
    check_placement(O, rays, tr, 64, stratified=False)
    gv = gpu_samples(tr)
    ref = O.render(rays, 64, stratified=False, given=gv)
    n = rays.shape[0]
    rng = np.random.default_rng(0)
    t_rgb = ref["rgb"] + rng.choice([-0.05, 0.05], size=(n, 3))
    t_depth = ref["depth"] + rng.choice([-0.1, 0.1], size=n)
    L, seeds = oracle.loss(ref["rgb"], ref["depth"], t_rgb, t_depth, 0.1)
    want = O.backward(rays, 64, seeds["rgb"], seeds["depth"], stratified=False, given=gv)
    G.zero_grad()
    loss = torch.empty(n, device="cuda")
    lsum = torch.empty(1, device="cuda")
    sdg.train_step_rays(G, rays.cuda(), torch.as_tensor(t_rgb, dtype=torch.float32, device="cuda"),
                        torch.as_tensor(t_depth, dtype=torch.float32, device="cuda"), n_samples=64,
                        stratified=False, loss=loss, loss_sum=lsum)
    torch.cuda.synchronize()
    assert lsum.item() == pytest.approx(L, rel=1e-4)
    assert lsum.item() == pytest.approx(loss.sum().item(), rel=1e-5)
    got = grad_arrays(G, G.num_blocks)
    assert_grad_close(got["sdf"], want["sdf"], what="sdf")
    assert_grad_close(got["rgb"], want["rgb"], what="rgb")
    # the unfused path (forward, loss kernel, backward) gives the same gradients
    G.zero_grad()
    o = sdg.render(G, rays.cuda(), 64, stratified=False, want_ctx=True)
    lv, gs = sdg.loss_l1(G, o["rgb"], o["depth"], torch.as_tensor(t_rgb, dtype=torch.float32, device="cuda"),
                         torch.as_tensor(t_depth, dtype=torch.float32, device="cuda"))
    sdg.backward(o["ctx"], gs["rgb"], gs["depth"])
    unf = grad_arrays(G, G.num_blocks)
    assert_grad_close(unf["sdf"], got["sdf"], rel=1e-5, floor=1e-5, what="unfused sdf")
    assert lv.sum().item() == pytest.approx(L, rel=1e-4)


# (layout, logits per voxel): the render program is unrolled for 20 semantic channels (n_sem <= 20) or for 32
# (n_sem 24-32); both capacities run in both colour layouts
SEM_CASES = [("bf16", 8), ("bf16", 20), ("f32", 20), ("bf16", 32), ("f32", 24)]


@pytest.mark.parametrize("layout,n_sem", SEM_CASES)
def test_semantics_match_oracle(sdg, layout, n_sem):
    sc, G, O, stored, vals = tiny_room(layout, n_sem)
    rays = _view(sc, 48, 32, seed=7)
    tr, _ = _all_rays(sdg, G, O, rays, 64, seed=4, ns=n_sem)
    n = len(rays)
    gen = torch.Generator().manual_seed(1)
    seeds = tuple(torch.randn(s, generator=gen) for s in ((n, 3), (n,), (n,), (n, n_sem)))
    G.zero_grad()
    o = sdg.render(G, rays.cuda(), 64, seed=4, want_ctx=True)
    sdg.backward(o["ctx"], *(x.cuda() for x in seeds))
    o["ctx"].release()
    torch.cuda.synchronize()
    got = grad_arrays(G, G.num_blocks)
    want = O.backward(rays.numpy(), 64, *(x.double().numpy() for x in seeds), seed=4, given=gpu_samples(tr))
    for k in ("sdf", "rgb", "sem"):
        assert_grad_close(got[k], want[k], what=k)


@pytest.mark.parametrize("layout,n_sem", [("bf16", 20), ("f32", 20), ("bf16", 32), ("f32", 24)])
def test_fused_semantic_train_step_matches_oracle(sdg, layout, n_sem):
    """Fused forward + L1 colour/depth + squared-L2 logit losses + backward (the precision variant's training pass)
    over every ray of a view, against the oracle's loss and backward over the GPU's samples."""
    sc, G, O, _, _ = tiny_room(layout, n_sem)
    rays = _view(sc, 48, 32, seed=9)
    tr = sdg.trace(G, rays.cuda(), 64, seed=5)
    check_placement(O, rays, tr, 64, seed=5)
    gv = gpu_samples(tr)
    ref = O.render(rays, 64, seed=5, given=gv)
    n = rays.shape[0]
    rng = np.random.default_rng(3)
    t_rgb = ref["rgb"] + rng.choice([-0.05, 0.05], size=(n, 3))
    t_depth = ref["depth"] + rng.choice([-0.1, 0.1], size=n)
    t_sem = ref["sem"] + rng.normal(0.0, 0.5, size=(n, n_sem))
    L, seeds = oracle.loss(ref["rgb"], ref["depth"], t_rgb, t_depth, 0.1, sem=ref["sem"], t_sem=t_sem, lam_s=0.1)
    want = O.backward(rays, 64, seeds["rgb"], seeds["depth"], np.zeros(n), seeds["sem"], seed=5, given=gv)
    G.zero_grad()
    loss = torch.empty(n, device="cuda")
    lsum = torch.empty(1, device="cuda")
    dev = lambda x: torch.as_tensor(x, dtype=torch.float32, device="cuda")  # noqa: E731
    sdg.train_step_rays(G, rays.cuda(), dev(t_rgb), dev(t_depth), dev(t_sem), n_samples=64, seed=5,
                        lambda_sem=0.1, loss=loss, loss_sum=lsum)
    torch.cuda.synchronize()
    assert lsum.item() == pytest.approx(L, rel=1e-4)
    got = grad_arrays(G, G.num_blocks)
    for k in ("sdf", "rgb", "sem"):
        assert_grad_close(got[k], want[k], what=k)


def test_bf16_precision_vs_unrounded_fp64(sdg):
    """Precision variant: BF16 colour/logit storage against the FP64 oracle on the unrounded values, every ray fed
    the GPU's samples (errors bounded by the BF16 quantisation of the inputs, ~2^-9 relative)."""
    sc, G, O, stored, vals = tiny_room("bf16", 20)
    Ofull = oracle.Grid(0.04, 0.02, 20).set(O.keys, vals["sdf"].astype(np.float32).astype(np.float64),
                                             vals["rgb"], vals["sem"])
    rays = _view(sc, 32, 24, seed=8)
    out = sdg.render(G, rays.cuda(), 64, seed=2)
    tr = sdg.trace(G, rays.cuda(), 64, seed=2)
    ref = Ofull.render(rays, 64, seed=2, given=gpu_samples(tr))
    e_rgb = np.abs(out["rgb"].double().cpu().numpy() - ref["rgb"]).max()
    e_sem = np.abs(out["sem"].double().cpu().numpy() - ref["sem"]).max()
    e_d = np.abs(out["depth"].double().cpu().numpy() - ref["depth"]).max()
    assert e_rgb < 2 ** -8 and e_sem < 5 * 2 ** -8 and e_d < TOL
