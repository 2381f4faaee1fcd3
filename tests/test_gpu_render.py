"""GPU parity of the rendering path (Sec. 3.5.1, Eq. 12-15; trilinear Eq. 17) against the FP64 oracle.

Tolerances (FP32 on the GPU vs FP64): rendered colour / depth / opacity max-abs 1e-4; gradients relative 1e-3
elementwise with a floor of 1e-5 of the channel's largest entry (FP32 atomics sum in arbitrary order).  Rays the
oracle flags degenerate (a sample within rounding of a skip-space joint or of a plane where its stencil's
validity flips) are excluded from the element-wise comparison and counted."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import assert_grad_close, grad_arrays, tiny_room

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
    for k in ("rgb", "depth", "opac"):
        got = out[k].double().cpu().numpy()
        d = np.abs(got - ref[k])[nd]
        assert d.max() <= TOL, (k, d.max())
    if ns:
        got = out["sem"].double().cpu().numpy()
        d = np.abs(got - ref["sem"])[nd]
        assert d.max() <= TOL * 10, ("sem", d.max())   # logits reach ~5 in magnitude


@pytest.mark.parametrize("stratified,bg", [(True, (0, 0, 0)), (False, (0.2, 0.5, 0.9)), (True, (1, 1, 1))])
def test_forward_matches_oracle(sdg, room, stratified, bg):
    sc, G, O, _, _ = room
    rays = _view(sc)
    out = sdg.render(G, rays.cuda(), 64, seed=5, stratified=stratified, bg=bg)
    ref = O.render(rays, 64, seed=5, stratified=stratified, bg=bg)
    nd = ~ref["degenerate"]
    assert nd.mean() > 0.97, nd.mean()
    assert ref["opac"].max() > 0.99 and ref["n_valid"].mean() > 30
    _cmp_forward(out, ref, nd)


@pytest.mark.parametrize("N", [1, 17, 48, 100, 128, 192, 256])
def test_forward_sample_counts(sdg, room, N):
    sc, G, O, _, _ = room
    rays = _view(sc, 24, 16, seed=1)
    out = sdg.render(G, rays.cuda(), N, seed=9)
    ref = O.render(rays, N, seed=9)
    nd = ~ref["degenerate"]
    assert nd.mean() > 0.9
    _cmp_forward(out, ref, nd)


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


def _runs(mask):
    """Contiguous runs [a, b) of True in mask."""
    runs, a = [], None
    for i, m in enumerate(list(mask) + [False]):
        if m and a is None:
            a = i
        if not m and a is not None:
            runs.append((a, i))
            a = None
    return runs


def _gpu_backward_runs(sdg, G, rays, runs, N, seed, stratified, bg, seeds, mode):
    G.zero_grad()
    gc, gd, go, gs = seeds
    for a, b in runs:
        sl = slice(a, b)
        o = sdg.render(G, rays[sl], N, seed=seed, ray_id0=a, stratified=stratified, bg=bg, want_ctx=True, mode=mode)
        sdg.backward(o["ctx"], gc[sl], gd[sl], go[sl], None if gs is None else gs[sl])
        o["ctx"].release()
    torch.cuda.synchronize()
    return grad_arrays(G, G.num_blocks)


def _oracle_backward_runs(O, rays, runs, N, seed, stratified, bg, seeds):
    gc, gd, go, gs = (None if s is None else s.double().cpu().numpy() for s in seeds)
    tot = None
    for a, b in runs:
        g = O.backward(rays[a:b], N, gc[a:b], gd[a:b], go[a:b], None if gs is None else gs[a:b], seed=seed,
                       ray_id0=a, stratified=stratified, bg=bg)
        g = {k: g[k] for k in ("sdf", "rgb", "sem", "beta") if k in g}  # per-voxel arrays and the scalar beta
        tot = g if tot is None else {k: tot[k] + g[k] for k in g}
    return tot


@pytest.mark.parametrize("mode", ["recompute", "store"])
@pytest.mark.parametrize("stratified", [True, False])
@pytest.mark.parametrize("N", [64, 192])  # 192: 6 samples per lane, where the forward reuses a cell's corners
def test_backward_matches_oracle(sdg, room, mode, stratified, N):
    sc, G, O, _, _ = room
    rays = _view(sc, seed=2)
    bg = (0.3, 0.1, 0.7)
    ref = O.render(rays, N, seed=3, stratified=stratified, bg=bg)
    runs = _runs(~ref["degenerate"])
    n = len(rays)
    gen = torch.Generator().manual_seed(0)
    seeds = tuple(torch.randn(s, generator=gen).cuda() for s in ((n, 3), (n,), (n,))) + (None,)
    got = _gpu_backward_runs(sdg, G, rays.cuda(), runs, N, 3, stratified, bg, seeds, mode)
    want = _oracle_backward_runs(O, rays.numpy(), runs, N, 3, stratified, bg, seeds)
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
        assert_grad_close(res["store"][k], res["recompute"][k], rel=1e-5, floor=1e-6, what=k)


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
    sc, G, O, _, _ = room
    rays = _view(sc, seed=6)
    ref = O.render(rays, 64, stratified=False)
    nd = ~ref["degenerate"]
    rays = rays[torch.as_tensor(nd)]
    ref = O.render(rays, 64, stratified=False)
    n = rays.shape[0]
    rng = np.random.default_rng(0)
    t_rgb = ref["rgb"] + rng.choice([-0.05, 0.05], size=(n, 3))
    t_depth = ref["depth"] + rng.choice([-0.1, 0.1], size=n)
    L, seeds = oracle.loss(ref["rgb"], ref["depth"], t_rgb, t_depth, 0.1)
    want = O.backward(rays, 64, seeds["rgb"], seeds["depth"], stratified=False)
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
    assert_grad_close(unf["sdf"], got["sdf"], rel=1e-5, floor=1e-6, what="unfused sdf")
    assert lv.sum().item() == pytest.approx(L, rel=1e-4)


@pytest.mark.parametrize("n_sem", [8, 20])
def test_bf16_and_semantics_match_oracle(sdg, n_sem):
    sc, G, O, stored, vals = tiny_room("bf16", n_sem)
    rays = _view(sc, 48, 32, seed=7)
    out = sdg.render(G, rays.cuda(), 64, seed=4)
    ref = O.render(rays, 64, seed=4)
    nd = ~ref["degenerate"]
    _cmp_forward(out, ref, nd, n_sem)
    runs = _runs(nd)
    n = len(rays)
    gen = torch.Generator().manual_seed(1)
    seeds = tuple(torch.randn(s, generator=gen).cuda() for s in ((n, 3), (n,), (n,), (n, n_sem)))
    got = _gpu_backward_runs(sdg, G, rays.cuda(), runs, 64, 4, True, (0, 0, 0), seeds, "recompute")
    want = _oracle_backward_runs(O, rays.numpy(), runs, 64, 4, True, (0, 0, 0), seeds)
    for k in ("sdf", "rgb", "sem"):
        assert_grad_close(got[k], want[k], what=k)


def test_bf16_precision_vs_unrounded_fp64(sdg):
    """Precision variant: BF16 colour/logit storage against the FP64 oracle on the unrounded values (errors
    reported; bounded by the BF16 quantisation of the inputs, ~2^-9 relative)."""
    sc, G, O, stored, vals = tiny_room("bf16", 20)
    Ofull = oracle.Grid(0.04, 0.02, 20).set(O.keys, vals["sdf"].astype(np.float32).astype(np.float64),
                                             vals["rgb"], vals["sem"])
    rays = _view(sc, 32, 24, seed=8)
    out = sdg.render(G, rays.cuda(), 64, seed=2)
    ref = Ofull.render(rays, 64, seed=2)
    nd = ~ref["degenerate"]
    e_rgb = np.abs(out["rgb"].double().cpu().numpy() - ref["rgb"])[nd].max()
    e_sem = np.abs(out["sem"].double().cpu().numpy() - ref["sem"])[nd].max()
    e_d = np.abs(out["depth"].double().cpu().numpy() - ref["depth"])[nd].max()
    assert e_rgb < 2 ** -8 and e_sem < 5 * 2 ** -8 and e_d < TOL
