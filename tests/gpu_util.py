"""Helpers shared by the GPU tests: build the same grid on the GPU (through the C ABI) and in the oracle."""
from __future__ import annotations

import numpy as np
import torch

import oracle
import synth


def fill_device_grid(G, vals, n_sem=0):
    """Writes float64 synth values (sdf [N,512], rgb [N,512,3], sem [N,512,ns]) into grid G's channels in index
    order.  Returns the values as the device stores them (float64, after any BF16 rounding)."""
    import paper_2305_13220_b300 as sdg
    A = sdg._abi
    N = vals["sdf"].shape[0]
    dev = f"cuda:{G.device}"
    sdf = torch.as_tensor(vals["sdf"], device=dev).to(torch.float32)
    rgb = torch.as_tensor(vals["rgb"], device=dev).to(torch.float32)
    stored = {}
    if G.rgb_dtype == "f32":
        geo = G.channel(A.GROUP_GEO)
        geo[:N, :, 0] = sdf
        geo[:N, :, 1:4] = rgb
        stored["rgb"] = rgb.double().cpu().numpy()
    else:
        G.channel(A.GROUP_SDF)[:N, :, 0] = sdf
        ch = G.channel(A.GROUP_RGB)
        ch[:N, :, 0:3] = rgb.to(torch.bfloat16)
        ch[:N, :, 3] = 0
        stored["rgb"] = ch[:N, :, 0:3].double().cpu().numpy()
    stored["sdf"] = sdf.double().cpu().numpy()
    if n_sem:
        sem = torch.as_tensor(vals["sem"], device=dev).to(torch.bfloat16)
        G.channel(A.GROUP_SEM)[:N] = sem
        stored["sem"] = sem.double().cpu().numpy()
    torch.cuda.synchronize()
    return stored


def make_pair(scene, keys, vs, band, beta, rgb_dtype="f32", n_sem=0, max_blocks=None, seed=0):
    """Returns (gpu Grid, oracle Grid, stored values) holding the same blocks and voxel values."""
    import paper_2305_13220_b300 as sdg
    keys = np.ascontiguousarray(keys, np.int32)
    G = sdg.Grid(vs, max_blocks or max(len(keys), 1), beta=beta, rgb_dtype=rgb_dtype, n_sem=n_sem)
    G.activate_keys(torch.as_tensor(keys, device="cuda"))
    gk = G.keys().cpu().numpy()
    vals = synth.fill_grid(scene, gk, vs, band, n_sem=n_sem, seed=seed)
    vals = {k: v.numpy() for k, v in vals.items()}
    stored = fill_device_grid(G, vals, n_sem)
    O = oracle.Grid(vs, beta, n_sem).set(gk, stored["sdf"], stored["rgb"], stored.get("sem"))
    return G, O, stored, vals


def tiny_room(rgb_dtype="f32", n_sem=0, seed=0):
    sc = synth.scene_tiny_room(seed)
    keys = synth.band_blocks(sc, 0.04, 3)
    G, O, stored, vals = make_pair(sc, keys, 0.04, 3, 0.02, rgb_dtype, n_sem)
    return sc, G, O, stored, vals


def grad_arrays(G, N):
    """Gradient channels of the first N blocks as float64 numpy: sdf [N,512], rgb [N,512,3], sem."""
    import paper_2305_13220_b300 as sdg
    A = sdg._abi
    out = {}
    if G.rgb_dtype == "f32":
        g = G.channel(A.GROUP_GEO, A.KIND_GRAD)[:N].double().cpu().numpy()
        out["sdf"], out["rgb"] = g[..., 0], g[..., 1:4]
    else:
        out["sdf"] = G.channel(A.GROUP_SDF, A.KIND_GRAD)[:N, :, 0].double().cpu().numpy()
        out["rgb"] = G.channel(A.GROUP_RGB, A.KIND_GRAD)[:N, :, 0:3].double().cpu().numpy()
    if G.n_sem:
        out["sem"] = G.channel(A.GROUP_SEM, A.KIND_GRAD)[:N].double().cpu().numpy()
    return out


def assert_grad_close(got, ref, rel=1e-3, floor=1e-5, what=""):
    """|got - ref| <= rel |ref| + floor * max|ref| elementwise (floor absorbs FP32 atomic-order noise on
    entries that are tiny relative to the channel)."""
    scale = np.abs(ref).max()
    assert scale > 0, f"{what}: reference gradient is zero"
    err = np.abs(got - ref)
    bound = rel * np.abs(ref) + floor * scale
    bad = err > bound
    assert not bad.any(), (f"{what}: {bad.sum()} of {bad.size} entries off; worst |d|={err.max():.3e}, "
                           f"scale={scale:.3e}")


# ----------------------------------------------------------------------------------------------------------------
# Every ray compared: the GPU's own sample placement (sdg_debug_trace) checked against the oracle's FP64
# traversal, then fed to the oracle so that each ray's outputs and gradient shares are compared -- including rays
# whose FP32 placement differs from the FP64 one only by rounding (Sec. 3.5.1 sampling in skip space).
# ----------------------------------------------------------------------------------------------------------------
PLACE_TOL = 2e-5  # metres: FP32 placement error of t_k (a few ulps of t ~ 5 m, and of the skip-space offsets)


def gpu_samples(tr):
    """The GPU's placement from a trace, as the oracle's given-samples dict."""
    return {"S": tr["S"].double().cpu().numpy(), "t": tr["t"].cpu().numpy(), "cell": tr["cell"].cpu().numpy()}


def _merge(segs, eps=1e-6):
    """Touching (t_in, t_out) stretches merged; stretches shorter than eps dropped."""
    out = []
    for a, b in segs:
        if b - a < eps:
            continue
        if out and abs(out[-1][1] - a) <= eps:
            out[-1][1] = b
        else:
            out.append([a, b])
    return out


def check_placement(O, rays, tr, N, seed=0, ray_id0=0, stratified=True, vs=None):
    """Asserts that every GPU sample lies where the oracle's FP64 traversal puts it, up to FP32 rounding: S and
    t_k within PLACE_TOL, except that a sample whose skip-space position falls on a joint between two allocated
    stretches (both precisions may pick either side) must sit at one of the joint's two ends; the cell must be
    floor(x / vs) of the GPU's own point, either side allowed where x / vs is within FP32 rounding of an integer;
    and the recorded cells of the traversal pass, merged, must be the oracle's stretches.  Returns the number of
    rays with a joint sample and with a cell tie (the rays the oracle's own placement would not reproduce)."""
    rays = np.asarray(rays.cpu() if hasattr(rays, "cpu") else rays, np.float32).reshape(-1, 8)
    vs = vs or O.vs
    S = tr["S"].double().cpu().numpy()
    t = tr["t"].double().cpu().numpy()
    cell = tr["cell"].cpu().numpy()
    nc = tr["n_cells"].cpu().numpy()
    seg = tr["seg"].double().cpu().numpy()
    ref = O.render(rays, N, seed=seed, ray_id0=ray_id0, stratified=stratified)
    assert np.all(np.abs(S - ref["S"]) <= 2e-6 + 1e-5 * ref["S"]), np.abs(S - ref["S"]).max()
    n_joint = n_tie = 0
    for i in range(len(rays)):
        if ref["S"][i] <= 0:
            assert S[i] == 0
            continue
        o, d = rays[i, :3].astype(np.float64), rays[i, 4:7].astype(np.float64)
        iv = O.traverse(rays[i])
        ends = np.array(iv)
        lens = ends[:, 1] - ends[:, 0]
        joints = np.cumsum(lens)[:-1]
        tro = O.trace(rays[i], N, seed=seed, ray_id=ray_id0 + i, stratified=stratified)
        dt = np.abs(t[i] - tro["t"])
        off = np.flatnonzero(dt > PLACE_TOL)
        for k in off:
            j = np.flatnonzero(np.abs(joints - tro["s"][k]) <= PLACE_TOL)
            assert len(j), (i, k, t[i, k], tro["t"][k])
            j = j[0]
            sides = (ends[j, 1], ends[j + 1, 0])
            assert min(abs(t[i, k] - sides[0]), abs(t[i, k] - sides[1])) <= PLACE_TOL, (i, k, t[i, k], sides)
        n_joint += len(off) > 0
        y = (o[None] + t[i][:, None] * d[None]) / vs
        fl = np.floor(y)
        near = np.abs(y - np.round(y)) < 1e-4
        ok = (cell[i] == fl) | (near & ((cell[i] == np.round(y)) | (cell[i] == np.round(y) - 1)))
        assert ok.all(), (i, np.argwhere(~ok)[:3])
        n_tie += bool(((cell[i] != fl) & near).any())
        if nc[i] >= 0:
            mine = _merge([(a, a + b) for a, b in seg[i, :nc[i]]])
            theirs = _merge([tuple(x) for x in ends])
            assert len(mine) == len(theirs), (i, mine, theirs)
            assert np.abs(np.array(mine) - np.array(theirs)).max() <= PLACE_TOL, (i, mine, theirs)
    return n_joint, n_tie


def assert_forward_all_rays(out, ref, tol=1e-4, ns=0, what=""):
    """Every ray's rgb, depth, opacity (and logits) within max-abs tol of the oracle."""
    for k in ("rgb", "depth", "opac") + (("sem",) if ns else ()):
        got = out[k].double().cpu().numpy()
        d = np.abs(got - ref[k]).max() if got.size else 0.0
        lim = tol * 10 if k == "sem" else tol   # logits reach ~5 in magnitude
        assert d <= lim, (what, k, d)


def assert_trace_equals_render(tr, out):
    """The trace's forward outputs are the render's, bit for bit (the trace runs the same placement code)."""
    import torch
    for k in ("rgb", "depth", "opac"):
        assert torch.equal(tr[k], out[k]), k
