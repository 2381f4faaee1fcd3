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
