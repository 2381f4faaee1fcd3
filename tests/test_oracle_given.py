"""Pins for the oracle's given-samples mode (the comparison of every ray, including those whose FP32 placement
differs from the FP64 one only by rounding at an interval joint or a block face, Sec. 3.5.1): the caller fixes S,
t_k and the trilinear cell of each sample, and the oracle computes s_k, delta_k and everything after the
placement.  Pinned two ways: (1) fed its own samples (t rounded to FP32, cells = floor(x / vs)) it reproduces its
own render and backward; (2) with one sample per ray its outputs are closed forms of that sample alone --
opac = 1 - exp(-sigma(d) S (1 - u)), rgb / opac = the trilinear colour of the given cell's corners at the given
point (whatever that cell is, so a mistake that ignores the given cell, or swaps its axes, fails), and depth /
opac = t."""
import numpy as np

import oracle
import synth


def _room():
    sc = synth.scene_tiny_room(0)
    keys = synth.band_blocks(sc, 0.04, 3)
    g = synth.fill_grid(sc, keys, 0.04, 3)
    G = oracle.Grid(0.04, 0.02).set(keys, g["sdf"], g["rgb"])
    return sc, keys, g, G


def _own_samples(G, rays, N, seed, vs):
    S = np.zeros(len(rays))
    t = np.zeros((len(rays), N), np.float32)
    cell = np.zeros((len(rays), N, 3), np.int32)
    for i, r in enumerate(rays):
        tr = G.trace(r, N, seed=seed, ray_id=i)
        if len(tr["t"]) == 0:
            continue
        S[i] = G.render(r[None], N, seed=seed, ray_id0=i)["S"][0]
        t[i] = tr["t"].astype(np.float32)
        x = r[None, :3].astype(np.float64) + t[i].astype(np.float64)[:, None] * r[None, 4:7].astype(np.float64)
        cell[i] = np.floor(x / vs).astype(np.int32)
    return {"S": S, "t": t, "cell": cell}


def test_given_own_samples_reproduce_render_and_backward():
    sc, keys, g, G = _room()
    rays = synth.view_rays(synth.random_poses(sc, 1, seed=4)[0], 16, 12, synth.intrinsics(16, 12)).numpy()
    N = 48
    gv = _own_samples(G, rays, N, 7, 0.04)
    ref = G.render(rays, N, seed=7)
    got = G.render(rays, N, seed=7, given=gv)
    nd = ~ref["degenerate"]
    assert nd.mean() > 0.9
    for k in ("rgb", "depth", "opac"):
        assert np.abs(got[k] - ref[k])[nd].max() < 1e-5, k
    np.testing.assert_allclose(got["S"], ref["S"], rtol=0, atol=0)
    rng = np.random.default_rng(0)
    n = len(rays)
    gc, gd = rng.normal(size=(n, 3)) * nd[:, None], rng.normal(size=n) * nd
    a = G.backward(rays, N, gc, gd, seed=7)
    b = G.backward(rays, N, gc, gd, seed=7, given=gv)
    scale = np.abs(a["sdf"]).max()
    assert scale > 0
    assert np.all(np.abs(a["sdf"] - b["sdf"]) <= 1e-4 * np.abs(a["sdf"]) + 1e-6 * scale)
    assert np.all(np.abs(a["rgb"] - b["rgb"]) <= 1e-4 * np.abs(a["rgb"]) + 1e-6 * np.abs(a["rgb"]).max())


def _trilinear(vals, index, c, f):
    """Trilinear combination of the 8 corner values of the cell with base corner c at fractions f (f may leave
    [0, 1]): corners c + (ex, ey, ez), weights prod over axes of f or 1 - f."""
    out = 0.0
    for ez in (0, 1):
        for ey in (0, 1):
            for ex in (0, 1):
                v = c + np.array([ex, ey, ez])
                b, l = v // 8, v % 8
                blk = index[tuple(b.tolist())]
                w = (f[0] if ex else 1 - f[0]) * (f[1] if ey else 1 - f[1]) * (f[2] if ez else 1 - f[2])
                out += w * vals[blk, l[2] * 64 + l[1] * 8 + l[0]]
    return out


def test_given_single_sample_closed_forms():
    sc, keys, g, G = _room()
    vs, beta = 0.04, 0.02
    index = {tuple(k.tolist()): i for i, k in enumerate(keys)}
    rays = synth.view_rays(synth.random_poses(sc, 1, seed=1)[0], 8, 6, synth.intrinsics(8, 6)).numpy()
    ref = G.render(rays, 1, seed=3)
    sel = np.flatnonzero(ref["S"] > 0)[:12]
    assert len(sel) >= 6
    rng = np.random.default_rng(2)
    checked = 0
    for i in sel:
        r = rays[i:i + 1]
        o, d = r[0, :3].astype(np.float64), r[0, 4:7].astype(np.float64)
        t = np.float32(G.trace(r[0], 1, seed=3, ray_id=i)["t"][0])
        x = o + float(t) * d
        c0 = np.floor(x / vs).astype(np.int64)
        for shift in ([0, 0, 0], [-1, 0, 0], [0, 1, 0], [0, 0, -1]):
            c = c0 + np.array(shift)
            if not all(tuple(((c + np.array(e)) // 8).tolist()) in index for e in np.ndindex(2, 2, 2)):
                continue
            S = float(ref["S"][i]) * (1.0 + 0.1 * rng.uniform())
            gv = {"S": [S], "t": [[t]], "cell": [[c.astype(np.int32)]]}
            out = G.render(r, 1, seed=3, ray_id0=int(i), given=gv)
            f = x / vs - c
            dd = _trilinear(g["sdf"].numpy() if hasattr(g["sdf"], "numpy") else g["sdf"], index, c, f)
            rgb = np.array([_trilinear((g["rgb"].numpy() if hasattr(g["rgb"], "numpy") else g["rgb"])[..., ch],
                                       index, c, f) for ch in range(3)])
            u = oracle.sample_u(3, int(i), 0)
            sigma = (0.5 * np.exp(-dd / beta) if dd >= 0 else 1 - 0.5 * np.exp(dd / beta)) / beta
            opac = 1 - np.exp(-sigma * S * (1 - u))
            assert abs(out["opac"][0] - opac) < 1e-12
            if opac > 1e-6:
                np.testing.assert_allclose(out["rgb"][0] / out["opac"][0], rgb, atol=1e-10)
                assert abs(out["depth"][0] / out["opac"][0] - float(t)) < 1e-10
            checked += 1
    assert checked >= 8
