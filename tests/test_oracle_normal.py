"""Pins of the oracle's rendered normal and normal loss (Eq. 14, with grad f of Eq. 17 at every sample).

A linear SDF has grad f = n everywhere, so the rendered normal is exactly the opacity times n; the backward with
normal seeds equals central differences of sum_i g_i . N_i in the stored SDF values; the L1 normal loss seeds equal
central differences of the loss."""
import numpy as np
import pytest

import oracle
import synth
from tests.test_oracle_render import BETA, VS, _fd_grid


def test_linear_field_renders_opacity_times_normal():
    nrm = np.array([0.2, -0.3, 0.9])
    nrm /= np.linalg.norm(nrm)
    keys, sdf, rgb = synth.plane_grid(nrm, 0.0, VS, extent_blocks=((-2, 2), (-2, 2), (-3, 3)), slab_blocks=2)
    G = oracle.Grid(VS, BETA).set(keys, sdf, rgb)
    rng = np.random.default_rng(0)
    o = np.stack([rng.uniform(-0.05, 0.05, 64), rng.uniform(-0.05, 0.05, 64), np.full(64, 0.12)], 1)
    d = np.stack([rng.uniform(-0.2, 0.2, 64), rng.uniform(-0.2, 0.2, 64), -np.ones(64)], 1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.concatenate([o, np.zeros((64, 1)), d, np.full((64, 1), 10.0)], 1).astype(np.float32)
    out = G.render(rays, 96, stratified=False)
    assert out["opac"].min() > 0.5
    np.testing.assert_allclose(out["normal"], out["opac"][:, None] * nrm[None], atol=1e-9)


def test_normal_backward_matches_central_differences():
    keys, sdf, rgb, _, rays = _fd_grid(0, seed=2)
    G = oracle.Grid(VS, BETA).set(keys, sdf, rgb)
    rng = np.random.default_rng(5)
    n = len(rays)
    gn = rng.normal(size=(n, 3))
    gc = np.zeros((n, 3))
    N = 16

    def L(s_):
        o = oracle.Grid(VS, BETA).set(keys, s_, rgb).render(rays, N, seed=5)
        return (o["normal"] * gn).sum()

    an = G.backward(rays, N, gc, seed=5, g_normal=gn)
    assert np.abs(an["sdf"]).max() > 0
    scale = np.abs(an["sdf"]).max()
    flat = sdf.reshape(-1)
    nz = np.flatnonzero(an["sdf"].reshape(-1))
    h = 1e-6
    for j in rng.choice(nz, 40, replace=False):
        p, m = flat.copy(), flat.copy()
        p[j] += h
        m[j] -= h
        fd = (L(p.reshape(sdf.shape)) - L(m.reshape(sdf.shape))) / (2 * h)
        a = an["sdf"].reshape(-1)[j]
        assert abs(fd - a) <= 1e-6 * abs(a) + 1e-7 * scale, (j, fd, a)


def test_normal_loss_seeds_match_finite_differences():
    rng = np.random.default_rng(4)
    Nr, Nt = rng.normal(size=(5, 3)), rng.normal(size=(5, 3))
    L, g = oracle.loss_normal(Nr, Nt, 0.05)
    assert L == pytest.approx(0.05 * np.abs(Nr - Nt).mean(), rel=1e-14)
    h = 1e-7
    for j in range(Nr.size):
        p, m = Nr.copy(), Nr.copy()
        p.reshape(-1)[j] += h
        m.reshape(-1)[j] -= h
        fd = (oracle.loss_normal(p, Nt, 0.05)[0] - oracle.loss_normal(m, Nt, 0.05)[0]) / (2 * h)
        assert fd == pytest.approx(g.reshape(-1)[j], rel=1e-6, abs=1e-12)
