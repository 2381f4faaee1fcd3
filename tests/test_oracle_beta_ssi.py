"""Pins of the oracle's Laplace-scale gradient dL/dbeta and of the scale/shift-invariant depth loss.

dL/dbeta: central differences of the rendered outputs in beta (grids rebuilt at beta +- h), against the
backward's accumulation of dL/dtau_k delta_k dsigma_k/dbeta.  The SSI depth loss (Eq. 13 with the per-batch least
squares scale and shift): zero for targets that are an affine image of the rendered depth, invariant to affine
changes of the targets, and its gradient equals central differences of the loss with (a, b) re-fitted at every
evaluation (the envelope theorem the closed form relies on)."""
import numpy as np
import pytest

import oracle
from tests.test_oracle_render import BETA, VS, _fd_grid


@pytest.mark.parametrize("bg", [(0, 0, 0), (0.3, 0.6, 0.1)])
def test_beta_gradient_matches_central_differences(bg):
    keys, sdf, rgb, sem, rays = _fd_grid(0)
    rng = np.random.default_rng(7)
    n = len(rays)
    gc, gd, go = rng.normal(size=(n, 3)), rng.normal(size=n), rng.normal(size=n)
    N = 16

    def L(beta):
        G = oracle.Grid(VS, beta).set(keys, sdf, rgb)
        o = G.render(rays, N, seed=5, bg=bg)
        return (o["rgb"] * gc).sum() + (o["depth"] * gd).sum() + (o["opac"] * go).sum(), o

    G = oracle.Grid(VS, BETA).set(keys, sdf, rgb)
    an = G.backward(rays, N, gc, gd, go, seed=5, bg=bg)
    _, o = L(BETA)
    assert o["n_valid"].min() > 0 and abs(an["beta"]) > 0
    h = 1e-7 * BETA
    fd = (L(BETA + h)[0] - L(BETA - h)[0]) / (2 * h)
    assert fd == pytest.approx(an["beta"], rel=1e-6)
    # per ray as well: each ray's seeds only move its own outputs
    for i in range(n):
        sel = np.zeros(n)
        sel[i] = 1

        def Li(beta):
            G2 = oracle.Grid(VS, beta).set(keys, sdf, rgb)
            o2 = G2.render(rays, N, seed=5, bg=bg)
            return (o2["rgb"][i] * gc[i]).sum() + o2["depth"][i] * gd[i] + o2["opac"][i] * go[i]
        fdi = (Li(BETA + h) - Li(BETA - h)) / (2 * h)
        assert abs(fdi - an["beta_per_ray"][i]) <= 1e-6 * abs(fdi) + 1e-9 * abs(an["beta"])


def test_ssi_loss_zero_for_affine_targets_and_invariant():
    rng = np.random.default_rng(0)
    D = rng.uniform(0.5, 4.0, 1000)
    t = (D - 0.3) / 2.5  # D = 2.5 t + 0.3
    L, g, (a, b) = oracle.depth_ssi(D, t, 0.1)
    assert L < 1e-20 and np.abs(g).max() < 1e-12
    assert a == pytest.approx(2.5, rel=1e-12) and b == pytest.approx(0.3, rel=1e-10)
    t2 = rng.uniform(0.5, 4.0, 1000)
    L1, g1, _ = oracle.depth_ssi(D, t2, 0.1)
    L2, g2, _ = oracle.depth_ssi(D, -3.0 * t2 + 7.0, 0.1)
    assert L1 > 0.01 and L2 == pytest.approx(L1, rel=1e-10)
    np.testing.assert_allclose(g2, g1, rtol=1e-8, atol=1e-14)
    # constant targets: the scale is undetermined; a = 1 and the loss is the variance of D
    L3, g3, (a3, b3) = oracle.depth_ssi(D, np.full(1000, 2.0), 0.1)
    assert a3 == 1.0 and L3 == pytest.approx(0.1 * D.var(), rel=1e-12)


def test_ssi_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    D = rng.uniform(0.5, 4.0, 200)
    t = 0.7 * D + 0.2 + rng.normal(0, 0.1, 200)
    L, g, _ = oracle.depth_ssi(D, t, 0.3)
    h = 1e-6
    for i in rng.choice(200, 30, replace=False):
        Dp, Dm = D.copy(), D.copy()
        Dp[i] += h
        Dm[i] -= h
        fd = (oracle.depth_ssi(Dp, t, 0.3)[0] - oracle.depth_ssi(Dm, t, 0.3)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * abs(g[i]) + 1e-10
