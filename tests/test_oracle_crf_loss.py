"""Pins of the oracle's CRF losses (Sec. 3.5.3, Eq. 22 read as the divergence between each property and its
message-passed value, a fixed target): zero loss and zero gradient when the target is the property itself;
KL >= 0; gradients equal central differences of the loss in the stored values."""
import numpy as np
import pytest

import oracle
from tests.test_oracle_eikonal import VS, cube_keys, interior_points


def grid(rng, ns=4):
    keys = cube_keys()
    N = len(keys)
    sdf = rng.normal(0, 0.05, (N, 512))
    rgb = rng.uniform(0, 1, (N, 512, 3))
    sem = rng.normal(0, 1, (N, 512, ns))
    return keys, sdf, rgb, sem


def make(keys, sdf, rgb, sem):
    return oracle.Grid(VS, 0.5 * VS, sem.shape[-1]).set(keys, sdf, rgb, sem)


def props(G, x):
    """Current property values at x: softmax(logits), colour, grad f."""
    f, gr, ok = G.query_grad(x)
    _, c, _ = G.query(x)
    return gr, c, ok


@pytest.mark.parametrize("prop", ["label", "color", "normal"])
def test_crf_loss_zero_at_target_and_matches_central_differences(prop):
    rng = np.random.default_rng({"label": 0, "color": 1, "normal": 2}[prop])
    keys, sdf, rgb, sem = grid(rng)
    G = make(keys, sdf, rgb, sem)
    x = interior_points(60, rng, keys, margin=1e-2)
    ns = sem.shape[-1]
    if prop == "label":
        t = rng.dirichlet(np.ones(ns), size=len(x))
    else:
        t = rng.normal(size=(len(x), 3))
    L, terms, g = G.crf_loss(prop, x, t, 0.3)
    assert L > 0 and np.all(terms >= 0) and abs(L - terms.sum()) < 1e-12
    arr = {"label": sem, "color": rgb, "normal": sdf}[prop]
    nz = np.flatnonzero(g.reshape(-1))
    assert len(nz) > 100
    h = 1e-6
    for j in rng.choice(nz, 30, replace=False):
        p, m = arr.copy(), arr.copy()
        p.reshape(-1)[j] += h
        m.reshape(-1)[j] -= h
        args = lambda a: {"label": (keys, sdf, rgb, a), "color": (keys, sdf, a, sem),
                          "normal": (keys, a, rgb, sem)}[prop]
        fd = (make(*args(p)).crf_loss(prop, x, t, 0.3)[0] - make(*args(m)).crf_loss(prop, x, t, 0.3)[0]) / (2 * h)
        assert abs(fd - g.reshape(-1)[j]) <= 1e-6 * abs(fd) + 1e-10, (prop, j, fd, g.reshape(-1)[j])


def test_crf_loss_vanishes_at_the_property_itself():
    rng = np.random.default_rng(5)
    keys, sdf, rgb, sem = grid(rng)
    G = make(keys, sdf, rgb, sem)
    x = interior_points(50, rng, keys, margin=1e-2)
    gr, c, ok = props(G, x)
    assert ok.all()
    for prop, t in (("color", c), ("normal", gr)):
        L, _, g = G.crf_loss(prop, x, t, 0.3)
        assert L < 1e-20 and np.abs(g).max() < 1e-12
    # labels: uniform logits make softmax uniform, so a uniform target gives KL = 0 and no gradient
    G0 = make(keys, sdf, rgb, np.full_like(sem, 0.7))
    L, terms, g = G0.crf_loss("label", x, np.full((len(x), sem.shape[-1]), 1.0 / sem.shape[-1]), 0.3)
    assert abs(L) < 1e-15 and np.abs(g).max() < 1e-15
    t = np.zeros((len(x), sem.shape[-1]))
    t[:, 1] = 1.0
    L, terms, g = G.crf_loss("label", x, t, 0.3)
    assert np.all(terms > 0)
