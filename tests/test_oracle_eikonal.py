"""Pins of the oracle's SDF-gradient query and Eikonal loss (Sec. 3.5.2-3.5.3, Eq. 16-17).

A linear SDF field is reproduced exactly by trilinear interpolation, so its analytic gradient is the field's
normal and the Eikonal loss is known in closed form; the analytic gradient equals central differences of the
interpolant; the Eikonal gradient with respect to the stored values equals central differences of the loss."""
import numpy as np

import oracle

VS = 0.05


def cube_keys(n=2):
    return np.array([(x, y, z) for z in range(n) for y in range(n) for x in range(n)], np.int32)


def voxel_xyz(keys):
    l = np.arange(512)
    loc = np.stack([l & 7, (l >> 3) & 7, l >> 6], -1)
    return (keys[:, None, :] * 8 + loc[None]) * VS


def grid_with(sdf, keys):
    return oracle.Grid(VS, 0.5 * VS).set(keys, sdf, np.zeros(sdf.shape + (3,)))


def interior_points(n, rng, keys, margin=1e-3):
    """Points strictly inside the allocated cube whose 8 grid points are allocated, away from cell faces."""
    lo, hi = keys.min(0) * 8 * VS, ((keys.max(0) + 1) * 8 - 1) * VS
    x = rng.uniform(lo, hi, size=(n, 3))
    f = x / VS - np.floor(x / VS)
    keep = np.all((f > margin) & (f < 1 - margin), axis=1)
    return x[keep]


def test_linear_field_gradient_and_eikonal_closed_forms():
    keys = cube_keys()
    rng = np.random.default_rng(0)
    nrm = np.array([0.36, -0.48, 0.8])  # unit normal
    xyz = voxel_xyz(keys)
    for scale in (1.0, 2.0):
        sdf = scale * (xyz @ nrm) - 0.1
        G = grid_with(sdf, keys)
        x = interior_points(400, rng, keys)
        f, g, ok = G.query_grad(x)
        assert ok.all()
        np.testing.assert_allclose(f, scale * (x @ nrm) - 0.1, atol=1e-12)
        np.testing.assert_allclose(g, np.broadcast_to(scale * nrm, g.shape), atol=1e-11)
        lam = 0.1
        L, terms, gs = G.eikonal(x, lam)
        assert abs(L - lam * (scale - 1.0) ** 2) < 1e-12
        if scale == 1.0:
            assert np.abs(gs).max() < 1e-12
    # a flat (truncated) region: |grad f| = 0, each point's term is lambda/n, and no gradient (its direction is
    # undefined below |grad f| = 1e-4)
    G0 = grid_with(np.full((len(keys), 512), 0.12), keys)
    x = interior_points(100, rng, keys)
    L, terms, gs = G0.eikonal(x, 0.1)
    assert abs(L - 0.1) < 1e-12 and np.all(gs == 0)
    # points outside the allocated cube are invalid and contribute nothing
    far = np.array([[5.0, 5.0, 5.0], [-1.0, 0.2, 0.2]])
    _, _, ok = G.query_grad(far)
    assert not ok.any()
    L, terms, gs = G.eikonal(far, 0.1)
    assert L == 0 and np.all(gs == 0)


def test_gradient_equals_central_differences_of_the_interpolant():
    keys = cube_keys()
    rng = np.random.default_rng(1)
    sdf = rng.normal(0, 0.05, size=(len(keys), 512))
    G = grid_with(sdf, keys)
    x = interior_points(300, rng, keys, margin=1e-2)
    _, g, ok = G.query_grad(x)
    assert ok.all()
    h = 1e-6 * VS
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fp, _, _ = G.query(x + e)
        fm, _, _ = G.query(x - e)
        np.testing.assert_allclose(g[:, a], (fp - fm) / (2 * h), rtol=1e-6, atol=1e-6)


def test_eikonal_gradient_equals_central_differences_of_the_loss():
    keys = cube_keys()
    rng = np.random.default_rng(2)
    xyz = voxel_xyz(keys)
    sdf = 1.7 * (xyz @ np.array([0.6, 0.0, 0.8])) - 0.2 + rng.normal(0, 0.01, size=(len(keys), 512))
    x = interior_points(200, rng, keys, margin=1e-2)
    lam = 0.3
    G = grid_with(sdf, keys)
    L, terms, gs = G.eikonal(x, lam)
    assert abs(L - terms.sum()) < 1e-14
    touched = np.argwhere(np.abs(gs) > 0)
    assert len(touched) > 500
    pick = touched[rng.choice(len(touched), 40, replace=False)]
    h = 1e-6
    for b, v in pick:
        s2 = sdf.copy()
        s2[b, v] += h
        Lp, _, _ = grid_with(s2, keys).eikonal(x, lam)
        s2[b, v] -= 2 * h
        Lm, _, _ = grid_with(s2, keys).eikonal(x, lam)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - gs[b, v]) <= 1e-6 * abs(gs[b, v]) + 1e-10, (b, v, fd, gs[b, v])
