"""Pins for the oracle's rendering path (Sec. 3.5: Eq. 12-15 and the trilinear interpolation of Sec. 3.5.2).

Checks against closed forms (linear-field reproduction, Laplace density limits, the plane's expected depth by
quadrature), invariants (partition of unity, transmittance monotone in [0,1], sum of weights = 1 - T_N),
brute force (traversal vs dense point classification) and finite differences (backward)."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
import synth

VS = 0.01
BETA = 0.005


def _plane(normal=(0.3, -0.5, 0.8), offset=0.013, vs=VS, slab=1):
    keys, sdf, rgb = synth.plane_grid(normal, offset, vs, slab_blocks=slab)
    return keys, sdf, rgb


def _interior_points(G, keys, vs, n, rng):
    """Random points whose 8 grid points are all allocated (brute-force membership test)."""
    ks = set(map(tuple, keys.tolist()))
    L = 8 * vs
    pts = []
    while len(pts) < n:
        b = keys[rng.integers(len(keys))]
        x = (b + rng.uniform(0, 1, 3)) * L
        c = np.floor(x / vs).astype(np.int64)
        if all(tuple(((c + np.array(e)) // 8).tolist()) in ks for e in np.ndindex(2, 2, 2)):
            pts.append(x)
    return np.array(pts)


def test_trilinear_reproduces_linear_field():
    keys, sdf, rgb = _plane()
    G = oracle.Grid(VS, BETA).set(keys, sdf, rgb)
    rng = np.random.default_rng(0)
    x = _interior_points(G, keys, VS, 400, rng)
    d, c, valid = G.query(x)
    assert valid.all()
    n = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    np.testing.assert_allclose(d, x @ n - 0.013, atol=1e-13)
    np.testing.assert_allclose(c[:, 0], 0.3 + 0.1 * x[:, 0], atol=1e-13)
    np.testing.assert_allclose(c[:, 2], 0.2 + 0.07 * x[:, 2], atol=1e-13)


def test_trilinear_partition_of_unity_and_corner_values():
    keys = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0], [0, 0, 1], [1, 0, 1], [0, 1, 1], [1, 1, 1]],
                    np.int32)
    N = len(keys)
    G = oracle.Grid(VS, BETA).set(keys, np.ones((N, 512)), np.zeros((N, 512, 3)))
    rng = np.random.default_rng(1)
    x = rng.uniform(0.0, 2 * 8 * VS - VS - 1e-9, size=(300, 3))
    d, _, valid = G.query(x)
    assert valid.all()
    np.testing.assert_allclose(d, 1.0, atol=1e-14)
    # at a grid point the interpolant equals that voxel's value (voxel (9,2,3) lives in block (1,0,0), local (1,2,3))
    sdf = rng.normal(size=(N, 512))
    G.set(keys, sdf, np.zeros((N, 512, 3)))
    d, _, _ = G.query(np.array([[9 * VS, 2 * VS, 3 * VS]]) + 1e-12)
    np.testing.assert_allclose(d[0], sdf[1, 3 * 64 + 2 * 8 + 1], atol=1e-9)


def test_missing_neighbour_makes_sample_invalid():
    keys = np.array([[0, 0, 0]], np.int32)
    G = oracle.Grid(VS, BETA).set(keys, np.zeros((1, 512)), np.zeros((1, 512, 3)))
    _, _, valid = G.query(np.array([[6.5 * VS, 3.5 * VS, 3.5 * VS], [7.5 * VS, 3.5 * VS, 3.5 * VS],
                                    [3.5 * VS, 3.5 * VS, 7.5 * VS], [-0.5 * VS, 1 * VS, 1 * VS]]))
    assert valid.tolist() == [True, False, False, False]


def test_laplace_density_closed_forms():
    b = 0.02
    assert oracle.density(0.0, b) == pytest.approx(1 / (2 * b), rel=1e-15)
    assert oracle.density(-1.0, b) == pytest.approx(1 / b, rel=1e-12)
    assert oracle.density(1.0, b) < 1e-20
    # Psi_beta(s) = 1 - 0.5 exp(-s/beta) for s > 0: d = -b ln 2 -> sigma = (1/b)(1 - 1/4)
    assert oracle.density(-b * math.log(2), b) == pytest.approx(0.75 / b, rel=1e-13)
    assert oracle.density(b * math.log(2), b) == pytest.approx(0.25 / b, rel=1e-13)
    # continuity and derivative vs central differences, monotone decreasing
    for d in (-0.05, -0.01, -1e-4, 1e-4, 0.003, 0.04):
        h = 1e-7
        fd = (oracle.density(d + h, b) - oracle.density(d - h, b)) / (2 * h)
        assert oracle.density_deriv(d, b) == pytest.approx(fd, rel=1e-6)
        assert oracle.density_deriv(d, b) < 0
    assert oracle.density(1e-12, b) == pytest.approx(oracle.density(-1e-12, b), rel=1e-9)


def test_sample_hash_uniform_and_stratified():
    us = np.array([oracle.sample_u(7, r, k) for r in range(64) for k in range(64)])
    assert us.min() >= 0 and us.max() < 1
    assert np.all(us * 2 ** 24 == np.floor(us * 2 ** 24))      # exactly 24-bit
    hist, _ = np.histogram(us, bins=16, range=(0, 1))
    chi2 = ((hist - len(us) / 16) ** 2 / (len(us) / 16)).sum()
    assert chi2 < 40                                          # 15 dof, p ~ 5e-4
    assert oracle.sample_u(7, 3, 5) != oracle.sample_u(8, 3, 5)
    assert oracle.sample_u(7, 3, 5) != oracle.sample_u(7, 4, 5)


def _tiny_room_grid(n_sem=0):
    sc = synth.scene_tiny_room(0)
    keys = synth.band_blocks(sc, 0.04, 3)
    g = synth.fill_grid(sc, keys, 0.04, 3, n_sem=n_sem)
    G = oracle.Grid(0.04, 0.02, n_sem).set(keys, g["sdf"], g["rgb"], g.get("sem"))
    return sc, keys, G


def test_traversal_matches_dense_classification():
    sc, keys, G = _tiny_room_grid()
    ks = set(map(tuple, keys.tolist()))
    rays = synth.random_rays_through(keys, 0.04, 40, seed=3).numpy()
    L = 0.32
    for r in rays:
        iv = G.traverse(r)
        o, d = r[:3].astype(np.float64), r[4:7].astype(np.float64)
        ts = np.linspace(0, 6.0, 60001)[1:]
        pts = o + ts[:, None] * d
        occ = np.array([tuple(np.floor(p / L).astype(int).tolist()) in ks for p in pts])
        inside = np.zeros_like(occ)
        for a, b in iv:
            inside |= (ts > a) & (ts < b)
        # points within 1e-6 of a block plane may go either way
        near = np.zeros_like(occ)
        for a in range(3):
            q = pts[:, a] / L
            near |= np.abs(q - np.round(q)) < 1e-6 / L
        assert np.all((occ == inside) | near)
        # intervals are disjoint, ordered, non-touching (merged)
        for (a0, b0), (a1, b1) in zip(iv[:-1], iv[1:]):
            assert b0 < a1


def test_stratified_sampling_and_deltas():
    sc, keys, G = _tiny_room_grid()
    rays = synth.view_rays(synth.random_poses(sc, 1)[0], 16, 12, synth.intrinsics(16, 12)).numpy()
    N = 64
    for i in (0, 37, 150):
        tr = G.trace(rays[i], N, seed=11, ray_id=i)
        S = G.render(rays[i:i + 1], N, seed=11, ray_id0=i)["S"][0]
        k = np.arange(N)
        assert np.all(tr["s"] >= k * S / N - 1e-12) and np.all(tr["s"] < (k + 1) * S / N + 1e-12)
        np.testing.assert_allclose(tr["delta"][:-1], np.diff(tr["s"]), atol=1e-14)
        assert tr["delta"][-1] == pytest.approx(S - tr["s"][-1], abs=1e-14)
        mid = G.trace(rays[i], N, stratified=False)
        np.testing.assert_allclose(mid["s"], (k + 0.5) * S / N, rtol=1e-14)
        # sample t lies in an allocated interval
        iv = G.traverse(rays[i])
        assert all(any(a - 1e-12 <= t <= b + 1e-12 for a, b in iv) for t in tr["t"])


def test_compositing_invariants():
    sc, keys, G = _tiny_room_grid()
    rays = synth.view_rays(synth.random_poses(sc, 1, seed=2)[0], 16, 12, synth.intrinsics(16, 12)).numpy()
    out = G.render(rays, 64, seed=3)
    for i in range(0, len(rays), 17):
        tr = G.trace(rays[i], 64, seed=3, ray_id=i)
        T = tr["T"]
        assert np.all((T >= 0) & (T <= 1)) and np.all(np.diff(T) <= 1e-15)
        assert tr["w"].sum() == pytest.approx(out["opac"][i], abs=1e-12)
        assert out["opac"][i] == pytest.approx(1 - out["T_N"][i], abs=1e-12)
        np.testing.assert_allclose(tr["w"], T * (1 - np.exp(-tr["sigma"] * tr["delta"])), atol=1e-15)
    # a constant colour field renders C = O * c (+ T_N * bg)
    N = G.n_blocks
    G2 = oracle.Grid(0.04, 0.02).set(keys, G.sdf, np.broadcast_to([0.2, 0.5, 0.9], (N, 512, 3)))
    o2 = G2.render(rays, 64, seed=3, bg=(1.0, 0.0, 0.5))
    np.testing.assert_allclose(o2["rgb"], o2["opac"][:, None] * [0.2, 0.5, 0.9] + o2["T_N"][:, None] * [1, 0, .5],
                               atol=1e-12)


def _plane_expected_depth(k, tstar, beta, ta, tb):
    """Continuous-limit expected depth for d(t) = k (t* - t) over [ta, tb], closed-form optical depth."""
    def tau(t):
        u = k * (t - tstar)
        return math.exp(u / beta) / (2 * k) if u <= 0 else (u + 0.5 * beta * math.exp(-u / beta)) / (beta * k)

    def sig(t):
        d = k * (tstar - t)
        return (0.5 * math.exp(-d / beta) if d >= 0 else 1 - 0.5 * math.exp(d / beta)) / beta

    t0 = tau(ta)
    f = lambda t: t * sig(t) * math.exp(-(tau(t) - t0))
    g = lambda t: sig(t) * math.exp(-(tau(t) - t0))
    pts = [tstar]
    D = integrate.quad(f, ta, tb, points=pts, limit=400, epsabs=1e-13, epsrel=1e-12)[0]
    O = integrate.quad(g, ta, tb, points=pts, limit=400, epsabs=1e-13, epsrel=1e-12)[0]
    return D, O


@pytest.mark.parametrize("beta", [0.004, 0.01])
def test_plane_depth_matches_quadrature_and_converges(beta):
    n = np.array([0.2, 0.3, 1.0])
    n /= np.linalg.norm(n)
    keys, sdf, rgb = synth.plane_grid(n, 0.0, VS, extent_blocks=((-3, 3), (-3, 3), (-3, 3)), slab_blocks=2)
    G = oracle.Grid(VS, beta).set(keys, sdf, rgb)
    o = np.array([0.01, -0.02, 0.2])
    d = np.array([0.1, 0.05, -1.0])
    d /= np.linalg.norm(d)
    ray = np.array([*o, 0.0, *d, 10.0], np.float32)
    o, d = ray[:3].astype(np.float64), ray[4:7].astype(np.float64)
    k = -(n @ d)
    tstar = -(n @ o) / (n @ d)
    iv = G.traverse(ray)
    assert len(iv) == 1
    ta, tb = iv[0]
    Dstar, Ostar = _plane_expected_depth(k, tstar, beta, ta, tb)
    errs = []
    for N in (64, 256, 1024):
        out = G.render(ray[None], N, stratified=False)
        assert out["n_valid"][0] >= N - 4 * N * (VS / (tb - ta))  # only slab-edge samples may be invalid
        errs.append(abs(out["depth"][0] - Dstar))
        delta = (tb - ta) / N
        assert errs[-1] <= 0.05 * delta
        assert out["opac"][0] == pytest.approx(Ostar, abs=1e-6)
    assert errs[2] < errs[0] / 50          # midpoint-rule (second-order) convergence
    # bias bound of the Laplace transform: |D* - t*| <= c beta / k (c = 2 is generous)
    assert abs(Dstar - tstar) <= 2 * beta / k


def test_plane_depth_sharp_limit():
    n = np.array([0.0, 0.0, 1.0])
    keys, sdf, rgb = synth.plane_grid(n, 0.0, VS, extent_blocks=((-2, 2), (-2, 2), (-3, 3)), slab_blocks=2)
    G = oracle.Grid(VS, 1e-5).set(keys, sdf, rgb)
    ray = np.array([0.003, 0.004, 0.15, 0.0, 0.0, 0.0, -1.0, 10.0], np.float32)
    N = 512
    out = G.render(ray[None], N, stratified=False)
    iv = G.traverse(ray)
    delta = (iv[-1][1] - iv[0][0]) / N
    assert out["depth"][0] == pytest.approx(0.15, abs=delta)
    assert out["opac"][0] == pytest.approx(1.0, abs=1e-9)


def _fd_grid(n_sem=0, seed=0):
    keys = np.array([[x, y, z] for z in (0, 1) for y in (0, 1) for x in (0, 1)], np.int32)
    x = synth.voxel_positions(keys, VS).numpy()
    rng = np.random.default_rng(seed)
    sdf = (x @ np.array([0.1, 0.2, 1.0]) - 0.08) * 0.9 + 0.002 * rng.normal(size=x.shape[:2])
    rgb = rng.uniform(0, 1, size=x.shape)
    sem = rng.normal(size=x.shape[:2] + (n_sem,)) if n_sem else None
    o = np.stack([rng.uniform(0.03, 0.13, 8), rng.uniform(0.03, 0.13, 8), np.full(8, 0.2)], 1)
    tgt = np.stack([rng.uniform(0.04, 0.12, 8), rng.uniform(0.04, 0.12, 8), np.full(8, 0.0)], 1)
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.concatenate([o, np.zeros((8, 1)), d, np.full((8, 1), 5.0)], 1).astype(np.float32)
    return keys, sdf, rgb, sem, rays


@pytest.mark.parametrize("n_sem,bg", [(0, (0, 0, 0)), (4, (0.3, 0.6, 0.1))])
def test_backward_matches_central_differences(n_sem, bg):
    keys, sdf, rgb, sem, rays = _fd_grid(n_sem)
    G = oracle.Grid(VS, BETA, n_sem)
    G.set(keys, sdf, rgb, sem)
    rng = np.random.default_rng(3)
    n = len(rays)
    gc, gd, go = rng.normal(size=(n, 3)), rng.normal(size=n), rng.normal(size=n)
    gs = rng.normal(size=(n, n_sem)) if n_sem else None
    N = 16

    def L(sdf_, rgb_, sem_):
        G.set(keys, sdf_, rgb_, sem_)
        o = G.render(rays, N, seed=5, bg=bg)
        v = (o["rgb"] * gc).sum() + (o["depth"] * gd).sum() + (o["opac"] * go).sum()
        if n_sem:
            v += (o["sem"] * gs).sum()
        return v

    G.set(keys, sdf, rgb, sem)
    assert G.render(rays, N, seed=5)["n_valid"].min() > 0
    an = G.backward(rays, N, gc, gd, go, gs, seed=5, bg=bg)
    assert np.abs(an["sdf"]).max() > 0
    h = 1e-6
    checks = [("sdf", sdf), ("rgb", rgb)] + ([("sem", sem)] if n_sem else [])
    for name, arr in checks:
        flat = arr.reshape(-1)
        nz = np.flatnonzero(an[name].reshape(-1))
        idx = np.concatenate([rng.choice(nz, min(40, len(nz)), replace=False), rng.integers(0, flat.size, 10)])
        scale = np.abs(an[name]).max()
        for j in idx:
            p = {"sdf": sdf.copy(), "rgb": rgb.copy(), "sem": None if sem is None else sem.copy()}
            m = {k: (None if v is None else v.copy()) for k, v in p.items()}
            p[name].reshape(-1)[j] += h
            m[name].reshape(-1)[j] -= h
            fd = (L(p["sdf"], p["rgb"], p["sem"]) - L(m["sdf"], m["rgb"], m["sem"])) / (2 * h)
            a = an[name].reshape(-1)[j]
            assert abs(fd - a) <= 1e-6 * abs(a) + 1e-7 * scale, (name, j, fd, a)


def test_loss_seeds_match_finite_differences():
    rng = np.random.default_rng(4)
    n, ns = 6, 3
    rgb, trgb = rng.uniform(size=(n, 3)), rng.uniform(size=(n, 3))
    dep, tdep = rng.uniform(1, 2, n), rng.uniform(1, 2, n)
    sem, tsem = rng.normal(size=(n, ns)), rng.normal(size=(n, ns))
    L, g = oracle.loss(rgb, dep, trgb, tdep, 0.1, sem, tsem, 0.1)
    expect = np.abs(rgb - trgb).mean() + 0.1 * np.abs(dep - tdep).mean() + 0.1 * ((sem - tsem) ** 2).sum(1).mean()
    assert L == pytest.approx(expect, rel=1e-14)
    h = 1e-7
    for arr, key in ((rgb, "rgb"), (dep, "depth"), (sem, "sem")):
        for j in range(arr.size):
            p, m = arr.copy(), arr.copy()
            p.reshape(-1)[j] += h
            m.reshape(-1)[j] -= h
            args = lambda a: {"rgb": (a, dep, sem), "depth": (rgb, a, sem), "sem": (rgb, dep, a)}[key]
            Lp = oracle.loss(args(p)[0], args(p)[1], trgb, tdep, 0.1, args(p)[2], tsem, 0.1)[0]
            Lm = oracle.loss(args(m)[0], args(m)[1], trgb, tdep, 0.1, args(m)[2], tsem, 0.1)[0]
            assert (Lp - Lm) / (2 * h) == pytest.approx(g[key].reshape(-1)[j], rel=1e-6, abs=1e-9)
    _, g0 = oracle.loss(trgb, tdep, trgb, tdep)
    assert np.all(g0["rgb"] == 0) and np.all(g0["depth"] == 0)


def test_adam_step_one_closed_form_and_torch():
    import torch
    rng = np.random.default_rng(6)
    g = rng.normal(size=50)
    th = rng.normal(size=50)
    t0, gg, m, v = th.copy(), g.copy(), np.zeros(50), np.zeros(50)
    oracle.adam(t0, gg, m, v, lr=1e-3, step=1)
    np.testing.assert_allclose(t0, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.all(gg == 0)
    # three steps against torch.optim.Adam in float64
    p = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    t1, m, v = th.copy(), np.zeros(50), np.zeros(50)
    for s in range(1, 4):
        gs = rng.normal(size=50)
        p.grad = torch.tensor(gs)
        opt.step()
        gg = gs.copy()
        oracle.adam(t1, gg, m, v, lr=1e-3, step=s)
    np.testing.assert_allclose(t1, p.detach().numpy(), rtol=0, atol=1e-14)


def test_rmsprop_matches_torch():
    import torch
    rng = np.random.default_rng(7)
    th = rng.normal(size=30)
    p = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.RMSprop([p], lr=1e-3, alpha=0.99, eps=1e-8)
    t1, v = th.copy(), np.zeros(30)
    for _ in range(3):
        gs = rng.normal(size=30)
        p.grad = torch.tensor(gs)
        opt.step()
        oracle.rmsprop(t1, gs.copy(), v, lr=1e-3, alpha=0.99, eps=1e-8)
    np.testing.assert_allclose(t1, p.detach().numpy(), rtol=0, atol=1e-14)


def test_view_rays_match_independent_pinhole():
    sc = synth.scene_tiny_room(0)
    T = synth.random_poses(sc, 1)[0]
    K = synth.intrinsics(20, 10)
    a = oracle.view_rays(10, 20, K, T)
    b = synth.view_rays(T, 20, 10, K).numpy()
    np.testing.assert_allclose(a, b, atol=2e-7)


def test_degenerate_rays_are_rare_on_tiny_room():
    sc, keys, G = _tiny_room_grid()
    rays = synth.view_rays(synth.random_poses(sc, 1)[0], 64, 48, synth.intrinsics(64, 48)).numpy()
    out = G.render(rays, 64, seed=1)
    assert out["degenerate"].mean() < 0.02
    assert np.all(np.isfinite(out["rgb"])) and np.all(out["opac"] <= 1 + 1e-12)


def test_lookup_present_and_absent():
    sc, keys, G = _tiny_room_grid()
    idx = G.lookup(keys)
    assert idx.tolist() == list(range(len(keys)))
    absent = keys + np.array([1000, 0, 0], np.int32)
    assert np.all(G.lookup(absent) == -1)
