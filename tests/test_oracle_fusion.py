"""Pins of the oracle's volumetric fusion (Sec. 3.4.2, Eq. 9-11; the supplement's truncation psi).

The fused SDF of a plane observed head-on is the true signed distance to the plane (truncated at mu in front,
rejected beyond mu behind): a geometric fact independent of the fusion formula.  Cameras are rotated by a
non-symmetric rotation and translated, so a transposed rotation or a dropped translation fails.  Averages,
normalisation, order independence and the pixel-centre convention are pinned by cases whose answer is known
without the formula."""
import numpy as np

import oracle

VS = 0.04
MU = 0.12
W, H = 64, 48
K = np.array([50.0, 50.0, 32.0, 24.0], np.float32)
# camera z -> world +x, camera x -> world +y, camera y -> world +z (not symmetric: R^T != R)
R = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])


def pose(t):
    T = np.zeros((3, 4), np.float32)
    T[:, :3] = R
    T[:, 3] = t
    return T


def plane_keys():
    """Blocks around the plane x = 2 m inside the cameras' frustum (block edge 0.32 m)."""
    ks = [(bx, by, bz) for bx in range(4, 9) for by in range(-3, 3) for bz in range(-3, 3)]
    return np.array(ks, np.int32)


def voxel_xyz(keys):
    l = np.arange(512)
    loc = np.stack([l & 7, (l >> 3) & 7, l >> 6], -1)
    v = keys[:, None, :] * 8 + loc[None]
    return v * np.float64(np.float32(VS))  # FP32 voxel size, as the fusion uses it


def test_plane_sdf_is_the_truncated_distance():
    keys = plane_keys()
    t = np.array([0.3, -0.2, 0.1], np.float32)
    depth = np.full((H, W), 2.0 - 0.3, np.float32)  # plane x = 2 seen head-on from x = 0.3
    out = oracle.fuse(keys, VS, depth, K, pose(t), MU)
    x = voxel_xyz(keys)
    d_true = 2.0 - x[..., 0]
    w = out["weight"]
    seen = w > 0
    assert seen.sum() > 2000
    # every kept voxel: the truncated true distance (FP32 projection: a few ulps of 2 m)
    np.testing.assert_allclose(out["sdf"][seen], np.minimum(d_true[seen], MU), atol=2e-6)
    # voxels beyond mu behind the plane are never kept; those in front of it by more than mu read mu
    assert not seen[d_true < -MU - 1e-5].any()
    far = seen & (d_true > MU + 1e-5)
    assert far.sum() > 500 and np.all(out["sdf"][far] == np.float32(MU))
    # the frustum: a voxel whose direction leaves the image is not kept
    ang = np.abs(x[..., 1] - t[1]) / (x[..., 0] - t[0])
    assert not seen[ang > 32.0 / 50.0 + 1e-3].any()
    assert np.all(out["weight"][~seen] == 0) and np.all(out["sdf"][~seen] == 0)


def test_two_views_agree_and_weights_count():
    keys = plane_keys()
    t1, t2 = np.array([0.0, 0.0, 0.0], np.float32), np.array([0.5, 0.1, -0.1], np.float32)
    depth = np.stack([np.full((H, W), 2.0, np.float32), np.full((H, W), 1.5, np.float32)])
    out = oracle.fuse(keys, VS, depth, K, np.stack([pose(t1), pose(t2)]), MU)
    d_true = 2.0 - voxel_xyz(keys)[..., 0]
    w = out["weight"]
    assert (w == 2).sum() > 1000 and (w == 1).sum() > 100
    seen = w > 0
    np.testing.assert_allclose(out["sdf"][seen], np.minimum(d_true[seen], MU), atol=2e-6)


def test_colour_is_the_mean_and_logits_are_normalised():
    keys = plane_keys()
    t1, t2 = np.array([0.0, 0.0, 0.0], np.float32), np.array([0.5, 0.1, -0.1], np.float32)
    depth = np.stack([np.full((H, W), 2.0, np.float32), np.full((H, W), 1.5, np.float32)])
    c1, c2 = np.array([0.25, 0.5, 1.0]), np.array([0.75, 0.0, 0.5])
    rgb = np.stack([np.broadcast_to(c1, (H, W, 3)), np.broadcast_to(c2, (H, W, 3))]).astype(np.float32)
    sem = np.zeros((2, H, W, 4), np.float32)
    sem[0, ..., 0], sem[0, ..., 2] = 1.5, 3.0
    sem[1, ..., 0], sem[1, ..., 2] = 1.5, 1.0
    out = oracle.fuse(keys, VS, depth, K, np.stack([pose(t1), pose(t2)]), MU, rgb=rgb, sem=sem)
    w = out["weight"]
    both, only1 = w == 2, w == 1
    np.testing.assert_allclose(out["rgb"][both], np.broadcast_to((c1 + c2) / 2, (both.sum(), 3)), atol=1e-15)
    # voxels kept by one view only: that view's colour
    one = out["rgb"][only1]
    assert np.all(np.isclose(one, c1).all(-1) | np.isclose(one, c2).all(-1))
    # mean logits (1.5, 0, 2, 0)/|.| where both views keep the voxel; unit norm everywhere it is kept
    s = out["sem"]
    np.testing.assert_allclose(s[both], np.broadcast_to(np.array([1.5, 0, 2, 0]) / 2.5, (both.sum(), 4)),
                               atol=1e-15)
    np.testing.assert_allclose(np.linalg.norm(s[w > 0], axis=-1), 1.0, atol=1e-12)
    assert np.all(s[w == 0] == 0)


def test_order_and_duplicates():
    keys = plane_keys()
    rng = np.random.default_rng(0)
    ts = [np.array([0.0, 0.0, 0.0], np.float32), np.array([0.5, 0.1, -0.1], np.float32),
          np.array([0.2, -0.3, 0.2], np.float32)]
    depth = (2.0 - np.array([t[0] for t in ts], np.float32))[:, None, None] \
        + rng.normal(0, 0.02, (3, H, W)).astype(np.float32)
    rgb = rng.uniform(0, 1, (3, H, W, 3)).astype(np.float32)
    T = np.stack([pose(t) for t in ts])
    a = oracle.fuse(keys, VS, depth, K, T, MU, rgb=rgb)
    b = oracle.fuse(keys, VS, depth[::-1], K, T[::-1], MU, rgb=rgb[::-1])
    for k in a:
        np.testing.assert_allclose(a[k], b[k], rtol=1e-14, atol=1e-15)
    c = oracle.fuse(keys, VS, np.concatenate([depth, depth]), K, np.concatenate([T, T]), MU,
                    rgb=np.concatenate([rgb, rgb]))
    np.testing.assert_array_equal(c["weight"], 2 * a["weight"])
    np.testing.assert_allclose(c["sdf"], a["sdf"], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(c["rgb"], a["rgb"], rtol=1e-14, atol=1e-15)


def test_pixel_centre_convention():
    """Pixel (u, v) covers [u, u+1) x [v, v+1) of the projected coordinate (centre at u + 0.5), the same
    convention as unprojection: a voxel on the optical axis projects to pu = cx = 32.0, pixel column 32."""
    keys = np.array([[6, -1, -1]], np.int32)  # block x in [1.92, 2.24), y, z in [-0.32, 0)
    depth = np.full((H, W), 2.0, np.float32)
    depth[:, 32:] = 2.1
    T = pose(np.zeros(3, np.float32))
    out = oracle.fuse(keys, VS, depth, K, T, MU)
    x = voxel_xyz(keys)[0]
    # local voxel (3, 7, 7): world (2.04, -0.04, -0.04), pu = 32 - 50 * 0.04 / 2.04 = 31.02 -> column 31 (2.0 m)
    l = 3 + 7 * 8 + 7 * 64
    pu = 50.0 * (-0.04 / x[l, 0]) + 32.0
    assert 31.0 < pu < 32.0
    np.testing.assert_allclose(out["sdf"][0, l], 2.0 - x[l, 0], atol=2e-6)
    # a voxel on the axis (y = 0 -> pu = 32.0 exactly) reads column 32 (the 2.1 m half)
    keys2 = np.array([[6, 0, -1]], np.int32)
    out2 = oracle.fuse(keys2, VS, depth, K, T, MU)
    x2 = voxel_xyz(keys2)[0]
    l2 = 3 + 0 * 8 + 7 * 64  # world (2.04, 0, -0.04)
    np.testing.assert_allclose(out2["sdf"][0, l2], 2.1 - x2[l2, 0], atol=2e-6)
    # local voxel (0, 7, 7) of block (13, -1, -1): world (4.16, -0.04, -0.04), pu = 31.52: floor -> column 31
    keys3 = np.array([[13, -1, -1]], np.int32)
    depth3 = np.full((H, W), 4.2, np.float32)
    depth3[:, 32:] = 4.3
    out3 = oracle.fuse(keys3, VS, depth3, K, T, MU)
    x3 = voxel_xyz(keys3)[0]
    l3 = 0 + 7 * 8 + 7 * 64
    assert 31.5 < 50.0 * (-0.04 / x3[l3, 0]) + 32.0 < 32.0
    np.testing.assert_allclose(out3["sdf"][0, l3], 4.2 - x3[l3, 0], atol=2e-6)
