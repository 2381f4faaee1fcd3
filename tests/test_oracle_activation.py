"""Pins for the oracle's block activation (Eq. 7-8 and the supplement's Dilate_R).

Each test checks the oracle against something other than itself: the analytic
surface a depth map was rendered from, a brute-force enumeration of the voxel
cube, hand-computed keys, or the block-level dilation definition."""
import itertools

import numpy as np
import pytest

import oracle
import synth


def test_unprojected_points_lie_on_the_surface():
    # Eq. 8 with phi = 1: a depth map rendered analytically must unproject back onto the scene surface.
    sc = synth.scene_room(3, size=(4.0, 3.5, 2.8), n_objects=4)
    poses = synth.random_poses(sc, 3, seed=1)
    W, H = 64, 48
    K = synth.intrinsics(W, H)
    for T in poses:
        dmap = synth.depth_map(sc, T, W, H, K)
        xyz, valid = oracle.unproject(dmap, K, T)
        assert valid.all()
        import torch
        d = synth.scene_sdf(sc, torch.tensor(xyz.astype(np.float64))).numpy()
        # FP32 unprojection of points a few metres away: error well below a micrometre per metre
        assert np.abs(d).max() < 5e-6 * max(1.0, float(dmap.max()))


def test_unproject_marks_bad_depth_invalid():
    depth = np.array([[1.0, 0.0, -2.0], [np.nan, np.inf, 3.0]], np.float32)
    T = np.concatenate([np.eye(3), np.zeros((3, 1))], 1)
    xyz, valid = oracle.unproject(depth, (100.0, 100.0, 1.5, 1.0), T)
    assert valid.tolist() == [1, 0, 0, 0, 0, 1]
    # pixel (u=0, v=0) at depth 1: x = (0.5 - 1.5)/100 = -0.01, y = (0.5 - 1)/100 = -0.005, z = 1
    np.testing.assert_allclose(xyz[0], [-0.01, -0.005, 1.0], rtol=1e-6)


def _brute_keys(xyz, vs, r):
    inv = np.float32(1.0) / np.float32(vs)
    out = set()
    for p in xyz:
        v = np.floor(p.astype(np.float32) * inv).astype(np.int64)
        for o in itertools.product(range(-r, r + 1), repeat=3):
            w = v + np.array(o)
            out.add(tuple(int(c) for c in (w // 8)))
    return sorted(out, key=lambda k: (k[2], k[1], k[0]))


@pytest.mark.parametrize("r", [0, 1, 3, 4, 9])
def test_activation_matches_voxel_cube_enumeration(r):
    rng = np.random.default_rng(r)
    xyz = rng.uniform(-0.7, 0.9, size=(150, 3)).astype(np.float32)
    ks = oracle.KeySet()
    ks.add_points(xyz, 0.01, r)
    got = [tuple(k) for k in ks.keys().tolist()]
    assert got == _brute_keys(xyz, 0.01, r)


@pytest.mark.parametrize("R", [1, 2])
def test_voxel_dilation_8R_is_block_dilation_R(R):
    # Supplement: Dilate_R grows the block of a point to the (2R+1)^3 block cube (L-inf reading).
    rng = np.random.default_rng(10 + R)
    xyz = rng.uniform(-0.5, 0.5, size=(60, 3)).astype(np.float32)
    ks = oracle.KeySet()
    ks.add_points(xyz, 0.015, 8 * R)
    inv = np.float32(1.0) / np.float32(0.015)
    expect = set()
    for p in xyz:
        b = np.floor(p * inv).astype(np.int64) // 8
        for o in itertools.product(range(-R, R + 1), repeat=3):
            expect.add(tuple(int(c) for c in b + np.array(o)))
    assert set(map(tuple, ks.keys().tolist())) == expect


def test_activation_floor_semantics_by_hand():
    # vs = 0.01: x = -0.001 -> voxel -1 -> block -1 (floor, not truncation); 0.079 -> voxel 7 -> block 0;
    # 0.081 -> voxel 8 -> block 1; -0.081 -> voxel -9 -> block -2.
    pts = np.array([[-0.001, 0.0, 0.079], [0.081, -0.081, 0.5]], np.float32)
    ks = oracle.KeySet()
    ks.add_points(pts, 0.01, 0)
    assert ks.keys().tolist() == [[-1, 0, 0], [1, -2, 6]]


def test_keys_sorted_unique_zyx():
    rng = np.random.default_rng(5)
    ks = oracle.KeySet()
    ks.add_points(rng.uniform(-1, 1, size=(500, 3)).astype(np.float32), 0.02, 3)
    k = ks.keys()
    packed = [(z, y, x) for x, y, z in k.tolist()]
    assert packed == sorted(set(packed))


def test_activation_skips_invalid_and_accumulates():
    ks = oracle.KeySet()
    ks.add_points(np.array([[0.0, 0.0, 0.0]], np.float32), 0.01, 0, valid=np.array([0], np.uint8))
    assert ks.keys().shape[0] == 0
    ks.add_points(np.array([[0.0, 0.0, 0.0]], np.float32), 0.01, 0)
    ks.add_points(np.array([[0.005, 0.0, 0.0]], np.float32), 0.01, 0)
    assert ks.keys().tolist() == [[0, 0, 0]]


def test_depth_activation_covers_surface_band():
    # Every block that contains a surface point seen by the camera must be active after activation.
    sc = synth.scene_tiny_room(1)
    T = synth.random_poses(sc, 1, seed=4)[0]
    K = synth.intrinsics(32, 24)
    dmap = synth.depth_map(sc, T, 32, 24, K)
    ks = oracle.KeySet()
    ks.add_depth(dmap, K, T, 0.04, 3)
    keys = set(map(tuple, ks.keys().tolist()))
    xyz, _ = oracle.unproject(dmap, K, T)
    own = {tuple(int(c) for c in np.floor(p / 0.32)) for p in xyz.astype(np.float64)}
    assert own <= keys
