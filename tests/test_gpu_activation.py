"""GPU parity of block activation (Eq. 7-8) and the block hash map against the oracle: bit-exact key sets,
index order, lookups, capacity behaviour and checkpoints."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sdg():
    import paper_2305_13220_b300 as m
    return m


@pytest.mark.parametrize("r", [0, 3, 4, 16])
def test_activate_points_bit_exact(sdg, r):
    rng = np.random.default_rng(100 + r)
    pts = np.concatenate([rng.uniform(-1.3, 2.1, size=(60000, 3)),
                          rng.normal(0.5, 0.01, size=(20000, 3))]).astype(np.float32)
    pts[:5] = [[np.nan, 0, 0], [np.inf, 1, 1], [0.0, -0.0, 0.079999995], [-1e-9, 0, 0], [1e30, 0, 0]]
    ks = oracle.KeySet()
    ks.add_points(pts, 0.01, r)
    want = ks.keys()
    G = sdg.Grid(0.01, len(want) + 10)
    n = G.activate_points(torch.as_tensor(pts, device="cuda"), r)
    assert n == len(want)
    np.testing.assert_array_equal(G.keys().cpu().numpy(), want)


def _expected_batches(views, K, vs, r):
    """Oracle index order: each activation batch appends its new keys in ascending (z, y, x) order."""
    ks = oracle.KeySet()
    order = np.zeros((0, 3), np.int32)
    for T, d in views:
        before = set(map(tuple, ks.keys().tolist()))
        ks.add_depth(d, K, T, vs, r)
        new = [k for k in ks.keys().tolist() if tuple(k) not in before]
        order = np.concatenate([order, np.array(new, np.int32).reshape(-1, 3)])
    return order


@pytest.mark.parametrize("which", ["tiny_room", "room_scale"])
def test_activate_depth_bit_exact(sdg, which):
    if which == "tiny_room":
        sc, vs, r, W, H, nv, cap = synth.scene_tiny_room(0), 0.04, 3, 64, 48, 4, 4096
    else:
        sc, vs, r, W, H, nv, cap = synth.scene_room(0), 0.01, 4, 640, 480, 3, 200000
    poses = synth.random_poses(sc, nv, seed=3)
    K = synth.intrinsics(W, H)
    views = [(T, synth.depth_map(sc, T, W, H, K)) for T in poses]
    G = sdg.Grid(vs, cap)
    total = sum(G.activate_depth(d.cuda(), K, T, r) for T, d in views)
    want = _expected_batches(views, K, vs, r)
    assert total == len(want) == G.num_blocks
    np.testing.assert_array_equal(G.keys().cpu().numpy(), want)


def test_activate_depth_frames_is_one_batch(sdg):
    """F depth maps in one call: the union of their blocks, indexed in ascending (z, y, x) order over the whole
    batch (the oracle's key set), the same block set as map-by-map calls, all-or-nothing on capacity."""
    sc, vs, r, W, H = synth.scene_tiny_room(0), 0.04, 3, 64, 48
    K = synth.intrinsics(W, H)
    poses = synth.random_poses(sc, 6, seed=5)
    views = [(T, synth.depth_map(sc, T, W, H, K)) for T in poses]
    depth = torch.stack([d for _, d in views]).cuda()
    Tw = np.stack([np.asarray(T, np.float64) for T, _ in views])
    ks = oracle.KeySet()
    for T, d in views[:4]:
        ks.add_depth(d, K, T, vs, r)
    first = ks.keys()
    G = sdg.Grid(vs, 4096)
    n = G.activate_depth_frames(depth[:4].contiguous(), K, Tw[:4], r)
    assert n == len(first) == G.num_blocks
    np.testing.assert_array_equal(G.keys().cpu().numpy(), first)
    # a second batch appends its new blocks, again in ascending order; zero maps add nothing
    for T, d in views[4:]:
        ks.add_depth(d, K, T, vs, r)
    old = set(map(tuple, first.tolist()))
    second = np.array([k for k in ks.keys().tolist() if tuple(k) not in old], np.int32).reshape(-1, 3)
    assert G.activate_depth_frames(depth[4:].contiguous(), K, Tw[4:], r) == len(second)
    np.testing.assert_array_equal(G.keys().cpu().numpy(), np.concatenate([first, second]))
    assert G.activate_depth_frames(depth[:0], K, Tw[:0], r) == 0
    # per-frame intrinsics: each frame unprojected with its own K, as map-by-map calls do
    Kf = np.tile(np.asarray(K, np.float64), (6, 1))
    Kf[1, 0] *= 1.25
    Kf[3, 1] *= 0.8
    Kf[4, 2] += 3.0
    Ga, Gb = sdg.Grid(vs, 4096), sdg.Grid(vs, 4096)
    Ga.activate_depth_frames(depth, Kf, Tw, r)
    for f, (T, d) in enumerate(views):
        Gb.activate_depth(d.cuda(), Kf[f], T, r)
    assert set(map(tuple, Ga.keys().cpu().numpy().tolist())) == set(map(tuple, Gb.keys().cpu().numpy().tolist()))
    # map by map: the same set
    G2 = sdg.Grid(vs, 4096)
    for T, d in views:
        G2.activate_depth(d.cuda(), K, T, r)
    assert set(map(tuple, G2.keys().cpu().numpy().tolist())) == set(map(tuple, ks.keys().tolist()))
    # one block short of the batch: nothing is added
    G3 = sdg.Grid(vs, len(first) - 1)
    with pytest.raises(sdg.SdgError):
        G3.activate_depth_frames(depth[:4].contiguous(), K, Tw[:4], r)
    assert G3.num_blocks == 0
    # a zero focal length in any frame is rejected before any work
    Kb = np.tile(np.asarray(K, np.float64), (4, 1))
    Kb[2, 0] = 0.0
    with pytest.raises(sdg.SdgError):
        G3.activate_depth_frames(depth[:4].contiguous(), Kb, Tw[:4], r)
    assert G3.num_blocks == 0


def test_lookup_present_and_absent(sdg):
    sc = synth.scene_tiny_room(0)
    keys = synth.band_blocks(sc, 0.04, 3)
    G = sdg.Grid(0.04, 2048)
    G.activate_keys(torch.as_tensor(keys, device="cuda"))
    gk = G.keys()
    idx = G.lookup(gk).cpu().numpy()
    np.testing.assert_array_equal(idx, np.arange(len(keys)))
    rng = np.random.default_rng(1)
    absent = rng.integers(-(1 << 20), 1 << 20, size=(1_000_000, 3)).astype(np.int32)
    O = oracle.Grid(0.04, 0.02).set(gk.cpu().numpy(), np.zeros((len(keys), 512)), np.zeros((len(keys), 512, 3)))
    want = O.lookup(absent)
    got = G.lookup(torch.as_tensor(absent, device="cuda")).cpu().numpy()
    np.testing.assert_array_equal(got, want)
    assert (got == -1).mean() > 0.999


def test_capacity_error_leaves_grid_unchanged(sdg):
    G = sdg.Grid(0.01, 100)
    rng = np.random.default_rng(2)
    small = torch.as_tensor(rng.uniform(0, 0.05, size=(50, 3)).astype(np.float32), device="cuda")
    n0 = G.activate_points(small, 0)
    k0 = G.keys().cpu().numpy()
    big = torch.as_tensor(rng.uniform(-5, 5, size=(5000, 3)).astype(np.float32), device="cuda")
    with pytest.raises(sdg.SdgError) as e:
        G.activate_points(big, 2)
    assert e.value.code == sdg._abi.ERR_CAPACITY
    assert G.num_blocks == n0
    np.testing.assert_array_equal(G.keys().cpu().numpy(), k0)
    # the de-duplication set was emptied: a fitting batch still activates exactly its new keys
    more = torch.as_tensor(np.array([[1.0, 1.0, 1.0]], np.float32), device="cuda")
    assert G.activate_points(more, 0) == 1
    assert G.num_blocks == n0 + 1


def test_block_bounding_box_limit_leaves_grid_unchanged(sdg):
    """The traversal keeps a 4-byte block index for every cell of the block AABB; a batch that would stretch the
    AABB beyond 2^31 cells is refused before anything is inserted."""
    G = sdg.Grid(0.01, 64)
    k0 = torch.tensor([[0, 0, 0], [1, 0, 0]], dtype=torch.int32, device="cuda")
    assert G.activate_keys(k0) == 2
    far = torch.tensor([[(1 << 20) - 1, (1 << 20) - 1, 0], [2, 0, 0]], dtype=torch.int32, device="cuda")
    with pytest.raises(sdg.SdgError) as e:
        G.activate_keys(far)  # AABB 2^20 x 2^20 x 1 cells
    assert e.value.code == sdg._abi.ERR_CAPACITY
    assert G.num_blocks == 2
    np.testing.assert_array_equal(G.lookup(k0).cpu().numpy(), [0, 1])
    assert G.activate_keys(torch.tensor([[2, 0, 0]], dtype=torch.int32, device="cuda")) == 1  # still usable


def test_activate_keys_duplicates_and_present(sdg):
    G = sdg.Grid(0.01, 64)
    k = torch.tensor([[0, 0, 0], [1, 0, 0], [0, 0, 0], [-3, 2, 1]], dtype=torch.int32, device="cuda")
    assert G.activate_keys(k) == 3
    assert G.activate_keys(k) == 0
    np.testing.assert_array_equal(G.keys().cpu().numpy(), [[0, 0, 0], [1, 0, 0], [-3, 2, 1]])
    bad = torch.tensor([[1 << 20, 0, 0]], dtype=torch.int32, device="cuda")
    with pytest.raises(sdg.SdgError):
        G.activate_keys(bad)
    assert G.num_blocks == 3


def test_empty_activation(sdg):
    G = sdg.Grid(0.01, 16)
    assert G.activate_points(torch.zeros((0, 3), device="cuda"), 3) == 0
    assert G.num_blocks == 0


def test_save_load_roundtrip(sdg, tmp_path):
    from tests.gpu_util import tiny_room
    sc, G, O, stored, vals = tiny_room()
    G.step = 7
    p = str(tmp_path / "g.sdg")
    G.save(p)
    H = sdg.Grid.load(p, max_blocks=G.max_blocks)
    assert H.num_blocks == G.num_blocks and H.step == 7
    np.testing.assert_array_equal(H.keys().cpu().numpy(), G.keys().cpu().numpy())
    A = sdg._abi
    N = G.num_blocks
    assert torch.equal(H.channel(A.GROUP_GEO)[:N], G.channel(A.GROUP_GEO)[:N])
    np.testing.assert_array_equal(H.lookup(G.keys()).cpu().numpy(), np.arange(N))
