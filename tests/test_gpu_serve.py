"""Serving loop: continuous batching across scenes and resolutions; each result must equal the same request
rendered alone (bit-for-bit: rays are computed independently of their batch mates) and match the oracle on every
pixel: the served view's rays and sample placement are exported by sdg_debug_trace_view (the serving kernel's own
ray and traversal code; its outputs equal the served result bit for bit), the placement is checked against the
oracle's FP64 traversal, and the oracle renders every pixel from those samples."""
import time

import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import check_placement, gpu_samples, make_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sdg():
    import paper_2305_13220_b300 as m
    return m


@pytest.fixture(scope="module")
def scenes():
    out = []
    for seed, dtype in ((0, "bf16"), (1, "bf16")):
        sc = synth.scene_room(seed, size=(2.0 + seed, 2.0, 2.0), n_objects=2)
        keys = synth.band_blocks(sc, 0.04, 3)
        G, O, stored, vals = make_pair(sc, keys, 0.04, 3, 0.02, dtype)
        out.append((sc, G, O))
    return out


def _req(sc, W, H, seed):
    T = synth.random_poses(sc, 1, seed=seed)[0]
    return T, synth.intrinsics(W, H)


def test_mix_equals_alone_and_oracle(sdg, scenes):
    srv = sdg.Server(hbm_budget_bytes=64 << 20, max_slots=6, n_streams=3, chunk_rays=1024, max_batch_rays=8192)
    ids = [srv.add_scene(G) for _, G, _ in scenes]
    reqs = []
    rng = np.random.default_rng(0)
    for i in range(12):
        s = int(rng.integers(0, 2))
        W, H = [(40, 30), (80, 60), (64, 48)][i % 3]
        T, K = _req(scenes[s][0], W, H, seed=i)
        reqs.append((s, W, H, T, K, 64 if i % 2 else 128, 100 + i))
    # alone: one at a time
    alone = []
    for s, W, H, T, K, N, seed in reqs:
        t = srv.submit(ids[s], H, W, K, T, n_samples=N, seed=seed)
        r = srv.wait(t, 60000)
        alone.append(srv.result_tensors(r))
        srv.release(t)
    # mixed: all at once
    tickets = [srv.submit(ids[s], H, W, K, T, n_samples=N, seed=seed) for s, W, H, T, K, N, seed in reqs]
    for t, ref in zip(tickets, alone):
        r = srv.wait(t, 60000)
        got = srv.result_tensors(r)
        for a, b in zip(got, ref):
            assert torch.equal(a, b)
        assert r.t_done_ms >= r.t_admit_ms >= r.t_submit_ms
        srv.release(t)
    st = srv.stats()
    assert st.completed == 24 and st.bytes_in_use == 0 and st.peak_bytes_in_use <= 64 << 20
    # oracle parity, every pixel, for two of the requests
    for i in (0, 7):
        s, W, H, T, K, N, seed = reqs[i]
        tr = sdg.trace_view(scenes[s][1], H, W, K, T, N, seed=seed)
        rgb, depth, opac = alone[i]
        assert torch.equal(tr["rgb"].reshape(rgb.shape), rgb) and torch.equal(tr["depth"].reshape(depth.shape), depth)
        assert torch.equal(tr["opac"].reshape(opac.shape), opac)
        rays = tr["rays"].cpu().numpy()
        np.testing.assert_allclose(rays, oracle.view_rays(H, W, K, T), atol=2e-6)  # the pinhole model itself
        check_placement(scenes[s][2], rays, tr, N, seed=seed)
        ref = scenes[s][2].render(rays, N, seed=seed, given=gpu_samples(tr))
        assert np.abs(rgb.double().cpu().numpy().reshape(-1, 3) - ref["rgb"]).max() < 1e-4
        assert np.abs(depth.double().cpu().numpy().reshape(-1) - ref["depth"]).max() < 1e-4
        assert np.abs(opac.double().cpu().numpy().reshape(-1) - ref["opac"]).max() < 1e-4
    srv.close()


def test_admission_by_memory_and_errors(sdg, scenes):
    one = 80 * 60 * 5 * 4
    srv = sdg.Server(hbm_budget_bytes=one + 4096, max_slots=8, n_streams=2, chunk_rays=512, max_batch_rays=4096)
    sid = srv.add_scene(scenes[0][1])
    T, K = _req(scenes[0][0], 80, 60, seed=3)
    ts = [srv.submit(sid, 60, 80, K, T, n_samples=64, seed=i) for i in range(5)]
    for t in ts:
        r = srv.wait(t, 60000)
        assert r.status == 0
        srv.release(t)
    st = srv.stats()
    assert st.peak_bytes_in_use <= one + 4096 and st.completed == 5
    with pytest.raises(sdg.SdgError) as e:
        srv.submit(sid, 600, 800, K, T)
    assert e.value.code == sdg._abi.ERR_CAPACITY
    with pytest.raises(sdg.SdgError):
        srv.submit(99, 10, 10, K, T)
    # cancel a queued request and time out on a wait of 0 ms
    t1 = srv.submit(sid, 60, 80, K, T, n_samples=256)
    t2 = srv.submit(sid, 60, 80, K, T, n_samples=256)
    srv.release(t2)
    with pytest.raises(sdg.SdgError):
        srv.poll(t2)
    try:
        srv.wait(t1, 0)
    except sdg.SdgError as err:
        assert err.code == sdg._abi.ERR_TIMEOUT
    assert srv.wait(t1, 60000).status == 0
    srv.close()


def test_served_grid_structure_is_fixed(sdg):
    """A grid registered with a server keeps its block structure until the server is destroyed: activation and
    destruction are refused (the scheduler reads the block tables without the grid's lock); value updates are
    allowed.  Mixed semantic channel counts are refused at registration."""
    sc = synth.scene_room(0, size=(2.0, 2.0, 2.0), n_objects=1)
    keys = synth.band_blocks(sc, 0.04, 3)
    G, O, stored, vals = make_pair(sc, keys, 0.04, 3, 0.02, "bf16", max_blocks=len(keys) + 64)
    srv = sdg.Server(hbm_budget_bytes=16 << 20, max_slots=2, n_streams=1, chunk_rays=256, max_batch_rays=1024)
    srv.add_scene(G)
    far = torch.as_tensor([[40, 40, 40]], dtype=torch.int32, device="cuda")
    with pytest.raises(sdg.SdgError) as e:
        G.activate_keys(far)
    assert e.value.code == sdg._abi.ERR_BUSY
    assert G.num_blocks == len(keys)
    rc = sdg._abi.lib().sdg_grid_destroy(G.handle)
    assert rc == sdg._abi.ERR_BUSY
    G.zero_grad()  # value updates stay allowed
    G4, _, _, _ = make_pair(sc, keys, 0.04, 3, 0.02, "bf16", n_sem=4)
    with pytest.raises(sdg.SdgError) as e:
        srv.add_scene(G4)
    assert e.value.code == sdg._abi.ERR_ARG
    srv.close()
    assert G.activate_keys(far) == 1  # structure free again once the server is gone


def test_served_rays_beyond_the_record_capacity(sdg):
    """Rays that cross more allocated block cells than the records kernel takes (32) are rendered by the serving
    loop's kernel over the mid list (their records two per lane), as sdg_debug_trace_view renders them: a view down
    a slab of 40 x 3 x 3 allocated blocks equals its trace bit for bit, and the oracle over the trace's samples on
    every pixel."""
    sc = synth.scene_room(0, size=(13.0, 2.0, 2.0), n_objects=0)
    keys = np.array([(x, y, z) for x in range(40) for y in range(3) for z in range(3)], np.int32)
    G, O, stored, vals = make_pair(sc, keys, 0.04, 3, 0.02, "bf16")
    # camera at x = 0.1 looking down +x (its z axis), centred in the slab's cross-section
    T = np.array([[0.0, 0.0, 1.0, 0.1], [1.0, 0.0, 0.0, 0.48], [0.0, 1.0, 0.0, 0.48]])
    H = W = 24
    K = synth.intrinsics(W, H, fov_deg=2.0)  # every ray stays inside the slab to its far end
    srv = sdg.Server(hbm_budget_bytes=16 << 20, max_slots=2, n_streams=1, chunk_rays=256, max_batch_rays=1024)
    sid = srv.add_scene(G)
    t = srv.submit(sid, H, W, K, T, n_samples=64, seed=5)
    r = srv.wait(t, 60000)
    rgb, depth, opac = srv.result_tensors(r)
    tr = sdg.trace_view(G, H, W, K, T, 64, seed=5)
    assert torch.equal(tr["rgb"].reshape(rgb.shape), rgb) and torch.equal(tr["depth"].reshape(depth.shape), depth)
    assert torch.equal(tr["opac"].reshape(opac.shape), opac)
    n_over = int((tr["n_cells"] < 0).sum())
    assert n_over >= H * W // 4, n_over  # a good part of the view beyond the records kernel (trace: n_cells -1)
    rays = tr["rays"].cpu().numpy()
    check_placement(O, rays, tr, 64, seed=5)
    ref = O.render(rays, 64, seed=5, given=gpu_samples(tr))
    assert np.abs(rgb.double().cpu().numpy().reshape(-1, 3) - ref["rgb"]).max() < 1e-4
    assert np.abs(depth.double().cpu().numpy().reshape(-1) - ref["depth"]).max() < 1e-4
    assert np.abs(opac.double().cpu().numpy().reshape(-1) - ref["opac"]).max() < 1e-4
    srv.release(t)
    srv.close()
