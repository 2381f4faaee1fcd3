"""Failure handling made on the host (no GPU fault is ever provoked): failing device allocations during grid
creation and activation, a request cancelled while in flight, and a wait that times out."""
import numpy as np
import pytest
import torch

import synth
from tests.gpu_util import make_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sdg():
    import paper_2305_13220_b300 as m
    return m


def test_allocation_failures_return_oom_and_leak_nothing(sdg):
    A = sdg._abi
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for n in range(0, 12):
        A.lib().sdg_debug_fail_alloc_after(n)
        try:
            G = sdg.Grid(0.01, 5000)
        except sdg.SdgError as e:
            assert e.code == A.ERR_OOM
            continue
        finally:
            A.lib().sdg_debug_fail_alloc_after(-1)
        G.close()  # creation got past the n-th allocation
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < (64 << 20)  # nothing of the failed creations stays allocated


def test_activation_allocation_failure_leaves_grid_usable(sdg):
    A = sdg._abi
    G = sdg.Grid(0.01, 5000)
    pts = torch.as_tensor(np.random.default_rng(0).uniform(0, 0.3, (500, 3)).astype(np.float32), device="cuda")
    A.lib().sdg_debug_fail_alloc_after(0)  # the block-index grid allocation of the first activation fails
    try:
        with pytest.raises(sdg.SdgError) as e:
            G.activate_points(pts, 2)
        assert e.value.code == A.ERR_OOM
    finally:
        A.lib().sdg_debug_fail_alloc_after(-1)
    assert G.num_blocks == 0            # all-or-nothing: nothing was inserted
    n = G.activate_points(pts, 2)       # and the grid still works
    assert n > 0 and G.num_blocks == n
    assert np.array_equal(G.lookup(G.keys()).cpu().numpy(), np.arange(n))


def test_cancel_in_flight_and_timeouts(sdg):
    sc = synth.scene_room(3, size=(3.0, 3.0, 2.5), n_objects=3)
    keys = synth.band_blocks(sc, 0.04, 3)
    G, O, _, _ = make_pair(sc, keys, 0.04, 3, 0.02)
    srv = sdg.Server(hbm_budget_bytes=256 << 20, max_slots=4, n_streams=2, chunk_rays=1024, max_batch_rays=8192)
    sid = srv.add_scene(G)
    T = synth.random_poses(sc, 1, seed=1)[0]
    K = synth.intrinsics(1280, 960)
    t = srv.submit(sid, 960, 1280, K, T, n_samples=256)
    srv.release(t)                       # cancelled while queued or in flight
    with pytest.raises(sdg.SdgError):
        srv.poll(t)
    t2 = srv.submit(sid, 960, 1280, K, T, n_samples=256)
    with pytest.raises(sdg.SdgError) as e:
        srv.wait(t2, 0)                  # not done immediately
    assert e.value.code == sdg._abi.ERR_TIMEOUT
    assert srv.wait(t2, 120000).status == 0
    srv.release(t2)
    import time
    for _ in range(200):                 # the cancelled request's memory comes back once its batches finish
        if srv.stats().bytes_in_use == 0:
            break
        time.sleep(0.01)
    assert srv.stats().bytes_in_use == 0
    srv.close()
