"""The allocation-free training entry point (sdg_train_step_rays_noalloc) gives what sdg_train_step_rays gives.

It exists for callers that cannot let the library allocate device memory (a device-memory budget owned by
another allocator, or a latency-critical loop that cannot afford cudaMalloc's device synchronisation).  It keeps
its per-ray loss scratch in a fixed array inside the library, so the test calls it through the C ABI twice in a
row (the second call on a smaller batch, so leftover contents of the shared array would show) and compares the
summed loss and the accumulated gradients with the allocating entry point's, within the tolerances the other
GPU tests use.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from tests.gpu_util import assert_grad_close, grad_arrays, tiny_room

pytestmark = pytest.mark.gpu


def _noalloc_fn(A):
    f = A.lib().sdg_train_step_rays_noalloc
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                  C.POINTER(A.RenderOpts), C.POINTER(A.LossOpts), C.c_void_p]
    f.restype = C.c_int
    return f


def _batch(sc, seed, W, H):
    T = synth.random_poses(sc, 1, seed=seed)[0]
    rays = synth.view_rays(T, W, H, synth.intrinsics(W, H)).cuda()
    g = torch.Generator(device="cuda").manual_seed(seed)
    t_rgb = torch.rand((rays.shape[0], 3), generator=g, device="cuda")
    t_depth = 2.0 * torch.rand(rays.shape[0], generator=g, device="cuda")
    return rays, t_rgb, t_depth


def test_noalloc_train_step_matches_allocating_entry_point():
    import paper_2305_13220_b300 as sdg
    A = sdg._abi
    sc, G, O, _, _ = tiny_room()
    f = _noalloc_fn(A)
    o = sdg.render_opts(64, seed=3)
    lo = A.LossOpts(lambda_depth=0.1, lambda_sem=0.1)
    for call, (W, H) in enumerate([(64, 48), (40, 24)]):   # two calls in a row, the second one smaller
        rays, t_rgb, t_depth = _batch(sc, 10 + call, W, H)
        n = rays.shape[0]
        G.zero_grad()
        ref_sum = torch.empty(1, device="cuda")
        sdg.train_step_rays(G, rays, t_rgb, t_depth, n_samples=64, seed=3, loss_sum=ref_sum)
        torch.cuda.synchronize()
        ref = grad_arrays(G, G.num_blocks)
        G.zero_grad()
        got_sum = torch.full((1,), float("nan"), device="cuda")
        rc = f(G.handle, rays.data_ptr(), n, t_rgb.data_ptr(), t_depth.data_ptr(), None, C.byref(o), C.byref(lo),
               got_sum.data_ptr())
        assert rc == A.OK, A.lib().sdg_last_error()
        torch.cuda.synchronize()
        got = grad_arrays(G, G.num_blocks)
        assert got_sum.item() == pytest.approx(ref_sum.item(), rel=1e-6)
        assert_grad_close(got["sdf"], ref["sdf"], what="sdf")
        assert_grad_close(got["rgb"], ref["rgb"], what="rgb")


def test_noalloc_rejects_batches_beyond_its_capacity():
    import paper_2305_13220_b300 as sdg
    A = sdg._abi
    sc, G, O, _, _ = tiny_room()
    f = _noalloc_fn(A)
    rays, t_rgb, t_depth = _batch(sc, 1, 8, 4)
    o = sdg.render_opts(64)
    lo = A.LossOpts(lambda_depth=0.1, lambda_sem=0.1)
    rc = f(G.handle, rays.data_ptr(), (1 << 20) + 1, t_rgb.data_ptr(), t_depth.data_ptr(), None, C.byref(o),
           C.byref(lo), None)
    assert rc == A.ERR_CAPACITY
    assert b"1048576" in A.lib().sdg_last_error()
    # dL/dbeta needs a per-ray buffer: learning beta is refused, not silently skipped
    lb = A.LossOpts(lambda_depth=0.1, lambda_sem=0.1, learn_beta=1)
    rc = f(G.handle, rays.data_ptr(), rays.shape[0], t_rgb.data_ptr(), t_depth.data_ptr(), None, C.byref(o),
           C.byref(lb), None)
    assert rc == A.ERR_ARG
    assert b"learn_beta" in A.lib().sdg_last_error()
