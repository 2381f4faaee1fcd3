"""GPU parity of the optimiser step (Sec. 3.5.4; Adam default, RMSProp flag) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from tests.gpu_util import tiny_room

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sdg():
    import paper_2305_13220_b300 as m
    return m


@pytest.mark.parametrize("algo", ["adam", "rmsprop"])
def test_f32_optimiser_matches_oracle(sdg, algo):
    sc, G, O, stored, vals = tiny_room()
    A = sdg._abi
    N = G.num_blocks
    geo, grad = G.channel(A.GROUP_GEO), G.channel(A.GROUP_GEO, A.KIND_GRAD)
    m, v = G.channel(A.GROUP_GEO, A.KIND_ADAM_M), G.channel(A.GROUP_GEO, A.KIND_ADAM_V)
    th = geo[:N].double().cpu().numpy().reshape(-1)
    mo, vo = np.zeros_like(th), np.zeros_like(th)
    gen = torch.Generator(device="cuda").manual_seed(0)
    b2 = 0.999 if algo == "adam" else 0.99
    for step in (1, 2, 3):
        g = torch.randn(grad[:N].shape, generator=gen, device="cuda") * 10 ** (-step)
        grad[:N] = g
        G.adam_step(lr=1e-3, beta2=b2, algo=algo)
        gg = g.double().cpu().numpy().reshape(-1).copy()
        if algo == "adam":
            oracle.adam(th, gg, mo, vo, lr=1e-3, step=step)
        else:
            oracle.rmsprop(th, gg, vo, lr=1e-3, alpha=b2)
    torch.cuda.synchronize()
    got = geo[:N].double().cpu().numpy().reshape(-1)
    # FP32 update of O(1) parameters by O(1e-3) steps: agreement to a few FP32 ulps of theta
    np.testing.assert_allclose(got, th, rtol=0, atol=4e-7 * max(1.0, np.abs(th).max()))
    assert torch.all(grad[:N] == 0)
    assert G.step == 3
    if algo == "adam":
        # m sums gradients of both signs: cancellation makes its relative error unbounded, so the
        # bound is a few FP32 ulps of the largest gradient fed in (0.1 * |N(0,1)| ~ 0.5)
        np.testing.assert_allclose(m[:N].double().cpu().numpy().reshape(-1), mo, rtol=1e-5, atol=1e-8)
    np.testing.assert_allclose(v[:N].double().cpu().numpy().reshape(-1), vo, rtol=1e-5, atol=1e-12)


def test_bf16_channels_round_to_nearest_even(sdg):
    sc, G, O, stored, vals = tiny_room("bf16", 8)
    A = sdg._abi
    N = G.num_blocks
    rgb0 = G.channel(A.GROUP_RGB)[:N].float().clone()
    sem0 = G.channel(A.GROUP_SEM)[:N].float().clone()
    g_rgb = torch.randn((N, 512, 4), device="cuda")
    g_rgb[..., 3] = 0
    g_sem = torch.randn((N, 512, 8), device="cuda")
    G.channel(A.GROUP_RGB, A.KIND_GRAD)[:N] = g_rgb
    G.channel(A.GROUP_SEM, A.KIND_GRAD)[:N] = g_sem
    G.adam_step(lr=1e-2, step=1)
    torch.cuda.synchronize()
    # step 1: theta - lr * g / (|g| + eps) in FP32, then rounded to nearest-even BF16
    exp_rgb = (rgb0 - 1e-2 * g_rgb / (g_rgb.abs() + 1e-8)).to(torch.bfloat16)
    exp_sem = (sem0 - 1e-2 * g_sem / (g_sem.abs() + 1e-8)).to(torch.bfloat16)
    got_rgb = G.channel(A.GROUP_RGB)[:N]
    assert (got_rgb[..., :3] != exp_rgb[..., :3]).float().mean() < 1e-3   # FP32 op-order ties only
    assert torch.all(got_rgb[..., 3] == 0)
    assert (G.channel(A.GROUP_SEM)[:N] != exp_sem).float().mean() < 1e-3
