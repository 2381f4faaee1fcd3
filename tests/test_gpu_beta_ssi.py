"""Learnable Laplace scale and the scale/shift-invariant depth loss on the GPU against the oracle.

dL/dbeta: the fused pass takes it through the identity dsigma/dbeta = -sigma/beta - (d/beta) dsigma/dd, the
oracle differentiates the two branches of sigma directly (and is pinned by finite differences in beta); both
must agree over every ray of the batch (the oracle fed the GPU's samples).  The optimiser then moves beta by the Adam step-1 closed form.
The SSI depth loss must match the oracle's FP64 least squares."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import assert_grad_close, check_placement, gpu_samples, grad_arrays, tiny_room

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sdg():
    import paper_2305_13220_b300 as m
    return m


def _batch(O, sc, seed, n_samples=64, G=None):
    """A whole view; with G, the oracle's render runs on the GPU's own samples (returned as ref["given"])."""
    import paper_2305_13220_b300 as sdg
    P = synth.random_poses(sc, 1, seed=seed)
    K = synth.intrinsics(64, 48)
    rays = synth.view_rays(P[0], 64, 48, K)
    gv = None
    if G is not None:
        tr = sdg.trace(G, rays.cuda(), n_samples, stratified=False)
        check_placement(O, rays, tr, n_samples, stratified=False)
        gv = gpu_samples(tr)
    ref = O.render(rays, n_samples, stratified=False, given=gv)
    ref["given"] = gv
    n = rays.shape[0]
    rng = np.random.default_rng(seed)
    t_rgb = ref["rgb"] + rng.choice([-0.05, 0.05], size=(n, 3))
    t_depth = ref["depth"] + rng.choice([-0.1, 0.1], size=n)
    return rays, ref, t_rgb, t_depth


def _dev(x):
    return torch.as_tensor(x, dtype=torch.float32, device="cuda")


def test_beta_gradient_matches_oracle_and_voxel_gradients_are_unchanged(sdg):
    sc, G, O, _, _ = tiny_room()
    rays, ref, t_rgb, t_depth = _batch(O, sc, seed=6, G=G)
    L, seeds = oracle.loss(ref["rgb"], ref["depth"], t_rgb, t_depth, 0.1)
    want = O.backward(rays, 64, seeds["rgb"], seeds["depth"], stratified=False, given=ref["given"])
    assert abs(want["beta"]) > 0
    G.zero_grad()
    sdg.train_step_rays(G, rays.cuda(), _dev(t_rgb), _dev(t_depth), n_samples=64, stratified=False)
    plain = grad_arrays(G, G.num_blocks)
    G.zero_grad()
    assert G.beta_grad() == 0.0
    sdg.train_step_rays(G, rays.cuda(), _dev(t_rgb), _dev(t_depth), n_samples=64, stratified=False,
                        learn_beta=True)
    got = G.beta_grad()
    assert got == pytest.approx(want["beta"], rel=1e-3)
    with_beta = grad_arrays(G, G.num_blocks)
    assert_grad_close(with_beta["sdf"], plain["sdf"], rel=1e-5, floor=1e-5, what="sdf (beta variant)")
    assert_grad_close(with_beta["rgb"], plain["rgb"], rel=1e-5, floor=1e-5, what="rgb (beta variant)")
    # a second pass accumulates
    sdg.train_step_rays(G, rays.cuda(), _dev(t_rgb), _dev(t_depth), n_samples=64, stratified=False,
                        learn_beta=True)
    assert G.beta_grad() == pytest.approx(2 * got, rel=1e-6)


def test_optimiser_moves_beta(sdg):
    sc, G, O, _, _ = tiny_room()
    rays, ref, t_rgb, t_depth = _batch(O, sc, seed=7)
    b0 = G.beta
    G.step = 0
    sdg.train_step_rays(G, rays.cuda(), _dev(t_rgb), _dev(t_depth), n_samples=64, stratified=False,
                        learn_beta=True)
    g = G.beta_grad()
    G.adam_step(lr=1e-3)
    # Adam step 1: m_hat = g, v_hat = g^2, so beta moves by -lr g / (|g| + eps)
    assert G.beta == pytest.approx(b0 - 1e-3 * g / (abs(g) + 1e-8), rel=1e-6)
    assert G.beta_grad() == 0.0
    # without learn_beta the scale stays put
    b1 = G.beta
    sdg.train_step_rays(G, rays.cuda(), _dev(t_rgb), _dev(t_depth), n_samples=64, stratified=False)
    G.adam_step(lr=1e-3)
    assert G.beta == b1
    G.beta = 0.03
    assert G.beta == pytest.approx(0.03)
    with pytest.raises(sdg.SdgError):
        G.beta = 0.0


def test_beta_moments_survive_a_checkpoint(sdg, tmp_path):
    sc, G1, O, _, _ = tiny_room()
    _, G2, _, _, _ = tiny_room()
    batches = [_batch(O, sc, seed=10 + s) for s in range(4)]

    def steps(G, lo, hi):
        for rays, ref, t_rgb, t_depth in batches[lo:hi]:
            sdg.train_step_rays(G, rays.cuda(), _dev(t_rgb), _dev(t_depth), n_samples=64, stratified=False,
                                learn_beta=True)
            G.adam_step(lr=1e-3)
        torch.cuda.synchronize()

    steps(G1, 0, 4)
    steps(G2, 0, 2)
    p = str(tmp_path / "beta.sdg")
    G2.save(p)
    G3 = sdg.Grid.load(p, max_blocks=G1.max_blocks)
    assert G3.beta == G2.beta and G3.step == 2
    steps(G3, 2, 4)
    # voxel gradients carry atomic-order noise from step to step, the beta moments do not depend on it much
    assert G3.beta == pytest.approx(G1.beta, rel=1e-5)


def test_ssi_depth_loss_matches_oracle(sdg):
    sc, G, O, _, _ = tiny_room()
    rng = np.random.default_rng(0)
    D = rng.uniform(0.5, 4.0, 20000).astype(np.float32)
    t = (0.6 * D + 0.3 + rng.normal(0, 0.05, D.shape)).astype(np.float32)
    loss, g, (a, b) = sdg.loss_depth_ssi(G, _dev(D), _dev(t), 0.2, want_ab=True)
    L, g_ref, (a_ref, b_ref) = oracle.depth_ssi(D.astype(np.float64), t.astype(np.float64), 0.2)
    assert a == pytest.approx(a_ref, rel=1e-9) and b == pytest.approx(b_ref, rel=1e-8, abs=1e-12)
    # FP32 residuals D - (a t + b) carry ~5e-7 absolute error (a few ulps of depths ~2 m)
    np.testing.assert_allclose(g.double().cpu().numpy(), g_ref, rtol=1e-4, atol=1e-5 * np.abs(g_ref).max())
    assert loss.sum().item() == pytest.approx(L, rel=1e-4)
    # constant targets: a = 1, b = mean(D - t)
    _, _, (a1, b1) = sdg.loss_depth_ssi(G, _dev(D), _dev(np.full_like(D, 2.0)), 0.2, want_ab=True)
    assert a1 == 1.0 and b1 == pytest.approx(float(D.astype(np.float64).mean() - 2.0), rel=1e-6)
