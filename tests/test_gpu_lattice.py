"""Permutohedral-lattice filter and the CRF mean-field update on the GPU against the oracle (Eq. 19-22).

The simplex search runs in FP32 in one fixed operation order on both sides, so the lattice (its size) must be
identical; splat / blur / slice run in FP32 on the GPU: outputs within 1e-5 of the output scale.  Features are
CRF-like: positions, colours and normals of surface samples of the tiny room, each divided by its bandwidth."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests.gpu_util import tiny_room

pytestmark = pytest.mark.gpu


def crf_features(n, seed):
    sc = synth.scene_tiny_room(0)
    P = synth.random_poses(sc, 4, seed=seed)
    K = synth.intrinsics(48, 36)
    rng = np.random.default_rng(seed)
    rows = []
    for T in P:
        fr = synth.rgbd_frame(sc, T, 48, 36, K, n_sem=4, seed=seed)
        rays = synth.view_rays(T, 48, 36, K).double()
        x = rays[:, :3] + fr["depth"].reshape(-1, 1).double() * rays[:, 4:7]
        rows.append(np.concatenate([x.numpy() / 0.1, fr["rgb"].reshape(-1, 3).numpy() / 0.2,
                                    fr["sem"].reshape(-1, 4).numpy()], 1))
    f = np.concatenate(rows)
    return f[rng.choice(len(f), n, replace=False)].astype(np.float32)


@pytest.mark.parametrize("d,normalize", [(3, False), (6, True), (10, False)])
def test_lattice_filter_matches_oracle(d, normalize):
    sc, G, O, _, _ = tiny_room()
    f = crf_features(3000, seed=d)[:, :d].copy()
    rng = np.random.default_rng(d)
    v = rng.normal(size=(3000, 5)).astype(np.float32)
    out, M = G.lattice_filter(torch.as_tensor(f, device="cuda"), torch.as_tensor(v, device="cuda"), normalize)
    ref, M_ref = oracle.lattice_filter(f.astype(np.float64), v.astype(np.float64), normalize)
    assert M == M_ref
    got = out.double().cpu().numpy()
    np.testing.assert_allclose(got, ref, atol=1e-5 * np.abs(ref).max(), rtol=1e-4)


@pytest.mark.parametrize("d", [2, 3, 9])
def test_filter_does_not_depend_on_point_order(d):
    """The memory order of the lattice rows follows the points that created them; permuting the points permutes
    the outputs and leaves the lattice size unchanged (values equal up to the order of FP32 splat atomics)."""
    sc, G, O, _, _ = tiny_room()
    f = crf_features(4000, seed=10 + d)[:, :d].copy()
    rng = np.random.default_rng(d)
    v = rng.normal(size=(4000, 6)).astype(np.float32)
    perm = rng.permutation(4000)
    out, M = G.lattice_filter(torch.as_tensor(f, device="cuda"), torch.as_tensor(v, device="cuda"), True)
    out_p, M_p = G.lattice_filter(torch.as_tensor(f[perm], device="cuda"), torch.as_tensor(v[perm], device="cuda"),
                                  True)
    assert M_p == M and M > 100
    a, b = out.double().cpu().numpy(), out_p.double().cpu().numpy()
    np.testing.assert_allclose(b, a[perm], atol=1e-5 * np.abs(a).max(), rtol=1e-4)


def test_meanfield_matches_oracle():
    sc, G, O, _, _ = tiny_room()
    f = crf_features(2000, seed=3)
    n, L = len(f), 4
    rng = np.random.default_rng(0)
    U = rng.normal(size=(n, L)).astype(np.float32)
    Q = np.exp(-U)
    Q = (Q / Q.sum(1, keepdims=True)).astype(np.float32)
    got = G.crf_meanfield(torch.as_tensor(f, device="cuda"), torch.as_tensor(U, device="cuda"),
                          torch.as_tensor(Q, device="cuda"), 0.5).double().cpu().numpy()
    ref = oracle.crf_meanfield(f.astype(np.float64), U.astype(np.float64), Q.astype(np.float64), 0.5)
    np.testing.assert_allclose(got, ref, atol=2e-5)
    np.testing.assert_allclose(got.sum(1), 1.0, atol=1e-5)


def test_bad_features_are_rejected():
    import paper_2305_13220_b300 as sdg
    sc, G, O, _, _ = tiny_room()
    f = torch.zeros((10, 3), device="cuda")
    f[3, 1] = float("nan")
    with pytest.raises(sdg.SdgError):
        G.lattice_filter(f, torch.ones((10, 1), device="cuda"))
    with pytest.raises(sdg.SdgError):
        G.lattice_filter(torch.zeros((10, 17), device="cuda"), torch.ones((10, 1), device="cuda"))
    out, M = G.lattice_filter(torch.zeros((0, 3), device="cuda"), torch.zeros((0, 2), device="cuda"))
    assert M == 0
