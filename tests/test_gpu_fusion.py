"""Volumetric fusion on the GPU (sdg_fuse_frames / sdg_fuse_finalize) against the oracle (Eq. 9-11).

Association decisions are taken in FP32 in the same order on both sides, so the per-voxel association counts
(the WEIGHT channel) must match bit for bit; the averages are FP32 running means on the GPU and FP64 means in the
oracle: |SDF error| <= 1e-6 (values within +-mu), colour <= 1e-5, and after rounding to BF16 one BF16 quantum."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

VS, BAND = 0.04, 3
MU = BAND * VS
W, H = 64, 48


@pytest.fixture(scope="module")
def sdg():
    import paper_2305_13220_b300 as m
    return m


def fresh_grid(sdg, keys, rgb_dtype="f32", n_sem=0):
    G = sdg.Grid(VS, max(len(keys), 1), beta=0.5 * VS, rgb_dtype=rgb_dtype, n_sem=n_sem)
    if len(keys):
        G.activate_keys(torch.as_tensor(keys, device="cuda"))
    return G, G.keys().cpu().numpy()


def frames(sc, n, seed, n_sem=0, W=W, H=H):
    P = synth.random_poses(sc, n, seed=seed)
    K = synth.intrinsics(W, H)
    fr = [synth.rgbd_frame(sc, p, W, H, K, n_sem=n_sem, seed=seed * 100 + i, device="cuda")
          for i, p in enumerate(P)]
    out = {k: torch.stack([f[k] for f in fr]).contiguous() for k in fr[0]}
    return out, P, K


def weights(sdg, G, N):
    return G.channel(sdg._abi.GROUP_WEIGHT)[:N, :, 0].double().cpu().numpy()


def test_fp32_grid_matches_oracle_over_two_calls(sdg):
    sc = synth.scene_tiny_room(0)
    G, gk = fresh_grid(sdg, synth.band_blocks(sc, VS, BAND))
    fr, P, K = frames(sc, 5, seed=3)
    G.fuse(fr["depth"][:2], K, P[:2], MU, rgb=fr["rgb"][:2])
    G.fuse(fr["depth"][2:], K, P[2:], MU, rgb=fr["rgb"][2:])
    G.fuse_finalize()  # no-op for an FP32 grid without logits
    torch.cuda.synchronize()
    ref = oracle.fuse(gk, VS, fr["depth"].cpu(), K, P, MU, rgb=fr["rgb"].cpu())
    N = len(gk)
    w = weights(sdg, G, N)
    np.testing.assert_array_equal(w, ref["weight"])
    assert (w > 0).mean() > 0.1 and w.max() >= 3
    geo = G.channel(sdg._abi.GROUP_GEO)[:N].double().cpu().numpy()
    np.testing.assert_allclose(geo[..., 0], ref["sdf"], atol=1e-6, rtol=0)
    np.testing.assert_allclose(geo[..., 1:4], ref["rgb"], atol=1e-5, rtol=0)
    assert np.all(geo[w == 0] == 0)  # voxels without association are not written


def test_bf16_grid_with_logits_matches_oracle(sdg):
    sc = synth.scene_tiny_room(1)
    ns = 8
    G, gk = fresh_grid(sdg, synth.band_blocks(sc, VS, BAND), rgb_dtype="bf16", n_sem=ns)
    fr, P, K = frames(sc, 4, seed=5, n_sem=ns)
    for i in range(4):  # one frame per call, as an online fusion loop would
        G.fuse(fr["depth"][i], K, P[i], MU, rgb=fr["rgb"][i], sem=fr["sem"][i])
    G.fuse_finalize()
    torch.cuda.synchronize()
    ref = oracle.fuse(gk, VS, fr["depth"].cpu(), K, P, MU, rgb=fr["rgb"].cpu(), sem=fr["sem"].cpu())
    N = len(gk)
    A = sdg._abi
    w = weights(sdg, G, N)
    np.testing.assert_array_equal(w, ref["weight"])
    sdf = G.channel(A.GROUP_SDF)[:N, :, 0].double().cpu().numpy()
    np.testing.assert_allclose(sdf, ref["sdf"], atol=1e-6, rtol=0)
    rgb = G.channel(A.GROUP_RGB)[:N, :, 0:3].double().cpu().numpy()
    q = 2.0 ** -8  # BF16 rounding: half a quantum of |x| < 2^-8 |x|
    assert np.all(np.abs(rgb - ref["rgb"]) <= q * np.abs(ref["rgb"]) + 1e-5)
    sem = G.channel(A.GROUP_SEM)[:N].double().cpu().numpy()
    assert np.all(np.abs(sem - ref["sem"]) <= q * np.abs(ref["sem"]) + 1e-5)
    kept = w > 0
    np.testing.assert_allclose(np.linalg.norm(sem[kept], axis=-1), 1.0, atol=8e-3)
    # the accumulators are released for training
    assert torch.all(G.channel(A.GROUP_RGB, A.KIND_GRAD)[:N] == 0)
    assert torch.all(G.channel(A.GROUP_SEM, A.KIND_GRAD)[:N] == 0)


def test_misaligned_logit_frames_take_the_scalar_path(sdg):
    """Logit frames that are not 16-byte aligned (a view at a 4-byte offset) are read channel by channel; the
    result is bit-identical to the float4 path on an aligned copy (same per-channel summation order)."""
    sc = synth.scene_tiny_room(1)
    ns = 8
    keys = synth.band_blocks(sc, VS, BAND)
    fr, P, K = frames(sc, 3, seed=11, n_sem=ns)
    sem = fr["sem"]
    buf = torch.empty(sem.numel() + 1, device="cuda")
    mis = buf[1:].view(sem.shape)
    mis.copy_(sem)
    assert mis.data_ptr() % 16 != 0 and mis.is_contiguous()
    out = []
    for s_in in (sem, mis):
        G, gk = fresh_grid(sdg, keys, rgb_dtype="bf16", n_sem=ns)
        G.fuse(fr["depth"], K, P, MU, rgb=fr["rgb"], sem=s_in)
        G.fuse_finalize()
        torch.cuda.synchronize()
        out.append(G.channel(sdg._abi.GROUP_SEM)[:len(gk)].float().cpu())
    assert torch.equal(out[0], out[1])
    assert out[0].abs().sum() > 0


def test_more_frames_than_one_launch_holds(sdg):
    """1100 small frames: the call is split into launches of at most 1024 frames."""
    sc = synth.scene_tiny_room(2)
    G, gk = fresh_grid(sdg, synth.band_blocks(sc, VS, BAND))
    fr, P, K = frames(sc, 1100, seed=7, W=8, H=6)
    G.fuse(fr["depth"], K, P, MU, rgb=fr["rgb"])
    torch.cuda.synchronize()
    ref = oracle.fuse(gk, VS, fr["depth"].cpu(), K, P, MU, rgb=fr["rgb"].cpu())
    N = len(gk)
    w = weights(sdg, G, N)
    np.testing.assert_array_equal(w, ref["weight"])
    geo = G.channel(sdg._abi.GROUP_GEO)[:N].double().cpu().numpy()
    np.testing.assert_allclose(geo[..., 0], ref["sdf"], atol=1e-6, rtol=0)
    np.testing.assert_allclose(geo[..., 1:4], ref["rgb"], atol=2e-5, rtol=0)


def test_invalid_depths_and_degenerate_calls(sdg):
    sc = synth.scene_tiny_room(0)
    G, gk = fresh_grid(sdg, synth.band_blocks(sc, VS, BAND))
    fr, P, K = frames(sc, 2, seed=9)
    d = fr["depth"].clone()
    d[0, ::3] = float("nan")
    d[0, 1::5] = 0.0
    d[1, :, ::4] = -1.0
    d[1, :, 1::7] = float("inf")
    G.fuse(d, K, P, MU)  # depth only: colour stays untouched
    G.fuse(d[:0], K, P[:0], MU)  # zero frames
    torch.cuda.synchronize()
    ref = oracle.fuse(gk, VS, d.cpu(), K, P, MU)
    N = len(gk)
    np.testing.assert_array_equal(weights(sdg, G, N), ref["weight"])
    geo = G.channel(sdg._abi.GROUP_GEO)[:N].double().cpu().numpy()
    np.testing.assert_allclose(geo[..., 0], ref["sdf"], atol=1e-6, rtol=0)
    assert np.all(geo[..., 1:4] == 0)
    # an empty grid accepts frames and does nothing
    E, _ = fresh_grid(sdg, np.zeros((0, 3), np.int32))
    E.fuse(fr["depth"], K, P, MU)
    torch.cuda.synchronize()


def test_bad_arguments_are_rejected(sdg):
    sc = synth.scene_tiny_room(0)
    G, gk = fresh_grid(sdg, synth.band_blocks(sc, VS, BAND))
    fr, P, K = frames(sc, 1, seed=1, n_sem=4)
    with pytest.raises(sdg.SdgError):
        G.fuse(fr["depth"], K, P, 0.0)  # mu must be positive
    with pytest.raises(sdg.SdgError):
        G.fuse(fr["depth"], [-50.0, 50.0, 32.0, 24.0], P, MU)  # fx must be positive
    with pytest.raises(sdg.SdgError):
        G.fuse(fr["depth"], K, P, MU, sem=fr["sem"])  # no semantic channel on this grid
