"""SDF + closed-form gradient query and the Eikonal loss on the GPU (sdg_query / sdg_eikonal) against the oracle
(Eq. 16-17, Sec. 3.5.3).

Points are drawn in and around the allocated blocks; points within 1e-3 of a cell face are left out, since FP32
and FP64 may put them in different cells, where the piecewise-linear interpolant has a different gradient.
Validity must match exactly (NaN on the GPU where the oracle reports an unallocated grid point); values within
FP32 rounding of the FP64 oracle."""
import numpy as np
import pytest
import torch

from tests.gpu_util import assert_grad_close, grad_arrays, tiny_room

pytestmark = pytest.mark.gpu

VS = 0.04


def points(gk, n, seed):
    """n points: most inside random allocated blocks (some reach past a block face into a missing neighbour),
    a few far outside, NaN and beyond the block-key range; none near a cell face."""
    rng = np.random.default_rng(seed)
    b = gk[rng.integers(0, len(gk), n)]
    x = (b * 8 + rng.uniform(0, 8, (n, 3))) * VS
    x[: n // 50] = rng.uniform(-20, 20, (n // 50, 3))
    x = x.astype(np.float32)
    f = x.astype(np.float64) / VS
    f = f - np.floor(f)
    x = x[np.all((f > 1e-3) & (f < 1 - 1e-3), axis=1)]
    extra = np.array([[np.nan, 0.1, 0.1], [1e9, 0.0, 0.0], [-3e5, 0.5, 0.5]], np.float32)
    return np.concatenate([x, extra])


@pytest.fixture(scope="module", params=["f32", "bf16"])
def room(request):
    import paper_2305_13220_b300 as sdg
    sc, G, O, stored, vals = tiny_room(rgb_dtype=request.param)
    return sdg, G, O, G.keys().cpu().numpy()


def test_query_matches_oracle(room):
    sdg, G, O, gk = room
    x = points(gk, 20000, 0)
    xt = torch.as_tensor(x, device="cuda")
    sdf, grad = G.query(xt)
    only_sdf, _ = G.query(xt, want_grad=False)
    torch.cuda.synchronize()
    sdf, grad, only_sdf = sdf.double().cpu().numpy(), grad.double().cpu().numpy(), only_sdf.double().cpu().numpy()
    f, g, ok = O.query_grad(x[:-3].astype(np.float64))
    ok = np.concatenate([ok, [False, False, False]])
    np.testing.assert_array_equal(~np.isnan(sdf), ok)
    assert np.isnan(grad[~ok]).all()
    assert ok.mean() > 0.5 and (~ok).sum() > 100
    v = ok[:-3]
    np.testing.assert_allclose(sdf[:-3][v], f[v], atol=1e-6, rtol=0)
    np.testing.assert_allclose(grad[:-3][v], g[v], atol=2e-5, rtol=0)
    np.testing.assert_array_equal(only_sdf[ok], sdf[ok])
    # the SDF of the band is a distance field where it is not truncated: |grad f| ~ 1 at the surface
    near = v & (np.abs(f) < 0.5 * VS)
    assert near.sum() > 100 and np.median(np.linalg.norm(g[near], axis=1)) == pytest.approx(1.0, abs=0.1)


def test_eikonal_matches_oracle(room):
    sdg, G, O, gk = room
    x = points(gk, 8000, 1)[:-3]
    xt = torch.as_tensor(x, device="cuda")
    n = len(x)
    terms = torch.empty(n, device="cuda")
    total = torch.zeros(1, device="cuda")
    G.zero_grad()
    G.eikonal(xt, 0.1, terms=terms, loss_sum=total)
    torch.cuda.synchronize()
    L, t_ref, g_ref = O.eikonal(x.astype(np.float64), 0.1)
    np.testing.assert_allclose(terms.double().cpu().numpy(), t_ref, atol=1e-9, rtol=1e-5)
    assert total.item() == pytest.approx(L, rel=1e-5)
    got = grad_arrays(G, len(gk))["sdf"]
    touched = np.abs(g_ref) > 0
    assert touched.sum() > 1000
    assert_grad_close(got, g_ref, what="eikonal sdf")
    # the loss sum alone (no per-point buffer) uses grid scratch and gives the same value
    total2 = torch.zeros(1, device="cuda")
    G.eikonal(xt, 0.1, loss_sum=total2)
    torch.cuda.synchronize()
    assert total2.item() == total.item()


def test_ragged_sizes_match_the_large_batch(room):
    """One point and 300 points (less than one wave of CTAs) give exactly what the same points give inside a batch
    of 20,000 (a grid of one resident wave, each thread looping)."""
    sdg, G, O, gk = room
    x = torch.as_tensor(points(gk, 20000, 4)[:-3], device="cuda")
    f_all, g_all = G.query(x)
    for m in (1, 300):
        f, g = G.query(x[:m].contiguous())
        torch.cuda.synchronize()
        assert torch.equal(torch.nan_to_num(f, nan=-7.0), torch.nan_to_num(f_all[:m], nan=-7.0))
        assert torch.equal(torch.nan_to_num(g, nan=-7.0), torch.nan_to_num(g_all[:m], nan=-7.0))


def test_empty_and_rejected_calls(room):
    sdg, G, O, gk = room
    empty = torch.zeros((0, 3), device="cuda")
    s, g = G.query(empty)
    total = torch.ones(1, device="cuda")
    G.eikonal(empty, 0.1, loss_sum=total)
    torch.cuda.synchronize()
    assert s.numel() == 0 and total.item() == 0.0
    with pytest.raises(ValueError):
        G.query(torch.zeros((4, 3), dtype=torch.float64, device="cuda"))
