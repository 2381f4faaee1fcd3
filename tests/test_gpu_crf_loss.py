"""CRF losses on the GPU (sdg_crf_loss) against the oracle: per-point terms and the gradients added to the label,
colour and SDF gradient channels, in both storage layouts (Sec. 3.5.3, Eq. 22)."""
import numpy as np
import pytest
import torch

from tests.gpu_util import assert_grad_close, grad_arrays, tiny_room
from tests.test_gpu_query import points

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("rgb_dtype", ["f32", "bf16"])
@pytest.mark.parametrize("prop", ["label", "color", "normal"])
def test_crf_loss_matches_oracle(rgb_dtype, prop):
    sc, G, O, stored, vals = tiny_room(rgb_dtype=rgb_dtype, n_sem=8)
    gk = G.keys().cpu().numpy()
    x = points(gk, 6000, 3)[:-3]
    rng = np.random.default_rng(4)
    t = rng.dirichlet(np.ones(8), size=len(x)) if prop == "label" else rng.normal(size=(len(x), 3))
    terms = torch.empty(len(x), device="cuda")
    total = torch.zeros(1, device="cuda")
    G.zero_grad()
    G.crf_loss(prop, torch.as_tensor(x, device="cuda"), torch.as_tensor(t, dtype=torch.float32, device="cuda"), 0.3,
               terms=terms, loss_sum=total)
    torch.cuda.synchronize()
    L, t_ref, g_ref = O.crf_loss(prop, x.astype(np.float64), t, 0.3)
    # (the target is rounded to FP32 on the GPU side; the terms are FP32)
    np.testing.assert_allclose(terms.double().cpu().numpy(), t_ref, rtol=2e-4, atol=1e-9)
    assert total.item() == pytest.approx(L, rel=1e-4)
    got = grad_arrays(G, len(gk))[{"label": "sem", "color": "rgb", "normal": "sdf"}[prop]]
    assert np.abs(g_ref).max() > 0
    assert_grad_close(got, g_ref, what=prop)
