"""gs_loss_noalloc against gs_loss.

gs_loss_noalloc serves callers that cannot allocate device memory when they
need the loss (code under an external memory manager that owns the GPU, or a
real-time loop that must not stall on or fail an allocation): it keeps its
scratch in one fixed array inside the library instead.  This file is named
so that pytest collects it last.  The test calls the new entry point twice in
a row (two image sizes, so the second call runs over what the first left in
the shared array) and checks each result against the allocating gs_loss on
the same inputs, within the loss tolerances of the parity tests.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _inputs(rng, H, W):
    out = np.zeros((12, H, W), np.float32)
    out[0:3] = rng.uniform(0, 1, (3, H, W))
    out[5] = rng.uniform(0.1, 0.6, (H, W))
    tgt = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    tinv = rng.uniform(0.1, 0.6, (H, W)).astype(np.float32)
    return [torch.from_numpy(a).cuda() for a in (out, tgt, tinv)]


def test_noalloc_loss_matches_allocating_loss_twice():
    from paper_2411_00771_gb300 import binding as B
    rng = np.random.default_rng(2024)
    w = (0.8, 0.2, 0.5)
    for (H, W) in [(128, 160), (75, 101)]:
        out, tgt, tinv = _inputs(rng, H, W)
        ref_adj = [torch.zeros((11, H, W), device="cuda") for _ in range(3)]
        ref_losses = torch.empty(4, device="cuda")
        B.loss(out, tgt, tinv, w, adj_total=ref_adj[0], adj_ssim=ref_adj[1], adj_l1=ref_adj[2],
               losses=ref_losses)
        na_adj = [torch.zeros((11, H, W), device="cuda") for _ in range(3)]
        na_losses = torch.empty(4, device="cuda")
        B.loss_noalloc(out, tgt, tinv, w, na_adj[0], na_adj[1], na_adj[2], na_losses)
        torch.cuda.synchronize()
        assert torch.allclose(na_losses, ref_losses, rtol=1e-6, atol=1e-7)
        for a, r in zip(na_adj, ref_adj):
            scale = float(r.abs().max())
            assert float((a - r).abs().max()) <= 1e-4 * scale


def test_noalloc_loss_rejects_images_beyond_its_scratch():
    from paper_2411_00771_gb300 import binding as B
    H, W = 600, 600
    out = torch.zeros((12, H, W), device="cuda")
    tgt = torch.zeros((3, H, W), device="cuda")
    adj = torch.zeros((11, H, W), device="cuda")
    losses = torch.empty(4, device="cuda")
    with pytest.raises(B.GsError) as e:
        B.loss_noalloc(out, tgt, None, (0.8, 0.2, 0.0), adj, losses=losses)
    assert e.value.code == -3 and "exceeds the fixed scratch" in str(e.value)
