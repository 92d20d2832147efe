"""Trim contribution (Sec. 3.3, Eq. 3-4) and percentile pruning on the GPU,
against the FP64 oracle.

Per surfel, the support count |P_k| is integer work and must match exactly;
the contribution sum within 1e-5 relative (FP32 accumulation of values in
(0, 1]).  Where the oracle reports a decision within a hair of its threshold
that the surfel's count or sum depends on, the FP32 path may legitimately
decide the other way; those surfels get a stated bound instead and must stay
a small fraction.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2411_00771_gb300 import synthetic as syn
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

SUM_RTOL, SUM_ATOL = 1e-5, 1e-6


def _gpu_view(scene, cam, gamma):
    sc, _ = gu.gpu_scene(scene)
    n = scene["mu"].shape[0]
    s = torch.full((n,), float("nan"), device="cuda")
    c = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    sc.contribution(cam, gamma=gamma, view_sum=s, view_count=c)
    torch.cuda.synchronize()
    return s.cpu().numpy().astype(np.float64), c.cpu().numpy().astype(np.int64)


def _compare(scene, cam, gamma, max_flag_frac=0.06):
    """Counts exact where the surfel's own support membership is not within a
    hair of rho_max; sums within tolerance where no decision at or in front of
    the surfel was near a threshold.  Elsewhere each uncertain pixel may move
    the count by one and the sum by at most 0.2 (a flipped pair's own term
    sqrt(alpha T) is at most ~0.1 at the stop or at rho_max; a flipped pair in
    front changes T by at most ~1 %)."""
    ref = oracle.contribution(scene, cam, gamma=gamma)
    s, c = _gpu_view(scene, cam, gamma)
    seen = ref["count"] > 0
    okc = ref["flag_count"] == 0
    oks = ref["flag_sum"] == 0
    assert (~oks & seen).sum() <= max_flag_frac * seen.sum(), (~oks & seen).sum()
    assert np.array_equal(c[okc], ref["count"][okc])
    assert np.all(np.abs(c - ref["count"]) <= ref["flag_count"])
    err = np.abs(s - ref["sum"])
    tol = SUM_ATOL + SUM_RTOL * np.abs(ref["sum"])
    assert np.all(err[oks] <= tol[oks]), err[oks].max()
    assert np.all(err <= tol + 0.2 * ref["flag_sum"])
    # outside the view: exactly zero
    assert np.all(c[~seen & okc] == 0) and np.all(s[~seen & oks] == 0)
    return ref, s, c


@pytest.mark.parametrize("gamma", [0.5, 0.3])
def test_contribution_matches_oracle_tiny(gamma):
    scene, cam, _, _ = syn.tiny_scene()
    ref, s, c = _compare(scene, cam, gamma)
    assert (ref["count"] > 0).sum() > 1000


@pytest.mark.parametrize("deg,W,H", [(0, 100, 75), (1, 67, 45), (2, 129, 97)])
def test_contribution_matches_oracle_ragged(deg, W, H):
    scene, cam, _, _ = syn.tiny_scene(seed=30 + deg, n=1500, width=W, height=H, fx=float(W),
                                      sh_degree=deg, log_scale_range=(-4.5, -1.5))
    _compare(scene, cam, 0.5)


def test_contribution_of_a_city_crop():
    """The aerial city at reduced size: deep lists, stopped pixels, elongated
    and tilted surfels.  Deep stacks put a near-threshold decision in front of
    more surfels (about 6 % have one tainted pixel, 0.07 % of support pixels)."""
    scene, info = syn.city_scene(n=200_000)
    cam = syn.aerial_camera(width=400, height=225)
    ref, s, c = _compare(scene, cam, 0.5, max_flag_frac=0.10)
    assert (ref["count"] > 0).sum() > 30_000


def test_weighted_accumulation_over_views():
    """Eq. 4: contrib accumulates weight * C_{n,k}; with weight 1/|V| over
    three views it is the average of the per-view contributions."""
    scene, cam, _, _ = syn.tiny_scene(seed=40, n=1200)
    cams = [cam]
    for yaw in (0.15, -0.2):
        cy, sy = math.cos(yaw), math.sin(yaw)
        c2 = dict(cam)
        c2["R"] = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
        cams.append(c2)
    sc, _ = gu.gpu_scene(scene)
    n = scene["mu"].shape[0]
    acc = torch.zeros(n, device="cuda")
    for c in cams:
        sc.contribution(c, gamma=0.5, weight=1.0 / len(cams), contrib=acc)
    torch.cuda.synchronize()
    refs = [oracle.contribution(scene, c, gamma=0.5) for c in cams]
    ok = np.all([(r["flag_sum"] == 0) & (r["flag_count"] == 0) for r in refs], axis=0)
    expect = sum(r["C"] for r in refs) / len(cams)
    got = acc.cpu().numpy().astype(np.float64)
    assert ok.mean() > 0.94
    assert np.all(np.abs(got - expect)[ok] <= SUM_ATOL + SUM_RTOL * expect[ok])


@pytest.mark.parametrize("n,ratio", [(1_000_000, 0.025), (1_000_000, 0.1), (1000, 0.5), (7, 0.0),
                                     (7, 1.0), (1, 0.3)])
def test_prune_bound_and_mask_bit_exact(n, ratio):
    from paper_2411_00771_gb300 import binding as B
    rng = np.random.default_rng(n + int(ratio * 1000))
    c = rng.exponential(0.05, n).astype(np.float32)
    c[rng.random(n) < 0.05] = 0.0                  # never observed
    c[rng.random(n) < 0.02] = np.float32(0.0125)   # ties
    keep, bound = B.prune_by_contribution(torch.from_numpy(c).cuda(), ratio)
    torch.cuda.synchronize()
    rb, rk = oracle.prune_bound(c, ratio)
    if rb is None:
        assert float(bound) == -math.inf
    else:
        assert float(bound) == float(rb)
    assert np.array_equal(keep.cpu().numpy().astype(bool), rk)


def test_contribution_rejects_bad_arguments():
    from paper_2411_00771_gb300 import binding as B
    scene, cam, _, _ = syn.tiny_scene(n=50)
    sc, _ = gu.gpu_scene(scene)
    acc = torch.zeros(50, device="cuda")
    with pytest.raises(B.GsError) as e:
        sc.contribution(cam, gamma=1.5, contrib=acc)
    assert e.value.code == -1
    with pytest.raises(B.GsError):
        sc.contribution(cam)  # no output
    with pytest.raises(B.GsError):
        B.prune_by_contribution(acc, 1.5)
