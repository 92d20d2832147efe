"""Visible frequency of points (Sec. 4, crop volume estimation) on the GPU
against the FP64 oracle: counts exact wherever no decision was within the
oracle's near-threshold margin, the keep mask and the height range exact."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2411_00771_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _cams(rng, k, sizes=((320, 180), (640, 360), (101, 77))):
    out = []
    for i in range(k):
        W, H = sizes[i % len(sizes)]
        out.append(syn.orbit_camera(rng, W, H, radius=rng.uniform(60, 140), altitude=rng.uniform(30, 90)))
    return out


def _compare(pts, sigma, cams, **kw):
    from paper_2411_00771_gb300 import binding as B
    d = torch.from_numpy(np.ascontiguousarray(pts, np.float32)).cuda()
    c = B.visibility_count(d, sigma, cams, **kw)
    torch.cuda.synchronize()
    ref, fl = oracle.visibility_count(np.asarray(pts, np.float32), sigma, cams, **{k: v for k, v in kw.items()
                                                                                 if k in ("lowpass",)})
    ok = fl == 0
    got = c.cpu().numpy().astype(np.int64)
    assert ok.mean() > 0.99
    assert np.array_equal(got[ok], ref[ok])
    assert np.all(np.abs(got - ref) <= fl)
    return d, c, ref


def test_counts_match_oracle_random_points():
    rng = np.random.default_rng(1)
    pts = rng.uniform([-80, -80, -5], [80, 80, 40], (50_000, 3))
    _, c, ref = _compare(pts, 0.4, _cams(rng, 30))
    assert 0 < ref.mean() < 30 and ref.min() < ref.max()


def test_counts_on_city_points_and_accumulation():
    from paper_2411_00771_gb300 import binding as B
    scene, _ = syn.city_scene(n=300_000)
    rng = np.random.default_rng(2)
    cams = [syn.orbit_camera(rng, 480, 270, radius=rng.uniform(150, 250), altitude=rng.uniform(150, 250))
            for _ in range(40)]
    d, c, ref = _compare(scene["mu"], 0.2, cams)
    B.visibility_count(d, 0.2, cams[:5], counts=c)  # accumulates
    ref5, fl5 = oracle.visibility_count(np.asarray(scene["mu"], np.float32), 0.2, cams[:5])
    torch.cuda.synchronize()
    ok = (fl5 == 0) & (oracle.visibility_count(np.asarray(scene["mu"], np.float32), 0.2, cams)[1] == 0)
    assert np.array_equal(c.cpu().numpy().astype(np.int64)[ok], (ref + ref5)[ok])


def test_keep_mask_and_height_range():
    from paper_2411_00771_gb300 import binding as B
    rng = np.random.default_rng(3)
    pts = rng.uniform([-60, -60, -3], [60, 60, 35], (20_000, 3)).astype(np.float32)
    cams = _cams(rng, 12)
    d, c, ref = _compare(pts, 0.3, cams)
    for m in (0, 3, 13):
        keep, zr = B.visibility_bounds(d, c, m)
        torch.cuda.synchronize()
        rk, (lo, hi) = oracle.visible_height_range(pts, c.cpu().numpy(), m)
        assert np.array_equal(keep.cpu().numpy().astype(bool), rk)
        z = zr.cpu().numpy()
        if lo is None:
            assert np.isnan(z).all()
        else:
            assert z[0] == np.float32(lo) and z[1] == np.float32(hi)


def test_visibility_edge_cases():
    from paper_2411_00771_gb300 import binding as B
    rng = np.random.default_rng(4)
    cams = _cams(rng, 3)
    empty = torch.zeros((0, 3), device="cuda")
    assert B.visibility_count(empty, 0.1, cams).numel() == 0
    pts = torch.zeros((5, 3), device="cuda")
    assert int(B.visibility_count(pts, 0.1, []).sum()) == 0
    with pytest.raises(B.GsError):
        B.visibility_count(pts, -1.0, cams)
