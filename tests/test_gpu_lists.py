"""Tile lists and ranges bit for bit (Eq. 1 composites each pixel's surfels
front to back; the tiles' sorted lists carry that order).

For each case the lists the CUDA path built are rebuilt independently: the
GPU's own per-surfel inputs of the binning (footprint shape, FP32 centre
depth, tile count; gs_frame_copy_cover) go through a numpy restatement of the
FP32 row rule (tests/rowrule.py), the (tile, depth bits, surfel index) keys
are sorted with numpy, and the GPU's sorted surfel indices and per-tile
ranges must equal the rebuilt ones exactly.  Separately, the GPU's FP32
depths must be the oracle's FP64 centre depths rounded to FP32, and every
tile's list must contain the oracle's exact FP64 cover (the row rule only
adds entries, within its rounding margin, never drops one)."""
import numpy as np
import pytest

import oracle
from paper_2411_00771_gb300 import synthetic as syn
from tests import gpu_util as gu
from tests import rowrule as rr

pytestmark = pytest.mark.gpu

RF = np.float32(np.sqrt(9.0 / 2.0))  # rf = sqrt(rho_max / screen_inv_sigma2), rounded once


def _elongated():
    scene, cam, _, _ = syn.tiny_scene(seed=21, n=3000, width=200, height=120, fx=150.0,
                                      log_scale_range=(-4.0, -1.5))
    rng = np.random.default_rng(21)
    k = rng.uniform(size=3000) < 0.33
    scene["scale"][k, 0] *= np.exp(rng.uniform(np.log(10), np.log(60), k.sum())).astype(np.float32)
    return scene, cam


def _ragged():
    scene, cam, _, _ = syn.tiny_scene(seed=44, n=1500, width=100, height=75, fx=90.0, sh_degree=3,
                                      log_scale_range=(-4.5, -1.5))
    return scene, cam


def _city():
    scene, info = syn.city_scene(n=1_000_000)
    return scene, syn.aerial_camera()


def _dense(n):
    """n surfels seen at 64x64: 16 tiles with lists of thousands of entries
    (30k: up to 6.7k entries; 60k: up to 13k)."""
    def make():
        scene, cam, _, _ = syn.tiny_scene(seed=77, n=n, width=64, height=64, fx=64.0, sh_degree=1,
                                          log_scale_range=(-4.0, -2.5))
        return scene, cam
    return make


CASES = {"ragged": _ragged, "elongated": _elongated, "city": _city, "dense30k": _dense(30000),
         "dense60k": _dense(60000)}


@pytest.mark.parametrize("case", list(CASES))
def test_lists_and_ranges_bit_exact(case):
    scene, cam = CASES[case]()
    sc, d, out, cnt, frame = gu.gpu_render(scene, cam)
    vals, ranges, rects = [t.cpu().numpy() for t in frame.lists()]
    geom, depth, tcount = [t.cpu().numpy() for t in frame.cover()]
    frame.release()
    W, H = int(cam["width"]), int(cam["height"])
    tiles_x, tiles_y = (W + 15) // 16, (H + 15) // 16
    vis = np.nonzero(tcount > 0)[0]

    # the GPU's FP32 centre depth is the oracle's FP64 depth rounded to FP32
    pre = oracle.preprocess(scene, cam)
    zk = pre["zkey"][vis].astype(np.float32)
    assert np.array_equal(depth[vis], zk), np.nonzero(depth[vis] != zk)[0][:10]

    # the row rule on the GPU's footprint shapes gives its instances ...
    surf, tile = rr.instances(geom, vis, tiles_x, RF)
    assert np.array_equal(np.bincount(surf, minlength=tcount.size), tcount)
    # ... and the stable (tile, depth bits, index) order its lists and ranges
    exp_vals, exp_ranges = rr.sorted_lists(surf, tile, depth.view(np.uint32), tiles_x * tiles_y)
    assert vals.shape == exp_vals.shape
    assert np.array_equal(vals, exp_vals)
    assert np.array_equal(ranges, exp_ranges)

    # every list contains the oracle's exact FP64 cover
    start, idx, _ = oracle.tile_lists(scene, cam)
    otile = np.repeat(np.arange(tiles_x * tiles_y), np.diff(start))
    got = set(zip(tile.tolist(), surf.tolist()))
    missing = [(t, s) for t, s in zip(otile.tolist(), idx.tolist()) if (t, s) not in got]
    assert not missing, missing[:10]
    assert len(surf) <= 1.02 * len(idx) + 16
