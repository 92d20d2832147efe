"""Large-scene stress: 25M surfels of the city distribution on a 500 m x 2 km
strip, SH degree 3, at 3840x2160, and a forward sweep over smaller prefixes of
the same scene.

The oracle cannot replay every pixel of a 25M-surfel 4K view in a test's time,
so the forward is compared on sampled pixels (the oracle renders any subset
of pixels exactly), and the backward through a window: the 4K backward with
adjoints that are zero outside a 256x256 window must equal the backward of a
crop camera over that window (the same pixels, the same surfels), which the
oracle checks in full."""
import numpy as np
import pytest
import torch

import oracle
from paper_2411_00771_gb300 import synthetic as syn
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

FLAG_ANY = oracle.FLAG_ALPHA | oracle.FLAG_RHO | oracle.FLAG_TSTOP | oracle.FLAG_MEDIAN
W4K, H4K = 3840, 2160


@pytest.fixture(scope="module")
def strip():
    scene, info = syn.city_scene(n=25_000_000, extent=(500.0, 2000.0), n_boxes=800)
    cam = syn.aerial_camera(width=W4K, height=H4K, altitude=250.0, azimuth_deg=-90.0)
    return scene, cam


def _subset(scene, n):
    return {k: (v[:n] if isinstance(v, np.ndarray) else v) for k, v in scene.items()}


def cond_scale(cond):
    """Tolerance factor of a pixel whose blended object-branch pairs have
    centred-Jacobian condition number up to k.  The plane coordinates
    (u, v) = Ji d come from an inverse Jacobian held in FP32, so their
    relative error is up to about k 2^-23; rho = u^2 + v^2 doubles it, and
    alpha = o exp(-rho / 2) turns it into a relative error of alpha of
    (rho / 2)(2 k 2^-23) <= 9 k 2^-23 (rho <= 9), which every weighted plane
    inherits.  Nearly edge-on surfels (large k) are common in an oblique 4K
    view of a dense scene; where that bound exceeds the 2e-5 of the render
    tolerance, the tolerance grows with it."""
    return np.maximum(1.0, 9.0 * cond * 2.0 ** -23 / gu.TOL_ABS)


def _compare_sampled(scene, cam, out, cnt, n_pix, seed):
    """Sampled pixels against the oracle with the render tolerances, scaled
    by cond_scale() at pixels with ill-conditioned pairs."""
    W, H = int(cam["width"]), int(cam["height"])
    pix = np.random.default_rng(seed).choice(W * H, n_pix, replace=False)
    ref = oracle.render(scene, cam, pixels=pix)
    bad = (ref["flags"] & FLAG_ANY) != 0
    assert bad.mean() < 0.01, bad.sum()
    g = np.asarray(out, np.float64).reshape(12, -1)[:, pix]
    scale = cond_scale(oracle.pixel_cond(scene, cam).reshape(-1)[pix])
    q = np.abs(g - ref["out"]) / (gu.plane_tolerance(ref["out"]) * scale[None, :])
    branch = (ref["flags"] & oracle.FLAG_BRANCH) != 0
    for p, name in enumerate(gu.PLANES):
        ok = ~bad & ~branch if p in gu.DEPTH_PLANES else ~bad
        e = q[p, ok].max() if ok.any() else 0.0
        assert e <= 1.0, (name, e)
    assert np.array_equal(cnt.reshape(-1)[pix][~bad], ref["count"][~bad])
    return ref


def test_strip_4k_forward_on_sampled_pixels(strip):
    scene, cam = strip
    sc, d, out, cnt, frame = gu.gpu_render(scene, cam)
    info = frame.info()
    frame.release()
    assert info["n_visible"] > 1_000_000 and info["n_instances"] > info["n_visible"]
    ref = _compare_sampled(scene, cam, out.cpu().numpy(), cnt.cpu().numpy(), 20_000, seed=1)
    assert (ref["count"] > 0).mean() > 0.5  # the samples land on the city, not on the sky


def _crop(cam, x0, y0, size):
    c = dict(cam)
    c["width"] = c["height"] = size
    c["cx"] = cam["cx"] - x0
    c["cy"] = cam["cy"] - y0
    return c


def test_strip_4k_backward_through_a_window(strip):
    scene, cam = strip
    x0, y0, S = 1808, 1040, 256  # a window near the image centre, not tile-aligned in y
    rng = np.random.default_rng(2)
    win = (rng.normal(size=(11, S, S)) * 1e-3).astype(np.float32)
    n = scene["mu"].shape[0]
    # 4K frame, adjoints only inside the window
    sc, d, out, cnt, frame = gu.gpu_render(scene, cam)
    adj = torch.zeros((11, H4K, W4K), device="cuda")
    adj[:, y0:y0 + S, x0:x0 + S] = torch.from_numpy(win).cuda()
    g4 = {k: torch.zeros_like(v) for k, v in d.items()}
    s4 = torch.zeros((1, n, 2), device="cuda")
    sc.backward(frame, [adj], [0x7FF], g4, s4)
    frame.release()
    # crop camera over the window
    cc = _crop(cam, x0, y0, S)
    out_c, frame_c = sc.render(cc)
    gc = {k: torch.zeros_like(v) for k, v in d.items()}
    scr = torch.zeros((1, n, 2), device="cuda")
    sc.backward(frame_c, [torch.from_numpy(win).cuda()], [0x7FF], gc, scr)
    frame_c.release()
    torch.cuda.synchronize()
    # the window of the 4K render is the crop render, up to pixels with a
    # decision at a threshold (pixel offsets are taken from different tile
    # origins, so they round differently)
    full = out[:, y0:y0 + S, x0:x0 + S].cpu().numpy().astype(np.float64)
    crop = out_c.cpu().numpy().astype(np.float64)
    rel = np.abs(full - crop) / np.maximum(1.0, np.abs(crop))
    assert (rel[:11] > 1e-4).any(axis=0).mean() <= 0.01
    for k in ("mu", "quat", "scale", "opacity", "sh"):
        e = gu.rel_err(g4[k].cpu().numpy(), gc[k].cpu().numpy())
        assert e <= 1e-3, (k, e)
    # the crop against the oracle, every pixel and every surfel
    ref = oracle.backward(scene, cc, win[None].astype(np.float64))
    for k in ("mu", "quat", "scale", "opacity", "sh"):
        e = gu.rel_err(gc[k].cpu().numpy(), ref[k].reshape(gc[k].shape))
        assert e <= 1e-3, (k, e)
    assert gu.rel_err(scr.cpu().numpy()[0], ref["screen"][0]) <= 1e-3


@pytest.mark.parametrize("n", [1_000_000, 5_000_000])
def test_forward_sweep_prefixes_on_sampled_pixels(strip, n):
    """Prefixes of the area-sampled strip are uniform subsamples: the same
    view at 1M and 5M surfels, sampled pixels against the oracle."""
    scene, cam = strip
    sub = _subset(scene, n)
    sc, d, out, cnt, frame = gu.gpu_render(sub, cam)
    frame.release()
    _compare_sampled(sub, cam, out.cpu().numpy(), cnt.cpu().numpy(), 8_000, seed=n)
