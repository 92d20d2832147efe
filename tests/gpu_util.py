"""Helpers for the GPU parity tests: upload seeded inputs, run the CUDA path
through the C ABI, compare with the oracle."""
import numpy as np
import torch

PLANES = ["r", "g", "b", "alpha", "depth", "invdepth", "median", "nx", "ny", "nz", "distortion",
          "T_final"]
DEPTH_PLANES = (4, 5, 6, 10)  # planes that switch value with the object/screen branch
TOL_ABS = 2e-5  # channel tolerance; planes whose values exceed 1 scale it by |value|


def to_dev(scene, device="cuda"):
    keys = ("mu", "quat", "scale", "opacity", "sh")
    return {k: torch.from_numpy(np.ascontiguousarray(scene[k], np.float32)).to(device) for k in keys}


def gpu_scene(scene, settings=None, device="cuda"):
    from paper_2411_00771_gb300 import binding as B
    d = to_dev(scene, device)
    s = B.default_settings(**(settings or {}))
    sc = B.Scene(d["mu"], d["quat"], d["scale"], d["opacity"], d["sh"], scene["sh_degree"], s)
    return sc, d


def gpu_render(scene, cam, settings=None):
    from paper_2411_00771_gb300 import binding as B
    sc, d = gpu_scene(scene, settings)
    H, W = cam["height"], cam["width"]
    cnt = torch.empty((H, W), dtype=torch.int32, device="cuda")
    out, frame = sc.render(cam, n_contrib=cnt)
    torch.cuda.synchronize()
    return sc, d, out, cnt, frame


U32 = 2.0 ** -24  # FP32 unit roundoff


def plane_tolerance(ref_out):
    """Per-pixel tolerance of each plane: 2e-5 x max(1, |value|).  The
    distortion plane adds 16 u Z (u the FP32 unit roundoff, Z the depth
    plane): every FP32 depth z_i carries a few roundings (|dz_i| <= 4 u z_i)
    and |dD/dz_i| <= 2 w_i, so the FP32 representation of the depths alone
    moves D by up to 8 u sum w_i z_i."""
    r = np.asarray(ref_out, np.float64)
    tol = TOL_ABS * np.maximum(1.0, np.abs(r))
    tol[10] = tol[10] + 16 * U32 * np.abs(r[4])
    return tol


def plane_violations(gpu_out, ref_out, mask):
    """Max over pixels in mask of |gpu - ref| / tolerance, per plane."""
    g = np.asarray(gpu_out, np.float64)
    r = np.asarray(ref_out, np.float64)
    q = np.abs(g - r) / plane_tolerance(r)
    q = q[:, mask]
    return q.max(axis=1) if q.size else np.zeros(g.shape[0])


def channel_errors(gpu_out, ref_out, mask=None):
    """Per-plane max |gpu - ref| / max(1, |ref|) over pixels in mask."""
    g = np.asarray(gpu_out, np.float64)
    r = np.asarray(ref_out, np.float64)
    e = np.abs(g - r) / np.maximum(1.0, np.abs(r))
    if mask is not None:
        e = e[:, mask]
    return e.reshape(e.shape[0], -1).max(axis=1) if e.size else np.zeros(g.shape[0])


def rel_err(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def visible(pre):
    """Surfels with a non-empty tile rectangle (the densification's
    'visible in this view')."""
    r = pre["rect"]
    return (pre["live"] > 0) & (r[:, 2] > r[:, 0]) & (r[:, 3] > r[:, 1])


# ---- sampled-pixel comparison of large views ----------------------------------

def compare_sampled(scene, cam, out, cnt, n_pix, seed):
    """Sampled pixels against the oracle at the plain render tolerances
    (plane_tolerance), counts bit-exact outside flagged pixels.  Returns the
    oracle's result for the samples, with "cond": the largest condition
    number of the centred Jacobian among each sampled pixel's blended
    object-space pairs (nearly edge-on or elongated disks make it large)."""
    import oracle
    W, H = int(cam["width"]), int(cam["height"])
    pix = np.random.default_rng(seed).choice(W * H, n_pix, replace=False)
    ref = oracle.render(scene, cam, pixels=pix)
    flag_any = oracle.FLAG_ALPHA | oracle.FLAG_RHO | oracle.FLAG_TSTOP | oracle.FLAG_MEDIAN
    bad = (ref["flags"] & flag_any) != 0
    assert bad.mean() < 0.01, bad.sum()
    g = np.asarray(out, np.float64).reshape(12, -1)[:, pix]
    q = np.abs(g - ref["out"]) / plane_tolerance(ref["out"])
    branch = (ref["flags"] & oracle.FLAG_BRANCH) != 0
    for p, name in enumerate(PLANES):
        ok = ~bad & ~branch if p in DEPTH_PLANES else ~bad
        e = q[p, ok].max() if ok.any() else 0.0
        assert e <= 1.0, (name, e)
    assert np.array_equal(cnt.reshape(-1)[pix][~bad], ref["count"][~bad])
    ref["cond"] = oracle.pixel_cond(scene, cam).reshape(-1)[pix]
    return ref


def crop_camera(cam, x0, y0, size):
    c = dict(cam)
    c["width"] = c["height"] = size
    c["cx"] = cam["cx"] - x0
    c["cy"] = cam["cy"] - y0
    return c


def check_window_backward(scene, cam, x0, y0, S, seed):
    """The backward through a window: the full view's backward with adjoints
    that are zero outside the S x S window at (x0, y0) must equal the backward
    of a crop camera over that window (the same pixels and surfels), which the
    oracle checks over every pixel and surfel (1e-3 relative).  The two renders
    agree up to pixels with a decision at a threshold (pixel offsets are taken
    from different tile origins, so they round differently)."""
    import oracle
    H, W = int(cam["height"]), int(cam["width"])
    rng = np.random.default_rng(seed)
    win = (rng.normal(size=(11, S, S)) * 1e-3).astype(np.float32)
    n = scene["mu"].shape[0]
    sc, d, out, cnt, frame = gpu_render(scene, cam)
    adj = torch.zeros((11, H, W), device="cuda")
    adj[:, y0:y0 + S, x0:x0 + S] = torch.from_numpy(win).cuda()
    gf = {k: torch.zeros_like(v) for k, v in d.items()}
    sf = torch.zeros((1, n, 2), device="cuda")
    sc.backward(frame, [adj], [0x7FF], gf, sf)
    frame.release()
    cc = crop_camera(cam, x0, y0, S)
    out_c, frame_c = sc.render(cc)
    gc = {k: torch.zeros_like(v) for k, v in d.items()}
    scr = torch.zeros((1, n, 2), device="cuda")
    sc.backward(frame_c, [torch.from_numpy(win).cuda()], [0x7FF], gc, scr)
    frame_c.release()
    torch.cuda.synchronize()
    full = out[:, y0:y0 + S, x0:x0 + S].cpu().numpy().astype(np.float64)
    crop = out_c.cpu().numpy().astype(np.float64)
    rel = np.abs(full - crop) / np.maximum(1.0, np.abs(crop))
    assert (rel[:11] > 1e-4).any(axis=0).mean() <= 0.01
    for k in ("mu", "quat", "scale", "opacity", "sh"):
        e = rel_err(gf[k].cpu().numpy(), gc[k].cpu().numpy())
        assert e <= 1e-3, (k, e)
    ref = oracle.backward(scene, cc, win[None].astype(np.float64))
    for k in ("mu", "quat", "scale", "opacity", "sh"):
        e = rel_err(gc[k].cpu().numpy(), ref[k].reshape(gc[k].shape))
        assert e <= 1e-3, (k, e)
    assert rel_err(scr.cpu().numpy()[0], ref["screen"][0]) <= 1e-3
