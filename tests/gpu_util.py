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
